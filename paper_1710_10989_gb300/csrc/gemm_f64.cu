// gemm_f64.cu -- FP64 dense product with the fused linear-combination epilogue.
//
// On GB300 the FP64 pipe issues about 1.6 DFMA per clock per SM (~1.0 TFLOP/s
// for the chip, measured; DMMA is no faster), roughly 1/70 of the FP32 rate. A
// product of the method (Section 1: the cost unit of scaling and squaring) is
// therefore bound by the FP64 pipe, not by HBM: with 64 x 64 tiles each operand
// element is re-read N/64 times from L2, far below what the FP64 pipe can
// consume. The kernel keeps the schedule simple: 64 x 64 x 16 tiles (32 x 32 up
// to N = 512 and 16 x 16 up to N = 256, to spread small matrices over more SMs),
// 256 threads, each thread a 4 x 4 (2 x 2, 1 x 1) register block with rows and
// columns strided by 16 so that shared memory reads are conflict-free and
// epilogue accesses coalesce, and the next K-slab prefetched into registers
// while the current one is multiplied. Every element sums k in the same order
// whatever the tile, so the tile choice changes no result.
#include "internal.h"

namespace bbc {
namespace {

constexpr int BK = 16;
constexpr int THREADS = 256;

template <int BM, int BN>
__global__ void __launch_bounds__(THREADS, 3)  // three blocks per SM keep the FP64 pipe fed
k_gemm_f64(const double* __restrict__ P, const double* __restrict__ Q, int64_t N, double alpha,
           const Epilogue e, int upper) {
  constexpr int TM = BM / 16, TN = BN / 16;
  constexpr int LP = BM * BK / THREADS;   // P elements per thread per slab
  constexpr int LQ = BK * BN / THREADS;   // Q elements per thread per slab
  constexpr int QROWS = THREADS / BN;     // Q rows covered by one pass of the block
  __shared__ double As[2][BK][BM];
  __shared__ double Bs[2][BK][BN];

  const int t = threadIdx.x;
  const int tx = t % 16, ty = t / 16;
  const int64_t m0 = (int64_t)blockIdx.y * BM, n0 = (int64_t)blockIdx.x * BN;

  double acc[TM][TN];
#pragma unroll
  for (int i = 0; i < TM; ++i)
#pragma unroll
    for (int j = 0; j < TN; ++j) acc[i][j] = 0.0;

  double rp[LP], rq[LQ];
  auto load = [&](int64_t k0) {
#pragma unroll
    for (int q = 0; q < LP; ++q) {
      const int64_t r = m0 + t / 16 + 16 * q, c = k0 + t % 16;
      rp[q] = (r < N && c < N) ? __ldg(P + r * N + c) : 0.0;
    }
#pragma unroll
    for (int q = 0; q < LQ; ++q) {
      const int64_t r = k0 + t / BN + QROWS * q, c = n0 + t % BN;
      rq[q] = (r < N && c < N) ? __ldg(Q + r * N + c) : 0.0;
    }
  };
  auto store = [&](int buf) {
#pragma unroll
    for (int q = 0; q < LP; ++q) As[buf][t % 16][t / 16 + 16 * q] = rp[q];
#pragma unroll
    for (int q = 0; q < LQ; ++q) Bs[buf][t / BN + QROWS * q][t % BN] = rq[q];
  };

  // K slabs to sum: all of them, or for upper triangular P and Q the slabs that
  // meet [m0, n0 + BN) (P_ik = 0 for k < i, Q_kj = 0 for k > j); none below the diagonal
  int64_t s0 = 0, s1 = (N + BK - 1) / BK;
  if (upper) {
    s0 = m0 / BK;
    s1 = min(s1, (n0 + BN + BK - 1) / BK);
  }
  if (s0 < s1) {
    load(s0 * BK);
    store(0);
  }
  __syncthreads();
  for (int64_t s = s0; s < s1; ++s) {
    const int buf = (int)((s - s0) & 1);
    if (s + 1 < s1) load((s + 1) * BK);
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      double a[TM], b[TN];
#pragma unroll
      for (int i = 0; i < TM; ++i) a[i] = As[buf][kk][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < TN; ++j) b[j] = Bs[buf][kk][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
    }
    if (s + 1 < s1) store(buf ^ 1);
    __syncthreads();
  }

  const bool zero_block = upper && n0 + BN <= m0;  // strictly below the diagonal: every output is 0
#pragma unroll
  for (int i = 0; i < TM; ++i) {
    const int64_t row = m0 + ty + 16 * i;
    if (row >= N) continue;
#pragma unroll
    for (int j = 0; j < TN; ++j) {
      const int64_t col = n0 + tx + 16 * j;
      if (col >= N) continue;
      if (zero_block) zero_epilogue(e, N, row, col);
      else apply_epilogue(e, N, row, col, alpha * acc[i][j]);
    }
  }
}

}  // namespace

cudaError_t gemm_f64(const double* P, const double* Q, int64_t N, double alpha, const Epilogue& e,
                     cudaStream_t st, bool upper) {
  if (N <= 256) {  // 16 x 16 tiles: a 64 x 64 product on 16 SMs, 256 x 256 on all of them
    dim3 grid((unsigned)((N + 15) / 16), (unsigned)((N + 15) / 16));
    k_gemm_f64<16, 16><<<grid, THREADS, 0, st>>>(P, Q, N, alpha, e, upper ? 1 : 0);
  } else if (N <= 512) {
    dim3 grid((unsigned)((N + 31) / 32), (unsigned)((N + 31) / 32));
    k_gemm_f64<32, 32><<<grid, THREADS, 0, st>>>(P, Q, N, alpha, e, upper ? 1 : 0);
  } else {
    dim3 grid((unsigned)((N + 63) / 64), (unsigned)((N + 63) / 64));
    k_gemm_f64<64, 64><<<grid, THREADS, 0, st>>>(P, Q, N, alpha, e, upper ? 1 : 0);
  }
  return cudaGetLastError();
}

}  // namespace bbc
