// pade.cu -- the linear solve of the diagonal Pade comparator: (v - u) R = u + v
// (eq. pade10 / eq. pade26). The paper counts it as 4/3 of a product: an LU
// factorisation with partial pivoting (1/3) and N forward / back substitutions (1).
//  N <= 112: the right-hand sides are independent once L, U and the pivots are
//    known, so each CTA of ceil(N / 4) factors M on its own in shared memory (the
//    same pivots everywhere: the choice is deterministic) and carries 4 of the
//    right-hand sides through the elimination and the back substitution (a warp
//    per right-hand side); no CTA waits for another.
//  N > 112: the blocked LU of lu_blocked.cu (panels factored by a thread-block
//    cluster, FP64 rank-32 updates of the trailing rows and of the right-hand sides).
#include <math.h>

#include <mutex>

#include "internal.h"

namespace bbc {
namespace {

constexpr int SMEM_SOLVE_THREADS = 512;
constexpr int SMEM_SOLVE_COLS = 4;      // right-hand sides per CTA
constexpr int SMEM_SOLVE_MAX_N = 112;   // (N^2 + 4 N) doubles fit the 227 KB of one CTA

__global__ void __launch_bounds__(SMEM_SOLVE_THREADS, 1)
k_lu_solve_smem(const double* __restrict__ M, double* __restrict__ B, int N, unsigned int* __restrict__ flag) {
  constexpr int T = SMEM_SOLVE_THREADS, C = SMEM_SOLVE_COLS;
  extern __shared__ double sh[];
  double* m = sh;          // N x N, row-major
  double* b = sh + N * N;  // C x N: this CTA's right-hand sides, each contiguous
  __shared__ int s_piv, s_singular;
  const int tid = threadIdx.x, c0 = blockIdx.x * C;
  const int nc = min(C, N - c0);
  for (int e = tid; e < N * N; e += T) m[e] = M[e];
  for (int e = tid; e < N * nc; e += T) b[(e % nc) * N + e / nc] = B[(int64_t)(e / nc) * N + c0 + e % nc];
  if (tid == 0) s_singular = 0;
  __syncthreads();
  for (int k = 0; k < N; ++k) {
    if (tid < 32) {  // pivot: largest |m_ik|, i >= k (ties to the smaller row)
      double best = -1.0;
      int bi = N;
      for (int i = k + tid; i < N; i += 32) {
        const double v = fabs(m[i * N + k]);
        if (v > best) { best = v; bi = i; }
      }
      for (int off = 16; off > 0; off >>= 1) {
        const double ov = __shfl_xor_sync(0xffffffffu, best, off);
        const int oi = __shfl_xor_sync(0xffffffffu, bi, off);
        if (ov > best || (ov == best && oi < bi)) { best = ov; bi = oi; }
      }
      if (tid == 0) {
        s_piv = bi;
        if (!(best > 0.0)) s_singular = 1;
      }
    }
    __syncthreads();
    const int piv = s_piv;
    if (piv != k && piv < N) {
      for (int j = tid; j < N + nc; j += T) {
        double* r0 = j < N ? m + k * N + j : b + (j - N) * N + k;
        double* r1 = j < N ? m + piv * N + j : b + (j - N) * N + piv;
        const double t = *r0;
        *r0 = *r1;
        *r1 = t;
      }
    }
    __syncthreads();
    const double d = m[k * N + k];
    for (int i = k + 1 + tid; i < N; i += T) m[i * N + k] /= d;
    __syncthreads();
    const int rows = N - k - 1, w = rows + nc;
    for (int e = tid; e < rows * w; e += T) {
      const int i = k + 1 + e / w, c = e % w;
      const double l = m[i * N + k];
      if (c < rows) m[i * N + k + 1 + c] -= l * m[k * N + k + 1 + c];
      else b[(c - rows) * N + i] -= l * b[(c - rows) * N + k];
    }
    __syncthreads();
  }
  // back substitution, one warp per right-hand side: x_i = (b_i - sum_{t > i} u_it x_t) / u_ii,
  // the lanes splitting the sum (a butterfly reduction leaves the same value in every lane)
  const int warp = tid >> 5, lane = tid & 31;
  if (warp < nc) {
    double* x = b + warp * N;  // solved in place
    bool bad = s_singular != 0;
    for (int i = N - 1; i >= 0; --i) {
      double acc = 0.0;
      for (int t = i + 1 + lane; t < N; t += 32) acc = fma(m[i * N + t], x[t], acc);
      for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
      const double xi = (x[i] - acc) / m[i * N + i];
      __syncwarp();
      if (lane == 0) x[i] = xi;
      __syncwarp();
      bad |= !isfinite(xi);
    }
    if (bad && lane == 0 && flag) atomicOr(flag, 1u);
  }
  __syncthreads();
  for (int e = tid; e < N * nc; e += T) B[(int64_t)(e / nc) * N + c0 + e % nc] = b[(e % nc) * N + e / nc];
}

}  // namespace

cudaError_t lu_solve_inplace(double* M, double* B, int64_t N, unsigned int* flag, cudaStream_t st,
                             double* scratch) {
  if (N < 1) return cudaErrorInvalidValue;
  if (N <= SMEM_SOLVE_MAX_N) {
    const size_t bytes = (size_t)(N * N + N * SMEM_SOLVE_COLS) * sizeof(double);
    static bool attr_set[64] = {};  // the shared-memory opt-in is per device
    int dev = 0;
    cudaError_t err = cudaGetDevice(&dev);
    if (err != cudaSuccess) return err;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    if (!attr_set[dev]) {
      err = cudaFuncSetAttribute(
          k_lu_solve_smem, cudaFuncAttributeMaxDynamicSharedMemorySize,
          (int)((SMEM_SOLVE_MAX_N * SMEM_SOLVE_MAX_N + SMEM_SOLVE_MAX_N * SMEM_SOLVE_COLS) * sizeof(double)));
      if (err != cudaSuccess) return err;
      attr_set[dev] = true;
    }
    const unsigned grid = (unsigned)((N + SMEM_SOLVE_COLS - 1) / SMEM_SOLVE_COLS);
    k_lu_solve_smem<<<grid, SMEM_SOLVE_THREADS, bytes, st>>>(M, B, (int)N, flag);
    return cudaGetLastError();
  }
  return lu_blocked_solve(M, B, N, flag, st, scratch);
}

}  // namespace bbc
