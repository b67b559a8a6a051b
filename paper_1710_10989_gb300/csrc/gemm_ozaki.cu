// gemm_ozaki.cu -- FP64 products computed exactly from BF16 slices on the
// tcgen05 tensor cores (an error-free splitting in the manner of Ozaki et al.).
//
// Why: the scaling-and-squaring cost is the number of dense products (Section 1,
// Section 4 of Bader-Blanes-Casas). GB300 runs FP64 at ~1.25 TFLOP/s but dense
// BF16 at ~2 PFLOP/s, so a product rebuilt from k^2/2 BF16 products is far
// faster than one FP64 product, and it is exact up to the slicing.
//
// Splitting. Row i of P gets a power-of-two scale 2^e_i with max_k |P_ik| < 2^(e_i-1);
// column j of Q gets 2^f_j likewise. Each scaled entry is rounded to a fixed-point
// integer with 8k fractional bits and cut into k balanced base-256 digits
// d_0..d_{k-1} (|d_0| <= 128, |d_p| <= 128): P_ik ~ sum_p d_p 2^(e_i - 8(p+1)).
// Digits are small integers, exact in BF16. The extraction is pure integer work
// on the FP64 bit pattern (no FP64 arithmetic: the FP64 pipe is the slow one).
//
// Diagonal deflation. The scheme's operands (B_j = b_0j I + ..., T = I + X + ...)
// are dominated by their diagonal, which would set the row and column scales
// and leave the off-diagonal entries ~10 fewer bits. So the diagonals are taken
// out before slicing (P = D_P + P', Q = D_Q + Q') and added back exactly in the
// epilogue: P Q = P'Q' + D_P Q + P D_Q - D_P D_Q (elementwise: P_ii Q_ij +
// P_ij Q_jj - [i = j] P_ii Q_jj).
//
// Exact products. Pairs (p, q) with g = p + q <= k - 1 are kept (the triangle),
// C_ij = 2^(e_i + f_j - 16) sum_g 2^(-8g) S_g with S_g = sum_{p+q=g} sum_k d^P d^Q,
// an error of order 2^(-8k) relative to the row and column scales.
//  * High groups g <= 4 carry weights down to 2^-32 and are summed exactly.
//    A product of digits is at most 2^14, so a sum of up to 1024 of them is an
//    integer below 2^24 and FP32 holds it exactly: the K loop of these pairs is
//    cut into 1024-wide chunks, and after each chunk the FP32 tile is drained from
//    TMEM, converted to int32 and added, shifted by 2^(8(4-g)), into an integer
//    accumulator R (two 32-bit TMEM planes; |R| < 2^60 for N <= 16384).
//  * Low groups g >= 5 weigh at most 2^-40. They accumulate in a second FP32 TMEM
//    tile over the whole K, Horner-style from the smallest weight up, the MMA
//    scaling the running sum by 2^-8 (scale-input-d) at each change of group.
//    That FP32 sum of up to ~10^5 terms loses roughly 2^-16 of itself, i.e. about
//    2^-56 of the result. (With the exact/FP32 boundary one group lower, at g = 4,
//    the same loss showed up as ~1e-14 relative error per product at N = 4096.)
//  C_ij = 2^(e_i + f_j - 48) (R + 2^-8 LOW).
//
// Kernel shape (one CTA per 128 x 128 output tile, 6 warps):
//   warp 0: TMA producer (3-D tensor maps over the slice planes, 128B swizzle),
//           6-stage ring of 128x64 BF16 A and B tiles;
//   warp 1: tcgen05.mma issuer (M=128, N=128, K=16, BF16 -> FP32 in TMEM). High
//           and low chunks are interleaved so each drain overlaps low-group MMAs;
//   warps 2-5: drain (tcgen05.ld / st) and the final FP64 epilogue.
//           with no low groups (k <= 5) the high accumulator is double-buffered;
// TMEM: [0,128) high accumulator, [128,256) low accumulator (or the second high
// buffer), [256,384) low and [384,512) high words of R.
// Every mbarrier wait is bounded in time; on expiry the kernel records a
// timeout in the status word, lets its copies and MMAs finish (bounded again),
// frees TMEM and returns.
#include <cuda.h>
#include <stdint.h>

#include <cstring>
#include <mutex>

#include "internal.h"

namespace bbc {
namespace {

constexpr int TILE = 128;          // M = N tile
constexpr int KSTEP = 64;          // BF16 elements per 128-byte swizzle row
constexpr int CHUNK_STEPS = 16;    // 16 x 64 = 1024 K per exact FP32 chunk
constexpr int STAGES = 6;
constexpr int STAGE_BYTES = TILE * KSTEP * 2;  // 16 KB per operand tile
constexpr int NUM_THREADS = 192;
constexpr int NUM_EPI = 128;
constexpr int G_EXACT = 5;         // groups 0..4 are summed exactly
constexpr unsigned long long TIMEOUT_NS = 2000000000ull;  // 2 s per wait
constexpr unsigned int STATUS_NONFINITE = 1u;  // bits of the handle's status word
constexpr unsigned int STATUS_TIMEOUT = 2u;

// ---------------------------------------------------------------- PTX helpers
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ unsigned long long globaltimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait. Returns false when the CTA already failed or the wait expired
// (then the CTA-wide flag is raised so that every other role stops too).
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, volatile int* cta_err) {
  if (mbar_try_wait(bar, parity)) return true;
  const unsigned long long t0 = globaltimer();
  for (uint32_t it = 1;; ++it) {
    if (mbar_try_wait(bar, parity)) return true;
    if ((it & 63) == 0) {
      if (*cta_err) return false;
      if (globaltimer() - t0 > TIMEOUT_NS) {
        *cta_err = 1;
        return false;
      }
    }
  }
}
__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, uint64_t* bar, int x, int y,
                                            int z) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4, %5}], "
      "[%2];" ::"r"(smem_u32(dst)),
      "l"(map), "r"(smem_u32(bar)), "r"(x), "r"(y), "r"(z)
      : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// Shared-memory matrix descriptor: K-major tile, rows of 128 bytes, 128-byte
// swizzle, 8-row core groups 1024 bytes apart.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr) {
  uint64_t d = 0;
  d |= (uint64_t)((addr & 0x3FFFF) >> 4);         // start address
  d |= (uint64_t)1 << 16;                          // leading byte offset (unused for this layout)
  d |= (uint64_t)(1024 >> 4) << 32;                // stride byte offset
  d |= (uint64_t)1 << 46;                          // descriptor version
  d |= (uint64_t)2 << 61;                          // 128-byte swizzle
  return d;
}
// Instruction descriptor, kind::f16: BF16 A and B, FP32 D, both K-major.
constexpr uint32_t IDESC = (1u << 4)                     // D = F32
                           | (1u << 7)                   // A = BF16
                           | (1u << 10)                  // B = BF16
                           | ((uint32_t)(TILE >> 3) << 17)   // N
                           | ((uint32_t)(TILE >> 4) << 24);  // M

__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(
          d_tmem),
      "l"(a), "l"(b), "r"(IDESC), "r"(accumulate)
      : "memory");
}
// D = A B + 2^-8 D (the running low-group sum moves one group down in weight)
__device__ __forceinline__ void mma_bf16_scaled(uint32_t d_tmem, uint64_t a, uint64_t b) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, 1, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p, 8;\n}\n" ::"r"(
          d_tmem),
      "l"(a), "l"(b), "r"(IDESC)
      : "memory");
}
__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}

#define TMEM_REGS32(r)                                                                                      \
  "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]), \
      "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]),   \
      "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),  \
      "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
#define TMEM_VALS32(r)                                                                                          \
  "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]), "r"(r[8]), "r"(r[9]), \
      "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]), "r"(r[15]), "r"(r[16]), "r"(r[17]),           \
      "r"(r[18]), "r"(r[19]), "r"(r[20]), "r"(r[21]), "r"(r[22]), "r"(r[23]), "r"(r[24]), "r"(r[25]),            \
      "r"(r[26]), "r"(r[27]), "r"(r[28]), "r"(r[29]), "r"(r[30]), "r"(r[31])

// 32 lanes x 32 consecutive 32-bit columns: thread t gets lane (base + t).
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&r)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,%18,"
      "%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : TMEM_REGS32(r)
      : "r"(taddr));
}
__device__ __forceinline__ void tmem_st32(uint32_t taddr, const uint32_t (&r)[32]) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,"
      "%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31,%32};" ::"r"(taddr),
      TMEM_VALS32(r)
      : "memory");
}
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }
__device__ __forceinline__ void tmem_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }

// ------------------------------------------------------------ digit extraction
// Biased exponent field of x; subnormals and zero report 1 and 0 respectively
// through the same rule max(E, 1) used below. Non-finite -> 0x7FF.
__device__ __forceinline__ int exp_field(double x) {
  return (int)((__double_as_longlong(x) >> 52) & 0x7FF);
}

// round(x * 2^(8k - e)) for |x| < 2^(e-1), with e = Emax - 1021 (Emax the largest
// biased exponent in the row/column): integer shift of the 53-bit significand.
__device__ __forceinline__ long long fixed_point(double x, int Emax, int k) {
  const unsigned long long bits = (unsigned long long)__double_as_longlong(x);
  int E = (int)((bits >> 52) & 0x7FF);
  unsigned long long M = bits & 0xFFFFFFFFFFFFFull;
  if (E == 0) E = 1; else M |= 1ull << 52;
  const int sh = 8 * k - 54 - (Emax - E);  // value * 2^(8k - e) = M * 2^sh
  long long X;
  if (sh >= 0) X = (long long)(M << sh);
  else if (sh > -60) X = (long long)((M + (1ull << (-sh - 1))) >> (-sh));
  else X = 0;
  return (bits >> 63) ? -X : X;
}

// Exact BF16 bit pattern of a small integer d (|d| <= 256).
__device__ __forceinline__ uint32_t bf16_of_int(int d) {
  const float f = __int_as_float(0x4B400000 + d) - 12582912.0f;  // exact for |d| < 2^22
  return (uint32_t)__float_as_uint(f) >> 16;
}

// Balanced base-256 digits, most significant first, as BF16 bit patterns.
template <int K>
__device__ __forceinline__ void digits(long long X, uint32_t (&out)[K]) {
#pragma unroll
  for (int p = K - 1; p >= 1; --p) {
    const long long low = ((X + 128) & 255) - 128;
    out[p] = bf16_of_int((int)low);
    X = (X - low) >> 8;
  }
  out[0] = bf16_of_int((int)X);
}

// P (N x N, row-major FP64) -> K slice planes [K][Rp][Kp] of BF16 digits with
// row exponents. One warp per row; padding rows/columns are written as zeros.
template <int K>
__global__ void __launch_bounds__(256)
k_split_rows(const double* __restrict__ P, int64_t N, int64_t Rp, int64_t Kp, uint16_t* __restrict__ planes,
             int* __restrict__ erow, double* __restrict__ pdiag, unsigned int* __restrict__ status) {
  const int64_t row = (int64_t)blockIdx.x * 8 + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (row >= Rp) return;
  const size_t plane = (size_t)Rp * Kp;
  uint32_t* out = reinterpret_cast<uint32_t*>(planes);  // bf16 pairs
  int Emax = 0;
  bool bad = false;
  if (row < N) {
    for (int64_t j = lane; j < N; j += 32) {
      const int E = (j == row) ? 0 : exp_field(__ldg(P + row * N + j));
      bad |= (E == 0x7FF);
      Emax = max(Emax, E);
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) Emax = max(Emax, __shfl_xor_sync(0xffffffffu, Emax, off));
    bad = __any_sync(0xffffffffu, bad);
  }
  if (bad == false && row < N) {  // the diagonal itself may be non-finite
    const int Ed = (lane == 0) ? exp_field(__ldg(P + row * N + row)) : 0;
    bad = __any_sync(0xffffffffu, Ed == 0x7FF);
  }
  if (bad && lane == 0) atomicOr(status, STATUS_NONFINITE);
  if (lane == 0) {
    erow[row] = (row < N && !bad) ? Emax - 1021 : 0;
    pdiag[row] = (row < N && !bad) ? __ldg(P + row * N + row) : 0.0;
  }
  Emax = max(Emax, 1);
  for (int64_t j = 2 * lane; j < Kp; j += 64) {
    uint32_t d0[K], d1[K];
    const double x0 = (row < N && j < N && j != row && !bad) ? __ldg(P + row * N + j) : 0.0;
    const double x1 = (row < N && j + 1 < N && j + 1 != row && !bad) ? __ldg(P + row * N + j + 1) : 0.0;
    digits<K>(fixed_point(x0, Emax, K), d0);
    digits<K>(fixed_point(x1, Emax, K), d1);
    const size_t idx = ((size_t)row * Kp + j) >> 1;
#pragma unroll
    for (int p = 0; p < K; ++p) out[p * (plane >> 1) + idx] = d0[p] | (d1[p] << 16);
  }
}

// Largest biased exponent per column of Q (fexp zeroed beforehand).
__global__ void __launch_bounds__(256)
k_col_maxexp(const double* __restrict__ Q, int64_t N, int64_t rows_per, int* __restrict__ fexp) {
  const int64_t j = (int64_t)blockIdx.x * 256 + threadIdx.x;
  if (j >= N) return;
  const int64_t r0 = (int64_t)blockIdx.y * rows_per;
  const int64_t r1 = min(N, r0 + rows_per);
  int m = 0;
  for (int64_t i = r0; i < r1; ++i) {
    const int E = exp_field(__ldg(Q + i * N + j));
    m = max(m, (i == j && E != 0x7FF) ? 0 : E);  // the diagonal is deflated (but still checked)
  }
  atomicMax(fexp + j, m);
}

// Q (N x N) -> K planes of Q^T digits [K][Rp][Kp] (plane row j holds column j of
// Q) with column exponents fcol. 32 x 32 tiles transposed through shared memory.
template <int K>
__global__ void __launch_bounds__(256)
k_split_cols(const double* __restrict__ Q, int64_t N, int64_t Rp, int64_t Kp, const int* __restrict__ fexp,
             uint16_t* __restrict__ planes, int* __restrict__ fcol, double* __restrict__ qdiag,
             unsigned int* __restrict__ status) {
  __shared__ uint16_t tile[K][32][34];
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  const int64_t i0 = (int64_t)blockIdx.x * 32;  // rows of Q (the K dimension)
  const int64_t j0 = (int64_t)blockIdx.y * 32;  // columns of Q
  const int64_t j = j0 + tx;
  const int Ej = (j < N) ? fexp[j] : 0;
  const bool bad = (Ej == 0x7FF);
  if (blockIdx.x == 0 && ty == 0 && j < Rp) {
    fcol[j] = (j < N && !bad) ? Ej - 1021 : 0;
    qdiag[j] = (j < N && !bad) ? __ldg(Q + j * N + j) : 0.0;
    if (bad) atomicOr(status, STATUS_NONFINITE);
  }
  const int Emax = max(Ej, 1);
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    const int il = ty + 8 * r;
    const int64_t i = i0 + il;
    const double x = (i < N && j < N && i != j && !bad) ? __ldg(Q + i * N + j) : 0.0;
    uint32_t d[K];
    digits<K>(fixed_point(x, Emax, K), d);
#pragma unroll
    for (int p = 0; p < K; ++p) tile[p][tx][il] = (uint16_t)d[p];
  }
  __syncthreads();
  const size_t plane = (size_t)Rp * Kp;
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    const int jl = ty + 8 * r;
    const int64_t jj = j0 + jl, ii = i0 + tx;
    if (jj < Rp && ii < Kp) {
#pragma unroll
      for (int p = 0; p < K; ++p) planes[p * plane + (size_t)jj * Kp + ii] = tile[p][jl][tx];
    }
  }
}

// ------------------------------------------------------------ the product kernel
struct Shared {
  uint64_t full[STAGES];
  uint64_t empty[STAGES];
  uint64_t acc_full[2];
  uint64_t acc_empty[2];
  uint64_t low_done;
  uint64_t mma_done;
  uint32_t tmem_base;
  int err;
};

// Work items: 1024-wide K chunks of slice pairs. High items (g <= 3) in order of
// increasing g; low items (g >= 4) in order of decreasing g (the Horner order).
struct Sched {
  int nslices, nch, nH, nL;
  __device__ Sched(int k, int nch_) : nslices(k), nch(nch_) {
    const int gh = min(k, G_EXACT);
    nH = gh * (gh + 1) / 2 * nch;
    nL = (k * (k + 1) / 2 - gh * (gh + 1) / 2) * nch;
  }
  __device__ void high(int i, int* g, int* p, int* c) const {
    int gg = 0, base = 0;
    while (i >= base + (gg + 1) * nch) { base += (gg + 1) * nch; ++gg; }
    *g = gg;
    *p = (i - base) / nch;
    *c = (i - base) % nch;
  }
  __device__ void low(int i, int* g, int* p, int* c) const {
    int gg = nslices - 1, base = 0;
    while (i >= base + (gg + 1) * nch) { base += (gg + 1) * nch; --gg; }
    *g = gg;
    *p = (i - base) / nch;
    *c = (i - base) % nch;
  }
  // idx-th item of the interleaved order H0 L0 H1 L1 ..., then the longer tail.
  // Returns true for a low item; *i is its index within its own list.
  __device__ bool item(int idx, int* i) const {
    const int m = min(nH, nL);
    if (idx < 2 * m) { *i = idx >> 1; return idx & 1; }
    *i = idx - m;
    return nL > nH;
  }
};

__global__ void __launch_bounds__(NUM_THREADS, 1)
k_ozaki_gemm(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
             const int* __restrict__ erow, const int* __restrict__ fcol, const double* __restrict__ P,
             const double* __restrict__ Q, const double* __restrict__ pdiag, const double* __restrict__ qdiag,
             int64_t N, double alpha, int nslices, int nksteps, const Epilogue e,
             unsigned int* __restrict__ status) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = smem_raw + ((1024 - (smem_u32(smem_raw) & 1023)) & 1023);
  uint8_t* smA = smem;
  uint8_t* smB = smem + STAGES * STAGE_BYTES;
  Shared* sh = reinterpret_cast<Shared*>(smem + 2 * STAGES * STAGE_BYTES);
  volatile int* cta_err = &sh->err;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t m0 = (int64_t)blockIdx.y * TILE, n0 = (int64_t)blockIdx.x * TILE;
  const int nch = (nksteps + CHUNK_STEPS - 1) / CHUNK_STEPS;
  const Sched sc(nslices, nch);
  const int nunits = sc.nH + sc.nL;
  const int nbuf = sc.nL > 0 ? 1 : 2;  // the low accumulator takes the second buffer

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) { mbar_init(&sh->full[s], 1); mbar_init(&sh->empty[s], 1); }
    for (int b = 0; b < 2; ++b) { mbar_init(&sh->acc_full[b], 1); mbar_init(&sh->acc_empty[b], NUM_EPI); }
    mbar_init(&sh->low_done, 1);
    mbar_init(&sh->mma_done, 1);
    sh->err = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;" ::"r"(smem_u32(&sh->tmem_base))
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = sh->tmem_base;

  if (warp == 0) {
    // ---------------- TMA producer
    if (lane == 0) {
      asm volatile("prefetch.tensormap [%0];" ::"l"(&tmA) : "memory");
      asm volatile("prefetch.tensormap [%0];" ::"l"(&tmB) : "memory");
      int it = 0;
      bool ok = true;
      for (int idx = 0; idx < nunits && ok; ++idx) {
        int i, g, p, c;
        if (sc.item(idx, &i)) sc.low(i, &g, &p, &c); else sc.high(i, &g, &p, &c);
        const int ks1 = min(nksteps, (c + 1) * CHUNK_STEPS);
        for (int ks = c * CHUNK_STEPS; ks < ks1; ++ks, ++it) {
          const int s = it % STAGES;
          const uint32_t ph = (uint32_t)(it / STAGES) & 1u;
          if (!mbar_wait(&sh->empty[s], ph ^ 1u, cta_err)) { ok = false; break; }
          mbar_arrive_expect_tx(&sh->full[s], 2 * STAGE_BYTES);
          tma_load_3d(smA + s * STAGE_BYTES, &tmA, &sh->full[s], ks * KSTEP, (int)m0, p);
          tma_load_3d(smB + s * STAGE_BYTES, &tmB, &sh->full[s], ks * KSTEP, (int)n0, g - p);
        }
      }
      if (!ok) {
        // let the copies already issued land before the CTA goes away (one
        // overall deadline; a stage whose phase moved on is simply skipped)
        const unsigned long long t0 = globaltimer();
        for (int back = 1; back <= STAGES && back <= it; ++back) {
          const int i2 = it - back;
          while (!mbar_try_wait(&sh->full[i2 % STAGES], (uint32_t)(i2 / STAGES) & 1u) &&
                 globaltimer() - t0 < TIMEOUT_NS / 16) {
          }
        }
      }
    }
  } else if (warp == 1) {
    // ---------------- MMA issuer
    if (lane == 0) {
      int it = 0;
      bool ok = true;
      for (int idx = 0; idx < nunits && ok; ++idx) {
        int i, g, p, c;
        const bool is_low = sc.item(idx, &i);
        uint32_t d_tmem;
        int b = 0;
        if (is_low) {
          sc.low(i, &g, &p, &c);
          d_tmem = tmem + (uint32_t)TILE;  // low-group accumulator
        } else {
          sc.high(i, &g, &p, &c);
          b = i % nbuf;
          if (!mbar_wait(&sh->acc_empty[b], ((uint32_t)(i / nbuf) & 1u) ^ 1u, cta_err)) { ok = false; break; }
          tc_fence_after();
          d_tmem = tmem + (uint32_t)(b * TILE);
        }
        const int ks0 = c * CHUNK_STEPS, ks1 = min(nksteps, (c + 1) * CHUNK_STEPS);
        for (int ks = ks0; ks < ks1; ++ks, ++it) {
          const int s = it % STAGES;
          if (!mbar_wait(&sh->full[s], (uint32_t)(it / STAGES) & 1u, cta_err)) { ok = false; break; }
          tc_fence_after();
          const uint64_t da = smem_desc(smem_u32(smA + s * STAGE_BYTES));
          const uint64_t db = smem_desc(smem_u32(smB + s * STAGE_BYTES));
#pragma unroll
          for (int kk = 0; kk < KSTEP / 16; ++kk) {  // +32 bytes per K=16 step inside the swizzle row
            const bool first = (ks == ks0 && kk == 0);
            if (!is_low) {
              mma_bf16(d_tmem, da + (uint64_t)(kk * 2), db + (uint64_t)(kk * 2), first ? 0u : 1u);
            } else if (first && i == 0) {                      // start of the low sum
              mma_bf16(d_tmem, da + (uint64_t)(kk * 2), db + (uint64_t)(kk * 2), 0u);
            } else if (first && p == 0 && c == 0) {            // next group: weight moves by 2^-8
              mma_bf16_scaled(d_tmem, da + (uint64_t)(kk * 2), db + (uint64_t)(kk * 2));
            } else {
              mma_bf16(d_tmem, da + (uint64_t)(kk * 2), db + (uint64_t)(kk * 2), 1u);
            }
          }
          mma_commit(&sh->empty[s]);
        }
        if (!ok) break;
        if (!is_low) mma_commit(&sh->acc_full[b]);
        else if (i == sc.nL - 1) mma_commit(&sh->low_done);
      }
      // no MMA may still be writing TMEM when the CTA frees it
      mma_commit(&sh->mma_done);
      const unsigned long long t0 = globaltimer();
      while (!mbar_try_wait(&sh->mma_done, 0u) && globaltimer() - t0 < TIMEOUT_NS) {
      }
    }
  } else {
    // ---------------- drain + epilogue (warps 2..5 cover TMEM lane quarters 2,3,0,1)
    const int q = warp & 3;
    const int row_in_tile = q * 32 + lane;
    const uint32_t lane_base = tmem + ((uint32_t)(q * 32) << 16);
    uint32_t z[32];
#pragma unroll
    for (int i = 0; i < 32; ++i) z[i] = 0u;
#pragma unroll
    for (int c4 = 0; c4 < 4; ++c4) {
      tmem_st32(lane_base + 256 + 32 * c4, z);
      tmem_st32(lane_base + 384 + 32 * c4, z);
    }
    tmem_wait_st();
    bool ok = true;
    for (int u = 0; u < sc.nH; ++u) {
      int g, p, c;
      sc.high(u, &g, &p, &c);
      const int b = u % nbuf;
      // warp-uniform outcome: the TMEM loads below are .sync.aligned
      ok = __all_sync(0xffffffffu, mbar_wait(&sh->acc_full[b], (uint32_t)(u / nbuf) & 1u, cta_err));
      if (!ok) break;
      tc_fence_after();
      const int shift = 8 * (G_EXACT - 1 - g);
#pragma unroll 1
      for (int c4 = 0; c4 < 4; ++c4) {
        uint32_t acc[32], lo[32], hi[32];
        tmem_ld32(lane_base + (uint32_t)(b * TILE + 32 * c4), acc);
        tmem_ld32(lane_base + 256 + 32 * c4, lo);
        tmem_ld32(lane_base + 384 + 32 * c4, hi);
        tmem_wait_ld();
        if (c4 == 3) {  // the accumulator buffer is free once all of it is in registers
          tc_fence_before();
          mbar_arrive(&sh->acc_empty[b]);
        }
#pragma unroll
        for (int i = 0; i < 32; ++i) {
          const long long a = (long long)__float2int_rn(__uint_as_float(acc[i])) << shift;
          unsigned long long r = ((unsigned long long)hi[i] << 32) | lo[i];
          r += (unsigned long long)a;
          lo[i] = (uint32_t)r;
          hi[i] = (uint32_t)(r >> 32);
        }
        tmem_st32(lane_base + 256 + 32 * c4, lo);
        tmem_st32(lane_base + 384 + 32 * c4, hi);
      }
      tmem_wait_st();
    }
    if (ok && sc.nL > 0)
      ok = __all_sync(0xffffffffu, mbar_wait(&sh->low_done, 0u, cta_err));
    if (ok) tc_fence_after();
    if (__all_sync(0xffffffffu, ok && !*cta_err)) {
      const int64_t row = m0 + row_in_tile;
      const int er = (row < N) ? erow[row] : 0;
      const double pii = (row < N) ? pdiag[row] : 0.0;
#pragma unroll 1
      for (int c4 = 0; c4 < 4; ++c4) {
        uint32_t lo[32], hi[32], lw[32];
        tmem_ld32(lane_base + 256 + 32 * c4, lo);
        tmem_ld32(lane_base + 384 + 32 * c4, hi);
        if (sc.nL > 0) tmem_ld32(lane_base + (uint32_t)TILE + 32 * c4, lw);
        tmem_wait_ld();
        if (row < N) {
#pragma unroll 4
          for (int i = 0; i < 32; ++i) {
            const int64_t col = n0 + 32 * c4 + i;
            if (col >= N) break;
            const long long r = (long long)(((unsigned long long)hi[i] << 32) | lo[i]);
            double v = (double)r;  // rounds to 53 bits when |R| >= 2^53
            if (sc.nL > 0) v = fma((double)__uint_as_float(lw[i]), 0.00390625, v);
            const int ex = er + fcol[col] - 16 - 8 * (G_EXACT - 1);
            const double scl = (ex >= -1022 && ex <= 1023) ? __longlong_as_double((long long)(ex + 1023) << 52)
                                                          : ldexp(1.0, ex);
            // the deflated diagonals: + P_ii Q_ij + P_ij Q_jj - [i = j] P_ii Q_jj
            const double qjj = qdiag[col];
            double d = fma(pii, __ldg(Q + row * N + col), (v * scl));
            d = fma(__ldg(P + row * N + col), qjj, d);
            if (row == col) d = fma(-pii, qjj, d);
            apply_epilogue(e, N, row, col, alpha * d);
          }
        }
      }
    }
  }

  tc_fence_before();
  __syncthreads();
  if (threadIdx.x == 0 && sh->err) atomicOr(status, STATUS_TIMEOUT);
  if (warp == 0) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" ::"r"(tmem) : "memory");
  }
}

// ------------------------------------------------------------ host side
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
  static EncodeTiledFn fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(p);
  });
  return fn;
}

bool make_map(CUtensorMap* m, void* base, int64_t Rp, int64_t Kp, int k) {
  EncodeTiledFn fn = encode_fn();
  if (!fn) return false;
  const cuuint64_t dims[3] = {(cuuint64_t)Kp, (cuuint64_t)Rp, (cuuint64_t)k};
  const cuuint64_t strides[2] = {(cuuint64_t)Kp * 2, (cuuint64_t)(Rp * Kp * 2)};
  const cuuint32_t box[3] = {KSTEP, TILE, 1};
  const cuuint32_t estr[3] = {1, 1, 1};
  return fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, base, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
            CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

int64_t padded(int64_t N) { return (N + TILE - 1) / TILE * TILE; }

constexpr size_t SMEM_BYTES = 2 * STAGES * STAGE_BYTES + sizeof(Shared) + 1024;

template <int K>
cudaError_t split_both(const double* P, const double* Q, int64_t N, int64_t Rp, uint16_t* Ps, uint16_t* Qs,
                       int* erow, int* fcol, int* fexp, double* pdiag, double* qdiag, unsigned int* status,
                       cudaStream_t st) {
  k_split_rows<K><<<(unsigned)((Rp + 7) / 8), 256, 0, st>>>(P, N, Rp, Rp, Ps, erow, pdiag, status);
  cudaError_t err = cudaMemsetAsync(fexp, 0, (size_t)N * sizeof(int), st);
  if (err != cudaSuccess) return err;
  const int64_t colblocks = (N + 255) / 256;
  int64_t slabs = (304 + colblocks - 1) / colblocks;
  slabs = std::min<int64_t>(slabs, (N + 63) / 64);
  const int64_t rows_per = (N + slabs - 1) / slabs;
  k_col_maxexp<<<dim3((unsigned)colblocks, (unsigned)slabs), 256, 0, st>>>(Q, N, rows_per, fexp);
  k_split_cols<K><<<dim3((unsigned)(Rp / 32), (unsigned)(Rp / 32)), 256, 0, st>>>(Q, N, Rp, Rp, fexp, Qs, fcol,
                                                                                   qdiag, status);
  return cudaGetLastError();
}

}  // namespace

bool ozaki_supported(int64_t N) { return N >= 1 && N <= 16384; }

// Layout of the workspace: 256 reserved bytes, erow[Rp], fcol[Rp], fexp[Rp], the
// deflated diagonals pdiag[Rp], qdiag[Rp], then the P planes and the Q^T planes,
// each k x Rp x Rp BF16.
size_t ozaki_workspace_bytes(int64_t N, int slices) {
  const int64_t Rp = padded(N);
  return 256 + 3 * (size_t)Rp * sizeof(int) + 256 + 2 * (size_t)Rp * sizeof(double) + 256 +
         2 * (size_t)slices * Rp * Rp * 2;
}

namespace {
struct OzLayout {
  int64_t Rp;
  int* erow;
  int* fcol;
  int* fexp;
  double* pdiag;
  double* qdiag;
  uint16_t* Ps;
  uint16_t* Qs;
};
OzLayout layout(void* work, int64_t N, int slices) {
  OzLayout L;
  L.Rp = padded(N);
  uint8_t* w = static_cast<uint8_t*>(work);
  L.erow = reinterpret_cast<int*>(w + 256);
  L.fcol = L.erow + L.Rp;
  L.fexp = L.fcol + L.Rp;
  size_t off = 256 + 3 * (size_t)L.Rp * sizeof(int);
  off = (off + 255) / 256 * 256;
  L.pdiag = reinterpret_cast<double*>(w + off);
  L.qdiag = L.pdiag + L.Rp;
  off += 2 * (size_t)L.Rp * sizeof(double);
  off = (off + 255) / 256 * 256;
  L.Ps = reinterpret_cast<uint16_t*>(w + off);
  L.Qs = L.Ps + (size_t)slices * L.Rp * L.Rp;
  return L;
}
}  // namespace

cudaError_t ozaki_split(const double* P, const double* Q, int64_t N, int slices, void* work, unsigned int* flag,
                        cudaStream_t st) {
  if (!ozaki_supported(N) || slices < 2 || slices > 8 || !work || !flag) return cudaErrorInvalidValue;
  const OzLayout L = layout(work, N, slices);
  switch (slices) {
    case 2: return split_both<2>(P, Q, N, L.Rp, L.Ps, L.Qs, L.erow, L.fcol, L.fexp, L.pdiag, L.qdiag, flag, st);
    case 3: return split_both<3>(P, Q, N, L.Rp, L.Ps, L.Qs, L.erow, L.fcol, L.fexp, L.pdiag, L.qdiag, flag, st);
    case 4: return split_both<4>(P, Q, N, L.Rp, L.Ps, L.Qs, L.erow, L.fcol, L.fexp, L.pdiag, L.qdiag, flag, st);
    case 5: return split_both<5>(P, Q, N, L.Rp, L.Ps, L.Qs, L.erow, L.fcol, L.fexp, L.pdiag, L.qdiag, flag, st);
    case 6: return split_both<6>(P, Q, N, L.Rp, L.Ps, L.Qs, L.erow, L.fcol, L.fexp, L.pdiag, L.qdiag, flag, st);
    case 7: return split_both<7>(P, Q, N, L.Rp, L.Ps, L.Qs, L.erow, L.fcol, L.fexp, L.pdiag, L.qdiag, flag, st);
    default: return split_both<8>(P, Q, N, L.Rp, L.Ps, L.Qs, L.erow, L.fcol, L.fexp, L.pdiag, L.qdiag, flag, st);
  }
}

cudaError_t ozaki_product(const double* P, const double* Q, int64_t N, double alpha, const Epilogue& e, int slices,
                          void* work, unsigned int* flag, cudaStream_t st) {
  if (!ozaki_supported(N) || slices < 2 || slices > 8 || !work || !flag) return cudaErrorInvalidValue;
  const OzLayout L = layout(work, N, slices);
  CUtensorMap ta, tb;
  if (!make_map(&ta, L.Ps, L.Rp, L.Rp, slices) || !make_map(&tb, L.Qs, L.Rp, L.Rp, slices))
    return cudaErrorNotSupported;
  cudaError_t err = cudaFuncSetAttribute(k_ozaki_gemm, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SMEM_BYTES);
  if (err != cudaSuccess) return err;
  const dim3 grid((unsigned)(L.Rp / TILE), (unsigned)(L.Rp / TILE));
  k_ozaki_gemm<<<grid, NUM_THREADS, SMEM_BYTES, st>>>(ta, tb, L.erow, L.fcol, P, Q, L.pdiag, L.qdiag, N, alpha,
                                                      slices, (int)(L.Rp / KSTEP), e, flag);
  return cudaGetLastError();
}

}  // namespace bbc
