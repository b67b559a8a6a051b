// slices.cu -- the operands of a split-precision product cut into BF16 slices
// (an error-free splitting in the manner of Ozaki et al.; the products that use
// them are in gemm_ozaki.cu).
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
// The literal split writes, instead of digits, K terms of the scaled value, each
// the rounding of what the earlier ones left: BF16 terms (BBC_PREC_SPLIT) or TF32
// terms (BBC_PREC_SPLIT_TF32, BBC_PREC_FP32), the latter as 32-bit words whose low
// 13 mantissa bits are zero, which the kind::tf32 MMAs read unchanged.
//
// Traffic per product: the two FP64 operands are read (Q twice: once for its column
// exponents) and 2 k BF16 planes written. At 6 slices the row and column kernels are
// bound by the integer (ALU) pipe, not by HBM: the digit extraction is their cost,
// which is why it works byte-wise on 32-bit words (digit_pairs).
#include <cuda_bf16.h>
#include <stdint.h>

#include <algorithm>
#include <type_traits>

#include "internal.h"
#include "slices.h"

namespace bbc {
namespace {

using slices::OzLayout;
using slices::layout;
using slices::STATUS_NONFINITE;
using slices::padded;

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

// Balanced base-256 digits of two fixed-point integers X0, X1 (|X| < 2^63), most
// significant first, as BF16 pairs (X0's digit in the low half of each word, the
// way the planes store neighbouring elements). The lower K - 1 digits lie in
// [-128, 127] and the top one takes the rest: X = sum_q d_q 256^q. Adding
// C = 128 (1 + 256 + ... + 256^(K-2)) turns them into plain bytes, d_q + 128 being
// byte q of X + C, and the top digit is floor((X + C) / 256^(K-1)). A byte b becomes
// the float 1.5 2^23 + b by one byte permute into that constant's low mantissa
// byte, and b - 128 by one exact FP32 subtraction; a small integer's float has at
// most 8 significant bits, so its upper 16 bits are its exact BF16 pattern. Integer
// work stays 32-bit after the one 64-bit addition per element.
template <int K>
__device__ __forceinline__ void digit_pairs(long long X0, long long X1, uint32_t (&out)[K]) {
  static_assert(K >= 2 && K <= 8, "2..8 digits");
  constexpr int LB = 8 * (K - 1);                                    // bits of the lower digits
  constexpr unsigned long long C = 0x8080808080808080ull >> (64 - LB);
  unsigned long long L0, L1;  // the lower digits + 128 in their low K - 1 bytes
  int T0, T1;                 // the top digits
  if constexpr (K <= 7) {     // |X| < 2^55: X + C is exact in 64 bits
    const long long Y0 = X0 + (long long)C, Y1 = X1 + (long long)C;
    L0 = (unsigned long long)Y0;
    L1 = (unsigned long long)Y1;
    T0 = (int)(Y0 >> LB);
    T1 = (int)(Y1 >> LB);
  } else {  // X + C may pass 2^63: X mod 2^LB + C stays below 2^(LB+1), its bit LB the carry
    constexpr unsigned long long MASK = (1ull << LB) - 1;
    L0 = ((unsigned long long)X0 & MASK) + C;
    L1 = ((unsigned long long)X1 & MASK) + C;
    T0 = (int)((X0 >> LB) + (long long)(L0 >> LB));
    T1 = (int)((X1 >> LB) + (long long)(L1 >> LB));
  }
#pragma unroll
  for (int q = 0; q < K - 1; ++q) {
    const uint32_t w0 = (q < 4) ? (uint32_t)L0 : (uint32_t)(L0 >> 32);
    const uint32_t w1 = (q < 4) ? (uint32_t)L1 : (uint32_t)(L1 >> 32);
    const uint32_t sel = 0x7650u | (uint32_t)(q & 3);  // byte q, then 0x00, 0x40, 0x4B
    const float f0 = __uint_as_float(__byte_perm(w0, 0x4B400000u, sel)) - 12583040.0f;
    const float f1 = __uint_as_float(__byte_perm(w1, 0x4B400000u, sel)) - 12583040.0f;
    out[K - 1 - q] = __byte_perm(__float_as_uint(f0), __float_as_uint(f1), 0x7632u);
  }
  const float t0 = __int_as_float(0x4B400000 + T0) - 12582912.0f;    // |T| <= 128
  const float t1 = __int_as_float(0x4B400000 + T1) - 12582912.0f;
  out[0] = __byte_perm(__float_as_uint(t0), __float_as_uint(t1), 0x7632u);
}

// The literal split (BBC_PREC_SPLIT): x scaled by the row's (column's) power of
// two 2^-(Emax - 1021), so |x| < 1/2, then K BF16 terms, each the rounding to
// nearest of what the earlier terms left (floating-point splitting, no common
// fixed point: each term keeps its own exponent).
template <int K>
__device__ __forceinline__ void float_terms(double x, int Emax, uint32_t (&out)[K]) {
  double r = ldexp(x, -(Emax - 1021));
#pragma unroll
  for (int p = 0; p < K; ++p) {
    const __nv_bfloat16 b = __double2bfloat16(r);
    out[p] = (uint32_t)__bfloat16_as_ushort(b);
    r -= (double)__bfloat162float(b);
  }
}
// TF32 rounding (to nearest, ties away from zero) of a binary32 value: the
// 32-bit word with the low 13 mantissa bits cleared.
__device__ __forceinline__ uint32_t tf32_rna(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return r;
}
// The literal split in TF32 terms: as float_terms, each term the TF32 rounding of
// (the binary32 rounding of) what the earlier terms left.
template <int K>
__device__ __forceinline__ void tf32_terms(double x, int Emax, uint32_t (&out)[K]) {
  double r = ldexp(x, -(Emax - 1021));
#pragma unroll
  for (int p = 0; p < K; ++p) {
    const uint32_t t = tf32_rna((float)r);
    out[p] = t;
    r -= (double)__uint_as_float(t);
  }
}
// Two neighbouring elements' BF16 slices packed per plane (x0 in the low half):
// MODE 0 exact digits, MODE 1 literal BF16 terms.
template <int K, int MODE>
__device__ __forceinline__ void bf16_pairs(double x0, double x1, int Emax, uint32_t (&w)[K]) {
  static_assert(MODE == 0 || MODE == 1, "BF16 planes");
  if constexpr (MODE == 0) {
    digit_pairs<K>(fixed_point(x0, Emax, K), fixed_point(x1, Emax, K), w);
  } else {
    uint32_t d0[K], d1[K];
    float_terms<K>(x0, Emax, d0);
    float_terms<K>(x1, Emax, d1);
#pragma unroll
    for (int p = 0; p < K; ++p) w[p] = d0[p] | (d1[p] << 16);
  }
}

// Writes elements 2 idx and 2 idx + 1 (x0, x1) of each of the K planes (plane: elements
// of one BF16 plane; a TF32 plane is twice its size, one 32-bit word per element).
template <int K, int MODE>
__device__ __forceinline__ void store_pair(uint16_t* __restrict__ planes, size_t plane, size_t idx, double x0,
                                           double x1, int Emax) {
  if constexpr (MODE == 2) {
    uint32_t d0[K], d1[K];
    tf32_terms<K>(x0, Emax, d0);
    tf32_terms<K>(x1, Emax, d1);
    uint2* out = reinterpret_cast<uint2*>(planes);
#pragma unroll
    for (int p = 0; p < K; ++p) out[p * (plane >> 1) + idx] = make_uint2(d0[p], d1[p]);
  } else {
    uint32_t w[K];
    bf16_pairs<K, MODE>(x0, x1, Emax, w);
    uint32_t* out = reinterpret_cast<uint32_t*>(planes);
#pragma unroll
    for (int p = 0; p < K; ++p) out[p * (plane >> 1) + idx] = w[p];
  }
}

// P (N x N, row-major FP64) -> K slice planes [K][Rp][Kp] of BF16 digits (or
// literal terms: BF16, or TF32 in 32-bit words) with row exponents. One warp per
// row; padding rows/columns are written as zeros. upper: P is upper triangular and
// the product reads row i only from column 256 floor(i / 256) on (its tile row's
// first K step), so the scan starts at the diagonal's warp-aligned column and the
// planes are written from that column on.
template <int K, int MODE, bool UPPER>
__global__ void __launch_bounds__(256)
k_split_rows(const double* __restrict__ P, int64_t N, int64_t Rp, int64_t Kp, uint16_t* __restrict__ planes,
             int* __restrict__ erow, double* __restrict__ pdiag, unsigned int* __restrict__ status) {
  const int64_t row = (int64_t)blockIdx.x * 8 + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (row >= Rp) return;
  const size_t plane = (size_t)Rp * Kp;
  int Emax = 0;
  bool bad = false;
  if (row < N) {
    const double* pr = P + row * N;
    int64_t j = (UPPER ? (row & ~(int64_t)31) : 0) + lane;
    for (; j + 96 < N; j += 128) {  // four independent loads in flight per lane
      const double a0 = __ldg(pr + j), a1 = __ldg(pr + j + 32), a2 = __ldg(pr + j + 64), a3 = __ldg(pr + j + 96);
      const int E0 = (j == row) ? 0 : exp_field(a0), E1 = (j + 32 == row) ? 0 : exp_field(a1);
      const int E2 = (j + 64 == row) ? 0 : exp_field(a2), E3 = (j + 96 == row) ? 0 : exp_field(a3);
      bad |= (E0 == 0x7FF) | (E1 == 0x7FF) | (E2 == 0x7FF) | (E3 == 0x7FF);
      Emax = max(max(Emax, max(E0, E1)), max(E2, E3));
    }
    for (; j < N; j += 32) {
      const int E = (j == row) ? 0 : exp_field(__ldg(pr + j));
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
  if (lane == 0) {  // the scale the digits are cut against: max(Emax, 1), as for subnormal-only rows
    erow[row] = (row < N && !bad) ? max(Emax, 1) - 1021 : 0;
    pdiag[row] = (row < N && !bad) ? __ldg(P + row * N + row) : 0.0;
  }
  Emax = max(Emax, 1);
  const bool live = row < N && !bad;
  auto elem = [&](int64_t c) -> double {
    return (live && c < N && c != row) ? __ldg(P + row * N + c) : 0.0;
  };
  const int64_t k0 = UPPER ? row / 256 * 256 : 0;
  for (int64_t j = k0 + 2 * lane; j < Kp; j += 128) {  // two pairs per lane per pass: four loads in flight
    const int64_t j2 = j + 64;
    const double x0 = elem(j), x1 = elem(j + 1);
    const double x2 = (j2 < Kp) ? elem(j2) : 0.0, x3 = (j2 < Kp) ? elem(j2 + 1) : 0.0;
    const size_t idx = ((size_t)row * Kp + j) >> 1;  // element pair (j, j + 1)
    store_pair<K, MODE>(planes, plane, idx, x0, x1, Emax);
    if (j2 < Kp) store_pair<K, MODE>(planes, plane, idx + 32, x2, x3, Emax);
  }
}

// As k_split_rows, for large rows (2048 < Kp <= 512 PPT): one block of 256 threads per
// row holds the whole row in registers (thread t owns the column pairs 2t + 512 i), so
// the row is read from memory once, not once for the exponent and once for the digits.
template <int K, int MODE, bool UPPER, int PPT>
__global__ void __launch_bounds__(256)
k_split_rows_reg(const double* __restrict__ P, int64_t N, int64_t Rp, int64_t Kp, uint16_t* __restrict__ planes,
                 int* __restrict__ erow, double* __restrict__ pdiag, unsigned int* __restrict__ status) {
  __shared__ int s_emax[8], s_bad[8];
  const int64_t row = blockIdx.x;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int64_t k0 = UPPER ? row / 256 * 256 : 0;   // first column a triangle product reads
  const bool real = row < N;
  double x[2 * PPT];
  int Emax = 0;
  bool bad = false;
#pragma unroll
  for (int i = 0; i < PPT; ++i) {
    const int64_t j = 2 * (int64_t)tid + 512 * (int64_t)i;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int64_t c = j + h;
      const double v = (real && c < N && c >= k0) ? __ldg(P + row * N + c) : 0.0;
      const int E = exp_field(v);
      bad |= (E == 0x7FF);                       // the diagonal too: it must be finite
      if (c != row) Emax = max(Emax, E);
      x[2 * i + h] = (c != row) ? v : 0.0;       // the diagonal is deflated
    }
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) Emax = max(Emax, __shfl_xor_sync(0xffffffffu, Emax, off));
  const bool wbad = __any_sync(0xffffffffu, bad);
  if (lane == 0) { s_emax[warp] = Emax; s_bad[warp] = wbad ? 1 : 0; }
  __syncthreads();
  Emax = s_emax[0];
  bad = s_bad[0] != 0;
#pragma unroll
  for (int w = 1; w < 8; ++w) { Emax = max(Emax, s_emax[w]); bad |= s_bad[w] != 0; }
  if (tid == 0) {
    if (bad) atomicOr(status, STATUS_NONFINITE);
    erow[row] = (real && !bad) ? max(Emax, 1) - 1021 : 0;
    pdiag[row] = (real && !bad) ? __ldg(P + row * N + row) : 0.0;
  }
  Emax = max(Emax, 1);
  const size_t plane = (size_t)Rp * Kp;
#pragma unroll
  for (int i = 0; i < PPT; ++i) {
    const int64_t j = 2 * (int64_t)tid + 512 * (int64_t)i;
    if (j >= Kp || j + 2 <= k0) continue;        // k0 is even: pairs never straddle it
    const double x0 = bad ? 0.0 : x[2 * i], x1 = bad ? 0.0 : x[2 * i + 1];
    store_pair<K, MODE>(planes, plane, ((size_t)row * Kp + j) >> 1, x0, x1, Emax);
  }
}

// Largest biased exponent per column of Q (fexp zeroed beforehand). upper: Q is upper
// triangular, so column j is scanned down to its diagonal only.
template <bool UPPER>
__global__ void __launch_bounds__(256)
k_col_maxexp(const double* __restrict__ Q, int64_t N, int64_t rows_per, int* __restrict__ fexp) {
  const int64_t j = (int64_t)blockIdx.x * 256 + threadIdx.x;
  if (j >= N) return;
  const int64_t r0 = (int64_t)blockIdx.y * rows_per;
  const int64_t r1 = min(UPPER ? j + 1 : N, r0 + rows_per);
  int m = 0;
  for (int64_t i = r0; i < r1; ++i) {
    const int E = exp_field(__ldg(Q + i * N + j));
    m = max(m, (i == j && E != 0x7FF) ? 0 : E);  // the diagonal is deflated (but still checked)
  }
  atomicMax(fexp + j, m);
}

// Q (N x N) -> K planes of Q^T digits [K][Rp][Kp] (plane row j holds column j of
// Q) with column exponents fcol. 64 x 32 tiles (rows x columns of Q) transposed
// through shared memory: each thread keeps eight loads in flight (rows in adjacent
// pairs, so a BF16 plane takes one 32-bit shared store per pair), and each warp
// writes a plane row's 64 digits as one 128-byte line.
// upper: Q is upper triangular and the product reads plane row j (column j of Q)
// only below K = 128 (floor(j / 128) + 1), the end of its tile column's K range:
// blocks wholly beyond it write nothing.
template <int K, int MODE, bool UPPER>
__global__ void __launch_bounds__(256)
k_split_cols(const double* __restrict__ Q, int64_t N, int64_t Rp, int64_t Kp, const int* __restrict__ fexp,
             uint16_t* __restrict__ planes, int* __restrict__ fcol, double* __restrict__ qdiag,
             unsigned int* __restrict__ status) {
  // [plane][column of Q][row of Q], rows padded; TF32 terms take a 32-bit word each
  using Elem = typename std::conditional<MODE == 2, uint32_t, uint16_t>::type;
  __shared__ __align__(16) Elem tile[K][32][MODE == 2 ? 65 : 66];
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  const int64_t i0 = (int64_t)blockIdx.x * 64;  // rows of Q (the K dimension)
  const int64_t j0 = (int64_t)blockIdx.y * 32;  // columns of Q
  const int64_t j = j0 + tx;
  const int Ej = (j < N) ? fexp[j] : 0;
  const bool bad = (Ej == 0x7FF);
  if (blockIdx.x == 0 && ty == 0 && j < Rp) {
    fcol[j] = (j < N && !bad) ? max(Ej, 1) - 1021 : 0;
    qdiag[j] = (j < N && !bad) ? __ldg(Q + j * N + j) : 0.0;
    if (bad) atomicOr(status, STATUS_NONFINITE);
  }
  if (UPPER && i0 >= (j0 / 128 + 1) * 128) return;  // block-uniform; no barrier has been reached
  const int Emax = max(Ej, 1);
  double x[8];  // rows 2 ty + 16 r + h of the tile, x[2 r + h]
#pragma unroll
  for (int r = 0; r < 4; ++r)
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int64_t i = i0 + 2 * ty + 16 * r + h;
      x[2 * r + h] = (i < N && j < N && i != j && !bad) ? __ldg(Q + i * N + j) : 0.0;
    }
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    const int il = 2 * ty + 16 * r;
    if constexpr (MODE == 2) {
      uint32_t d0[K], d1[K];
      tf32_terms<K>(x[2 * r], Emax, d0);
      tf32_terms<K>(x[2 * r + 1], Emax, d1);
#pragma unroll
      for (int p = 0; p < K; ++p) {
        tile[p][tx][il] = d0[p];
        tile[p][tx][il + 1] = d1[p];
      }
    } else {  // row stride 66 halfwords = 33 words: the warp's 32 stores hit 32 banks
      uint32_t w[K];
      bf16_pairs<K, MODE>(x[2 * r], x[2 * r + 1], Emax, w);
#pragma unroll
      for (int p = 0; p < K; ++p) *reinterpret_cast<uint32_t*>(&tile[p][tx][il]) = w[p];
    }
  }
  __syncthreads();
  const size_t plane = (size_t)Rp * Kp;
  uint32_t* out = reinterpret_cast<uint32_t*>(planes);
  uint2* out2 = reinterpret_cast<uint2*>(planes);
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    const int jl = ty + 8 * r;
    const int64_t jj = j0 + jl, ii = i0 + 2 * tx;
    if (jj < Rp && ii < Kp) {
#pragma unroll
      for (int p = 0; p < K; ++p) {
        if (MODE == 2)
          out2[(p * plane + (size_t)jj * Kp + ii) >> 1] =
              make_uint2((uint32_t)tile[p][jl][2 * tx], (uint32_t)tile[p][jl][2 * tx + 1]);
        else
          out[(p * plane + (size_t)jj * Kp + ii) >> 1] = *reinterpret_cast<const uint32_t*>(&tile[p][jl][2 * tx]);
      }
    }
  }
}

template <int K, int MODE, bool UPPER>
cudaError_t split_both_t(const double* P, const double* Q, int64_t N, int64_t Rp, uint16_t* Ps, uint16_t* Qs,
                         int* erow, int* fcol, int* fexp, double* pdiag, double* qdiag, unsigned int* status,
                         cudaStream_t st) {
  if (Rp > 2048 && Rp <= 4096)
    k_split_rows_reg<K, MODE, UPPER, 8><<<(unsigned)Rp, 256, 0, st>>>(P, N, Rp, Rp, Ps, erow, pdiag, status);
  else if (Rp > 4096 && Rp <= 8192)
    k_split_rows_reg<K, MODE, UPPER, 16><<<(unsigned)Rp, 256, 0, st>>>(P, N, Rp, Rp, Ps, erow, pdiag, status);
  else
    k_split_rows<K, MODE, UPPER><<<(unsigned)((Rp + 7) / 8), 256, 0, st>>>(P, N, Rp, Rp, Ps, erow, pdiag, status);
  cudaError_t err = cudaMemsetAsync(fexp, 0, (size_t)N * sizeof(int), st);
  if (err != cudaSuccess) return err;
  const int64_t colblocks = (N + 255) / 256;
  int64_t slabs = (1216 + colblocks - 1) / colblocks;  // ~8 blocks per SM: enough loads in flight
  slabs = std::min<int64_t>(slabs, (N + 63) / 64);
  const int64_t rows_per = (N + slabs - 1) / slabs;
  k_col_maxexp<UPPER><<<dim3((unsigned)colblocks, (unsigned)slabs), 256, 0, st>>>(Q, N, rows_per, fexp);
  k_split_cols<K, MODE, UPPER><<<dim3((unsigned)(Rp / 64), (unsigned)(Rp / 32)), 256, 0, st>>>(
      Q, N, Rp, Rp, fexp, Qs, fcol, qdiag, status);
  return cudaGetLastError();
}

template <int K, int MODE>
cudaError_t split_both(const double* P, const double* Q, int64_t N, int64_t Rp, uint16_t* Ps, uint16_t* Qs,
                       int* erow, int* fcol, int* fexp, double* pdiag, double* qdiag, unsigned int* status,
                       cudaStream_t st, int upper) {
  return upper ? split_both_t<K, MODE, true>(P, Q, N, Rp, Ps, Qs, erow, fcol, fexp, pdiag, qdiag, status, st)
               : split_both_t<K, MODE, false>(P, Q, N, Rp, Ps, Qs, erow, fcol, fexp, pdiag, qdiag, status, st);
}

}  // namespace

bool ozaki_supported(int64_t N) { return N >= 1 && N <= 16384; }

// Bytes of the layout in slices.h.
size_t ozaki_workspace_bytes(int64_t N, int slices) {
  const int64_t Rp = padded(N);
  return 256 + 3 * (size_t)Rp * sizeof(int) + 256 + 2 * (size_t)Rp * sizeof(double) + 256 +
         2 * (size_t)slices * Rp * Rp * 2;
}


template <int MODE>
cudaError_t split_k(const double* P, const double* Q, int64_t N, int slices, const OzLayout& L, unsigned int* flag,
                    cudaStream_t st, int upper) {
#define BBC_SPLIT_CASE(k) \
  case k:                  \
    return split_both<k, MODE>(P, Q, N, L.Rp, L.Ps, L.Qs, L.erow, L.fcol, L.fexp, L.pdiag, L.qdiag, flag, st, upper);
  if (MODE == 2) {  // TF32 terms: 2..4
    switch (slices) {
      BBC_SPLIT_CASE(2)
      BBC_SPLIT_CASE(3)
      default: return split_both<4, MODE>(P, Q, N, L.Rp, L.Ps, L.Qs, L.erow, L.fcol, L.fexp, L.pdiag, L.qdiag,
                                          flag, st, upper);
    }
  }
  switch (slices) {
    BBC_SPLIT_CASE(2)
    BBC_SPLIT_CASE(3)
    BBC_SPLIT_CASE(4)
    BBC_SPLIT_CASE(5)
    BBC_SPLIT_CASE(6)
    BBC_SPLIT_CASE(7)
    default:
      return split_both<8, MODE>(P, Q, N, L.Rp, L.Ps, L.Qs, L.erow, L.fcol, L.fexp, L.pdiag, L.qdiag, flag, st, upper);
  }
#undef BBC_SPLIT_CASE
}

// mode: 0 exact BF16 digits, 1 literal BF16 terms, 2 literal TF32 terms (whose planes
// take two BF16 planes' room each: the layout is that of 2 x slices BF16 planes).
cudaError_t ozaki_split(const double* P, const double* Q, int64_t N, int slices, void* work, unsigned int* flag,
                        cudaStream_t st, int mode, bool upper) {
  const int kmax = (mode == 2) ? 4 : 8;
  if (!ozaki_supported(N) || slices < 2 || slices > kmax || !work || !flag || mode < 0 || mode > 2)
    return cudaErrorInvalidValue;
  const OzLayout L = layout(work, N, mode == 2 ? 2 * slices : slices);
  const int up = upper ? 1 : 0;
  if (mode == 2) return split_k<2>(P, Q, N, slices, L, flag, st, up);
  return mode == 1 ? split_k<1>(P, Q, N, slices, L, flag, st, up) : split_k<0>(P, Q, N, slices, L, flag, st, up);
}

}  // namespace bbc
