// batched.cu -- exp(A) for many independent matrices of uneven sizes (N <= 256)
// in one persistent launch.
//
// Each CTA takes matrices from a device work queue (an atomic counter over the
// caller's order; callers put the most expensive first) and runs the whole
// method on each one: ||A||_1 (Section 4), the (m, s) selection by the
// backward-error thresholds (eq. theta, Table 2/3) on the device, the Taylor
// program of the reduced-product scheme (Section 3) with the scaling 2^-s folded
// into its coefficients, and s squarings (eq. eses). There is no host round trip
// between matrices and no inter-CTA wait, so the launch is one memset plus one
// kernel and can be captured in a CUDA graph.
//
// Intermediates are binary64 matrices in a per-CTA slice of a workspace reserved
// beforehand (bbc_batch_reserve): 12 slots of N_max^2 doubles per resident CTA;
// for N <= 256 a CTA's slots stay within a few MiB, mostly L2-resident.
//
// Products: the CTA's 256 threads compute alpha * (P Q) in 64 x 64 output tiles
// on the FP64 pipe (4 x 4 register blocks, 16-deep shared-memory K slabs), each
// element then passing through the same fused linear-combination epilogue as
// the single-matrix path (internal.h).
//
// Selection modes (per launch):
//  plain    (m, s) from ||A||_1 and theta_m(u) (the paper's rule);
//  learned  a small MLP proposes (m, s) from cheap features (log ||A||_1, FP32
//           estimates of log ||A^k||_1^(1/k) for k = 2, 3, 4 from random-sign
//           mat-vec chains, log N). The proposal is used only if certified: by
//           ||A||_1 / 2^s <= theta_m, else by alpha_2 / 2^s <= theta_m with
//           alpha_2 = max(||A^2||^(1/2), ||A^3||^(1/3)) from exact FP64 powers
//           (which T12 / T18 then reuse); otherwise the plain rule runs;
//  alpha    always compute A^2, A^3 and take the cheapest (m, s) certified by
//           either bound (the closed-form rule the network is compared with);
//  data     no exponential: features and exact ||A^k||_1, k = 1..3, for training.
#include <math.h>

#include <algorithm>
#include <stdint.h>

#include "bbcexpm.h"
#include "internal.h"
#include "schemes.h"
#include "squarings.h"

namespace bbc {

constexpr int BATCH_THREADS = 256;
constexpr int BATCH_MAX_N = 512;     // largest matrix the batched path serves
constexpr int MLP_MAX = 256;         // widest hidden / output layer of in-kernel inference
constexpr int BATCH_SLOTS = 12;      // W0..W9 (W9 = squaring buffer), A64, T
constexpr int BSL_A = 10, BSL_T = 11;
constexpr int BATCH_MAX_STEPS = 8;
constexpr int BATCH_PROGS = 6;       // m = 1, 2, 4, 8, 12, 18

struct BOut {
  int dst, nt;
  double cv, cI;
  int slot[MAX_TERMS];
  double c[MAX_TERMS];
  int sigma_pow[MAX_TERMS];          // coefficient carries (2^-s)^pow
};
struct BStep {
  int P, Q;                          // slots; P < 0: no product
  int alpha_pow;                     // alpha = (2^-s)^alpha_pow
  int nout;
  BOut o[MAX_OUT];
};
struct BProg {
  int m, products, nsteps;
  BStep st[BATCH_MAX_STEPS];
};

__constant__ BProg c_progs[BATCH_PROGS];
__constant__ BProg c_progs_pre[2];  // T12, T18 starting from A^2 (W0) and A^3 (W1), unscaled
__constant__ BProg c_progs_pade[2]; // numerator and denominator of r_10 and r_26 (eq. pade10, eq. pade26)

constexpr int NFEAT = 5;
enum { MODE_PLAIN = 0, MODE_LEARNED = 1, MODE_ALPHA = 2, MODE_DATA = 3 };
// bbc_info.selector values
enum { SEL_PLAIN = 0, SEL_LEARNED_NORM = 2, SEL_LEARNED_ALPHA = 3, SEL_LEARNED_REJECTED = 4, SEL_ALPHA = 5 };

struct BatchArgs {
  const void* const* A;    // device array of device pointers
  const void* const* B;    // may be null; else Out_i = exp(A_i) B_i (same type and size as A_i)
  void* const* Out;
  const int64_t* Ns;
  int64_t count;
  int64_t nmax;            // reserved N_max
  int dtype;               // 0 binary64, 1 binary32
  double theta[BATCH_PROGS];
  int deg[BATCH_PROGS], prod[BATCH_PROGS];
  double* work;            // per-CTA slices of BATCH_SLOTS * nmax^2 doubles
  unsigned int* counter;   // work queue head (zeroed by the launch)
  bbc_info* info;          // may be null
  int mode;
  const float* mlp;        // learned mode: parameters W1 b1 W2 b2 W3 b3
  int mlp_hid, mlp_out, mlp_S;   // classes: m index * mlp_S + s
  float mu[NFEAT], sd[NFEAT];    // feature normalisation
  float* feat_out;         // data mode: count x NFEAT
  double* norms_out;       // data mode: count x 4
  int prec;                // 0: products on the FP64 pipe; 1: 4-slice BF16 mma.sync products (N <= 256)
  uint32_t split_mask;     // prec 1: bit b set = matrices with (N - 1) / 8 == b use split products
  BatchShapes shapes;      // per size bucket: FP64 output tile and split warp-task height (autotuned)
  uint32_t* ozwork;        // per-CTA slice scratch, OZB_WORDS words each (prec 1)
  int csize;               // CTAs per matrix: 1, or the size of the thread-block cluster sharing it
  int pade;                // 0: Taylor (the paper's scheme); 1: Pade r_10 or r_26 by cost; 2: r_26 only
  double theta_pade[2];    // theta_10, theta_26 (Pade thresholds)
};

namespace {

// Slot matrices are rewritten during the launch (by other CTAs of a cluster
// too), so they are read with ordinary loads, which the barriers' release /
// acquire order after those writes, never through the read-only (.nc) path,
// which nothing orders (hence no __ldg and no const __restrict__ on slot
// pointers in this file).
__device__ __forceinline__ double ldslot(const double* p) { return *p; }

// The fused epilogue of the batched path: the same arithmetic as
// apply_epilogue, with the matrices the outputs read loaded together (one L2
// round trip instead of one per term). An output that overwrites a matrix that a
// later output of the same element reads updates the loaded value, which is what
// reading it in order would give.
struct EpiMasks {
  unsigned used;             // bit k: some output reads Y[k]
  unsigned alias[MAX_OUT];   // bit k: output o writes the matrix Y[k]
};
__device__ __forceinline__ EpiMasks epi_masks(const Epilogue& e) {
  EpiMasks m = {};
  for (int o = 0; o < e.nout; ++o)
    for (int t = 0; t < e.o[o].nt; ++t) m.used |= 1u << e.o[o].slot[t];
  for (int o = 0; o < e.nout; ++o)
    for (int k = 0; k < MAX_Y; ++k)
      if (((m.used >> k) & 1u) && e.Y[k] == e.o[o].out) m.alias[o] |= 1u << k;
  return m;
}
__device__ __forceinline__ void epi_batched(const Epilogue& e, const EpiMasks& m, int64_t N, int64_t row,
                                            int64_t col, double v) {
  const int64_t idx = row * N + col;
  double y[MAX_Y];
#pragma unroll
  for (int k = 0; k < MAX_Y; ++k) y[k] = ((m.used >> k) & 1u) ? ldslot(e.Y[k] + idx) : 0.0;
  bool bad = false;
#pragma unroll 1
  for (int o = 0; o < e.nout; ++o) {
    const EpiOut& q = e.o[o];
    double r = q.cv * v;
    if (row == col) r += q.cI;
#pragma unroll 1
    for (int t = 0; t < q.nt; ++t) {
      const int sl = q.slot[t];
      double yv = y[0];
#pragma unroll
      for (int k = 1; k < MAX_Y; ++k) yv = (sl == k) ? y[k] : yv;
      r = fma(q.c[t], yv, r);
    }
    q.out[idx] = r;
    bad |= !isfinite(r);
#pragma unroll
    for (int k = 0; k < MAX_Y; ++k)
      if ((m.alias[o] >> k) & 1u) y[k] = r;
  }
  if (bad && e.flag) atomicOr(e.flag, 1u);
}

// Output tiles of T x T (T = 64, 32 or 16), 16-deep K slabs, 256 threads
// (R x R each with R = T / 16, stride 16); the next slab's loads are issued
// before the current slab's FMAs. Tiles part, part + parts, ... of the product:
// a cluster of `parts` CTAs shares one matrix. Every element sums k in the same
// order whatever T, so the result does not depend on the partition.
struct GemmSmem {
  double As[16][64];
  double Bs[16][64];
  EpiMasks em;               // of the epilogue of the product in flight
};

template <int T>
__device__ void block_gemm_f64_t(const double* P, const double* Q, int N, double alpha, const Epilogue& e,
                                 GemmSmem& sm, int part, int parts) {
  constexpr int R = T / 16;
  const int t = threadIdx.x, tx = t % 16, ty = t / 16;
  const int tiles = (N + T - 1) / T;
  const EpiMasks& em = sm.em;
  for (int tile = part; tile < tiles * tiles; tile += parts) {
    const int m0 = (tile / tiles) * T, n0 = (tile % tiles) * T;
    double acc[R][R];
#pragma unroll
    for (int i = 0; i < R; ++i)
#pragma unroll
      for (int j = 0; j < R; ++j) acc[i][j] = 0.0;
    double pa[R], pb[R];
    auto fetch = [&](int k0) {
#pragma unroll
      for (int q = 0; q < R; ++q) {
        const int r = t / 16 + 16 * q, c = t % 16;  // P tile T x 16
        pa[q] = (m0 + r < N && k0 + c < N) ? ldslot(P + (int64_t)(m0 + r) * N + k0 + c) : 0.0;
        const int r2 = t / T + (256 / T) * q, c2 = t % T;  // Q tile 16 x T
        pb[q] = (k0 + r2 < N && n0 + c2 < N) ? ldslot(Q + (int64_t)(k0 + r2) * N + n0 + c2) : 0.0;
      }
    };
    fetch(0);
    for (int k0 = 0; k0 < N; k0 += 16) {
#pragma unroll
      for (int q = 0; q < R; ++q) {
        sm.As[t % 16][t / 16 + 16 * q] = pa[q];
        sm.Bs[t / T + (256 / T) * q][t % T] = pb[q];
      }
      __syncthreads();
      if (k0 + 16 < N) fetch(k0 + 16);
#pragma unroll
      for (int kk = 0; kk < 16; ++kk) {
        double a[R], b[R];
#pragma unroll
        for (int i = 0; i < R; ++i) a[i] = sm.As[kk][ty + 16 * i];
#pragma unroll
        for (int j = 0; j < R; ++j) b[j] = sm.Bs[kk][tx + 16 * j];
#pragma unroll
        for (int i = 0; i < R; ++i)
#pragma unroll
          for (int j = 0; j < R; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
      }
      __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < R; ++i) {
      const int row = m0 + ty + 16 * i;
      if (row >= N) continue;
#pragma unroll
      for (int j = 0; j < R; ++j) {
        const int col = n0 + tx + 16 * j;
        if (col < N) epi_batched(e, em, N, row, col, alpha * acc[i][j]);
      }
    }
  }
}

// The largest tile that still gives every CTA of the cluster a tile, or a smaller one
// when the autotuner found it faster for this size (tile_max = 32 or 16; 0: no limit).
__device__ void block_gemm_f64(const double* P, const double* Q, int N, double alpha,
                               const Epilogue& e, GemmSmem& sm, int part, int parts, int tile_max) {
  const int t64 = (N + 63) / 64, t32 = (N + 31) / 32;
  if (t64 * t64 >= parts && tile_max != 32 && tile_max != 16)
    block_gemm_f64_t<64>(P, Q, N, alpha, e, sm, part, parts);
  else if (t32 * t32 >= parts && tile_max != 16)
    block_gemm_f64_t<32>(P, Q, N, alpha, e, sm, part, parts);
  else
    block_gemm_f64_t<16>(P, Q, N, alpha, e, sm, part, parts);
}

// ---------------------------------------------------------------------------
// Split-precision products inside a CTA (N <= 256): 4 BF16 slices per operand
// and warp-level mma.sync m16n8k16 (BF16 in, FP32 accumulate). With K <= 256
// and digits of at most 2^7 in magnitude, a slice group g = p + q (at most 4
// pairs) sums to at most 4 * 256 * 2^14 = 2^24 in magnitude, so FP32 holds every
// group sum exactly and no chunking is needed; the groups combine exactly in an
// int64. The diagonals are deflated as in the single-matrix path
// (P Q = P'Q' + D_P Q + P D_Q - D_P D_Q). Products carry ~32 significant bits.
// ---------------------------------------------------------------------------
constexpr int OZB_K = 4;          // slices
constexpr int OZB_NMAX = 256;     // largest N served by these products
constexpr size_t OZB_WORDS = 2 * (size_t)OZB_K * OZB_NMAX * (OZB_NMAX / 2);  // per-CTA slice scratch

struct OzbSmem {
  int rexp[OZB_NMAX], cexp[OZB_NMAX];      // largest biased exponent of each row of P' / column of Q' (>= 1)
  double pdiag[OZB_NMAX], qdiag[OZB_NMAX];
  int bad;
};

__device__ __forceinline__ int ozb_expf(double x) { return (int)((__double_as_longlong(x) >> 52) & 0x7FF); }

// round(x * 2^(32 - e)), e = Emax - 1021 (|x| < 2^(e-1)): an integer below 2^31
__device__ __forceinline__ long long ozb_fixed(double x, int Emax) {
  const unsigned long long bits = (unsigned long long)__double_as_longlong(x);
  int E = (int)((bits >> 52) & 0x7FF);
  unsigned long long M = bits & 0xFFFFFFFFFFFFFull;
  if (E == 0) E = 1; else M |= 1ull << 52;
  const int sh = 8 * OZB_K - 54 - (Emax - E);
  long long X;
  if (sh >= 0) X = (long long)(M << sh);
  else if (sh > -60) X = (long long)((M + (1ull << (-sh - 1))) >> (-sh));
  else X = 0;
  return (bits >> 63) ? -X : X;
}

__device__ __forceinline__ uint32_t ozb_bf16(int d) {  // exact for |d| <= 256
  return (uint32_t)__float_as_uint(__int_as_float(0x4B400000 + d) - 12582912.0f) >> 16;
}

__device__ __forceinline__ void ozb_digits(long long X, uint32_t (&d)[OZB_K]) {
#pragma unroll
  for (int p = OZB_K - 1; p >= 1; --p) {
    const long long low = ((X + 128) & 255) - 128;
    d[p] = ozb_bf16((int)low);
    X = (X - low) >> 8;
  }
  d[0] = ozb_bf16((int)X);
}

// P' rows -> Ps[p][Np][Np/2] and Q' columns -> Qt[q][Np][Np/2] (words of two BF16
// digits, K contiguous). Returns false (CTA-uniformly) if an operand is not finite.
__device__ bool block_split_oz(const double* P, const double* Q, int N, int Np, uint32_t* Ps, uint32_t* Qt,
                               OzbSmem& o) {
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int half = Np / 2;
  const size_t plane = (size_t)Np * half;
  if (tid == 0) o.bad = 0;
  __syncthreads();
  for (int i = warp; i < Np; i += BATCH_THREADS / 32) {
    int em = 0;
    bool bad = false;
    if (i < N)
      for (int j = lane; j < N; j += 32) {
        const int E = ozb_expf(ldslot(P + (int64_t)i * N + j));
        bad |= (E == 0x7FF);
        if (j != i) em = max(em, E);
      }
    for (int off = 16; off > 0; off >>= 1) em = max(em, __shfl_xor_sync(0xffffffffu, em, off));
    bad = __any_sync(0xffffffffu, bad);
    if (lane == 0) {
      if (bad) o.bad = 1;
      o.rexp[i] = max(em, 1);
      o.pdiag[i] = (i < N) ? ldslot(P + (int64_t)i * N + i) : 0.0;
    }
  }
  for (int j = tid; j < Np; j += BATCH_THREADS) {
    int em = 0;
    bool bad = false;
    if (j < N)
      for (int i = 0; i < N; ++i) {
        const int E = ozb_expf(ldslot(Q + (int64_t)i * N + j));
        bad |= (E == 0x7FF);
        if (i != j) em = max(em, E);
      }
    if (bad) o.bad = 1;
    o.cexp[j] = max(em, 1);
    o.qdiag[j] = (j < N) ? ldslot(Q + (int64_t)j * N + j) : 0.0;
  }
  __syncthreads();
  if (o.bad) return false;
  for (int idx = tid; idx < Np * half; idx += BATCH_THREADS) {
    const int i = idx / half, j = 2 * (idx % half);
    const double x0 = (i < N && j < N && j != i) ? ldslot(P + (int64_t)i * N + j) : 0.0;
    const double x1 = (i < N && j + 1 < N && j + 1 != i) ? ldslot(P + (int64_t)i * N + j + 1) : 0.0;
    uint32_t d0[OZB_K], d1[OZB_K];
    ozb_digits(ozb_fixed(x0, o.rexp[i]), d0);
    ozb_digits(ozb_fixed(x1, o.rexp[i]), d1);
#pragma unroll
    for (int p = 0; p < OZB_K; ++p) Ps[p * plane + idx] = d0[p] | (d1[p] << 16);
  }
  for (int idx = tid; idx < Np * half; idx += BATCH_THREADS) {
    const int j = idx / half, i = 2 * (idx % half);
    const double x0 = (i < N && j < N && i != j) ? ldslot(Q + (int64_t)i * N + j) : 0.0;
    const double x1 = (i + 1 < N && j < N && i + 1 != j) ? ldslot(Q + (int64_t)(i + 1) * N + j) : 0.0;
    uint32_t d0[OZB_K], d1[OZB_K];
    ozb_digits(ozb_fixed(x0, o.cexp[j]), d0);
    ozb_digits(ozb_fixed(x1, o.cexp[j]), d1);
#pragma unroll
    for (int q = 0; q < OZB_K; ++q) Qt[q * plane + idx] = d0[q] | (d1[q] << 16);
  }
  __syncthreads();
  return true;
}

__device__ __forceinline__ void ozb_mma(float (&c)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// alpha * (P Q) with the fused epilogue, from the slices of block_split_oz.
// Warp tasks of (16 MT) x 16 outputs (MT m16 x two n8 tiles; MT = 2 or, for sizes
// where the autotuner found it faster, 1), 10 slice pairs. Every output sums the
// same slice products in the same order whatever MT.
template <int MT>
__device__ void block_gemm_oz(const uint32_t* Ps, const uint32_t* Qt, const double* P, const double* Q, int N, int Np,
                              double alpha, const Epilogue& e, const EpiMasks& em, const OzbSmem& o, int part,
                              int parts) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, gid = lane >> 2, tig = lane & 3;
  const int half = Np / 2;
  const size_t plane = (size_t)Np * half;
  const int tn = Np / 16, tasks = (Np / (16 * MT)) * tn;
  constexpr int WARPS = BATCH_THREADS / 32;
  for (int task = part * WARPS + warp; task < tasks; task += parts * WARPS) {
    const int i0 = (task / tn) * (16 * MT), j0 = (task % tn) * 16;
    float acc[OZB_K][MT][2][4];
#pragma unroll
    for (int g = 0; g < OZB_K; ++g)
#pragma unroll
      for (int mt = 0; mt < MT; ++mt)
#pragma unroll
        for (int nt = 0; nt < 2; ++nt)
#pragma unroll
          for (int r = 0; r < 4; ++r) acc[g][mt][nt][r] = 0.f;
    for (int k0 = 0; k0 < Np; k0 += 16) {
      const int kw = (k0 >> 1) + tig;
      uint32_t a[OZB_K][MT][4], b[OZB_K][2][2];
#pragma unroll
      for (int p = 0; p < OZB_K; ++p)
#pragma unroll
        for (int mt = 0; mt < MT; ++mt) {
          const uint32_t* base = Ps + p * plane + (size_t)(i0 + 16 * mt + gid) * half + kw;
          a[p][mt][0] = base[0];
          a[p][mt][1] = base[8 * half];
          a[p][mt][2] = base[4];
          a[p][mt][3] = base[8 * half + 4];
        }
#pragma unroll
      for (int q = 0; q < OZB_K; ++q)
#pragma unroll
        for (int nt = 0; nt < 2; ++nt) {
          const uint32_t* base = Qt + q * plane + (size_t)(j0 + 8 * nt + gid) * half + kw;
          b[q][nt][0] = base[0];
          b[q][nt][1] = base[4];
        }
#pragma unroll
      for (int p = 0; p < OZB_K; ++p)
#pragma unroll
        for (int q = 0; q + p < OZB_K; ++q)
#pragma unroll
          for (int mt = 0; mt < MT; ++mt)
#pragma unroll
            for (int nt = 0; nt < 2; ++nt) ozb_mma(acc[p + q][mt][nt], a[p][mt], b[q][nt][0], b[q][nt][1]);
    }
#pragma unroll
    for (int mt = 0; mt < MT; ++mt)
#pragma unroll
      for (int nt = 0; nt < 2; ++nt)
#pragma unroll
        for (int r = 0; r < 4; ++r) {
          const int row = i0 + 16 * mt + gid + 8 * (r >> 1);
          const int col = j0 + 8 * nt + 2 * tig + (r & 1);
          if (row >= N || col >= N) continue;
          long long R = 0;
#pragma unroll
          for (int g = 0; g < OZB_K; ++g)
            R += (long long)__float2int_rn(acc[g][mt][nt][r]) << (8 * (OZB_K - 1 - g));
          const int ex = (o.rexp[row] - 1021) + (o.cexp[col] - 1021) - 16 - 8 * (OZB_K - 1);
          const double scl = (ex >= -1022 && ex <= 1023) ? __longlong_as_double((long long)(ex + 1023) << 52)
                                                        : ldexp(1.0, ex);
          const double pii = o.pdiag[row], qjj = o.qdiag[col];
          double v = fma(pii, ldslot(Q + (int64_t)row * N + col), (double)R * scl);
          v = fma(ldslot(P + (int64_t)row * N + col), qjj, v);
          if (row == col) v = fma(-pii, qjj, v);
          epi_batched(e, em, N, row, col, alpha * v);
        }
  }
}

__device__ void block_lincomb(int N, const Epilogue& e, GemmSmem& sm, int part, int parts) {
  if (threadIdx.x == 0) sm.em = epi_masks(e);
  __syncthreads();
  const EpiMasks& em = sm.em;
  for (int idx = part * BATCH_THREADS + threadIdx.x; idx < N * N; idx += parts * BATCH_THREADS)
    epi_batched(e, em, N, idx / N, idx % N, 0.0);
}

// One product of the program: split precision when asked and N <= 256 (and the
// operands are finite), else the FP64 pipe. In a cluster, CTA `part` of `parts`
// forms its share of the output tiles (each CTA splits the operands into its own
// scratch, so no slice plane crosses CTAs).
__device__ void block_product(const BatchArgs& a, const double* P, const double* Q, int N, double alpha,
                              const Epilogue& e, GemmSmem& sm, OzbSmem& oz, int part, int parts) {
  if (threadIdx.x == 0) sm.em = epi_masks(e);
  __syncthreads();
  if (a.prec == 1 && N <= OZB_NMAX && ((a.split_mask >> ((N - 1) >> 3)) & 1u)) {
    const int Np = (N + 31) / 32 * 32;
    uint32_t* Ps = a.ozwork + (size_t)blockIdx.x * OZB_WORDS;
    uint32_t* Qt = Ps + OZB_WORDS / 2;
    if (block_split_oz(P, Q, N, Np, Ps, Qt, oz)) {
      if ((a.shapes.split_task16 >> ((N - 1) >> 3)) & 1u)
        block_gemm_oz<1>(Ps, Qt, P, Q, N, Np, alpha, e, sm.em, oz, part, parts);
      else
        block_gemm_oz<2>(Ps, Qt, P, Q, N, Np, alpha, e, sm.em, oz, part, parts);
      return;
    }
  }
  const int b = (N - 1) >> 3;
  const int tile_max = (b < 32 && ((a.shapes.f64_tile16 >> b) & 1u)) ? 16
                       : (b < 32 && ((a.shapes.f64_tile32 >> b) & 1u)) ? 32 : 0;
  block_gemm_f64(P, Q, N, alpha, e, sm, part, parts, tile_max);
}

// Barrier over the CTAs sharing a matrix (the CTA itself when csize == 1). The
// cluster barrier's release / acquire orders each CTA's global-memory writes
// before the other CTAs' reads.
__device__ __forceinline__ void csync(int csize) {
  if (csize > 1)
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
  else
    __syncthreads();
}

// 32-bit word at `p` in the shared memory of CTA `rank` of this cluster.
__device__ __forceinline__ uint32_t cluster_map(const void* p, int rank) {
  uint32_t remote;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;"
               : "=r"(remote)
               : "r"((uint32_t)__cvta_generic_to_shared(p)), "r"(rank));
  return remote;
}
__device__ __forceinline__ int cluster_load(const int* p, int rank) {
  int v;
  asm volatile("ld.shared::cluster.s32 %0, [%1];" : "=r"(v) : "r"(cluster_map(p, rank)) : "memory");
  return v;
}
__device__ __forceinline__ void cluster_or(unsigned int* p, int rank, unsigned int v) {
  asm volatile("red.shared::cluster.or.b32 [%0], %1;" ::"r"(cluster_map(p, rank)), "r"(v) : "memory");
}

// max_j sum_i |M_ij| over an N x N binary64 matrix (one column per thread).
__device__ double block_norm1(const double* M, int N, double* red) {
  double best = 0.0;
  for (int j = threadIdx.x; j < N; j += BATCH_THREADS) {
    double s = 0.0;
    for (int i = 0; i < N; ++i) s += fabs(ldslot(M + (int64_t)i * N + j));
    best = (s > best || isnan(s)) ? s : best;
  }
  for (int off = 16; off > 0; off >>= 1) {
    const double o = __shfl_xor_sync(0xffffffffu, best, off);
    best = (o > best || isnan(o)) ? o : best;
  }
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = best;
  __syncthreads();
  double r = 0.0;
  for (int w = 0; w < BATCH_THREADS / 32; ++w) r = (red[w] > r || isnan(red[w])) ? red[w] : r;
  __syncthreads();
  return r;
}

// Cheap features: est_k = max over 4 random-sign vectors x of ||A^k x||_1 / ||x||_1
// (a lower bound of ||A^k||_1), from FP32 mat-vec chains, one warp per row.
// f = [log ||A||_1, log est_2 / 2, log est_3 / 3, log est_4 / 4, log N].
__device__ void block_features(const double* A, int N, double norm1, float* y0, float* y1, float* est, float* f) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int e = threadIdx.x; e < 4 * N; e += BATCH_THREADS) {
    const unsigned h = (unsigned)(e >> 2) * 2654435761u ^ (unsigned)(e & 3) * 40503u;
    y0[e] = ((h >> 15) & 1u) ? 1.f : -1.f;  // x[j][v] at e = 4 j + v
  }
  __syncthreads();
  float* src = y0;
  float* dst = y1;
  for (int k = 1; k <= 4; ++k) {
    for (int i = warp; i < N; i += BATCH_THREADS / 32) {
      float a0 = 0.f, a1 = 0.f, a2 = 0.f, a3 = 0.f;
      for (int j = lane; j < N; j += 32) {
        const float a = (float)ldslot(A + (int64_t)i * N + j);
        a0 = fmaf(a, src[4 * j + 0], a0);
        a1 = fmaf(a, src[4 * j + 1], a1);
        a2 = fmaf(a, src[4 * j + 2], a2);
        a3 = fmaf(a, src[4 * j + 3], a3);
      }
      for (int off = 16; off > 0; off >>= 1) {
        a0 += __shfl_xor_sync(0xffffffffu, a0, off);
        a1 += __shfl_xor_sync(0xffffffffu, a1, off);
        a2 += __shfl_xor_sync(0xffffffffu, a2, off);
        a3 += __shfl_xor_sync(0xffffffffu, a3, off);
      }
      if (lane == 0) { dst[4 * i] = a0; dst[4 * i + 1] = a1; dst[4 * i + 2] = a2; dst[4 * i + 3] = a3; }
    }
    __syncthreads();
    if (threadIdx.x < 4) {
      float sum = 0.f;
      for (int i = 0; i < N; ++i) sum += fabsf(dst[4 * i + threadIdx.x]);
      est[(k - 1) * 4 + threadIdx.x] = sum / (float)N;
    }
    __syncthreads();
    float* t = src; src = dst; dst = t;
  }
  if (threadIdx.x == 0) {
    f[0] = (float)log(fmax(norm1, 1e-300));
    for (int k = 2; k <= 4; ++k) {
      const float* e4 = est + (k - 1) * 4;
      const float e = fmaxf(fmaxf(e4[0], e4[1]), fmaxf(e4[2], e4[3]));
      f[k - 1] = (float)(log(fmax((double)e, 1e-300)) / k);
    }
    f[4] = (float)log((double)N);
  }
  __syncthreads();
}

// argmax of the network's logits on one feature vector (all threads take part)
__device__ int block_mlp_argmax(const BatchArgs& a, const float* f, float* h1, float* h2, float* lg) {
  const int hid = a.mlp_hid, out = a.mlp_out;
  const float *W1 = a.mlp, *b1 = W1 + hid * NFEAT, *W2 = b1 + hid, *b2 = W2 + hid * hid;
  const float *W3 = b2 + hid, *b3 = W3 + out * hid;
  for (int t = threadIdx.x; t < hid; t += BATCH_THREADS) {
    float acc = b1[t];
    for (int i = 0; i < NFEAT; ++i) acc = fmaf(W1[t * NFEAT + i], (f[i] - a.mu[i]) / a.sd[i], acc);
    h1[t] = fmaxf(acc, 0.f);
  }
  __syncthreads();
  for (int t = threadIdx.x; t < hid; t += BATCH_THREADS) {
    float acc = b2[t];
    for (int j = 0; j < hid; ++j) acc = fmaf(W2[t * hid + j], h1[j], acc);
    h2[t] = fmaxf(acc, 0.f);
  }
  __syncthreads();
  for (int t = threadIdx.x; t < out; t += BATCH_THREADS) {
    float acc = b3[t];
    for (int j = 0; j < hid; ++j) acc = fmaf(W3[t * hid + j], h2[j], acc);
    lg[t] = acc;
  }
  __syncthreads();
  int best = 0;
  for (int t = 1; t < out; ++t) best = lg[t] > lg[best] ? t : best;
  __syncthreads();
  return best;
}

// The Pade comparator's solve (-u + v) R = u + v in one CTA: Gaussian
// elimination with partial pivoting (largest |m_ik|, ties to the smaller row)
// applied to M and the N right-hand sides B alike, then back substitution with
// one right-hand side per thread; R overwrites B, M is destroyed. The paper
// counts it as 4/3 of a product (Section 1). flag (may be null) is set when the
// result is not finite.
__device__ __noinline__ void block_lu_solve(double* M, double* B, int N, double* red, int* redi,
                                            unsigned int* flag) {
  __shared__ int s_piv, s_sing;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (tid == 0) s_sing = 0;
  for (int k = 0; k < N; ++k) {
    double best = -1.0;
    int bi = N;
    for (int i = k + tid; i < N; i += BATCH_THREADS) {
      const double v = fabs(ldslot(M + (int64_t)i * N + k));
      if (v > best) { best = v; bi = i; }
    }
    for (int off = 16; off > 0; off >>= 1) {
      const double ov = __shfl_xor_sync(0xffffffffu, best, off);
      const int oi = __shfl_xor_sync(0xffffffffu, bi, off);
      if (ov > best || (ov == best && oi < bi)) { best = ov; bi = oi; }
    }
    if (lane == 0) { red[warp] = best; redi[warp] = bi; }
    __syncthreads();
    if (tid == 0) {
      double bv = -1.0;
      int bb = N;
      for (int w = 0; w < BATCH_THREADS / 32; ++w)
        if (red[w] > bv || (red[w] == bv && redi[w] < bb)) { bv = red[w]; bb = redi[w]; }
      s_piv = bb;
      if (!(bv > 0.0)) s_sing = 1;
    }
    __syncthreads();
    const int piv = s_piv;
    if (piv != k && piv < N) {
      for (int j = tid; j < 2 * N; j += BATCH_THREADS) {
        double* base = j < N ? M : B;
        const int c = j < N ? j : j - N;
        const double t = base[(int64_t)k * N + c];
        base[(int64_t)k * N + c] = base[(int64_t)piv * N + c];
        base[(int64_t)piv * N + c] = t;
      }
    }
    __syncthreads();
    const double d = M[(int64_t)k * N + k];
    for (int i = k + 1 + tid; i < N; i += BATCH_THREADS) M[(int64_t)i * N + k] /= d;
    __syncthreads();
    const int rows = N - k - 1, w = rows + N;
    for (int e = tid; e < rows * w; e += BATCH_THREADS) {
      const int i = k + 1 + e / w, c = e % w;
      const double l = M[(int64_t)i * N + k];
      if (c < rows) M[(int64_t)i * N + k + 1 + c] -= l * M[(int64_t)k * N + k + 1 + c];
      else B[(int64_t)i * N + (c - rows)] -= l * B[(int64_t)k * N + (c - rows)];
    }
    __syncthreads();
  }
  bool bad = s_sing != 0;
  for (int j = tid; j < N; j += BATCH_THREADS) {
    for (int i = N - 1; i >= 0; --i) {
      double x = B[(int64_t)i * N + j];
      for (int t = i + 1; t < N; ++t) x -= M[(int64_t)i * N + t] * B[(int64_t)t * N + j];
      x /= M[(int64_t)i * N + i];
      B[(int64_t)i * N + j] = x;
      bad |= !isfinite(x);
    }
  }
  if (bad && flag) atomicOr(flag, 1u);
  __syncthreads();
}

}  // namespace

__global__ void __launch_bounds__(BATCH_THREADS, 2) k_batched_expm(const BatchArgs args) {

  __shared__ GemmSmem sm;
  __shared__ Epilogue s_epi;
  __shared__ double s_red[BATCH_THREADS / 32];
  __shared__ int s_redi[BATCH_THREADS / 32];
  __shared__ int s_idx, s_m, s_s, s_prog, s_status, s_sel, s_pre;
  __shared__ double s_norm;
  __shared__ unsigned int s_flag;
  __shared__ float s_feat[NFEAT];
  __shared__ float s_h1[MLP_MAX], s_h2[MLP_MAX], s_lg[MLP_MAX];
  __shared__ float s_y[2][4 * BATCH_MAX_N];
  __shared__ float s_est[16];
  __shared__ double s_pnorm[4];
  __shared__ int s_pow, s_prop_m, s_prop_s;
  __shared__ OzbSmem s_oz;

  const int tid = threadIdx.x;
  // csize CTAs (one thread-block cluster) share each matrix: the cluster's slots,
  // its queue entry taken by rank 0, every product and element-wise pass split
  // by rank; the scalar work (norms, selection, features) is done by each CTA
  // from the same data, so all agree without exchanging it.
  const int csize = args.csize, rank = (int)(blockIdx.x % csize);
  const size_t nn_max = (size_t)args.nmax * args.nmax;
  double* slots = args.work + (size_t)(blockIdx.x / csize) * BATCH_SLOTS * nn_max;

  while (true) {
    if (tid == 0 && rank == 0) s_idx = (int)atomicAdd(args.counter, 1u);
    csync(csize);
    if (csize > 1) {
      if (tid == 0 && rank != 0) s_idx = cluster_load(&s_idx, 0);
      csync(csize);  // rank 0's entry is read everywhere before it changes (or its CTA exits)
    }
    const int64_t idx = s_idx;
    if (idx >= args.count) break;
    const int64_t N64 = args.Ns[idx];
    if (N64 < 1 || N64 > args.nmax) {  // not served: report and move on
      if (tid == 0 && rank == 0 && args.info) {
        bbc_info inf = {};
        inf.status = BBC_INVALID_ARG;
        args.info[idx] = inf;
      }
      __syncthreads();
      continue;
    }
    const int N = (int)N64;
    double* A64 = slots + (size_t)BSL_A * nn_max;

    // ---- a1: load A as binary64 and take ||A||_1. G threads share a column
    // (G = 4, 2, 1 for N <= 64, 128, larger; thread g sums rows g, g + G, ...,
    // then the G partial sums add in order), and each thread issues 8 loads
    // before its stores: a store may alias the next load for all the compiler
    // knows, so one load per store would cost a memory round trip per element.
    const int G = N <= 64 ? 4 : (N <= 128 ? 2 : 1);
    const int CW = BATCH_THREADS / G;  // columns per pass
    const int g = tid / CW, jj = tid % CW;
    double* colpart = reinterpret_cast<double*>(&s_y[0][0]);  // G x CW partial sums
    const void* Ain = args.A[idx];
    double colmax = 0.0;
    for (int j0 = 0; j0 < N; j0 += CW) {
      const int j = j0 + jj;
      double s = 0.0;
      if (j < N) {
        const bool own = (j % csize) == rank;
        for (int i0 = g; i0 < N; i0 += 8 * G) {
          double v[8];
#pragma unroll
          for (int u = 0; u < 8; ++u) {
            const int64_t e = (int64_t)(i0 + u * G) * N + j;
            v[u] = i0 + u * G >= N ? 0.0
                   : args.dtype == 1 ? (double)static_cast<const float*>(Ain)[e]
                                     : static_cast<const double*>(Ain)[e];
          }
#pragma unroll
          for (int u = 0; u < 8; ++u) {
            const int i = i0 + u * G;
            if (i < N) {
              if (own) A64[(int64_t)i * N + j] = v[u];
              s += fabs(v[u]);
            }
          }
        }
      }
      if (G > 1) {
        colpart[g * CW + jj] = s;
        __syncthreads();
        if (g == 0)
          for (int k = 1; k < G; ++k) s += colpart[k * CW + jj];
        __syncthreads();
      }
      if (g == 0 && j < N) colmax = (s > colmax || isnan(s)) ? s : colmax;
    }
    for (int off = 16; off > 0; off >>= 1) {
      const double o = __shfl_xor_sync(0xffffffffu, colmax, off);
      colmax = (o > colmax || isnan(o)) ? o : colmax;
    }
    if ((tid & 31) == 0) s_red[tid >> 5] = colmax;
    __syncthreads();

    // ---- a2: select (m, s) on the device
    if (tid == 0) {
      double nrm = 0.0;
      for (int w = 0; w < BATCH_THREADS / 32; ++w) nrm = (s_red[w] > nrm || isnan(s_red[w])) ? s_red[w] : nrm;
      s_norm = nrm;
      s_flag = 0u;
      s_pre = 0;
      s_pow = 0;
      s_sel = SEL_PLAIN;
      s_status = isfinite(nrm) ? BBC_OK : BBC_NONFINITE_INPUT;
    }
    csync(csize);  // A64 complete
    if (s_status == BBC_OK && (args.mode == MODE_LEARNED || args.mode == MODE_DATA))
      block_features(A64, N, s_norm, s_y[0], s_y[1], s_est, s_feat);
    if (s_status == BBC_OK && args.mode == MODE_LEARNED) {
      const int c = block_mlp_argmax(args, s_feat, s_h1, s_h2, s_lg);
      if (tid == 0) {
        s_prop_m = c / args.mlp_S;
        s_prop_s = c % args.mlp_S;
        // the paper's own bound already certifies the proposal: no powers needed
        s_pow = !(s_prop_m < BATCH_PROGS && ldexp(s_norm, -s_prop_s) <= args.theta[s_prop_m]);
      }
    }
    if (tid == 0 && s_status == BBC_OK && (args.mode == MODE_ALPHA || args.mode == MODE_DATA)) s_pow = 1;
    __syncthreads();
    // exact powers A^2 -> W0, A^3 -> W1 when a bound (or the training data) needs them
    if (s_status == BBC_OK && s_pow) {
      double* W0p = slots;
      const int npow = 2;
      for (int k = 0; k < npow; ++k) {
        if (tid == 0) {
          s_epi.nout = 1;
          s_epi.flag = nullptr;
          s_epi.o[0].out = slots + (size_t)k * nn_max;
          s_epi.o[0].cv = 1.0;
          s_epi.o[0].cI = 0.0;
          s_epi.o[0].nt = 0;
        }
        __syncthreads();
        // A^2 = A A, A^3 = A^2 A (split products in split mode; FP64 for training data)
        block_product(args, k == 0 ? A64 : W0p, A64, N, 1.0, s_epi, sm, s_oz, rank, csize);
        csync(csize);
        const double nk = block_norm1(slots + (size_t)k * nn_max, N, s_red);
        if (tid == 0) s_pnorm[k + 1] = nk;
      }
    }
    __syncthreads();
    if (tid == 0 && s_status == BBC_OK && args.mode != MODE_DATA) {
      const double nrm = s_norm;
      // the margin covers the rounding of the computed powers (~2^-30 relative for split products)
      const double margin = (args.prec == 1 && N <= OZB_NMAX) ? 1e-6 : 1e-12;
      const double alpha2 = s_pow ? fmax(sqrt(s_pnorm[1]), cbrt(s_pnorm[2])) * (1.0 + margin) : INFINITY;
      int bm = 0, bs = 0, bc = 1 << 30;
      bool done = false;
      if (args.pade) {  // r_10 (3 products) or r_26 (6); the solve is common to both
        for (int i = args.pade == 2 ? 1 : 0; i < 2; ++i) {
          const int si = least_squarings(nrm, args.theta_pade[i]);
          const int cost = (i ? 6 : 3) + si;
          if (cost < bc || (cost == bc && si < bs)) { bc = cost; bm = i; bs = si; }
        }
        done = true;
      }
      if (args.mode == MODE_LEARNED && s_prop_m < BATCH_PROGS) {
        if (ldexp(nrm, -s_prop_s) <= args.theta[s_prop_m]) {
          bm = s_prop_m; bs = s_prop_s; done = true; s_sel = SEL_LEARNED_NORM;
        } else if (ldexp(alpha2, -s_prop_s) <= args.theta[s_prop_m]) {
          bm = s_prop_m; bs = s_prop_s; done = true; s_sel = SEL_LEARNED_ALPHA;
        } else {
          s_sel = SEL_LEARNED_REJECTED;
        }
      }
      if (!done) {
        for (int i = 0; i < BATCH_PROGS; ++i) {
          int si = least_squarings(nrm, args.theta[i]);
          if (args.mode == MODE_ALPHA) si = min(si, least_squarings(alpha2, args.theta[i]));
          const int cost = args.prod[i] + si;
          if (cost < bc || (cost == bc && si < bs)) { bc = cost; bm = i; bs = si; }
        }
        if (args.mode == MODE_ALPHA) s_sel = SEL_ALPHA;
      }
      s_prog = bm;
      s_m = args.pade ? (bm ? 26 : 10) : args.deg[bm];
      s_s = bs;
      s_pre = (!args.pade && s_pow && (args.deg[bm] == 12 || args.deg[bm] == 18)) ? 1 : 0;
    }
    __syncthreads();
    if (args.mode == MODE_DATA) {
      if (tid == 0 && rank == 0) {
        const bool ok = s_status == BBC_OK;
        args.norms_out[idx * 4 + 0] = ok ? s_norm : NAN;
        for (int k = 1; k < 3; ++k) args.norms_out[idx * 4 + k] = ok ? s_pnorm[k] : NAN;
        args.norms_out[idx * 4 + 3] = NAN;  // ||A^4|| is not computed
        for (int k = 0; k < NFEAT; ++k) args.feat_out[idx * NFEAT + k] = ok ? s_feat[k] : NAN;
        if (args.info) {
          bbc_info inf = {};
          inf.norm1 = s_norm;
          inf.products = ok ? 2 : 0;
          inf.status = s_status;
          args.info[idx] = inf;
        }
      }
      __syncthreads();
      continue;
    }
    if (s_status != BBC_OK) {
      if (tid == 0 && rank == 0 && args.info) {
        bbc_info inf = {};
        inf.norm1 = s_norm;
        inf.status = s_status;
        args.info[idx] = inf;
      }
      __syncthreads();
      continue;
    }
    const int s = s_s;
    const double sig = ldexp(1.0, -s);
    const BProg& prog = args.pade ? c_progs_pade[s_prog] : s_pre ? c_progs_pre[s_m == 18 ? 1 : 0] : c_progs[s_prog];
    const int extra_products = s_pow ? 2 : 0;
    double* Tslot = slots + (size_t)BSL_T * nn_max;
    double* SQ = slots + (size_t)SL_SQ * nn_max;

    // ---- a3..a8: the Taylor program with 2^-s folded into its coefficients
    for (int k = 0; k < prog.nsteps; ++k) {
      const BStep& st = prog.st[k];
      if (tid == 0) {
        s_epi.nout = st.nout;
        s_epi.flag = (k + 1 == prog.nsteps && s == 0) ? &s_flag : nullptr;
        int ny = 0;
        for (int o = 0; o < st.nout; ++o) {
          const BOut& q = st.o[o];
          const int dslot = q.dst == SL_T ? BSL_T : q.dst;
          s_epi.o[o].out = slots + (size_t)dslot * nn_max;
          s_epi.o[o].cv = q.cv;
          s_epi.o[o].cI = q.cI;
          s_epi.o[o].nt = q.nt;
          for (int tt = 0; tt < q.nt; ++tt) {
            const int sl = q.slot[tt] == SL_A ? BSL_A : q.slot[tt];
            const double* y = slots + (size_t)sl * nn_max;
            int yi = 0;
            while (yi < ny && s_epi.Y[yi] != y) ++yi;
            if (yi == ny) s_epi.Y[ny++] = y;
            s_epi.o[o].slot[tt] = yi;
            double c = q.c[tt];
            for (int p = 0; p < q.sigma_pow[tt]; ++p) c *= sig;
            s_epi.o[o].c[tt] = c;
          }
        }
      }
      __syncthreads();
      if (st.P < 0) {
        block_lincomb(N, s_epi, sm, rank, csize);
      } else {
        double alpha = 1.0;
        for (int p = 0; p < st.alpha_pow; ++p) alpha *= sig;
        const double* P = slots + (size_t)(st.P == SL_A ? BSL_A : st.P) * nn_max;
        const double* Q = slots + (size_t)(st.Q == SL_A ? BSL_A : st.Q) * nn_max;
        block_product(args, P, Q, N, alpha, s_epi, sm, s_oz, rank, csize);
      }
      csync(csize);
    }

    // Pade: W8 holds -u + v and T holds u + v; r = (-u + v)^-1 (u + v) overwrites T
    // (one CTA of a cluster solves, the others wait)
    if (args.pade) {
      if (rank == 0) block_lu_solve(slots + (size_t)8 * nn_max, Tslot, N, s_red, s_redi, s == 0 ? &s_flag : nullptr);
      csync(csize);
    }

    // ---- a9: s squarings, ping-pong between T and the squaring slot
    double* src = Tslot;
    for (int k = 0; k < s; ++k) {
      double* dst = (src == Tslot) ? SQ : Tslot;
      if (tid == 0) {
        s_epi.nout = 1;
        s_epi.flag = (k + 1 == s) ? &s_flag : nullptr;
        s_epi.o[0].out = dst;
        s_epi.o[0].cv = 1.0;
        s_epi.o[0].cI = 0.0;
        s_epi.o[0].nt = 0;
      }
      __syncthreads();
      block_product(args, src, src, N, 1.0, s_epi, sm, s_oz, rank, csize);
      csync(csize);
      src = dst;
    }

    // ---- exp(A) B (the step of an exponential integrator): B_i copied into the
    // A slot, free once the program has run (a copy, so Out_i may be B_i), then
    // one more product into the other ping-pong buffer
    int applied = 0;
    if (args.B) {
      const void* Bin = args.B[idx];
      const int NN = N * N, step = csize * BATCH_THREADS;
      for (int e0 = rank * BATCH_THREADS + tid; e0 < NN; e0 += 8 * step) {
        double v[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          const int e = e0 + u * step;
          v[u] = e >= NN ? 0.0
                 : args.dtype == 1 ? (double)static_cast<const float*>(Bin)[e] : static_cast<const double*>(Bin)[e];
        }
#pragma unroll
        for (int u = 0; u < 8; ++u)
          if (e0 + u * step < NN) A64[e0 + u * step] = v[u];
      }
      csync(csize);
      double* dst = (src == Tslot) ? SQ : Tslot;
      if (tid == 0) {
        s_epi.nout = 1;
        s_epi.flag = &s_flag;
        s_epi.o[0].out = dst;
        s_epi.o[0].cv = 1.0;
        s_epi.o[0].cI = 0.0;
        s_epi.o[0].nt = 0;
      }
      __syncthreads();
      block_product(args, src, A64, N, 1.0, s_epi, sm, s_oz, rank, csize);
      csync(csize);
      src = dst;
      applied = 1;
    }

    // ---- a10: output in the caller's type, status, info
    {
      void* outp = args.Out[idx];
      const int NN = N * N, step = csize * BATCH_THREADS;
      for (int e0 = rank * BATCH_THREADS + tid; e0 < NN; e0 += 8 * step) {
        double v[8];  // 8 loads in flight before the stores (as in a1)
#pragma unroll
        for (int u = 0; u < 8; ++u) v[u] = e0 + u * step < NN ? ldslot(src + e0 + u * step) : 0.0;
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          const int e = e0 + u * step;
          if (e >= NN) break;
          if (args.dtype == 1) {
            const float f = (float)v[u];
            static_cast<float*>(outp)[e] = f;
            if (!isfinite(f)) s_flag = 1u;
          } else {
            static_cast<double*>(outp)[e] = v[u];
          }
        }
      }
    }
    __syncthreads();
    if (csize > 1) {  // overflow seen by any CTA of the cluster -> rank 0's flag
      if (tid == 0 && rank != 0 && s_flag) cluster_or(&s_flag, 0, 1u);
      csync(csize);
    }
    if (tid == 0 && rank == 0 && args.info) {
      bbc_info inf = {};
      inf.m = s_m;
      inf.s = s;
      inf.products = prog.products + s + extra_products + applied;
      inf.selector = s_sel;
      inf.norm1 = s_norm;
      inf.status = s_flag ? BBC_OVERFLOW : BBC_OK;
      args.info[idx] = inf;
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
size_t batched_workspace_bytes(int64_t nmax, int ctas, bool split) {
  return (size_t)ctas * BATCH_SLOTS * nmax * nmax * sizeof(double) + 256 +
         (split ? (size_t)ctas * OZB_WORDS * sizeof(uint32_t) : 0);
}

// Two resident CTAs per SM (128 registers, ~43 KB shared memory each): while one
// waits on its loads the other computes.
int batched_ctas(int device) {
  int sms = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess || sms <= 0) sms = 152;
  return 2 * sms;
}

namespace {
// s = 0 coefficients with the powers of 2^-s each coefficient / alpha carries:
// given explicitly (sp, ap >= 0) or, for the plain programs, one per use of A.
bool to_device_program(const Program& p, int m, BProg* out) {
  if ((int)p.steps.size() > BATCH_MAX_STEPS) return false;
  out->m = m;
  out->products = p.products;
  out->nsteps = (int)p.steps.size();
  for (size_t k = 0; k < p.steps.size(); ++k) {
    const StepS& st = p.steps[k];
    BStep& b = out->st[k];
    b.P = st.P;
    b.Q = st.Q;
    b.alpha_pow = st.ap >= 0 ? st.ap : (st.P == SL_A) + (st.Q == SL_A);
    b.nout = st.nout;
    for (int o = 0; o < st.nout; ++o) {
      b.o[o].dst = st.o[o].dst;
      b.o[o].cv = st.o[o].cv;
      b.o[o].cI = st.o[o].cI;
      b.o[o].nt = st.o[o].nt;
      for (int t = 0; t < st.o[o].nt; ++t) {
        const TermS& ts = st.o[o].t[t];
        b.o[o].slot[t] = ts.slot;
        b.o[o].c[t] = ts.c;
        b.o[o].sigma_pow[t] = ts.sp >= 0 ? ts.sp : (ts.slot == SL_A ? 1 : 0);
      }
    }
  }
  return true;
}
}  // namespace

// Upload the reduced-product programs: plain ones and T12 / T18 that start from
// precomputed A^2, A^3.
cudaError_t batched_upload_programs() {
  static const int deg[BATCH_PROGS] = {1, 2, 4, 8, 12, 18};
  BProg h[BATCH_PROGS] = {};
  for (int i = 0; i < BATCH_PROGS; ++i) {
    Program p;
    if (!make_program(BBC_SCHEME_NEW, deg[i], 0, &p) || !to_device_program(p, deg[i], &h[i]))
      return cudaErrorInvalidValue;
  }
  cudaError_t e = cudaMemcpyToSymbol(c_progs, h, sizeof h);
  if (e != cudaSuccess) return e;
  BProg pre[2] = {};
  const int pm[2] = {12, 18};
  for (int i = 0; i < 2; ++i) {
    Program p;
    int a2, a3;
    if (!make_prefilled_program(pm[i], &p, &a2, &a3) || a2 != 0 || a3 != 1 || !to_device_program(p, pm[i], &pre[i]))
      return cudaErrorInvalidValue;
  }
  e = cudaMemcpyToSymbol(c_progs_pre, pre, sizeof pre);
  if (e != cudaSuccess) return e;
  BProg pd[2] = {};
  const int pdeg[2] = {10, 26};
  for (int i = 0; i < 2; ++i) {
    Program p;
    if (!make_program(BBC_SCHEME_PADE, pdeg[i], 0, &p) || !to_device_program(p, pdeg[i], &pd[i]))
      return cudaErrorInvalidValue;
  }
  return cudaMemcpyToSymbol(c_progs_pade, pd, sizeof pd);
}

// Cluster shapes for small batches: a dynamic shared-memory request that leaves
// room for one CTA per SM (the CTAs of a cluster then sit on distinct SMs, each
// with its own FP64 pipe) and how many clusters of 2, 4, 8, 16 CTAs fit at once.
// Called outside stream capture (at reservation).
cudaError_t batched_cluster_probe(int device, BatchClusters* out) {
  *out = BatchClusters{};
  int sms = 0, smem_sm = 0, optin = 0;
  cudaError_t e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, device);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, device);
  cudaFuncAttributes fa = {};
  if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, k_batched_expm);
  if (e != cudaSuccess) return e;
  const int stat = (int)fa.sharedSizeBytes;
  const int dyn = smem_sm / 2 + 1024 - stat;
  if (dyn < 0 || stat + dyn > optin) return cudaSuccess;  // no cluster mode
  e = cudaFuncSetAttribute(k_batched_expm, cudaFuncAttributeMaxDynamicSharedMemorySize, dyn);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_batched_expm, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return cudaSuccess;
  }
  out->sms = sms;
  out->dyn_smem = dyn;
  for (int lg = 1; lg <= 4; ++lg) {
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute at = {};
    at.id = cudaLaunchAttributeClusterDimension;
    at.val.clusterDim.x = 1u << lg;
    at.val.clusterDim.y = 1;
    at.val.clusterDim.z = 1;
    cfg.gridDim = dim3(1u << lg);
    cfg.blockDim = dim3(BATCH_THREADS);
    cfg.dynamicSmemBytes = (size_t)dyn;
    cfg.attrs = &at;
    cfg.numAttrs = 1;
    int n = 0;
    if (cudaOccupancyMaxActiveClusters(&n, k_batched_expm, &cfg) != cudaSuccess) {
      cudaGetLastError();
      n = 0;
    }
    out->max_active[lg] = n;
  }
  return cudaSuccess;
}

// CTAs per matrix for a batch of `count`: the cluster size (1, 2, 4, 8, 16) with
// the fewest FP64-pipe rounds, ceil(count / clusters) / size, counting only
// batches that leave SMs idle at one CTA per matrix. *grid gets the CTA count.
int batched_cluster_size(const BatchClusters* cl, int64_t count, int ctas, int* grid) {
  *grid = ctas;
  if (!cl || cl->sms <= 0 || count < 1 || count > cl->sms / 2) return 1;
  int best_c = 1;
  double best = (double)((count + ctas - 1) / ctas);
  for (int lg = 1; lg <= 4; ++lg) {
    const int c = 1 << lg;
    const int64_t ncl = std::min<int64_t>(std::min<int64_t>(count, cl->max_active[lg]), ctas / c);
    if (ncl < 1) continue;
    const double cost = (double)((count + ncl - 1) / ncl) / c;
    if (cost < best) {
      best = cost;
      best_c = c;
      *grid = (int)(ncl * c);
    }
  }
  return best_c;
}

cudaError_t batched_launch(const void* const* A, void* const* Out, const int64_t* Ns, int64_t count, int64_t nmax,
                           int dtype, const double* theta, void* work, int ctas, bbc_info* info, cudaStream_t st,
                           const BatchSelector* sel, bool split, uint32_t split_mask, const BatchClusters* cl,
                           const void* const* B, int pade, const double* theta_pade, const BatchShapes* shapes) {
  static const int deg[BATCH_PROGS] = {1, 2, 4, 8, 12, 18};
  static const int prod[BATCH_PROGS] = {0, 1, 2, 3, 4, 5};
  BatchArgs a = {};
  a.A = A;
  a.B = B;
  a.pade = pade;
  if (pade) {
    if (!theta_pade) return cudaErrorInvalidValue;
    a.theta_pade[0] = theta_pade[0];
    a.theta_pade[1] = theta_pade[1];
  }
  a.Out = Out;
  a.Ns = Ns;
  a.count = count;
  a.nmax = nmax;
  a.dtype = dtype;
  for (int i = 0; i < BATCH_PROGS; ++i) { a.theta[i] = theta[i]; a.deg[i] = deg[i]; a.prod[i] = prod[i]; }
  a.counter = static_cast<unsigned int*>(work);
  a.work = reinterpret_cast<double*>(static_cast<char*>(work) + 256);
  a.info = info;
  a.prec = split ? 1 : 0;
  a.split_mask = split_mask;
  if (shapes) a.shapes = *shapes;
  a.ozwork = split ? reinterpret_cast<uint32_t*>(static_cast<char*>(work) + 256 +
                                                 (size_t)ctas * BATCH_SLOTS * nmax * nmax * sizeof(double))
                   : nullptr;
  a.mode = MODE_PLAIN;
  if (sel) {
    a.mode = sel->mode;
    a.mlp = sel->params;
    a.mlp_hid = sel->hid;
    a.mlp_out = sel->out;
    a.mlp_S = sel->S > 0 ? sel->S : 1;
    for (int i = 0; i < NFEAT; ++i) { a.mu[i] = sel->mu[i]; a.sd[i] = sel->sd[i] != 0.f ? sel->sd[i] : 1.f; }
    a.feat_out = sel->feat_out;
    a.norms_out = sel->norms_out;
    if (a.mode == MODE_LEARNED && (!a.mlp || a.mlp_hid < 1 || a.mlp_hid > MLP_MAX || a.mlp_out < 1 ||
                                   a.mlp_out > MLP_MAX))
      return cudaErrorInvalidValue;
    if (a.mode == MODE_DATA && (!a.feat_out || !a.norms_out)) return cudaErrorInvalidValue;
  }
  int grid = ctas;
  a.csize = batched_cluster_size(cl, count, ctas, &grid);
  cudaError_t err = cudaMemsetAsync(a.counter, 0, sizeof(unsigned int), st);
  if (err != cudaSuccess) return err;
  if (a.csize == 1) {
    k_batched_expm<<<ctas, BATCH_THREADS, 0, st>>>(a);
    return cudaGetLastError();
  }
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute at = {};
  at.id = cudaLaunchAttributeClusterDimension;
  at.val.clusterDim.x = (unsigned)a.csize;
  at.val.clusterDim.y = 1;
  at.val.clusterDim.z = 1;
  cfg.gridDim = dim3((unsigned)grid);
  cfg.blockDim = dim3(BATCH_THREADS);
  cfg.dynamicSmemBytes = (size_t)cl->dyn_smem;
  cfg.stream = st;
  cfg.attrs = &at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k_batched_expm, a);
}

// Calibration matrices for the batched autotuner: count matrices of size N with
// entries uniform on [-1, 1) from a counter-based hash (splitmix64 of seed and
// index), scaled so that every column sum of |a_ij| is about 2 norm1 / N * N / 2
// = norm1 (the 1-norm, hence (m, s), sits near the chosen value).
__global__ void k_calibration(double* out, int64_t N, int64_t count, uint64_t seed, double norm1) {
  const int64_t total = N * N * count;
  const double scale = 2.0 * norm1 / (double)N;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    uint64_t z = seed + 0x9E3779B97F4A7C15ull * (uint64_t)(i + 1);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z ^= z >> 31;
    out[i] = scale * ((double)(z >> 11) * 0x1.0p-53 * 2.0 - 1.0);
  }
}

cudaError_t calibration_matrices(double* out, int64_t N, int64_t count, uint64_t seed, double norm1, cudaStream_t st) {
  k_calibration<<<1216, 256, 0, st>>>(out, N, count, seed, norm1);
  return cudaGetLastError();
}

}  // namespace bbc
