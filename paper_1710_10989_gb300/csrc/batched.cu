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
#include <math.h>
#include <stdint.h>

#include "bbcexpm.h"
#include "internal.h"
#include "schemes.h"

namespace bbc {

constexpr int BATCH_THREADS = 256;
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

struct BatchArgs {
  const void* const* A;    // device array of device pointers
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
};

namespace {

__device__ int least_squarings_dev(double norm, double th) {
  if (!(norm > th)) return 0;
  int s = (int)ceil(log2(norm / th));
  if (s < 0) s = 0;
  while (ldexp(norm, -s) > th) ++s;
  while (s > 0 && ldexp(norm, -(s - 1)) <= th) --s;
  return s;
}

// 64 x 64 output tiles, 16-deep K slabs, 256 threads (4 x 4 each, stride 16).
struct GemmSmem {
  double As[16][64];
  double Bs[16][64];
};

__device__ void block_gemm_f64(const double* __restrict__ P, const double* __restrict__ Q, int N, double alpha,
                               const Epilogue& e, GemmSmem& sm) {
  const int t = threadIdx.x, tx = t % 16, ty = t / 16;
  const int tiles = (N + 63) / 64;
  for (int tile = 0; tile < tiles * tiles; ++tile) {
    const int m0 = (tile / tiles) * 64, n0 = (tile % tiles) * 64;
    double acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) acc[i][j] = 0.0;
    for (int k0 = 0; k0 < N; k0 += 16) {
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int r = t / 16 + 16 * q, c = t % 16;  // P tile 64 x 16
        sm.As[c][r] = (m0 + r < N && k0 + c < N) ? P[(int64_t)(m0 + r) * N + k0 + c] : 0.0;
        const int r2 = t / 64 + 4 * q, c2 = t % 64;  // Q tile 16 x 64
        sm.Bs[r2][c2] = (k0 + r2 < N && n0 + c2 < N) ? Q[(int64_t)(k0 + r2) * N + n0 + c2] : 0.0;
      }
      __syncthreads();
#pragma unroll
      for (int kk = 0; kk < 16; ++kk) {
        double a[4], b[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) a[i] = sm.As[kk][ty + 16 * i];
#pragma unroll
        for (int j = 0; j < 4; ++j) b[j] = sm.Bs[kk][tx + 16 * j];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
      }
      __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int row = m0 + ty + 16 * i;
      if (row >= N) continue;
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int col = n0 + tx + 16 * j;
        if (col < N) apply_epilogue(e, N, row, col, alpha * acc[i][j]);
      }
    }
  }
}

__device__ void block_lincomb(int N, const Epilogue& e) {
  for (int idx = threadIdx.x; idx < N * N; idx += BATCH_THREADS) apply_epilogue(e, N, idx / N, idx % N, 0.0);
}

}  // namespace

__global__ void __launch_bounds__(BATCH_THREADS, 1) k_batched_expm(const BatchArgs args) {
  __shared__ GemmSmem sm;
  __shared__ Epilogue s_epi;
  __shared__ double s_red[BATCH_THREADS / 32];
  __shared__ int s_idx, s_m, s_s, s_prog, s_status;
  __shared__ double s_norm;
  __shared__ unsigned int s_flag;

  const int tid = threadIdx.x;
  const size_t nn_max = (size_t)args.nmax * args.nmax;
  double* slots = args.work + (size_t)blockIdx.x * BATCH_SLOTS * nn_max;

  while (true) {
    if (tid == 0) s_idx = (int)atomicAdd(args.counter, 1u);
    __syncthreads();
    const int64_t idx = s_idx;
    if (idx >= args.count) break;
    const int64_t N64 = args.Ns[idx];
    if (N64 < 1 || N64 > args.nmax) {  // not served: report and move on
      if (tid == 0 && args.info) {
        bbc_info inf = {};
        inf.status = BBC_INVALID_ARG;
        args.info[idx] = inf;
      }
      __syncthreads();
      continue;
    }
    const int N = (int)N64;
    double* A64 = slots + (size_t)BSL_A * nn_max;

    // ---- a1: load A as binary64 and take ||A||_1 (one column per thread)
    double colmax = 0.0;
    for (int j = tid; j < N; j += BATCH_THREADS) {
      double s = 0.0;
      for (int i = 0; i < N; ++i) {
        const double v = args.dtype == 1 ? (double)((const float*)args.A[idx])[(int64_t)i * N + j]
                                         : ((const double*)args.A[idx])[(int64_t)i * N + j];
        A64[(int64_t)i * N + j] = v;
        s += fabs(v);
      }
      colmax = (s > colmax || isnan(s)) ? s : colmax;
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
      if (!isfinite(nrm)) {
        s_status = BBC_NONFINITE_INPUT;
      } else {
        s_status = BBC_OK;
        int bm = 0, bs = 0, bc = 1 << 30;
        for (int i = 0; i < BATCH_PROGS; ++i) {
          const int si = least_squarings_dev(nrm, args.theta[i]);
          const int cost = args.prod[i] + si;
          if (cost < bc || (cost == bc && si < bs)) { bc = cost; bm = i; bs = si; }
        }
        s_prog = bm;
        s_m = args.deg[bm];
        s_s = bs;
      }
    }
    __syncthreads();
    if (s_status != BBC_OK) {
      if (tid == 0 && args.info) {
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
    const BProg& prog = c_progs[s_prog];
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
        block_lincomb(N, s_epi);
      } else {
        double alpha = 1.0;
        for (int p = 0; p < st.alpha_pow; ++p) alpha *= sig;
        const double* P = slots + (size_t)(st.P == SL_A ? BSL_A : st.P) * nn_max;
        const double* Q = slots + (size_t)(st.Q == SL_A ? BSL_A : st.Q) * nn_max;
        block_gemm_f64(P, Q, N, alpha, s_epi, sm);
      }
      __syncthreads();
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
      block_gemm_f64(src, src, N, 1.0, s_epi, sm);
      __syncthreads();
      src = dst;
    }

    // ---- a10: output in the caller's type, status, info
    for (int e = tid; e < N * N; e += BATCH_THREADS) {
      const double v = src[e];
      if (args.dtype == 1) {
        const float f = (float)v;
        ((float*)args.Out[idx])[e] = f;
        if (!isfinite(f)) s_flag = 1u;
      } else {
        ((double*)args.Out[idx])[e] = v;
      }
    }
    __syncthreads();
    if (tid == 0 && args.info) {
      bbc_info inf = {};
      inf.m = s_m;
      inf.s = s;
      inf.products = prog.products + s;
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
size_t batched_workspace_bytes(int64_t nmax, int ctas) {
  return (size_t)ctas * BATCH_SLOTS * nmax * nmax * sizeof(double) + 256;
}

int batched_ctas(int device) {
  int sms = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess || sms <= 0) sms = 152;
  return sms;
}

// Upload the reduced-product programs (s = 0 coefficients with sigma powers).
cudaError_t batched_upload_programs() {
  static const int deg[BATCH_PROGS] = {1, 2, 4, 8, 12, 18};
  BProg h[BATCH_PROGS] = {};
  for (int i = 0; i < BATCH_PROGS; ++i) {
    Program p;
    if (!make_program(BBC_SCHEME_NEW, deg[i], 0, &p) || (int)p.steps.size() > BATCH_MAX_STEPS)
      return cudaErrorInvalidValue;
    h[i].m = deg[i];
    h[i].products = p.products;
    h[i].nsteps = (int)p.steps.size();
    for (size_t k = 0; k < p.steps.size(); ++k) {
      const StepS& st = p.steps[k];
      BStep& b = h[i].st[k];
      b.P = st.P;
      b.Q = st.Q;
      b.alpha_pow = (st.P == SL_A) + (st.Q == SL_A);
      b.nout = st.nout;
      for (int o = 0; o < st.nout; ++o) {
        b.o[o].dst = st.o[o].dst;
        b.o[o].cv = st.o[o].cv;
        b.o[o].cI = st.o[o].cI;
        b.o[o].nt = st.o[o].nt;
        for (int t = 0; t < st.o[o].nt; ++t) {
          b.o[o].slot[t] = st.o[o].t[t].slot;
          b.o[o].c[t] = st.o[o].t[t].c;
          b.o[o].sigma_pow[t] = st.o[o].t[t].slot == SL_A ? 1 : 0;
        }
      }
    }
  }
  return cudaMemcpyToSymbol(c_progs, h, sizeof h);
}

cudaError_t batched_launch(const void* const* A, void* const* Out, const int64_t* Ns, int64_t count, int64_t nmax,
                           int dtype, const double* theta, void* work, int ctas, bbc_info* info, cudaStream_t st) {
  static const int deg[BATCH_PROGS] = {1, 2, 4, 8, 12, 18};
  static const int prod[BATCH_PROGS] = {0, 1, 2, 3, 4, 5};
  BatchArgs a = {};
  a.A = A;
  a.Out = Out;
  a.Ns = Ns;
  a.count = count;
  a.nmax = nmax;
  a.dtype = dtype;
  for (int i = 0; i < BATCH_PROGS; ++i) { a.theta[i] = theta[i]; a.deg[i] = deg[i]; a.prod[i] = prod[i]; }
  a.counter = static_cast<unsigned int*>(work);
  a.work = reinterpret_cast<double*>(static_cast<char*>(work) + 256);
  a.info = info;
  cudaError_t err = cudaMemsetAsync(a.counter, 0, sizeof(unsigned int), st);
  if (err != cudaSuccess) return err;
  k_batched_expm<<<ctas, BATCH_THREADS, 0, st>>>(a);
  return cudaGetLastError();
}

}  // namespace bbc
