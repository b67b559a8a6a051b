// pade.cu -- the linear solve of the diagonal Pade comparator: (v - u) R = u + v
// (eq. pade10 / eq. pade26). The paper counts it as 4/3 of a product: an LU
// factorisation with partial pivoting (1/3) and N forward / back substitutions (1).
//  N <= 112: the right-hand sides are independent once L, U and the pivots are
//    known, so each CTA of ceil(N / 4) factors M on its own in shared memory (the
//    same pivots everywhere: the choice is deterministic) and carries 4 of the
//    right-hand sides through the elimination and the back substitution (a warp
//    per right-hand side); no CTA waits for another.
//  N <= 1024: Gaussian elimination with partial pivoting on the N right-hand
//    sides at once in one CTA of 1024 threads, in global memory.
//  N > 1024: cuSOLVER's getrf / getrs (FP64), loaded at run time; the comparator
//    then fails with BBC_UNSUPPORTED where the library is absent. Row-major M is
//    the column-major M^T, so getrf factors M^T and getrs with op = T solves
//    M Z = B for B given column-major (a transpose on each side of the solve).
#include <dlfcn.h>
#include <math.h>

#include <mutex>

#include "internal.h"

namespace bbc {
namespace {

constexpr int SOLVE_THREADS = 1024;

__global__ void __launch_bounds__(SOLVE_THREADS, 1)
k_lu_solve(double* __restrict__ M, double* __restrict__ B, int N, unsigned int* __restrict__ flag) {
  __shared__ double s_val[SOLVE_THREADS / 32];
  __shared__ int s_idx[SOLVE_THREADS / 32];
  __shared__ int s_piv;
  __shared__ int s_singular;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (tid == 0) s_singular = 0;
  for (int k = 0; k < N; ++k) {
    // pivot: largest |M_ik|, i >= k (ties to the smaller row)
    double best = -1.0;
    int bi = N;
    for (int i = k + tid; i < N; i += SOLVE_THREADS) {
      const double v = fabs(M[(int64_t)i * N + k]);
      if (v > best) { best = v; bi = i; }
    }
    for (int off = 16; off > 0; off >>= 1) {
      const double ov = __shfl_xor_sync(0xffffffffu, best, off);
      const int oi = __shfl_xor_sync(0xffffffffu, bi, off);
      if (ov > best || (ov == best && oi < bi)) { best = ov; bi = oi; }
    }
    if (lane == 0) { s_val[warp] = best; s_idx[warp] = bi; }
    __syncthreads();
    if (tid == 0) {
      double bv = -1.0;
      int bb = N;
      for (int w = 0; w < SOLVE_THREADS / 32; ++w)
        if (s_val[w] > bv || (s_val[w] == bv && s_idx[w] < bb)) { bv = s_val[w]; bb = s_idx[w]; }
      s_piv = bb;
      if (!(bv > 0.0)) s_singular = 1;
    }
    __syncthreads();
    const int piv = s_piv;
    if (piv != k && piv < N) {
      for (int j = tid; j < 2 * N; j += SOLVE_THREADS) {
        double* base = j < N ? M : B;
        const int c = j < N ? j : j - N;
        const double t = base[(int64_t)k * N + c];
        base[(int64_t)k * N + c] = base[(int64_t)piv * N + c];
        base[(int64_t)piv * N + c] = t;
      }
    }
    __syncthreads();
    const double d = M[(int64_t)k * N + k];
    for (int i = k + 1 + tid; i < N; i += SOLVE_THREADS) M[(int64_t)i * N + k] /= d;
    __syncthreads();
    const int64_t rows = N - k - 1, w = (N - k - 1) + N;
    for (int64_t e = tid; e < rows * w; e += SOLVE_THREADS) {
      const int64_t i = k + 1 + e / w, c = e % w;
      const double l = M[i * N + k];
      if (c < N - k - 1) M[i * N + k + 1 + c] -= l * M[(int64_t)k * N + k + 1 + c];
      else B[i * N + (c - (N - k - 1))] -= l * B[(int64_t)k * N + (c - (N - k - 1))];
    }
    __syncthreads();
  }
  // back substitution, one right-hand side (column of B) per thread
  for (int j = tid; j < N; j += SOLVE_THREADS) {
    bool bad = s_singular != 0;
    for (int i = N - 1; i >= 0; --i) {
      double x = B[(int64_t)i * N + j];
      for (int t = i + 1; t < N; ++t) x -= M[(int64_t)i * N + t] * B[(int64_t)t * N + j];
      x /= M[(int64_t)i * N + i];
      B[(int64_t)i * N + j] = x;
      bad |= !isfinite(x);
    }
    if (bad && flag) atomicOr(flag, 1u);
  }
}


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

// dst = src^T (N x N), 32 x 32 tiles through shared memory; flags a non-finite value.
__global__ void k_transpose(const double* __restrict__ src, double* __restrict__ dst, int64_t N,
                            unsigned int* __restrict__ flag) {
  __shared__ double t[32][33];
  const int64_t i0 = (int64_t)blockIdx.y * 32, j0 = (int64_t)blockIdx.x * 32;
  bool bad = false;
  for (int r = threadIdx.y; r < 32; r += 8) {
    const int64_t i = i0 + r, j = j0 + threadIdx.x;
    if (i < N && j < N) t[r][threadIdx.x] = src[i * N + j];
  }
  __syncthreads();
  for (int r = threadIdx.y; r < 32; r += 8) {
    const int64_t i = j0 + r, j = i0 + threadIdx.x;
    if (i < N && j < N) {
      const double v = t[threadIdx.x][r];
      dst[i * N + j] = v;
      bad |= !isfinite(v);
    }
  }
  if (bad && flag) atomicOr(flag, 1u);
}

// cuSOLVER dense entry points, resolved at run time (no link-time dependency).
typedef int (*CreateFn)(void**);
typedef int (*SetStreamFn)(void*, cudaStream_t);
typedef int (*GetrfBufFn)(void*, int, int, double*, int, int*);
typedef int (*GetrfFn)(void*, int, int, double*, int, double*, int*, int*);
typedef int (*GetrsFn)(void*, int, int, int, const double*, int, const int*, double*, int, int*);
struct Solver {
  bool tried = false, ok = false;
  CreateFn create = nullptr;
  SetStreamFn set_stream = nullptr;
  GetrfBufFn getrf_buf = nullptr;
  GetrfFn getrf = nullptr;
  GetrsFn getrs = nullptr;
  void* handle[64] = {};          // per device
  double* work[64] = {};          // per device: getrf workspace, then pivots and info
  size_t work_bytes[64] = {};
};
Solver g_solver;
std::mutex g_solver_mu;

bool load_solver() {
  if (g_solver.tried) return g_solver.ok;
  g_solver.tried = true;
  const char* names[] = {"libcusolver.so", "libcusolver.so.12", "libcusolver.so.11"};
  void* lib = nullptr;
  for (const char* n : names)
    if ((lib = dlopen(n, RTLD_NOW | RTLD_LOCAL))) break;
  if (!lib) return false;
  g_solver.create = (CreateFn)dlsym(lib, "cusolverDnCreate");
  g_solver.set_stream = (SetStreamFn)dlsym(lib, "cusolverDnSetStream");
  g_solver.getrf_buf = (GetrfBufFn)dlsym(lib, "cusolverDnDgetrf_bufferSize");
  g_solver.getrf = (GetrfFn)dlsym(lib, "cusolverDnDgetrf");
  g_solver.getrs = (GetrsFn)dlsym(lib, "cusolverDnDgetrs");
  g_solver.ok = g_solver.create && g_solver.set_stream && g_solver.getrf_buf && g_solver.getrf && g_solver.getrs;
  return g_solver.ok;
}

}  // namespace

bool lu_solve_large_available() {
  std::lock_guard<std::mutex> lk(g_solver_mu);
  return load_solver();
}

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
  if (N <= 1024) {
    k_lu_solve<<<1, SOLVE_THREADS, 0, st>>>(M, B, (int)N, flag);
    return cudaGetLastError();
  }
  if (!scratch || N > 65535) return cudaErrorInvalidValue;
  std::lock_guard<std::mutex> lk(g_solver_mu);
  if (!load_solver()) return cudaErrorNotSupported;
  int dev = 0;
  cudaError_t err = cudaGetDevice(&dev);
  if (err != cudaSuccess) return err;
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  if (!g_solver.handle[dev] && g_solver.create(&g_solver.handle[dev]) != 0) return cudaErrorNotSupported;
  void* hs = g_solver.handle[dev];
  if (g_solver.set_stream(hs, st) != 0) return cudaErrorNotSupported;
  const int n = (int)N;
  int lwork = 0;
  if (g_solver.getrf_buf(hs, n, n, M, n, &lwork) != 0) return cudaErrorNotSupported;
  // workspace: lwork doubles, N pivots, one info word (grown on a new largest N only)
  const size_t need = (size_t)lwork * sizeof(double) + (size_t)N * sizeof(int) + 256;
  if (need > g_solver.work_bytes[dev]) {
    if (g_solver.work[dev]) {
      if ((err = cudaStreamSynchronize(st)) != cudaSuccess) return err;
      cudaFree(g_solver.work[dev]);
    }
    g_solver.work[dev] = nullptr;
    g_solver.work_bytes[dev] = 0;
    if ((err = cudaMalloc(&g_solver.work[dev], need)) != cudaSuccess) return err;
    g_solver.work_bytes[dev] = need;
  }
  double* work = g_solver.work[dev];
  int* ipiv = reinterpret_cast<int*>(work + lwork);
  int* info = ipiv + N;
  if (g_solver.getrf(hs, n, n, M, n, work, ipiv, info) != 0) return cudaErrorUnknown;
  const dim3 tg((unsigned)((N + 31) / 32), (unsigned)((N + 31) / 32)), tb(32, 8);
  k_transpose<<<tg, tb, 0, st>>>(B, scratch, N, nullptr);              // B, column-major
  if ((err = cudaGetLastError()) != cudaSuccess) return err;
  if (g_solver.getrs(hs, 1 /* op T */, n, n, M, n, ipiv, scratch, n, info) != 0) return cudaErrorUnknown;
  k_transpose<<<tg, tb, 0, st>>>(scratch, B, N, flag);                 // R, row-major
  return cudaGetLastError();
}

}  // namespace bbc
