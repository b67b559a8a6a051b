// pade.cu -- the linear solve of the diagonal Pade comparator: (v - u) R = u + v
// (eq. pade10 / eq. pade26), by Gaussian elimination with partial pivoting on the
// N right-hand sides at once. One CTA of 1024 threads: the paper counts this
// step as 4/3 of a product, but at the sizes the comparator serves (N <= 1024)
// a single SM suffices; a blocked multi-CTA factorisation is the way to scale.
#include <math.h>

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

}  // namespace

cudaError_t lu_solve_inplace(double* M, double* B, int64_t N, unsigned int* flag, cudaStream_t st) {
  if (N < 1 || N > 1024) return cudaErrorInvalidValue;
  k_lu_solve<<<1, SOLVE_THREADS, 0, st>>>(M, B, (int)N, flag);
  return cudaGetLastError();
}

}  // namespace bbc
