// complex.cu -- complex A through its real form.
//
// The paper states the problem for A in C^{N x N} (Section 2). The map
// Z -> [[Re Z, -Im Z], [Im Z, Re Z]] sends sums to sums and products to
// products, so exp of the 2N x 2N real form of A is the real form of exp(A):
// the real path (every product kernel, the epilogues, the squarings) runs on
// E = [[Re A, -Im A], [Im A, Re A]] unchanged, and exp(A) is read back from the
// left column blocks. (m, s) still come from the complex ||A||_1 (moduli), as
// the theta rule (eq. theta) asks; this costs twice the flops of complex
// products written out with four real ones, and needs no second set of kernels.
//
// The 1-norm is deterministic: per row slab a partial column sum of moduli,
// then the slabs of each column added in order and the maximum taken.
#include <math.h>

#include <algorithm>

#include "internal.h"

namespace bbc {
namespace {

constexpr int CN_THREADS = 256;
constexpr int CN_MAX_SLABS = 64;

int slabs_of(int64_t N) { return (int)std::min<int64_t>(CN_MAX_SLABS, (N + 63) / 64); }

// partial[s * N + j] = sum of |a_ij| over the rows of slab s
__global__ void k_complex_colsum(const double2* __restrict__ A, int64_t N, int S, double* __restrict__ partial) {
  const int64_t j = (int64_t)blockIdx.x * CN_THREADS + threadIdx.x;
  const int s = blockIdx.y;
  if (j >= N) return;
  const int64_t rows = (N + S - 1) / S, i0 = s * rows, i1 = min(N, i0 + rows);
  double acc = 0.0;
  for (int64_t i = i0; i < i1; ++i) {
    const double2 a = A[i * N + j];
    acc += hypot(a.x, a.y);
  }
  partial[(int64_t)s * N + j] = acc;
}

// *dNorm = max_j sum_s partial[s][j] (a NaN anywhere gives NaN)
__global__ void k_complex_colmax(const double* __restrict__ partial, int64_t N, int S, double* __restrict__ dNorm) {
  __shared__ double red[32];
  double best = 0.0;
  for (int64_t j = threadIdx.x; j < N; j += blockDim.x) {
    double t = 0.0;
    for (int s = 0; s < S; ++s) t += partial[(int64_t)s * N + j];
    best = (t > best || isnan(t)) ? t : best;
  }
  for (int off = 16; off > 0; off >>= 1) {
    const double o = __shfl_xor_sync(0xffffffffu, best, off);
    best = (o > best || isnan(o)) ? o : best;
  }
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = best;
  __syncthreads();
  if (threadIdx.x == 0) {
    double r = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) r = (red[w] > r || isnan(red[w])) ? red[w] : r;
    *dNorm = r;
  }
}

// E (2N x 2N) = [[Re A, -Im A], [Im A, Re A]]
__global__ void k_complex_embed(const double2* __restrict__ A, int64_t N, double* __restrict__ E) {
  const int64_t n2 = 2 * N, total = N * N;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / N, j = e % N;
    const double2 a = A[e];
    E[i * n2 + j] = a.x;
    E[i * n2 + N + j] = -a.y;
    E[(N + i) * n2 + j] = a.y;
    E[(N + i) * n2 + N + j] = a.x;
  }
}

// out = top-left block + i * bottom-left block of E; flags a non-finite value
__global__ void k_complex_extract(const double* __restrict__ E, int64_t N, double2* __restrict__ out,
                                  unsigned int* __restrict__ flag) {
  const int64_t n2 = 2 * N, total = N * N;
  bool bad = false;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / N, j = e % N;
    const double2 v = make_double2(E[i * n2 + j], E[(N + i) * n2 + j]);
    out[e] = v;
    bad |= !isfinite(v.x) || !isfinite(v.y);
  }
  if (bad && flag) atomicOr(flag, 1u);
}

unsigned grid_for(int64_t total) {
  return (unsigned)std::max<int64_t>(1, std::min<int64_t>((total + 255) / 256, 152 * 16));
}

}  // namespace

int64_t complex_norm_partial_len(int64_t N) { return (int64_t)slabs_of(N) * N; }

cudaError_t complex_norm1(const double* A, int64_t N, double* partial, double* dNorm, cudaStream_t st) {
  const int S = slabs_of(N);
  dim3 grid((unsigned)((N + CN_THREADS - 1) / CN_THREADS), (unsigned)S);
  k_complex_colsum<<<grid, CN_THREADS, 0, st>>>(reinterpret_cast<const double2*>(A), N, S, partial);
  k_complex_colmax<<<1, 1024, 0, st>>>(partial, N, S, dNorm);
  return cudaGetLastError();
}

cudaError_t complex_embed(const double* A, int64_t N, double* E, cudaStream_t st) {
  k_complex_embed<<<grid_for(N * N), 256, 0, st>>>(reinterpret_cast<const double2*>(A), N, E);
  return cudaGetLastError();
}

cudaError_t complex_extract(const double* E, int64_t N, double* out, unsigned int* flag, cudaStream_t st) {
  k_complex_extract<<<grid_for(N * N), 256, 0, st>>>(E, N, reinterpret_cast<double2*>(out), flag);
  return cudaGetLastError();
}

}  // namespace bbc
