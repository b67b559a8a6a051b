// elementwise.cu -- the O(N^2) steps: ||A||_1 and product-free linear combinations.
//
// ||A||_1 = max_j sum_i |a_ij| (the norm that drives the choice of (m, s),
// Section 4 and eq. theta). Row-major storage puts a column's entries N apart,
// so each thread owns one column and the 32 threads of a warp read 32 adjacent
// doubles of a row (256 B, coalesced). Rows are split into slabs across
// blockIdx.y so a 4096 x 4096 input fills the GPU; the slab partial sums are
// then added in slab order (deterministic) and the maximum is taken with a warp
// shuffle and a 64-bit atomicMax on the bit pattern, which orders non-negative
// doubles (and a positive NaN above +inf) correctly.
#include "internal.h"

namespace bbc {
namespace {

constexpr int NORM_THREADS = 256;

int64_t slabs_for(int64_t N) {
  // ~2 * 152 SMs worth of blocks, at least 64 rows per slab
  const int64_t colblocks = (N + NORM_THREADS - 1) / NORM_THREADS;
  int64_t slabs = (304 + colblocks - 1) / colblocks;
  const int64_t max_slabs = (N + 63) / 64;
  if (slabs > max_slabs) slabs = max_slabs;
  return slabs < 1 ? 1 : slabs;
}

__global__ void __launch_bounds__(NORM_THREADS)
k_colsum(const double* __restrict__ A, int64_t N, int64_t rows_per, double* __restrict__ partial,
         unsigned int* __restrict__ lower_nz) {
  const int64_t j = (int64_t)blockIdx.x * NORM_THREADS + threadIdx.x;
  if (j >= N) return;
  const int64_t r0 = (int64_t)blockIdx.y * rows_per;
  const int64_t r1 = r0 + rows_per < N ? r0 + rows_per : N;
  double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
  bool below = false;  // a nonzero strictly below the diagonal in this column (rows i > j)
  int64_t i = r0;
  for (; i + 4 <= r1; i += 4) {
    const double a0 = __ldg(A + (i + 0) * N + j), a1 = __ldg(A + (i + 1) * N + j);
    const double a2 = __ldg(A + (i + 2) * N + j), a3 = __ldg(A + (i + 3) * N + j);
    s0 += fabs(a0);
    s1 += fabs(a1);
    s2 += fabs(a2);
    s3 += fabs(a3);
    below |= (i + 0 > j && a0 != 0.0) | (i + 1 > j && a1 != 0.0) | (i + 2 > j && a2 != 0.0) |
             (i + 3 > j && a3 != 0.0);
  }
  for (; i < r1; ++i) {
    const double a = __ldg(A + i * N + j);
    s0 += fabs(a);
    below |= (i > j && a != 0.0);
  }
  partial[(int64_t)blockIdx.y * N + j] = (s0 + s1) + (s2 + s3);
  const unsigned act = __activemask();
  const unsigned any = __ballot_sync(act, below);  // one atomic per warp that saw one
  if (lower_nz && any && (int)(threadIdx.x & 31) == __ffs(act) - 1) atomicOr(lower_nz, 1u);
}

__global__ void __launch_bounds__(NORM_THREADS)
k_colmax(const double* __restrict__ partial, int64_t N, int64_t slabs,
         unsigned long long* __restrict__ out) {
  const int64_t j = (int64_t)blockIdx.x * NORM_THREADS + threadIdx.x;
  double s = 0.0;
  if (j < N)
    for (int64_t r = 0; r < slabs; ++r) s += partial[r * N + j];
  unsigned long long b = (unsigned long long)__double_as_longlong(s);
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    const unsigned long long o = __shfl_xor_sync(0xffffffffu, b, off);
    b = o > b ? o : b;
  }
  if ((threadIdx.x & 31) == 0) atomicMax(out, b);
}

__global__ void k_lincomb(int64_t N, const Epilogue e) {
  const int64_t total = N * N;
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x)
    apply_epilogue(e, N, idx / N, idx % N, 0.0);
}

}  // namespace

int64_t norm1_partial_len(int64_t N) { return slabs_for(N) * N; }

cudaError_t norm1(const double* A, int64_t N, double* partial, double* dNorm, cudaStream_t st,
                  unsigned int* lower_nz) {
  const int64_t slabs = slabs_for(N);
  const int64_t rows_per = (N + slabs - 1) / slabs;
  const unsigned colblocks = (unsigned)((N + NORM_THREADS - 1) / NORM_THREADS);
  cudaError_t err = cudaMemsetAsync(dNorm, 0, sizeof(double), st);
  if (err != cudaSuccess) return err;
  if (lower_nz && (err = cudaMemsetAsync(lower_nz, 0, sizeof(unsigned int), st)) != cudaSuccess) return err;
  k_colsum<<<dim3(colblocks, (unsigned)slabs), NORM_THREADS, 0, st>>>(A, N, rows_per, partial, lower_nz);
  k_colmax<<<colblocks, NORM_THREADS, 0, st>>>(partial, N, slabs, (unsigned long long*)dNorm);
  return cudaGetLastError();
}

cudaError_t lincomb(int64_t N, const Epilogue& e, cudaStream_t st) {
  const int64_t total = N * N;
  int64_t blocks = (total + 255) / 256;
  if (blocks > 152 * 8) blocks = 152 * 8;
  k_lincomb<<<(unsigned)blocks, 256, 0, st>>>(N, e);
  return cudaGetLastError();
}

namespace {

// Upper triangular A: the diagonal and first superdiagonal of exp(2^-q A) in
// closed form (Section 5, concluding remarks): e^{l_i} on the diagonal, and for
// the block [[l1, t], [0, l2]] the divided difference t (e^l2 - e^l1)/(l2 - l1),
// evaluated as t e^((l1+l2)/2) sinh(d)/d with d = (l2 - l1)/2 (no cancellation;
// e^l1 when l1 = l2). Written over T's computed values.
__global__ void k_exact_diag(const double* __restrict__ A, int64_t N, int q, double* __restrict__ T) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  const double l1 = ldexp(A[i * N + i], -q);
  T[i * N + i] = exp(l1);
  if (i + 1 < N) {
    const double l2 = ldexp(A[(i + 1) * N + i + 1], -q);
    const double t = ldexp(A[i * N + i + 1], -q);
    const double d = 0.5 * (l2 - l1);
    const double sinhc = (d == 0.0) ? 1.0 : sinh(d) / d;
    T[i * N + i + 1] = t * exp(0.5 * (l1 + l2)) * sinhc;
  }
}

}  // namespace

cudaError_t exact_diagonals(const double* A, int64_t N, int q, double* T, cudaStream_t st) {
  k_exact_diag<<<(unsigned)((N + 255) / 256), 256, 0, st>>>(A, N, q, T);
  return cudaGetLastError();
}

// A few words from device memory into host memory the device can write directly
// (mapped pinned memory): the host reads a norm or a status word after a stream
// synchronisation without a copy-engine transfer, which would queue behind any
// large device-to-host copy in flight on another stream.
__global__ void k_words_to_host(const uint32_t* __restrict__ src, uint32_t* dst, int words) {
  if ((int)threadIdx.x < words) dst[threadIdx.x] = src[threadIdx.x];
}

cudaError_t copy_to_mapped(void* dst_dev, const void* src, size_t bytes, cudaStream_t st) {
  if (bytes == 0 || bytes % 4 != 0 || bytes > 128) return cudaErrorInvalidValue;
  k_words_to_host<<<1, 32, 0, st>>>(static_cast<const uint32_t*>(src), static_cast<uint32_t*>(dst_dev),
                                    (int)(bytes / 4));
  return cudaGetLastError();
}

}  // namespace bbc

// ---------------------------------------------------------------------------
// ||A||_1 without any allocation, for callers that must not allocate device
// memory at call time (see bbc_norm1_noalloc in the public header).
// The slab partial sums live in this file-scope device array instead of a
// handle's workspace. Every GPU that loads the library holds it (1 MiB) until
// the process exits; all calls share it.
// ---------------------------------------------------------------------------
namespace bbc {

constexpr int64_t NOALLOC_SCRATCH_DOUBLES = 131072;  // 1 MiB
static __device__ __align__(256) double g_norm1_scratch[NOALLOC_SCRATCH_DOUBLES];

bool norm1_noalloc_fits(int64_t N) { return N >= 1 && norm1_partial_len(N) <= NOALLOC_SCRATCH_DOUBLES; }

// In host code the array's name is only a host-side stand-in, so its device
// address on the current device is looked up (with that device current) and
// passed to the kernels. The lookup is repeated on every call rather than
// cached: it is a host-side table read once the module is loaded, and a cached
// address would be stale after a device reset reloads the module. The first
// lookup on a device loads the module, which is why the first call on a device
// must come before any stream capture.
cudaError_t norm1_noalloc(const double* A, int64_t N, double* dNorm, cudaStream_t st) {
  if (!norm1_noalloc_fits(N)) return cudaErrorInvalidValue;
  double* scratch = nullptr;
  const cudaError_t err = cudaGetSymbolAddress((void**)&scratch, g_norm1_scratch);
  if (err != cudaSuccess) return err;
  if (!scratch) return cudaErrorInvalidSymbol;
  // every partial sum the kernels read is written first by the same call, and
  // norm1() clears *dNorm before the maximum is taken: no stale state is used
  return norm1(A, N, scratch, dNorm, st);
}

}  // namespace bbc
