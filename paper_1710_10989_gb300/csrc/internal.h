// internal.h -- declarations shared by the translation units of libbbcexpm.so.
//
// The central abstraction is the fused linear-combination epilogue: every dense
// product of the method is followed by up to MAX_OUT outputs, each a linear
// combination of the product value v, the identity and up to MAX_TERMS matrices
// that are already resident (X, X2, X3, B_j, ...). This is how the reduced-product
// scheme of Section 3 (eq. Algorithm83eA, eq. poly12, eq. poly.18) runs with no
// standalone linear-combination pass: e.g. for T18 the product X6 = X3 X3 emits
// B1..B5 directly, and B1 B5 emits both A9 = B1 B5 + B4 and B3 + A9.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "bbcexpm.h"

namespace bbc {

constexpr int MAX_Y = 6;      // distinct matrices an epilogue may read
constexpr int MAX_OUT = 6;    // outputs one epilogue may write
constexpr int MAX_TERMS = 5;  // matrix terms per output

struct EpiOut {
  double* out;             // destination, N x N row-major
  double cv;               // coefficient of the product value v
  double cI;               // coefficient of the identity
  int nt;                  // number of matrix terms
  int slot[MAX_TERMS];     // index into Epilogue::Y
  double c[MAX_TERMS];     // coefficients
};

struct Epilogue {
  const double* Y[MAX_Y];  // matrices read element-wise by the epilogue
  int ny;                  // how many of Y are used (Y[0..ny-1])
  int nout;
  EpiOut o[MAX_OUT];
  unsigned int* flag;      // if non-null: set to 1 when any output is not finite
};

// Element (row, col) of every output of the epilogue, given v = alpha * (P Q)_rc.
// TERMS = false: the outputs have no matrix terms (e.ny == 0: a squaring, a plain
// product). TERMS = true: the element of every matrix the outputs read is loaded
// once, all loads issued together, before any output is formed (a step such as
// T18's X6 = X3 X3, whose five outputs B1..B5 read X, X2, X3 three terms each, then
// waits for three loads in flight instead of fifteen one after another); an output
// written to one of those matrices is seen by the outputs after it.
template <bool TERMS>
__device__ __forceinline__ void apply_epilogue_t(const Epilogue& e, int64_t N, int64_t row, int64_t col, double v) {
  const int64_t idx = row * N + col;
  double y[MAX_Y];
  if (TERMS) {
#pragma unroll
    for (int k = 0; k < MAX_Y; ++k) y[k] = (k < e.ny) ? __ldg(e.Y[k] + idx) : 0.0;
  }
  bool bad = false;
#pragma unroll 1
  for (int o = 0; o < e.nout; ++o) {
    const EpiOut& q = e.o[o];
    double r = q.cv * v;
    if (row == col) r += q.cI;
    if (TERMS) {
#pragma unroll 1
      for (int t = 0; t < q.nt; ++t) {
        const int sl = q.slot[t];
        double yv = y[0];
#pragma unroll
        for (int k = 1; k < MAX_Y; ++k) yv = (sl == k) ? y[k] : yv;
        r = fma(q.c[t], yv, r);
      }
    }
    q.out[idx] = r;
    bad |= !isfinite(r);
    if (TERMS) {
#pragma unroll
      for (int k = 0; k < MAX_Y; ++k)
        if (k < e.ny && e.Y[k] == q.out) y[k] = r;
    }
  }
  if (bad && e.flag) atomicOr(e.flag, 1u);
}

// Either form, chosen per element at run time (kernels where the choice is not a
// template parameter).
__device__ __forceinline__ void apply_epilogue(const Epilogue& e, int64_t N, int64_t row, int64_t col, double v) {
  if (e.ny == 0) apply_epilogue_t<false>(e, N, row, col, v);
  else apply_epilogue_t<true>(e, N, row, col, v);
}

// Element (row, col) of every output when it is known to be zero: below the
// diagonal of a product of upper triangular matrices, where v, the identity and
// every matrix term of an epilogue vanish.
__device__ __forceinline__ void zero_epilogue(const Epilogue& e, int64_t N, int64_t row, int64_t col) {
  const int64_t idx = row * N + col;
#pragma unroll 1
  for (int o = 0; o < e.nout; ++o) e.o[o].out[idx] = 0.0;
}

// FP64 DFMA product with fused epilogue: v = alpha * (P Q). upper: P and Q are
// upper triangular, so entry (i, j) sums k over [i, j] only and blocks strictly
// below the diagonal skip the sum (their outputs come from the epilogue alone).
cudaError_t gemm_f64(const double* P, const double* Q, int64_t N, double alpha, const Epilogue& e,
                     cudaStream_t st, bool upper = false);

// Element-wise linear combination (no product): outputs of `e` with v = 0.
cudaError_t lincomb(int64_t N, const Epilogue& e, cudaStream_t st);

// ||A||_1 into *dNorm (device). `partial` must hold norm1_partial_len(N) doubles.
// lower_nz (device word, may be null) is set to 1 if A has a nonzero strictly
// below the diagonal, 0 otherwise.
int64_t norm1_partial_len(int64_t N);
cudaError_t norm1(const double* A, int64_t N, double* partial, double* dNorm, cudaStream_t st,
                  unsigned int* lower_nz = nullptr);

// `bytes` (a multiple of 4, at most 128) from device memory `src` to `dst_dev`, the
// device address of mapped pinned host memory, by a one-warp kernel on `st`.
cudaError_t copy_to_mapped(void* dst_dev, const void* src, size_t bytes, cudaStream_t st);

// Upper triangular A: overwrite the diagonal and first superdiagonal of T with
// those of exp(2^-q A), known in closed form (Section 5, concluding remarks).
cudaError_t exact_diagonals(const double* A, int64_t N, int q, double* T, cudaStream_t st);

// ||A||_1 with the slab sums in a static device array instead of a workspace
// (no allocation); false / cudaErrorInvalidValue when N exceeds its capacity.
bool norm1_noalloc_fits(int64_t N);
cudaError_t norm1_noalloc(const double* A, int64_t N, double* dNorm, cudaStream_t st);

// Ozaki split products on tcgen05 (gemm_ozaki.cu). `flag` is the handle's
// status word: bit 0 = an operand held a non-finite value, bit 1 = a bounded
// device wait expired.
// ozaki_split writes the slice planes and scales of P (rows) and Q (columns)
// into `work`; ozaki_product then forms alpha * (P Q) from them with the
// fused epilogue.
// `slices` counts BF16 planes; a TF32 plane takes the room of two.
size_t ozaki_workspace_bytes(int64_t N, int slices);
// Split modes: the exact BF16 digits, or the plain floating-point split (each term
// the rounding of the remainder: BF16 for BBC_PREC_SPLIT, TF32 for
// BBC_PREC_SPLIT_TF32 and BBC_PREC_FP32) with every term product accumulated in FP32.
enum SplitMode { SPLIT_EXACT = 0, SPLIT_LITERAL_BF16 = 1, SPLIT_LITERAL_TF32 = 2 };
// upper: P and Q are upper triangular; only the plane regions a triangle product reads are
// written (rows of P from their tile row's first K step, columns of Q to their tile
// column's last), and the exponent scans skip the zero triangles.
cudaError_t ozaki_split(const double* P, const double* Q, int64_t N, int slices, void* work,
                        unsigned int* flag, cudaStream_t st, int mode = SPLIT_EXACT, bool upper = false);
cudaError_t ozaki_product(const double* P, const double* Q, int64_t N, double alpha, const Epilogue& e,
                          int slices, void* work, unsigned int* flag, cudaStream_t st, bool upper = false,
                          int mode = SPLIT_EXACT);
bool ozaki_supported(int64_t N);
// One warp waits, with the product kernel's bounded wait, on an mbarrier that
// nothing arrives at; about 2 s later bit 1 (timeout) of *status is set.
cudaError_t wait_selftest(unsigned int* status, cudaStream_t st);

// Complex A (interleaved real and imaginary parts, N x N row-major, 16-byte
// aligned) through its real form E = [[Re A, -Im A], [Im A, Re A]] (complex.cu).
// complex_norm1 needs complex_norm_partial_len(N) doubles of `partial`.
int64_t complex_norm_partial_len(int64_t N);
cudaError_t complex_norm1(const double* A, int64_t N, double* partial, double* dNorm, cudaStream_t st);
cudaError_t complex_embed(const double* A, int64_t N, double* E, cudaStream_t st);
cudaError_t complex_extract(const double* E, int64_t N, double* out, unsigned int* flag, cudaStream_t st);

// Solve M X = B in place (X overwrites B, M is destroyed) (pade.cu). N > 112 runs
// the blocked LU (lu_blocked.cu), which keeps its N pivot indices in `scratch`
// (at least N ints; an N x N matrix of the workspace serves). No allocation.
cudaError_t lu_solve_inplace(double* M, double* B, int64_t N, unsigned int* flag, cudaStream_t st,
                             double* scratch = nullptr);
// The blocked LU with partial pivoting and both triangular solves (lu_blocked.cu);
// lu_blocked_max_n: the largest N its cluster-resident panels allow on this device.
cudaError_t lu_blocked_solve(double* M, double* B, int64_t N, unsigned int* flag, cudaStream_t st, void* scratch);
int64_t lu_blocked_max_n();
// Whether the blocked LU's one-time device set-up (kernel attributes, cluster
// occupancy) has run on the current device; it must run outside any stream capture.
bool lu_blocked_ready();

// The (m, s)-proposing MLP (mlp.cu).
int64_t mlp_param_count(int n_in, int hid, int n_out);
int64_t mlp_workspace_floats(int hid, int n_out, int64_t B);
cudaError_t mlp_forward(const float* P, int n_in, int hid, int n_out, const float* X, int64_t B, float* logits,
                        float* ws, cudaStream_t st);
cudaError_t mlp_grad(const float* P, int n_in, int hid, int n_out, const float* X, const int* y, int64_t B,
                     float* grad, float* loss, float* ws, cudaStream_t st);
cudaError_t mlp_adam(float* P, const float* g, float* m, float* v, int64_t n, float lr, float b1, float b2,
                     float eps, int step, cudaStream_t st);

// Persistent batched exp(A) (batched.cu).
size_t batched_workspace_bytes(int64_t nmax, int ctas, bool split);
int batched_ctas(int device);
cudaError_t batched_upload_programs();
struct BatchSelector {
  int mode;                 // 1 learned, 2 alpha rule, 3 training data
  const float* params;      // network parameters (learned)
  int hid, out, S;          // hidden width, classes, s values per degree
  float mu[5], sd[5];       // feature normalisation
  float* feat_out;          // training data: count x 5
  double* norms_out;        // training data: count x 4
};
// Small batches (at most half as many matrices as SMs) may run with a cluster of
// CTAs per matrix; the shapes that fit are probed once, outside stream capture.
struct BatchClusters {
  int sms = 0;              // 0: no cluster mode
  int dyn_smem = 0;         // dynamic shared memory per CTA that keeps one CTA per SM
  int max_active[5] = {};   // resident clusters of 2^i CTAs (index 0 unused)
};
cudaError_t batched_cluster_probe(int device, BatchClusters* out);
// Product shapes per size bucket b = (N - 1) / 8 (bit b of each mask), chosen by the
// autotuner; all zero = the defaults. Results do not depend on them (every output
// element sums the same terms in the same order).
struct BatchShapes {
  uint32_t f64_tile16 = 0;     // FP64 products in 16 x 16 output tiles
  uint32_t f64_tile32 = 0;     // FP64 products in 32 x 32 output tiles (unless tile16)
  uint32_t split_task16 = 0;   // split products in 16 x 16 warp tasks (default 32 x 16)
};
int batched_cluster_size(const BatchClusters* cl, int64_t count, int ctas, int* grid);
cudaError_t batched_launch(const void* const* A, void* const* Out, const int64_t* Ns, int64_t count,
                           int64_t nmax, int dtype, const double* theta, void* work, int ctas,
                           bbc_info* info, cudaStream_t st, const BatchSelector* sel = nullptr,
                           bool split = false, uint32_t split_mask = 0xFFFFFFFFu,
                           const BatchClusters* cl = nullptr, const void* const* B = nullptr,
                           int pade = 0, const double* theta_pade = nullptr, const BatchShapes* shapes = nullptr);
// count N x N binary64 calibration matrices (uniform entries, 1-norm about norm1).
cudaError_t calibration_matrices(double* out, int64_t N, int64_t count, uint64_t seed, double norm1, cudaStream_t st);

}  // namespace bbc
