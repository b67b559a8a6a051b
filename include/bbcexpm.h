/*
 * bbcexpm.h -- C ABI of libbbcexpm.so, a GB300 (sm_103a) matrix exponential.
 *
 * Method: Bader, Blanes and Casas, "An improved algorithm to compute the
 * exponential of a matrix" (arXiv:1710.10989). exp(A) = (T_m(A/2^s))^(2^s)
 * (Section 1, eq. eses), with the Taylor polynomial T_m evaluated by the
 * reduced-product scheme of Section 3 (T8 in 3 products, eq. Algorithm83eA;
 * T12 in 4, eq. poly12; T18 in 5, eq. poly.18; T1, T2, T4 in 0, 1, 2) and
 * (m, s) chosen from ||A||_1 and the backward-error thresholds theta_m(u)
 * (eq. theta, Table 2) to minimise the number of products (Table 3).
 *
 * Conventions for every entry point:
 *  - Matrices are square, N x N, row-major, contiguous, IEEE binary64
 *    (unless a dtype argument says otherwise).
 *  - "d" pointers are device pointers on the handle's device; "h" pointers
 *    are host pointers. The caller owns every buffer it passes in.
 *  - Outputs may not alias inputs (BBC_INVALID_ARG, output untouched).
 *  - Work is enqueued on `stream` (a cudaStream_t; NULL = the legacy default
 *    stream). Calls that return a host-side result (bbc_info, a norm) wait
 *    for the stream once at the point that result is needed.
 *  - Every function returns a bbc_status; nothing throws across the ABI.
 *  - The library allocates device memory only in bbc_create, bbc_batch_reserve
 *    and a call whose N (or precision) needs a larger workspace than the
 *    handle holds (it grows then); never inside a stream capture.
 */
#ifndef BBCEXPM_H
#define BBCEXPM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  BBC_OK = 0,
  BBC_INVALID_ARG = 1,      /* null pointer, N <= 0, tol out of range, aliasing, bad flags */
  BBC_NONFINITE_INPUT = 2,  /* A holds a NaN or an infinity (||A||_1 not finite) */
  BBC_OVERFLOW = 3,         /* the result holds a non-finite value */
  BBC_CUDA_ERROR = 4,       /* a CUDA call failed; bbc_last_error() has the text */
  BBC_TIMEOUT = 5,          /* a bounded device-side wait gave up */
  BBC_UNSUPPORTED = 6       /* valid request the library or device cannot serve */
} bbc_status;

/* flags: scheme in bits 0-3, product precision in bits 4-11. */
#define BBC_SCHEME_NEW 0x0     /* reduced-product Taylor, degrees {1,2,4,8,12,18} (Section 3) */
#define BBC_SCHEME_PS 0x1      /* Paterson-Stockmeyer Taylor, degrees {1,2,4,6,9,12,16} (eq. poli9) */
#define BBC_SCHEME_PADE26 0x2  /* diagonal Pade r_26 (eq. pade26), the paper's comparator; its solve
                                  (v - u) R = u + v is an LU with partial pivoting and both triangular
                                  solves on the GPU (the library's own kernels; BBC_UNSUPPORTED beyond
                                  the N whose panels fit a 16-CTA cluster's shared memory, about 13,000) */
#define BBC_SCHEME_PADE 0x3    /* diagonal Pade r_10 (eq. pade10, 3 products) or r_26 (6), whichever costs
                                  fewer products + squarings (the solve is common to both), ties to
                                  the smaller s */
#define BBC_SCHEME_MASK 0xF
#define BBC_PREC_FP64 0x00     /* every product on the FP64 pipe (DFMA) */
#define BBC_PREC_OZAKI 0x10    /* products as exact BF16 slice products on tcgen05 tensor cores,
                                  accumulated exactly; bits 8-11 = slice count k (0 -> 7) */
#define BBC_PREC_SPLIT 0x20    /* the literal split: each operand (row / column scaled by a power of
                                  two) written as k BF16 terms, each the rounding of what the
                                  earlier terms left; the k(k+1)/2 term products with p + q < k
                                  accumulated in FP32 on the tensor cores (bits 8-11 = k, 0 -> 3).
                                  About 8k significant bits per product, no better than FP32 sums
                                  allow (~1e-7 relative); kept to report the plain split beside
                                  the exact one */
#define BBC_PREC_SPLIT_BF16 BBC_PREC_SPLIT
#define BBC_PREC_SPLIT_TF32 0x30  /* the literal split in TF32 terms (the precision config's 2-term TF32
                                     form): each scaled operand written as k TF32 terms (10 explicit
                                     mantissa bits each), the term products with p + q < k accumulated
                                     in FP32 by tcgen05 kind::tf32 MMAs (bits 8-11 = k in 2..4, 0 -> 2).
                                     About 22 significant bits per product at k = 2 */
#define BBC_PREC_FP32 0x40     /* products at binary32 accuracy: three TF32 terms per operand with
                                  FP32 accumulation on the tensor cores (as BBC_PREC_SPLIT_TF32 with
                                  k = 3; the slice-count bits must be 0) */
#define BBC_PREC_MASK 0xF0
/* The four split precisions serve N <= 16384 (2N <= 16384 for bbc_expm_complex, which runs
 * the 2N x 2N real form); beyond it the calls return BBC_UNSUPPORTED before any work. */
#define BBC_OZAKI_SLICES(k) (((k) & 0xF) << 8)
/* bits 16-19: the last n squarings run on the FP64 pipe whatever the product precision
 * (the squarings amplify a product's error 2^s-fold) */
#define BBC_SQUARE_FP64_LAST(n) (((n) & 0xF) << 16)
/* selection of (m, s) (bits 12-13; default: the paper's rule) in bbc_expm_batched and in
 * bbc_expm. bbc_expm runs such a call as a batch of one through the persistent batched
 * kernel (which computes the power-norm estimates, the network and the certificate):
 * it needs bbc_batch_reserve(max_n >= N) (N <= 512), scheme NEW and FP64 products
 * (BBC_UNSUPPORTED otherwise), and for BBC_SELECT_LEARNED an installed network;
 * bbc_info.selector then reports 2 certified by ||A||_1, 3 by alpha_2, 4 fallback to
 * the paper's rule, 5 the alpha rule; no triangular structure is detected there. */
#define BBC_SELECT_LEARNED 0x1000  /* network proposal, certified, else the paper's rule */
#define BBC_SELECT_ALPHA 0x2000    /* cheapest (m, s) certified by ||A|| or alpha_2 (computes A^2, A^3) */
#define BBC_SELECT_MASK 0x3000
/* structure (bits 14-15). By default bbc_expm, bbc_expm_fixed and the host-buffer
 * calls find out, in the 1-norm pass, whether A is upper triangular; if it is,
 * every product runs on the triangles only (entry (i, j) sums k over [i, j]:
 * about a sixth of the dense flops) and the computed diagonal and first
 * superdiagonal are replaced by the exact ones of exp(2^-q A), after the
 * polynomial and after every squaring (Section 5, concluding remarks: the
 * diagonal of exp(A) is exp(a_ii), the superdiagonal a divided difference of
 * exp). bbc_info.structure reports which path ran. The Pade comparator stays dense. */
#define BBC_DENSE 0x4000   /* treat A as dense: no structure detection */
#define BBC_UPPER 0x8000   /* bbc_gemm and bbc_expm_fixed_async only: the caller guarantees
                              the operands are upper triangular; products then sum only k in [i, j] */

typedef struct bbc_handle_s* bbc_handle;

typedef struct {
  int m;          /* degree used: Taylor m, or 2m of the Pade approximant r_2m */
  int s;          /* squarings used */
  int products;   /* dense N x N products performed */
  int selector;   /* 0 = theta rule, 1 = caller-fixed (m, s) */
  double norm1;   /* ||A||_1 as computed on the device */
  int status;     /* bbc_status of this evaluation */
  int structure;  /* 0 dense, 1 upper triangular path */
} bbc_info;

/* Create a handle bound to CUDA device `device`; allocates its device state.
 * Returns BBC_CUDA_ERROR when the device cannot be used. */
int bbc_create(bbc_handle* h, int device);

/* Release a handle and all device memory it owns (NULL is accepted). */
int bbc_destroy(bbc_handle h);

/* Device bytes the handle needs to serve an N x N call with `flags`
 * (dtype is reserved: pass 0 for binary64). */
int bbc_workspace_size(bbc_handle h, int64_t N, int dtype, int flags, size_t* bytes);

/* theta_m(u) for the Taylor polynomial T_m (eq. theta: the root of
 * f(theta)/theta = u, f the 150-term majorant of log(e^-x T_m(x))).
 * Host-only; m in 1..30, u in [2^-60, 2^-5]. */
int bbc_theta(int m, double u, double* theta);

/* theta_2m(u) for the diagonal Pade approximant r_2m (eq. theta with eq. 24,
 * Table 1), 2m even in 2..30. Host-only. */
int bbc_theta_pade(int two_m, double u, double* theta);

/* (m, s) selection (Section 4, Table 2, Table 3): minimise products(m) + s
 * subject to norm1 / 2^s <= theta_m(u), ties to the smaller s. Host-only.
 * `scheme` is BBC_SCHEME_NEW or BBC_SCHEME_PS; BBC_SCHEME_PADE26 gives m = 26
 * and the least s with norm1 / 2^s <= theta_26 (the paper's reference rule);
 * BBC_SCHEME_PADE chooses r_10 (3 products) or r_26 (6) the same way on the
 * Pade thresholds (m = 10 or 26). */
int bbc_select(double norm1, double u, int scheme, int* m, int* s);

/* ||A||_1 = max_j sum_i |a_ij| on the device. Writes the result to host
 * memory *hNorm (waits for the stream). */
int bbc_norm1(bbc_handle h, const double* dA, int64_t N, void* stream, double* hNorm);

/* ||A||_1 into device memory, allocating nothing. The paper has no
 * counterpart: this is a service entry point for callers that must not
 * allocate device memory at call time, for instance a service whose device
 * memory is entirely reserved up front by its own pool, or a latency-critical
 * path where cudaMalloc's implicit synchronisation, or its failure under
 * memory pressure, cannot be tolerated. It needs no handle.
 *  dA     device, N x N row-major binary64 (read only)
 *  dNorm  device, one double; receives ||A||_1 (cleared by the call itself)
 *  N      1 <= N <= 65536; larger N returns BBC_INVALID_ARG before any work
 * Scratch: a fixed 1 MiB array compiled into the library (held on every GPU
 * that loads it until the process exits). Every call looks up that array's
 * device address on the current device; the first lookup on a device loads
 * the library's device code there, so make the first call on a device before
 * any stream capture. All calls share the array:
 * calls that may overlap on the GPU (other streams, other host threads) race
 * and must be serialised by the caller. Returns without waiting for the stream. */
int bbc_norm1_noalloc(const double* dA, int64_t N, double* dNorm, void* stream);

/* dB <- dM^-1 dB: the Pade comparator's linear solve (v - u) R = u + v (eq. pade26,
 * Section 1: "4/3 of a product"), as bbc_expm runs it, exposed for testing and
 * reuse. LU factorisation with partial pivoting (ties to the smaller row) of dM,
 * forward substitution of the N right-hand sides, back substitution: for N <= 112
 * in shared memory, one CTA per 4 right-hand sides; beyond, blocked (32-column
 * panels factored by a thread-block cluster, FP64 rank-32 updates).
 *  dM  device, N x N row-major binary64; overwritten by its LU factors
 *  dB  device, N x N row-major binary64; overwritten by the solution
 * The handle keeps the N pivot indices (allocated on the first call with this N or a
 * larger one). Waits for the stream. BBC_OVERFLOW when dM is singular to working precision or
 * the solution is not finite; BBC_UNSUPPORTED beyond the N the panel clusters hold
 * (about 13,000 on a GPU with 227 KB of shared memory per CTA). */
int bbc_solve(bbc_handle h, double* dM, double* dB, int64_t N, void* stream);

/* dC = dP * dQ (one dense product) with the precision in `flags`. With a split
 * precision (BBC_PREC_OZAKI, BBC_PREC_SPLIT, BBC_PREC_SPLIT_TF32, BBC_PREC_FP32) the
 * call waits for the stream and reports a non-finite operand (BBC_OVERFLOW) or an
 * expired device wait (BBC_TIMEOUT). */
int bbc_gemm(bbc_handle h, const double* dP, const double* dQ, int64_t N, double* dC,
             int flags, void* stream);

/* dT = T_m(2^-s dA) by the scheme in `flags` (no squaring). m must be a
 * degree of that scheme. `products` (may be NULL) receives the count. */
int bbc_taylor(bbc_handle h, const double* dA, int64_t N, int m, int s, double* dT, int flags,
               void* stream, int* products);

/* dOut = exp(dA). tol is the backward-error target u (eq. theta);
 * tol <= 0 selects u = 2^-53. info (may be NULL) receives the outcome.
 * With BBC_SELECT_LEARNED or BBC_SELECT_ALPHA see the selection flags above.
 * Range: the scaling 2^-s is folded into the coefficients, so the first product is
 * formed from A itself; beyond ||A||_1 of about 1.3e154 it overflows and the call
 * returns BBC_OVERFLOW even where exp(A) is finite: scale such an A first,
 * exp(A) = exp(2^-t A)^(2^t). */
int bbc_expm(bbc_handle h, const double* dA, int64_t N, double* dOut, double tol, int flags,
             void* stream, bbc_info* info);

/* Failure-detection self-test: one warp waits, with the bounded wait of the
 * split-product kernel, on a device barrier that nothing ever completes. The
 * wait gives up after about 2 s and reports it through the handle's status
 * word, as a product whose partner CTA never arrived would; *status receives
 * the outcome (BBC_TIMEOUT when the bound works) and the context stays usable.
 * Returns BBC_OK when the call itself ran. Synchronises `stream`. */
int bbc_selftest_wait(bbc_handle h, void* stream, int* status);

/* dOut = exp(dA) for complex A (Section 2 states the problem over C):
 * dA, dOut hold N x N complex numbers row-major with real and imaginary parts
 * interleaved (C99 double complex, numpy / torch complex128), 16-byte aligned,
 * device memory, not overlapping. (m, s) follow the theta rule on the complex
 * 1-norm (column sums of moduli); the products run on the 2N x 2N real form
 * [[Re A, -Im A], [Im A, Re A]] in the precision and scheme of `flags` (real
 * paths unchanged: about twice the flops of complex products), and exp(A) is
 * read back from its left column blocks. bbc_info.norm1 is the complex 1-norm;
 * bbc_info.products counts products of the real form.
 * Errors as bbc_expm; BBC_UPPER is rejected (no triangular path for complex A). */
int bbc_expm_complex(bbc_handle h, const double* dA, int64_t N, double* dOut, double tol, int flags,
                     void* stream, bbc_info* info);

/* As bbc_expm_fixed with no host synchronisation and no allocation while the
 * stream is being captured, so that it can be replayed from a CUDA graph
 * (call it once outside the capture to size the workspace for N and the
 * precision). No norm is read and no structure detected: A is dense unless
 * flags hold BBC_UPPER (the caller's guarantee). dStatus (device word, may be
 * NULL) receives, stream-ordered, bit 0 = a non-finite value in the result
 * (a non-finite input ends there too), bit 1 = a bounded device wait expired.
 * BBC_INVALID_ARG for a capture with too small a workspace, or for a captured
 * Pade comparator (N > 112) on a device where no such solve has run outside a
 * capture yet (its kernels' one-time set-up). */
int bbc_expm_fixed_async(bbc_handle h, const double* dA, int64_t N, double* dOut, int m, int s, int flags,
                         void* stream, unsigned int* dStatus);

/* As bbc_expm with (m, s) fixed by the caller instead of selected. */
int bbc_expm_fixed(bbc_handle h, const double* dA, int64_t N, double* dOut, int m, int s,
                   int flags, void* stream, bbc_info* info);

/* dOut = exp(A) for HOST buffers hA, hOut (pinned memory recommended): the
 * input is copied to the device on `stream`, evaluated as by bbc_expm, and
 * the result copied back; returns after the result is in hOut. The device
 * copies live in the handle's workspace. */
int bbc_expm_host(bbc_handle h, const double* hA, int64_t N, double* hOut, double tol, int flags,
                  void* stream, bbc_info* info);

/* exp(A_i) for `count` matrices in HOST memory (pinned memory recommended),
 * pipelined: while matrix i is evaluated on `stream` (as by bbc_expm), matrix
 * i + 1 is copied to the device and matrix i - 1 back to the host on two copy
 * streams the handle owns, so the copies hide behind the computation.
 *  hA, hOut  host arrays of `count` host pointers; A_i and Out_i are N_i x N_i
 *            row-major binary64 and must not overlap.
 *  Ns        host array of the `count` sizes (N_i >= 1; they may differ).
 *  info      host array of `count` bbc_info, or NULL.
 * The device staging (four max N_i x max N_i buffers) lives in the handle and
 * grows on demand. Stops at the first matrix that fails and returns its status
 * (earlier results are in hOut); returns after every started copy has finished. */
int bbc_expm_host_many(bbc_handle h, const double* const* hA, const int64_t* Ns, int64_t count,
                       double* const* hOut, double tol, int flags, void* stream, bbc_info* info);

/* Element types of bbc_expm_batched. */
#define BBC_DTYPE_F64 0
#define BBC_DTYPE_F32 1

/* Reserve the device workspace bbc_expm_batched needs for matrices up to
 * max_n x max_n (1 <= max_n <= 512) with `flags`, and probe which cluster
 * shapes fit. Allocates; call it before any stream capture of bbc_expm_batched. */
int bbc_batch_reserve(bbc_handle h, int64_t max_n, int flags);

/* Host helper: an order of the `count` matrices with sizes hNs (host array)
 * that puts the largest first (cost grows as N^3), for the work queue of
 * bbc_expm_batched (longest-processing-time-first). hOrder: host, count entries. */
int bbc_batch_order(const int64_t* hNs, int64_t count, int64_t* hOrder);

/* exp(A_i) for `count` independent matrices in one persistent launch (Section 1,
 * eq. eses, per matrix; (m, s) chosen on the device as in bbc_expm).
 *  dA, dOut  DEVICE arrays of `count` device pointers; A_i and Out_i are
 *            N_i x N_i row-major of type dtype (BBC_DTYPE_F32 / F64); the
 *            work runs in binary64 whatever the storage type.
 *  dNs       DEVICE array of the `count` sizes N_i (1 <= N_i <= reserved max_n).
 *  dInfo     DEVICE array of `count` bbc_info (may be NULL): per-matrix m, s,
 *            products, ||A_i||_1 and status (BBC_INVALID_ARG for an N_i beyond
 *            the reservation, BBC_NONFINITE_INPUT, BBC_OVERFLOW).
 * Matrices are taken in array order by whichever CTA is free: put expensive
 * ones first (bbc_batch_order). A batch of at most half as many matrices as
 * SMs runs with a thread-block cluster of 2 to 16 CTAs per matrix, each CTA
 * forming part of every product (bbc_batch_launch_shape reports the choice;
 * the results are bit-identical either way). Needs bbc_batch_reserve first; performs no
 * allocation and no host synchronisation (one memset and one kernel on
 * `stream`), so it can be captured in a CUDA graph. Schemes NEW, and the Pade
 * comparators PADE (r_10 or r_26 by cost) and PADE26, whose solve runs as
 * Gaussian elimination with partial pivoting in one CTA per matrix; the
 * learned and alpha selections serve scheme NEW only.
 * Products: FP64 (BBC_PREC_FP64), or with BBC_PREC_OZAKI (reserved with the
 * same flag) 4 BF16 slices on warp-level tensor-core MMAs with exact FP32
 * slice-group sums (about 32 significant bits per product; N_i <= 256, larger
 * matrices use FP64 products). */
int bbc_expm_batched(bbc_handle h, const void* const* dA, const int64_t* dNs, int64_t count, void* const* dOut,
                     int dtype, double tol, int flags, void* stream, bbc_info* dInfo);

/* Out_i = exp(A_i) B_i for every i: one step Y <- exp(h Omega) Y of an
 * exponential (Lie-group / Magnus) integrator per matrix, in the same
 * persistent launch as bbc_expm_batched (arguments and semantics as there).
 * dB: device array of count device pointers, B_i of the same size and type as
 * A_i. B_i is read before Out_i is written, so Out_i may be B_i (the update in
 * place); Out_i must not overlap A_i. The product with B_i runs in the same
 * precision as the others and counts in bbc_info.products. */
int bbc_expm_apply_batched(bbc_handle h, const void* const* dA, const void* const* dB, const int64_t* dNs,
                           int64_t count, void* const* dOut, int dtype, double tol, int flags, void* stream,
                           bbc_info* dInfo);

/* Autotuner of bbc_expm_batched (needs bbc_batch_reserve with BBC_PREC_OZAKI).
 * Times, on this GPU, calibration batches the library generates itself (entries
 * uniform on [-1, 1), 1-norm about 5, two matrices per resident CTA per size):
 *  1. for every size bucket ((N - 1) / 8 for N <= min(max_n, 256)) the fastest of
 *     split products (32 x 16 or 16 x 16 warp tasks) and FP64 products (64 x 64,
 *     32 x 32 or 16 x 16 output tiles), and
 *  2. the persistent grid, one or two CTAs per SM, on a largest-first mix of all
 *     buckets (eight matrices per resident CTA) with the choices of 1.
 * Keeps the result in the handle for later split-precision batched calls and
 * returns the product family and grid (split_mask: bit b set = bucket b uses split
 * products; ctas: CTA count; the shapes through bbc_batch_get_shapes), so that
 * callers can cache them and restore them with bbc_batch_set_tuning and
 * bbc_batch_set_shapes.
 * Allocates and frees temporary device memory (about 1 GB for max_n = 256 on a
 * 152-SM GPU) and waits for the stream; takes seconds. */
int bbc_batch_tune(bbc_handle h, int64_t max_n, double tol, void* stream, uint32_t* split_mask, int* ctas);

/* Install a tuning (from bbc_batch_tune, possibly cached): ctas 0 = the reserved count. */
int bbc_batch_set_tuning(bbc_handle h, uint32_t split_mask, int ctas);

/* Product shapes of the batched kernel per size bucket b = (N - 1) / 8 (bit b of each
 * mask), as bbc_batch_tune chose them alongside the split mask: for every bucket it
 * times split products in 32 x 16 and 16 x 16 warp tasks and FP64 products in
 * 64 x 64, 32 x 32 and 16 x 16 output tiles and keeps the fastest.
 *  masks[0]  FP64 products in 16 x 16 output tiles
 *  masks[1]  FP64 products in 32 x 32 output tiles (where masks[0] is clear)
 *  masks[2]  split products in 16 x 16 warp tasks (default 32 x 16)
 * All zero: the defaults (the largest tile that gives every CTA sharing a matrix a
 * tile). Results are bit-identical whatever the shapes. host arrays of 3 words; set
 * with NULL restores the defaults. */
int bbc_batch_get_shapes(bbc_handle h, uint32_t* masks);
int bbc_batch_set_shapes(bbc_handle h, const uint32_t* masks);

/* How bbc_expm_batched would launch a batch of `count` matrices (host query, no
 * GPU work): *csize = CTAs sharing each matrix (1, or a thread-block cluster of
 * 2, 4, 8 or 16 CTAs on distinct SMs when the batch is small enough to leave SMs
 * idle at one CTA per matrix) and *grid = CTAs launched. Needs
 * bbc_batch_reserve; BBC_INVALID_ARG for count < 1 or null outputs. */
int bbc_batch_launch_shape(bbc_handle h, int64_t count, int* csize, int* grid);

/* ---- the (m, s)-proposing network (an extension of the method: the paper selects
 * (m, s) from ||A||_1 alone; a proposal is only ever used once the backward-error
 * bound certifies it). A 2-hidden-layer ReLU MLP in FP32 with parameters as one
 * flat device array: W1[hid][in], b1[hid], W2[hid][hid], b2[hid], W3[out][hid],
 * b3[out], row-major. Inputs X are [B][in] row-major; labels are class indices. */

/* Number of floats of the parameter array, and of the activation workspace a
 * batch of B needs (device, caller-owned). */
int bbc_mlp_sizes(int in, int hid, int out, int64_t B, int64_t* n_params, int64_t* ws_floats);

/* dLogits[B][out] = network(dX). dWs: workspace of bbc_mlp_sizes' ws_floats. */
int bbc_mlp_forward(const float* dParams, int in, int hid, int out, const float* dX, int64_t B, float* dLogits,
                    float* dWs, void* stream);

/* Mean softmax cross-entropy over the batch: dGrad (n_params floats) receives its
 * gradient, dLoss[B] the per-sample losses. */
int bbc_mlp_grad(const float* dParams, int in, int hid, int out, const float* dX, const int* dLabels, int64_t B,
                 float* dGrad, float* dLoss, float* dWs, void* stream);

/* One Adam step (bias-corrected, step >= 1) on n parameters in place. */
int bbc_mlp_adam(float* dParams, const float* dGrad, float* dM, float* dV, int64_t n, float lr, float beta1,
                 float beta2, float eps, int step, void* stream);

/* (m, s) certified by the power norms norms3 = {||A||_1, ||A^2||_1, ||A^3||_1}:
 * the cheapest choice with ||A||/2^s <= theta_m or alpha_2/2^s <= theta_m,
 * alpha_2 = max(||A^2||^(1/2), ||A^3||^(1/3)) (a sharper sufficient condition
 * for the same backward-error bound, from the work the paper builds on; the
 * paper itself uses ||A|| only). Host-only. */
int bbc_select_certified(const double* norms3, double u, int scheme, int* m, int* s);

/* Install the network that BBC_SELECT_LEARNED uses on this handle: dParams as
 * for bbc_mlp_forward with in = 5 features [log ||A||_1, three FP32 estimates
 * of log ||A^k||_1^(1/k) for k = 2, 3, 4, log N], normalised as (f - mu) / sd
 * (host arrays of 5); out = 6 * S classes, class c meaning degree index c / S
 * of {1, 2, 4, 8, 12, 18} and s = c % S. The parameters stay caller-owned. */
int bbc_batch_set_selector(bbc_handle h, const float* dParams, int hid, int out, int S, const float* hMu,
                           const float* hSd);

/* Training data for the network, in one persistent launch: per matrix the 5
 * features (dFeat, count x 5 floats) and the exact ||A^k||_1, k = 1..3 from
 * FP64 products (dNorms, count x 4 doubles; the fourth entry is NaN).
 * Arguments as bbc_expm_batched. */
int bbc_selector_data_batched(bbc_handle h, const void* const* dA, const int64_t* dNs, int64_t count, int dtype,
                              float* dFeat, double* dNorms, void* stream, bbc_info* dInfo);

/* Kernel classes for bbc_profile_read. */
#define BBC_KERNEL_PRODUCT 0   /* dense products (with fused epilogues) */
#define BBC_KERNEL_NORM 1      /* the two 1-norm kernels, counted as one class */
#define BBC_KERNEL_LINCOMB 2   /* product-free linear combinations */
#define BBC_KERNEL_SPLIT 3     /* Ozaki slice extraction */
#define BBC_KERNEL_BATCHED 4   /* the persistent batched kernel */
#define BBC_KERNEL_ALL -1

/* Start (enable != 0) or stop per-kernel timing on this handle and reset its
 * counters. While enabled, every kernel launch of the handle is bracketed by a
 * pair of CUDA events recorded on the launch's stream. */
int bbc_profile_enable(bbc_handle h, int enable);

/* Launch count and summed event-measured duration (ms) of one kernel class
 * since bbc_profile_enable; waits for the recorded events. total_ms may be
 * NULL. Launches are counted whether or not timing is enabled. */
int bbc_profile_read(bbc_handle h, int kind, int64_t* launches, double* total_ms);

/* Algorithmic flops of one kernel class since bbc_profile_enable: for products
 * (BBC_KERNEL_PRODUCT) 2 N^3 per dense product and N (N+1) (N+2) / 3 per
 * product of upper triangular operands, whatever precision ran them. */
int bbc_profile_flops(bbc_handle h, int kind, double* flops);

/* Text of the last error on this thread ("" if none). */
const char* bbc_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* BBCEXPM_H */
