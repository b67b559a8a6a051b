// api.cu -- the C ABI of libbbcexpm.so (include/bbcexpm.h): handle and
// workspace, backward-error thresholds, (m, s) selection, program execution and
// the squaring chain of scaling and squaring (eq. eses).
#include <cmath>
#include <cstddef>
#include <cstdio>
#include <cstring>
#include <algorithm>
#include <map>
#include <mutex>
#include <string>
#include <utility>
#include <vector>

#include "bbcexpm.h"
#include "internal.h"
#include "schemes.h"
#include "squarings.h"

using namespace bbc;

struct bbc_handle_s {
  int device = 0;
  int64_t slots_n = 0;            // N the work slots are sized for
  double* work = nullptr;         // NUM_WORK_SLOTS * N * N doubles
  int64_t partial_len = 0;
  double* partial = nullptr;      // norm slab sums
  double* dnorm = nullptr;        // device ||A||_1
  unsigned int* dflag = nullptr;  // device non-finite flag
  unsigned int* dlower = nullptr; // device: A has a nonzero below its diagonal
  void* hstage = nullptr;         // mapped pinned host staging: [0] norm, [1] flag, [2] lower flag
  void* hstage_dev = nullptr;     // its device address (null: not mapped, copies go through memcpy)
  void* ozaki = nullptr;          // Ozaki slice workspace
  size_t ozaki_bytes = 0;
  // profiling: launch counters per kernel class and, when enabled, event pairs
  int64_t launches[5] = {0, 0, 0, 0, 0};
  double flops[5] = {0, 0, 0, 0, 0};   // algorithmic FP64-product flops per class
  bool prof = false;
  struct Rec { int kind; cudaEvent_t a, b; };
  std::vector<Rec> recs;       // recorded in this profiling window
  std::vector<cudaEvent_t> pool;
  int64_t batch_nmax = 0;         // reservation of the batched workspace
  BatchSelector selector = {};    // network for BBC_SELECT_LEARNED (mode 0: none installed)
  int batch_ctas = 0;
  bool batch_split = false;       // reservation includes the split-precision scratch
  uint32_t batch_split_mask = 0xFFFFFFFFu;  // tuned: size buckets ((N-1)/8) that use split products
  int batch_grid = 0;                       // tuned persistent CTA count (0: the reserved count)
  BatchShapes batch_shapes;                 // tuned product shapes per size bucket
  BatchClusters batch_cl;                   // cluster shapes for small batches
  double* cplx = nullptr;         // complex calls: two (2N)^2 real forms and the norm partials
  int64_t cplx_n = 0;
  void* batch_work = nullptr;
  // bbc_expm with a certified selection runs as a batch of one: its device descriptor
  // (pointers, size, bbc_info) and the pinned host copy it is filled from
  void* one_dev = nullptr;
  void* one_host = nullptr;
  int* piv = nullptr;             // bbc_solve: the blocked LU's N pivot indices
  int64_t piv_n = 0;
  int64_t io_n = 0;               // N the host-call staging buffers are sized for
  double* io = nullptr;           // 4 * N * N doubles: device copies of two inputs and two outputs
  cudaStream_t copy_in = nullptr;   // host-call pipeline: host -> device copies
  cudaStream_t copy_out = nullptr;  // host-call pipeline: device -> host copies
  cudaEvent_t ev_in[2] = {nullptr, nullptr};
  cudaEvent_t ev_out[2] = {nullptr, nullptr};
  std::mutex mu;
};

namespace {

thread_local std::string g_err;

// Descriptor of a batch of one (bbc_expm with a certified selection).
struct OneDesc {
  const void* a;
  void* out;
  int64_t n;
  bbc_info info;
};
constexpr size_t ONE_DESC_BYTES = 256;
static_assert(sizeof(OneDesc) <= ONE_DESC_BYTES, "descriptor room");
int batched_locked(bbc_handle h, const void* const* dA, const void* const* dB, const int64_t* dNs, int64_t count,
                   void* const* dOut, int dtype, double u, int flags, cudaStream_t st, bbc_info* dInfo);

// Products rebuilt from slices on the tensor cores: the exact form (BBC_PREC_OZAKI,
// default 7 BF16 slices) or the literal split in BF16 terms (BBC_PREC_SPLIT, default 3)
// or TF32 terms (BBC_PREC_SPLIT_TF32, default 2; BBC_PREC_FP32 = 3 TF32 terms).
bool split_prec(int flags) {
  const int prec = flags & BBC_PREC_MASK;
  return prec == BBC_PREC_OZAKI || prec == BBC_PREC_SPLIT || prec == BBC_PREC_SPLIT_TF32 || prec == BBC_PREC_FP32;
}
int split_mode(int flags) {
  const int prec = flags & BBC_PREC_MASK;
  if (prec == BBC_PREC_SPLIT_TF32 || prec == BBC_PREC_FP32) return SPLIT_LITERAL_TF32;
  return prec == BBC_PREC_SPLIT ? SPLIT_LITERAL_BF16 : SPLIT_EXACT;
}
int split_slices(int flags) {
  const int prec = flags & BBC_PREC_MASK;
  if (prec == BBC_PREC_FP32) return 3;
  const int k = (flags >> 8) & 0xF;
  if (k) return k;
  return prec == BBC_PREC_SPLIT ? 3 : prec == BBC_PREC_SPLIT_TF32 ? 2 : 7;
}
// Workspace room in BF16 planes (a TF32 plane takes two).
int split_planes(int flags) {
  return split_slices(flags) * (split_mode(flags) == SPLIT_LITERAL_TF32 ? 2 : 1);
}

int fail(int code, const std::string& msg) {
  g_err = msg;
  return code;
}

int cuda_fail(cudaError_t e, const char* where) {
  return fail(BBC_CUDA_ERROR, std::string(where) + ": " + cudaGetErrorString(e));
}

#define BBC_CUDA(call)                                     \
  do {                                                     \
    cudaError_t e_ = (call);                               \
    if (e_ != cudaSuccess) return cuda_fail(e_, #call);    \
  } while (0)

// ---------------------------------------------------------------------------
// theta_m(u), eq. (theta): theta is the root of f(theta)/theta = u where
// f(x) = sum |c_i| x^i majorises rho(x) = log(e^-x T_m(x)) = sum c_i x^i,
// truncated to the 150 terms i = m+1 .. m+150.
// Series of h(x) = e^-x T_m(x): h_0 = 1, h_j = 0 for 1 <= j <= m, and for j > m
//   h_j = (-1)^(j+m) / (j * m! * (j-1-m)!)
// (the partial alternating binomial sum identity); rho = log h by the usual
// recurrence n rho_n = n h_n - sum_{k=1}^{n-1} k rho_k h_{n-k}.
// ---------------------------------------------------------------------------
double factorial(int n) {  // n <= 181 stays finite in binary64
  double f = 1.0;
  for (int k = 2; k <= n; ++k) f *= k;
  return f;
}

double compute_theta(int m, double u) {
  const int K = m + 151;
  std::vector<double> h(K, 0.0), g(K, 0.0);
  h[0] = 1.0;
  const double mf = factorial(m);
  for (int j = m + 1; j < K; ++j) {
    const double mag = 1.0 / ((double)j * mf * factorial(j - 1 - m));
    h[j] = ((j + m) % 2 == 0) ? mag : -mag;
  }
  for (int n = 1; n < K; ++n) {
    double acc = n * h[n];
    for (int k = m + 1; k < n; ++k) acc -= k * g[k] * h[n - k];
    g[n] = acc / n;
  }
  auto f_over_x = [&](double x) {
    double acc = 0.0, p = std::pow(x, m);  // x^(i-1) at i = m+1
    for (int i = m + 1; i < K; ++i) {
      acc += std::fabs(g[i]) * p;
      p *= x;
    }
    return acc;
  };
  double lo = 0.0, hi = 1.0;
  while (f_over_x(hi) < u) hi *= 2.0;
  for (int it = 0; it < 200; ++it) {
    const double mid = 0.5 * (lo + hi);
    if (mid == lo || mid == hi) break;
    if (f_over_x(mid) < u) lo = mid; else hi = mid;
  }
  return lo;
}

// ---------------------------------------------------------------------------
// theta_2m(u) for the diagonal Pade approximant r_2m (eq. 24, eq. theta). The
// series rho(x) = log(e^-x r_2m(x)) starts at x^(2m+1), and its coefficients come
// from a sum whose terms cancel by ~10 orders of magnitude for m = 13, so they
// are formed in double-double arithmetic (deterministic on every host):
//   N(x) = e^-x p_m(x) - p_m(-x) (first term at x^(2m+1)), q = N / p_m(-x),
//   rho = log(1 + q) = q - q^2/2 + ...  (q^3 starts beyond the 150 terms used).
// ---------------------------------------------------------------------------
struct DD { double hi, lo; };
DD dd_two_sum(double a, double b) {
  const double s = a + b, bb = s - a;
  return {s, (a - (s - bb)) + (b - bb)};
}
DD dd_norm(double hi, double lo) {
  const double s = hi + lo;
  return {s, lo - (s - hi)};
}
DD dd_add(DD a, DD b) {
  DD s = dd_two_sum(a.hi, b.hi);
  return dd_norm(s.hi, s.lo + a.lo + b.lo);
}
DD dd_mul(DD a, DD b) {
  const double p = a.hi * b.hi;
  const double e = std::fma(a.hi, b.hi, -p);
  return dd_norm(p, e + (a.hi * b.lo + a.lo * b.hi));
}
DD dd_div(DD a, double d) {  // a / d for an exact double d
  const double q1 = a.hi / d;
  const double r = std::fma(-q1, d, a.hi) + a.lo;
  return dd_norm(q1, r / d);
}
DD dd_neg(DD a) { return {-a.hi, -a.lo}; }

double compute_theta_pade(int two_m, double u) {
  const int m = two_m / 2;
  const int K = two_m + 151;
  std::vector<DD> invf(K + 1), p(m + 1), n(K, DD{0, 0}), q(K, DD{0, 0});
  invf[0] = {1.0, 0.0};
  for (int k = 1; k <= K; ++k) invf[k] = dd_div(invf[k - 1], (double)k);
  for (int j = 0; j <= m; ++j) {  // p_j = prod_{t<j} (m-t)/(2m-t) / j!
    DD v = invf[j];
    for (int t = 0; t < j; ++t) v = dd_div(dd_mul(v, DD{(double)(m - t), 0.0}), (double)(2 * m - t));
    p[j] = v;
  }
  for (int k = two_m + 1; k < K; ++k) {
    DD acc = {0.0, 0.0};
    for (int j = 0; j <= m; ++j) {
      const DD t = dd_mul(p[j], invf[k - j]);
      acc = dd_add(acc, ((k - j) % 2) ? dd_neg(t) : t);
    }
    n[k] = acc;
  }
  for (int k = 0; k < K; ++k) {  // q = N / p(-x), p(-x)_j = (-1)^j p_j
    DD acc = n[k];
    for (int j = 1; j <= m && j <= k; ++j) {
      const DD t = dd_mul(p[j], q[k - j]);
      acc = dd_add(acc, (j % 2) ? t : dd_neg(t));
    }
    q[k] = acc;
  }
  std::vector<double> rho(K, 0.0);
  for (int i = 0; i < K; ++i) rho[i] = q[i].hi;
  for (int i = two_m + 1; i < K; ++i)
    for (int j = two_m + 1; i + j < K; ++j) rho[i + j] -= 0.5 * q[i].hi * q[j].hi;
  auto f_over_x = [&](double x) {
    double acc = 0.0, pw = std::pow(x, two_m);  // x^(i-1) at i = 2m+1
    for (int i = two_m + 1; i < K; ++i) {
      acc += std::fabs(rho[i]) * pw;
      pw *= x;
    }
    return acc;
  };
  double lo = 0.0, hi = 1.0;
  while (f_over_x(hi) < u) hi *= 2.0;
  for (int it = 0; it < 200; ++it) {
    const double mid = 0.5 * (lo + hi);
    if (mid == lo || mid == hi) break;
    if (f_over_x(mid) < u) lo = mid; else hi = mid;
  }
  return lo;
}

std::mutex g_theta_mu;
std::map<std::pair<int, double>, double> g_theta_cache;

// m > 0: Taylor degree m; m < 0: Pade order 2|m|... encoded as -two_m
double theta_cached(int m, double u) {
  std::lock_guard<std::mutex> lk(g_theta_mu);
  auto key = std::make_pair(m, u);
  auto it = g_theta_cache.find(key);
  if (it != g_theta_cache.end()) return it->second;
  const double t = m > 0 ? compute_theta(m, u) : compute_theta_pade(-m, u);
  g_theta_cache[key] = t;
  return t;
}

bool valid_u(double u) { return std::isfinite(u) && u >= std::ldexp(1.0, -60) && u <= std::ldexp(1.0, -5); }

int select_ms(double norm, double u, int scheme, int* m, int* s) {
  if (scheme == BBC_SCHEME_PADE26) {  // the paper's reference method: r_26, s from theta_26
    *m = 26;
    *s = least_squarings(norm, theta_cached(-26, u));
    return BBC_OK;
  }
  const bool pade = scheme == BBC_SCHEME_PADE;  // thresholds of r_2m, negative keys in the cache
  const int *deg, *prod;
  const int cnt = scheme_degrees(scheme, &deg, &prod);
  int bm = -1, bs = 0, bc = 1 << 30;
  for (int i = 0; i < cnt; ++i) {
    const int si = least_squarings(norm, theta_cached(pade ? -deg[i] : deg[i], u));
    const int cost = prod[i] + si;
    if (cost < bc || (cost == bc && si < bs)) { bc = cost; bm = deg[i]; bs = si; }
  }
  *m = bm;
  *s = bs;
  return BBC_OK;
}

// ---------------------------------------------------------------------------
// workspace
// ---------------------------------------------------------------------------
int ensure_workspace(bbc_handle h, int64_t N, int flags) {
  if (split_prec(flags) && !ozaki_supported(N))
    return fail(BBC_UNSUPPORTED, "split-precision products take N <= 16384");
  BBC_CUDA(cudaSetDevice(h->device));
  if (N > h->slots_n) {
    if (h->work) BBC_CUDA(cudaFree(h->work));
    if (h->partial) BBC_CUDA(cudaFree(h->partial));
    h->work = nullptr;
    h->partial = nullptr;
    h->slots_n = 0;
    BBC_CUDA(cudaMalloc(&h->work, (size_t)NUM_WORK_SLOTS * N * N * sizeof(double)));
    h->partial_len = norm1_partial_len(N);
    BBC_CUDA(cudaMalloc(&h->partial, (size_t)h->partial_len * sizeof(double)));
    h->slots_n = N;
  }
  if (split_prec(flags)) {
    const size_t need = ozaki_workspace_bytes(N, split_planes(flags));
    if (need > h->ozaki_bytes) {
      if (h->ozaki) BBC_CUDA(cudaFree(h->ozaki));
      h->ozaki = nullptr;
      h->ozaki_bytes = 0;
      BBC_CUDA(cudaMalloc(&h->ozaki, need));
      h->ozaki_bytes = need;
    }
  }
  return BBC_OK;
}

cudaEvent_t take_event(bbc_handle h) {
  if (!h->pool.empty()) {
    cudaEvent_t e = h->pool.back();
    h->pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
  return e;
}

// Brackets one kernel launch: counts it and, if profiling, records events.
struct LaunchScope {
  bbc_handle h;
  int kind;
  cudaStream_t st;
  cudaEvent_t a = nullptr;
  LaunchScope(bbc_handle h_, int kind_, cudaStream_t st_) : h(h_), kind(kind_), st(st_) {
    // the 1-norm is two kernels; a split is three (row split, column maxima, column split)
    h->launches[kind] += (kind == BBC_KERNEL_NORM) ? 2 : (kind == BBC_KERNEL_SPLIT) ? 3 : 1;
    if (h->prof && (a = take_event(h))) cudaEventRecord(a, st);
  }
  ~LaunchScope() {
    if (!a) return;
    cudaEvent_t b = take_event(h);
    if (!b) { h->pool.push_back(a); return; }
    cudaEventRecord(b, st);
    h->recs.push_back({kind, a, b});
  }
};

double* slot_ptr(bbc_handle h, int slot, int64_t N, const double* A, double* T) {
  if (slot == SL_A) return const_cast<double*>(A);
  if (slot == SL_T) return T;
  return h->work + (size_t)slot * N * N;
}

// One dense product alpha * (P Q) with its fused epilogue, at the precision in flags.
int launch_product(bbc_handle h, const double* P, const double* Q, int64_t N, double alpha, const Epilogue& e,
                   int flags, cudaStream_t stream, bool upper) {
  cudaError_t err;
  // algorithmic work: 2 N^3, or for upper triangular operands 2 sum_{i<=j} (j - i + 1) = N(N+1)(N+2)/3
  const double n = (double)N;
  h->flops[BBC_KERNEL_PRODUCT] += upper ? n * (n + 1) * (n + 2) / 3.0 : 2.0 * n * n * n;
  if (split_prec(flags)) {
    const int k = split_slices(flags);
    const int mode = split_mode(flags);
    {
      LaunchScope scope(h, BBC_KERNEL_SPLIT, stream);
      err = ozaki_split(P, Q, N, k, h->ozaki, h->dflag, stream, mode, upper);
    }
    if (err != cudaSuccess) return cuda_fail(err, "split launch");
    LaunchScope scope(h, BBC_KERNEL_PRODUCT, stream);
    err = ozaki_product(P, Q, N, alpha, e, k, h->ozaki, h->dflag, stream, upper, mode);
  } else {
    LaunchScope scope(h, BBC_KERNEL_PRODUCT, stream);
    err = gemm_f64(P, Q, N, alpha, e, stream, upper);
  }
  if (err != cudaSuccess) return cuda_fail(err, "product launch");
  return BBC_OK;
}

// One product (or linear combination) with its fused epilogue.
int run_step(bbc_handle h, const StepS& st, int64_t N, const double* A, double* T, int flags,
             unsigned int* flag, cudaStream_t stream, bool upper = false) {
  Epilogue e{};
  int ny = 0;
  e.nout = st.nout;
  e.flag = flag;
  for (int o = 0; o < st.nout; ++o) {
    const OutS& q = st.o[o];
    e.o[o].out = slot_ptr(h, q.dst, N, A, T);
    e.o[o].cv = q.cv;
    e.o[o].cI = q.cI;
    e.o[o].nt = q.nt;
    for (int t = 0; t < q.nt; ++t) {
      const double* y = slot_ptr(h, q.t[t].slot, N, A, T);
      int k = 0;
      while (k < ny && e.Y[k] != y) ++k;
      if (k == ny) {
        if (ny == MAX_Y) return fail(BBC_INVALID_ARG, "epilogue reads too many matrices");
        e.Y[ny++] = y;
      }
      e.o[o].slot[t] = k;
      e.o[o].c[t] = q.t[t].c;
    }
  }
  e.ny = ny;
  if (st.P < 0) {
    LaunchScope scope(h, BBC_KERNEL_LINCOMB, stream);
    const cudaError_t err = lincomb(N, e, stream);
    if (err != cudaSuccess) return cuda_fail(err, "lincomb launch");
    return BBC_OK;
  }
  const double* P = slot_ptr(h, st.P, N, A, T);
  const double* Q = slot_ptr(h, st.Q, N, A, T);
  return launch_product(h, P, Q, N, st.alpha, e, flags, stream, upper);
}

int check_flags(int flags) {
  const int scheme = flags & BBC_SCHEME_MASK;
  const int prec = flags & BBC_PREC_MASK;
  if (scheme != BBC_SCHEME_NEW && scheme != BBC_SCHEME_PS && scheme != BBC_SCHEME_PADE26 && scheme != BBC_SCHEME_PADE)
    return fail(BBC_INVALID_ARG, "unknown scheme");
  if (prec != BBC_PREC_FP64 && prec != BBC_PREC_OZAKI && prec != BBC_PREC_SPLIT && prec != BBC_PREC_SPLIT_TF32 &&
      prec != BBC_PREC_FP32)
    return fail(BBC_INVALID_ARG, "unknown precision");
  if (flags & ~0xFFFFF) return fail(BBC_INVALID_ARG, "unknown flag bits");
  if ((flags & BBC_SELECT_MASK) == BBC_SELECT_MASK) return fail(BBC_INVALID_ARG, "two selectors requested");
  if (prec == BBC_PREC_OZAKI || prec == BBC_PREC_SPLIT) {
    const int k = (flags >> 8) & 0xF;
    if (k != 0 && (k < 2 || k > 8)) return fail(BBC_INVALID_ARG, "slice count must be 2..8");
  }
  if (prec == BBC_PREC_SPLIT_TF32) {
    const int k = (flags >> 8) & 0xF;
    if (k != 0 && (k < 2 || k > 4)) return fail(BBC_INVALID_ARG, "TF32 term count must be 2..4");
  }
  if (prec == BBC_PREC_FP32 && ((flags >> 8) & 0xF)) return fail(BBC_INVALID_ARG, "BBC_PREC_FP32 takes no term count");
  return BBC_OK;
}

bool overlaps(const double* a, const double* b, int64_t N) {
  const char* pa = (const char*)a;
  const char* pb = (const char*)b;
  const size_t bytes = (size_t)N * N * sizeof(double);
  return pa < pb + bytes && pb < pa + bytes;
}

// T_m(2^-s A) into T, then s squarings ending in Out. The final write sets
// the non-finite flag if any entry of the result is not finite.
// upper: A is upper triangular. Every product then runs on the triangles only,
// and the exact diagonal and first superdiagonal of exp(2^-q A) replace the
// computed ones after the polynomial (q = s) and after every squaring (Section
// 5, concluding remarks). Not used for the Pade comparator (dense solve).
int run_expm(bbc_handle h, const double* A, int64_t N, double* Out, int m, int s, int flags,
             cudaStream_t stream, bbc_info* info, bool upper = false) {
  Program prog;
  if (!make_program(flags & BBC_SCHEME_MASK, m, s, &prog))
    return fail(BBC_INVALID_ARG, "degree not available in this scheme");
  if (s < 0 || s > 1100) return fail(BBC_INVALID_ARG, "squarings out of range");
  const bool pade = (flags & BBC_SCHEME_MASK) == BBC_SCHEME_PADE26 || (flags & BBC_SCHEME_MASK) == BBC_SCHEME_PADE;
  if (pade && N > 112 && N > lu_blocked_max_n())
    return fail(BBC_UNSUPPORTED, "the Pade comparator's solve: N beyond what the panel clusters hold");
  if (pade) upper = false;
  auto exact = [&](double* T, int q) -> int {
    if (!upper) return BBC_OK;
    LaunchScope scope(h, BBC_KERNEL_LINCOMB, stream);
    const cudaError_t e = exact_diagonals(A, N, q, T, stream);
    return e == cudaSuccess ? BBC_OK : cuda_fail(e, "exact diagonals");
  };
  double* tmp = h->work + (size_t)SL_SQ * N * N;
  double* T = (s % 2 == 0) ? Out : tmp;  // the ping-pong ends in Out
  for (size_t i = 0; i < prog.steps.size(); ++i) {
    const bool last = (s == 0 && i + 1 == prog.steps.size() && !pade);
    const int rc = run_step(h, prog.steps[i], N, A, T, flags, last ? h->dflag : nullptr, stream, upper);
    if (rc) return rc;
  }
  if (int rc = exact(T, s)) return rc;
  if (pade) {  // (-u + v) r_26 = u + v: W8 holds -u + v, T holds u + v
    LaunchScope scope(h, BBC_KERNEL_LINCOMB, stream);
    double* scratch = (T == Out) ? tmp : Out;  // whichever of the two is not holding u + v
    const cudaError_t e =
        lu_solve_inplace(h->work + (size_t)8 * N * N, T, N, s == 0 ? h->dflag : nullptr, stream, scratch);
    if (e != cudaSuccess) return cuda_fail(e, "Pade solve");
  }
  double* src = T;
  for (int k = 0; k < s; ++k) {
    double* dst = (src == Out) ? tmp : Out;
    StepS sq{};
    sq.P = SL_A; sq.Q = SL_A; sq.alpha = 1.0; sq.nout = 1;
    sq.o[0].dst = SL_T; sq.o[0].cv = 1.0; sq.o[0].cI = 0.0; sq.o[0].nt = 0;
    // SL_A -> src and SL_T -> dst for this step; the last n_fp64 squarings on the FP64 pipe
    const int n_fp64 = (flags >> 16) & 0xF;
    const int fl = (k >= s - n_fp64) ? ((flags & ~BBC_PREC_MASK & ~0xF00) | BBC_PREC_FP64) : flags;
    const int rc = run_step(h, sq, N, src, dst, fl, (k + 1 == s) ? h->dflag : nullptr, stream, upper);
    if (rc) return rc;
    if (int rc2 = exact(dst, s - k - 1)) return rc2;
    src = dst;
  }
  if (info) {
    info->m = m;
    info->s = s;
    info->products = prog.products + s;
    info->structure = upper ? 1 : 0;
  }
  return BBC_OK;
}

// The batched path serves scheme NEW, with FP64 products or 4-slice split products.
int batch_flags_ok(int flags) {
  const int scheme = flags & BBC_SCHEME_MASK;
  if (scheme != BBC_SCHEME_NEW && scheme != BBC_SCHEME_PADE && scheme != BBC_SCHEME_PADE26)
    return fail(BBC_UNSUPPORTED, "batched path: schemes NEW, PADE and PADE26");
  if (scheme != BBC_SCHEME_NEW && (flags & BBC_SELECT_MASK))
    return fail(BBC_UNSUPPORTED, "batched path: the learned and alpha selections serve scheme NEW");
  const int prec = flags & BBC_PREC_MASK;
  if (prec != BBC_PREC_FP64 && prec != BBC_PREC_OZAKI)
    return fail(BBC_UNSUPPORTED, "batched path: FP64 products or BBC_PREC_OZAKI split products");
  if (prec == BBC_PREC_OZAKI) {
    const int k = (flags >> 8) & 0xF;
    if (k != 0 && k != 4) return fail(BBC_UNSUPPORTED, "batched split products use 4 slices");
  }
  return BBC_OK;
}

int begin(bbc_handle h) {
  if (!h) return fail(BBC_INVALID_ARG, "null handle");
  g_err.clear();
  BBC_CUDA(cudaSetDevice(h->device));
  return BBC_OK;
}

// A few bytes of device state into the handle's host staging `dst` (inside hstage):
// written by a kernel through the mapped address, so that no copy engine is involved
// (a large device-to-host copy in flight on another stream would hold it up), or by
// cudaMemcpyAsync where the staging is not mapped.
cudaError_t to_host(bbc_handle h, void* dst, const void* src, size_t bytes, cudaStream_t st) {
  if (h->hstage_dev) {
    char* d = static_cast<char*>(h->hstage_dev) + (static_cast<char*>(dst) - static_cast<char*>(h->hstage));
    return copy_to_mapped(d, src, bytes, st);
  }
  return cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToHost, st);
}

// ||A||_1 to the host; with `upper` non-null also whether A is upper triangular
// (found in the same pass over A).
int read_norm(bbc_handle h, const double* A, int64_t N, cudaStream_t st, double* norm, bool* upper = nullptr) {
  cudaError_t e;
  {
    LaunchScope scope(h, BBC_KERNEL_NORM, st);
    e = bbc::norm1(A, N, h->partial, h->dnorm, st, upper ? h->dlower : nullptr);
  }
  if (e != cudaSuccess) return cuda_fail(e, "norm1");
  double* hs = (double*)h->hstage;
  unsigned int* hl = (unsigned int*)(hs + 2);
  BBC_CUDA(to_host(h, hs, h->dnorm, sizeof(double), st));
  if (upper) BBC_CUDA(to_host(h, hl, h->dlower, sizeof(unsigned int), st));
  BBC_CUDA(cudaStreamSynchronize(st));
  *norm = hs[0];
  if (upper) *upper = (*hl == 0) && N > 1;
  return BBC_OK;
}

int finish_status(bbc_handle h, cudaStream_t st, int* status) {
  unsigned int* hf = (unsigned int*)((double*)h->hstage + 1);
  BBC_CUDA(to_host(h, hf, h->dflag, sizeof(unsigned int), st));
  BBC_CUDA(cudaStreamSynchronize(st));
  *status = (*hf & 2u) ? BBC_TIMEOUT : (*hf != 0) ? BBC_OVERFLOW : BBC_OK;
  return BBC_OK;
}

}  // namespace

extern "C" {

const char* bbc_last_error(void) { return g_err.c_str(); }

int bbc_create(bbc_handle* out, int device) {
  if (!out) return fail(BBC_INVALID_ARG, "null handle pointer");
  *out = nullptr;
  int count = 0;
  BBC_CUDA(cudaGetDeviceCount(&count));
  if (device < 0 || device >= count) return fail(BBC_INVALID_ARG, "no such device");
  BBC_CUDA(cudaSetDevice(device));
  bbc_handle h = new bbc_handle_s();
  h->device = device;
  cudaError_t e = cudaMalloc(&h->dnorm, sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&h->dflag, sizeof(unsigned int));
  if (e == cudaSuccess) e = cudaMalloc(&h->dlower, sizeof(unsigned int));
  if (e == cudaSuccess) e = cudaHostAlloc(&h->hstage, 64, cudaHostAllocMapped | cudaHostAllocPortable);
  if (e == cudaSuccess && cudaHostGetDevicePointer(&h->hstage_dev, h->hstage, 0) != cudaSuccess) {
    cudaGetLastError();
    h->hstage_dev = nullptr;
  }
  if (e != cudaSuccess) {
    bbc_destroy(h);
    return cuda_fail(e, "bbc_create");
  }
  *out = h;
  return BBC_OK;
}

int bbc_destroy(bbc_handle h) {
  if (!h) return BBC_OK;
  cudaSetDevice(h->device);
  cudaFree(h->work);
  cudaFree(h->partial);
  cudaFree(h->dnorm);
  cudaFree(h->dflag);
  cudaFree(h->dlower);
  cudaFree(h->ozaki);
  cudaFree(h->io);
  cudaFree(h->batch_work);
  cudaFree(h->one_dev);
  cudaFree(h->piv);
  if (h->one_host) cudaFreeHost(h->one_host);
  cudaFree(h->cplx);
  if (h->copy_in) cudaStreamDestroy(h->copy_in);
  if (h->copy_out) cudaStreamDestroy(h->copy_out);
  for (int k = 0; k < 2; ++k) {
    if (h->ev_in[k]) cudaEventDestroy(h->ev_in[k]);
    if (h->ev_out[k]) cudaEventDestroy(h->ev_out[k]);
  }
  for (auto& r : h->recs) { h->pool.push_back(r.a); h->pool.push_back(r.b); }
  for (cudaEvent_t e : h->pool) cudaEventDestroy(e);
  if (h->hstage) cudaFreeHost(h->hstage);
  delete h;
  return BBC_OK;
}

int bbc_workspace_size(bbc_handle h, int64_t N, int dtype, int flags, size_t* bytes) {
  (void)h;
  if (N <= 0 || !bytes || dtype != 0) return fail(BBC_INVALID_ARG, "bad workspace query");
  int rc = check_flags(flags);
  if (rc) return rc;
  size_t b = (size_t)NUM_WORK_SLOTS * N * N * sizeof(double) + norm1_partial_len(N) * sizeof(double);
  if (split_prec(flags)) b += ozaki_workspace_bytes(N, split_planes(flags));
  *bytes = b;
  return BBC_OK;
}

int bbc_profile_enable(bbc_handle h, int enable) {
  int rc = begin(h);
  if (rc) return rc;
  std::lock_guard<std::mutex> lk(h->mu);
  for (auto& r : h->recs) { h->pool.push_back(r.a); h->pool.push_back(r.b); }
  h->recs.clear();
  for (auto& l : h->launches) l = 0;
  for (auto& f : h->flops) f = 0.0;
  h->prof = enable != 0;
  return BBC_OK;
}

int bbc_profile_flops(bbc_handle h, int kind, double* flops) {
  int rc = begin(h);
  if (rc) return rc;
  if (!flops || kind < -1 || kind > 4) return fail(BBC_INVALID_ARG, "bad profile query");
  std::lock_guard<std::mutex> lk(h->mu);
  double f = 0.0;
  for (int k = 0; k < 5; ++k)
    if (kind == -1 || kind == k) f += h->flops[k];
  *flops = f;
  return BBC_OK;
}

int bbc_profile_read(bbc_handle h, int kind, int64_t* launches, double* total_ms) {
  int rc = begin(h);
  if (rc) return rc;
  if (!launches || kind < -1 || kind > 4) return fail(BBC_INVALID_ARG, "bad profile query");
  std::lock_guard<std::mutex> lk(h->mu);
  int64_t n = 0;
  for (int k = 0; k < 5; ++k)
    if (kind == -1 || kind == k) n += h->launches[k];
  *launches = n;
  if (total_ms) {
    double ms = 0.0;
    for (auto& r : h->recs) {
      if (kind != -1 && r.kind != kind) continue;
      BBC_CUDA(cudaEventSynchronize(r.b));
      float t = 0.f;
      BBC_CUDA(cudaEventElapsedTime(&t, r.a, r.b));
      ms += t;
    }
    *total_ms = ms;
  }
  return BBC_OK;
}

int bbc_theta(int m, double u, double* theta) {
  if (!theta || m < 1 || m > 30 || !valid_u(u)) return fail(BBC_INVALID_ARG, "bad theta query");
  *theta = theta_cached(m, u);
  return BBC_OK;
}

int bbc_theta_pade(int two_m, double u, double* theta) {
  if (!theta || two_m < 2 || two_m > 30 || two_m % 2 || !valid_u(u)) return fail(BBC_INVALID_ARG, "bad Pade theta query");
  *theta = theta_cached(-two_m, u);
  return BBC_OK;
}

int bbc_select(double norm1, double u, int scheme, int* m, int* s) {
  if (!m || !s || !valid_u(u)) return fail(BBC_INVALID_ARG, "bad selection query");
  if (scheme != BBC_SCHEME_NEW && scheme != BBC_SCHEME_PS && scheme != BBC_SCHEME_PADE26 && scheme != BBC_SCHEME_PADE)
    return fail(BBC_INVALID_ARG, "unknown scheme");
  if (!std::isfinite(norm1) || norm1 < 0) return fail(BBC_NONFINITE_INPUT, "norm not finite");
  return select_ms(norm1, u, scheme, m, s);
}

int bbc_norm1(bbc_handle h, const double* dA, int64_t N, void* stream, double* hNorm) {
  int rc = begin(h);
  if (rc) return rc;
  if (!dA || !hNorm || N <= 0) return fail(BBC_INVALID_ARG, "bad norm1 arguments");
  std::lock_guard<std::mutex> lk(h->mu);
  rc = ensure_workspace(h, N, 0);
  if (rc) return rc;
  return read_norm(h, dA, N, (cudaStream_t)stream, hNorm);
}

int bbc_norm1_noalloc(const double* dA, int64_t N, double* dNorm, void* stream) {
  g_err.clear();
  if (N <= 0 || !norm1_noalloc_fits(N))
    return fail(BBC_INVALID_ARG, "bbc_norm1_noalloc: N must be in 1..65536 (fixed 1 MiB scratch)");
  if (!dA || !dNorm) return fail(BBC_INVALID_ARG, "bbc_norm1_noalloc: null pointer");
  const cudaError_t e = norm1_noalloc(dA, N, dNorm, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "bbc_norm1_noalloc");
  return BBC_OK;
}

int bbc_solve(bbc_handle h, double* dM, double* dB, int64_t N, void* stream) {
  int rc = begin(h);
  if (rc) return rc;
  if (!dM || !dB || N <= 0) return fail(BBC_INVALID_ARG, "bad solve arguments");
  if (overlaps(dM, dB, N)) return fail(BBC_INVALID_ARG, "M and B overlap");
  if (N > 112 && N > lu_blocked_max_n()) return fail(BBC_UNSUPPORTED, "N beyond what the panel clusters hold");
  std::lock_guard<std::mutex> lk(h->mu);
  BBC_CUDA(cudaSetDevice(h->device));
  if (N > h->piv_n) {  // the blocked LU's only scratch: N pivot indices (grown on demand)
    if (h->piv) BBC_CUDA(cudaFree(h->piv));
    h->piv = nullptr;
    h->piv_n = 0;
    BBC_CUDA(cudaMalloc(&h->piv, (size_t)N * sizeof(int)));
    h->piv_n = N;
  }
  cudaStream_t st = (cudaStream_t)stream;
  BBC_CUDA(cudaMemsetAsync(h->dflag, 0, sizeof(unsigned int), st));
  {
    LaunchScope scope(h, BBC_KERNEL_LINCOMB, st);
    const cudaError_t e = lu_solve_inplace(dM, dB, N, h->dflag, st, reinterpret_cast<double*>(h->piv));
    if (e != cudaSuccess) return cuda_fail(e, "solve");
  }
  int status = BBC_OK;
  if ((rc = finish_status(h, st, &status))) return rc;
  if (status) return fail(status, "singular or non-finite system");
  return BBC_OK;
}

int bbc_gemm(bbc_handle h, const double* dP, const double* dQ, int64_t N, double* dC, int flags,
             void* stream) {
  int rc = begin(h);
  if (rc) return rc;
  if (!dP || !dQ || !dC || N <= 0) return fail(BBC_INVALID_ARG, "bad gemm arguments");
  if (overlaps(dC, dP, N) || overlaps(dC, dQ, N)) return fail(BBC_INVALID_ARG, "output aliases an input");
  if ((rc = check_flags(flags))) return rc;
  std::lock_guard<std::mutex> lk(h->mu);
  if ((rc = ensure_workspace(h, N, flags))) return rc;
  Epilogue e{};
  e.nout = 1;
  e.o[0].out = dC;
  e.o[0].cv = 1.0;
  cudaStream_t st = (cudaStream_t)stream;
  const bool ozaki = split_prec(flags);
  if (ozaki) BBC_CUDA(cudaMemsetAsync(h->dflag, 0, sizeof(unsigned int), st));
  if ((rc = launch_product(h, dP, dQ, N, 1.0, e, flags, st, (flags & BBC_UPPER) != 0))) return rc;
  if (ozaki) {  // report a non-finite operand or an expired device wait
    int status = BBC_OK;
    if ((rc = finish_status(h, st, &status))) return rc;
    if (status) return fail(status, status == BBC_TIMEOUT ? "device wait timed out" : "non-finite operand");
  }
  return BBC_OK;
}

int bbc_taylor(bbc_handle h, const double* dA, int64_t N, int m, int s, double* dT, int flags,
               void* stream, int* products) {
  int rc = begin(h);
  if (rc) return rc;
  if (!dA || !dT || N <= 0 || s < 0 || s > 1100) return fail(BBC_INVALID_ARG, "bad taylor arguments");
  if (overlaps(dA, dT, N)) return fail(BBC_INVALID_ARG, "output aliases the input");
  if ((rc = check_flags(flags))) return rc;
  Program prog;
  if (!make_program(flags & BBC_SCHEME_MASK, m, s, &prog))
    return fail(BBC_INVALID_ARG, "degree not available in this scheme");
  std::lock_guard<std::mutex> lk(h->mu);
  if ((rc = ensure_workspace(h, N, flags))) return rc;
  for (const StepS& st : prog.steps)
    if ((rc = run_step(h, st, N, dA, dT, flags, nullptr, (cudaStream_t)stream))) return rc;
  if (products) *products = prog.products;
  return BBC_OK;
}

int bbc_expm_fixed(bbc_handle h, const double* dA, int64_t N, double* dOut, int m, int s, int flags,
                   void* stream, bbc_info* info) {
  int rc = begin(h);
  if (rc) return rc;
  if (!dA || !dOut || N <= 0) return fail(BBC_INVALID_ARG, "bad expm arguments");
  if (overlaps(dA, dOut, N)) return fail(BBC_INVALID_ARG, "output aliases the input");
  if ((rc = check_flags(flags))) return rc;
  std::lock_guard<std::mutex> lk(h->mu);
  if ((rc = ensure_workspace(h, N, flags))) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  bbc_info loc{};
  bbc_info* inf = info ? info : &loc;
  memset(inf, 0, sizeof *inf);
  inf->selector = 1;
  bool upper = false;
  if ((rc = read_norm(h, dA, N, st, &inf->norm1, (flags & BBC_DENSE) ? nullptr : &upper))) return rc;
  if (!std::isfinite(inf->norm1)) {
    inf->status = BBC_NONFINITE_INPUT;
    return fail(BBC_NONFINITE_INPUT, "input holds a non-finite value");
  }
  BBC_CUDA(cudaMemsetAsync(h->dflag, 0, sizeof(unsigned int), st));
  if ((rc = run_expm(h, dA, N, dOut, m, s, flags, st, inf, upper))) return rc;
  if ((rc = finish_status(h, st, &inf->status))) return rc;
  if (inf->status) return fail(inf->status, "result holds a non-finite value");
  return BBC_OK;
}

int bbc_expm_fixed_async(bbc_handle h, const double* dA, int64_t N, double* dOut, int m, int s, int flags,
                         void* stream, unsigned int* dStatus) {
  int rc = begin(h);
  if (rc) return rc;
  if (!dA || !dOut || N <= 0) return fail(BBC_INVALID_ARG, "bad expm arguments");
  if (overlaps(dA, dOut, N)) return fail(BBC_INVALID_ARG, "output aliases the input");
  if ((rc = check_flags(flags))) return rc;
  std::lock_guard<std::mutex> lk(h->mu);
  cudaStream_t st = (cudaStream_t)stream;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  BBC_CUDA(cudaStreamIsCapturing(st, &cs));
  if (cs != cudaStreamCaptureStatusNone) {  // nothing may be allocated inside a capture
    if (split_prec(flags) && !ozaki_supported(N))
      return fail(BBC_UNSUPPORTED, "split-precision products take N <= 16384");
    if (N > h->slots_n || (split_prec(flags) && ozaki_workspace_bytes(N, split_planes(flags)) > h->ozaki_bytes))
      return fail(BBC_INVALID_ARG, "workspace too small: run this N and precision once before the capture");
    if (((flags & BBC_SCHEME_MASK) == BBC_SCHEME_PADE26 || (flags & BBC_SCHEME_MASK) == BBC_SCHEME_PADE) && N > 112 &&
        !lu_blocked_ready())
      return fail(BBC_INVALID_ARG, "run the Pade comparator once (N > 112) before capturing it on this device");
  } else if ((rc = ensure_workspace(h, N, flags))) {
    return rc;
  }
  BBC_CUDA(cudaMemsetAsync(h->dflag, 0, sizeof(unsigned int), st));
  if ((rc = run_expm(h, dA, N, dOut, m, s, flags, st, nullptr, (flags & BBC_UPPER) != 0))) return rc;
  if (dStatus)
    BBC_CUDA(cudaMemcpyAsync(dStatus, h->dflag, sizeof(unsigned int), cudaMemcpyDeviceToDevice, st));
  return BBC_OK;
}

int bbc_selftest_wait(bbc_handle h, void* stream, int* status) {
  int rc = begin(h);
  if (rc) return rc;
  if (!status) return fail(BBC_INVALID_ARG, "null status");
  std::lock_guard<std::mutex> lk(h->mu);
  cudaStream_t st = (cudaStream_t)stream;
  BBC_CUDA(cudaMemsetAsync(h->dflag, 0, sizeof(unsigned int), st));
  BBC_CUDA(wait_selftest(h->dflag, st));
  return finish_status(h, st, status);
}

int bbc_expm_complex(bbc_handle h, const double* dA, int64_t N, double* dOut, double tol, int flags,
                     void* stream, bbc_info* info) {
  int rc = begin(h);
  if (rc) return rc;
  if (!dA || !dOut || N <= 0) return fail(BBC_INVALID_ARG, "bad expm arguments");
  if ((reinterpret_cast<uintptr_t>(dA) | reinterpret_cast<uintptr_t>(dOut)) & 15)
    return fail(BBC_INVALID_ARG, "complex arrays must be 16-byte aligned");
  {
    const char* pa = (const char*)dA;
    const char* pb = (const char*)dOut;
    const size_t bytes = (size_t)2 * N * N * sizeof(double);
    if (pa < pb + bytes && pb < pa + bytes) return fail(BBC_INVALID_ARG, "output aliases the input");
  }
  const double u = tol > 0 ? tol : std::ldexp(1.0, -53);
  if (!valid_u(u)) return fail(BBC_INVALID_ARG, "tol out of range [2^-60, 2^-5]");
  if ((rc = check_flags(flags))) return rc;
  if (flags & BBC_UPPER) return fail(BBC_INVALID_ARG, "BBC_UPPER is not defined for complex calls");
  std::lock_guard<std::mutex> lk(h->mu);
  if ((rc = ensure_workspace(h, 2 * N, flags))) return rc;
  if (N > h->cplx_n) {
    if (h->cplx) BBC_CUDA(cudaFree(h->cplx));
    h->cplx = nullptr;
    h->cplx_n = 0;
    BBC_CUDA(cudaMalloc(&h->cplx, ((size_t)8 * N * N + (size_t)complex_norm_partial_len(N)) * sizeof(double)));
    h->cplx_n = N;
  }
  double* E = h->cplx;
  double* Eout = E + (size_t)4 * N * N;
  double* partial = Eout + (size_t)4 * N * N;
  cudaStream_t st = (cudaStream_t)stream;
  bbc_info loc{};
  bbc_info* inf = info ? info : &loc;
  memset(inf, 0, sizeof *inf);
  {
    LaunchScope scope(h, BBC_KERNEL_NORM, st);
    const cudaError_t e = complex_norm1(dA, N, partial, h->dnorm, st);
    if (e != cudaSuccess) return cuda_fail(e, "complex norm1");
  }
  double* hs = (double*)h->hstage;
  BBC_CUDA(to_host(h, hs, h->dnorm, sizeof(double), st));
  BBC_CUDA(cudaStreamSynchronize(st));
  inf->norm1 = hs[0];
  if (!std::isfinite(inf->norm1)) {
    inf->status = BBC_NONFINITE_INPUT;
    return fail(BBC_NONFINITE_INPUT, "input holds a non-finite value");
  }
  int m, s;
  select_ms(inf->norm1, u, flags & BBC_SCHEME_MASK, &m, &s);
  BBC_CUDA(cudaMemsetAsync(h->dflag, 0, sizeof(unsigned int), st));
  {
    LaunchScope scope(h, BBC_KERNEL_LINCOMB, st);
    const cudaError_t e = complex_embed(dA, N, E, st);
    if (e != cudaSuccess) return cuda_fail(e, "complex embedding");
  }
  if ((rc = run_expm(h, E, 2 * N, Eout, m, s, flags, st, inf, false))) return rc;
  {
    LaunchScope scope(h, BBC_KERNEL_LINCOMB, st);
    const cudaError_t e = complex_extract(Eout, N, dOut, h->dflag, st);
    if (e != cudaSuccess) return cuda_fail(e, "complex extraction");
  }
  if ((rc = finish_status(h, st, &inf->status))) return rc;
  if (inf->status) return fail(inf->status, "result holds a non-finite value");
  return BBC_OK;
}

int bbc_expm(bbc_handle h, const double* dA, int64_t N, double* dOut, double tol, int flags,
             void* stream, bbc_info* info) {
  int rc = begin(h);
  if (rc) return rc;
  if (!dA || !dOut || N <= 0) return fail(BBC_INVALID_ARG, "bad expm arguments");
  if (overlaps(dA, dOut, N)) return fail(BBC_INVALID_ARG, "output aliases the input");
  const double u = tol > 0 ? tol : std::ldexp(1.0, -53);
  if (!valid_u(u)) return fail(BBC_INVALID_ARG, "tol out of range [2^-60, 2^-5]");
  if ((rc = check_flags(flags))) return rc;
  if (flags & BBC_SELECT_MASK) {
    // A certified (m, s) proposal (learned network, or the alpha_2 bound) needs the
    // power-norm estimates and the network the persistent batched kernel carries:
    // the matrix runs there as a batch of one.
    if ((flags & BBC_SCHEME_MASK) != BBC_SCHEME_NEW || (flags & BBC_PREC_MASK) != BBC_PREC_FP64)
      return fail(BBC_UNSUPPORTED, "bbc_expm: the learned and alpha selections run scheme NEW with FP64 products");
    std::lock_guard<std::mutex> lk(h->mu);
    if (!h->batch_work || !h->one_dev || N > h->batch_nmax)
      return fail(BBC_INVALID_ARG, "bbc_expm with a certified selection: call bbc_batch_reserve(max_n >= N) first");
    cudaStream_t st = (cudaStream_t)stream;
    OneDesc* host = static_cast<OneDesc*>(h->one_host);
    OneDesc* dev = static_cast<OneDesc*>(h->one_dev);
    host->a = dA;
    host->out = dOut;
    host->n = N;
    BBC_CUDA(cudaMemcpyAsync(dev, host, offsetof(OneDesc, info), cudaMemcpyHostToDevice, st));
    if ((rc = batched_locked(h, &dev->a, nullptr, &dev->n, 1, &dev->out, BBC_DTYPE_F64, u, flags, st, &dev->info)))
      return rc;
    BBC_CUDA(cudaMemcpyAsync(&host->info, &dev->info, sizeof(bbc_info), cudaMemcpyDeviceToHost, st));
    BBC_CUDA(cudaStreamSynchronize(st));
    if (info) *info = host->info;
    if (host->info.status) return fail(host->info.status, "certified-selection exp(A) failed");
    return BBC_OK;
  }
  std::lock_guard<std::mutex> lk(h->mu);
  if ((rc = ensure_workspace(h, N, flags))) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  bbc_info loc{};
  bbc_info* inf = info ? info : &loc;
  memset(inf, 0, sizeof *inf);
  bool upper = false;
  if ((rc = read_norm(h, dA, N, st, &inf->norm1, (flags & BBC_DENSE) ? nullptr : &upper))) return rc;
  if (!std::isfinite(inf->norm1)) {
    inf->status = BBC_NONFINITE_INPUT;
    return fail(BBC_NONFINITE_INPUT, "input holds a non-finite value");
  }
  int m, s;
  select_ms(inf->norm1, u, flags & BBC_SCHEME_MASK, &m, &s);
  BBC_CUDA(cudaMemsetAsync(h->dflag, 0, sizeof(unsigned int), st));
  if ((rc = run_expm(h, dA, N, dOut, m, s, flags, st, inf, upper))) return rc;
  if ((rc = finish_status(h, st, &inf->status))) return rc;
  if (inf->status) return fail(inf->status, "result holds a non-finite value");
  return BBC_OK;
}

namespace {
// Device staging for the host-buffer calls: four N x N slots (two inputs, two
// outputs), grown on demand. Caller holds no lock.
int ensure_io(bbc_handle h, int64_t N) {
  std::lock_guard<std::mutex> lk(h->mu);
  if (N <= h->io_n) return BBC_OK;
  if (h->io) BBC_CUDA(cudaFree(h->io));
  h->io = nullptr;
  h->io_n = 0;
  BBC_CUDA(cudaMalloc(&h->io, (size_t)4 * N * N * sizeof(double)));
  h->io_n = N;
  return BBC_OK;
}
}  // namespace

int bbc_expm_host(bbc_handle h, const double* hA, int64_t N, double* hOut, double tol, int flags,
                  void* stream, bbc_info* info) {
  int rc = begin(h);
  if (rc) return rc;
  if (!hA || !hOut || N <= 0) return fail(BBC_INVALID_ARG, "bad expm arguments");
  if (overlaps(hA, hOut, N)) return fail(BBC_INVALID_ARG, "output aliases the input");
  if ((rc = ensure_io(h, N))) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  const size_t bytes = (size_t)N * N * sizeof(double);
  double* dA = h->io;
  double* dOut = h->io + (size_t)2 * h->io_n * h->io_n;
  BBC_CUDA(cudaMemcpyAsync(dA, hA, bytes, cudaMemcpyHostToDevice, st));
  rc = bbc_expm(h, dA, N, dOut, tol, flags, stream, info);
  if (rc) return rc;
  BBC_CUDA(cudaMemcpyAsync(hOut, dOut, bytes, cudaMemcpyDeviceToHost, st));
  BBC_CUDA(cudaStreamSynchronize(st));
  return BBC_OK;
}

int bbc_expm_host_many(bbc_handle h, const double* const* hA, const int64_t* Ns, int64_t count,
                       double* const* hOut, double tol, int flags, void* stream, bbc_info* info) {
  int rc = begin(h);
  if (rc) return rc;
  if (!hA || !Ns || !hOut || count < 0) return fail(BBC_INVALID_ARG, "bad expm_host_many arguments");
  int64_t nmax = 0;
  for (int64_t i = 0; i < count; ++i) {
    if (!hA[i] || !hOut[i] || Ns[i] <= 0) return fail(BBC_INVALID_ARG, "bad matrix in expm_host_many");
    if (overlaps(hA[i], hOut[i], Ns[i])) return fail(BBC_INVALID_ARG, "an output aliases its input");
    nmax = std::max(nmax, Ns[i]);
  }
  if (count == 0) return BBC_OK;
  if ((rc = ensure_io(h, nmax))) return rc;
  {
    std::lock_guard<std::mutex> lk(h->mu);
    if (!h->copy_in) {
      BBC_CUDA(cudaStreamCreateWithFlags(&h->copy_in, cudaStreamNonBlocking));
      BBC_CUDA(cudaStreamCreateWithFlags(&h->copy_out, cudaStreamNonBlocking));
      for (int k = 0; k < 2; ++k) {
        BBC_CUDA(cudaEventCreateWithFlags(&h->ev_in[k], cudaEventDisableTiming));
        BBC_CUDA(cudaEventCreateWithFlags(&h->ev_out[k], cudaEventDisableTiming));
      }
    }
  }
  cudaStream_t st = (cudaStream_t)stream;
  const size_t slot = (size_t)h->io_n * h->io_n;
  double* din[2] = {h->io, h->io + slot};
  double* dout[2] = {h->io + 2 * slot, h->io + 3 * slot};
  // Matrix i computes on `stream` (bbc_expm returns once it is done) while the
  // copy streams bring in matrix i + 1 and take out matrix i - 1.
  BBC_CUDA(cudaMemcpyAsync(din[0], hA[0], (size_t)Ns[0] * Ns[0] * sizeof(double), cudaMemcpyHostToDevice,
                           h->copy_in));
  BBC_CUDA(cudaEventRecord(h->ev_in[0], h->copy_in));
  int first_err = BBC_OK;
  for (int64_t i = 0; i < count && !first_err; ++i) {
    const int b = (int)(i & 1);
    if (i + 1 < count) {  // slot (i+1)&1 was last read by matrix i-1, which has finished
      BBC_CUDA(cudaMemcpyAsync(din[b ^ 1], hA[i + 1], (size_t)Ns[i + 1] * Ns[i + 1] * sizeof(double),
                               cudaMemcpyHostToDevice, h->copy_in));
      BBC_CUDA(cudaEventRecord(h->ev_in[b ^ 1], h->copy_in));
    }
    BBC_CUDA(cudaStreamWaitEvent(st, h->ev_in[b], 0));
    if (i >= 2) BBC_CUDA(cudaStreamWaitEvent(st, h->ev_out[b], 0));  // matrix i-2 has left dout[b]
    first_err = bbc_expm(h, din[b], Ns[i], dout[b], tol, flags, stream, info ? info + i : nullptr);
    if (first_err) break;
    BBC_CUDA(cudaMemcpyAsync(hOut[i], dout[b], (size_t)Ns[i] * Ns[i] * sizeof(double), cudaMemcpyDeviceToHost,
                             h->copy_out));
    BBC_CUDA(cudaEventRecord(h->ev_out[b], h->copy_out));
  }
  const std::string err = g_err;
  BBC_CUDA(cudaStreamSynchronize(h->copy_in));
  BBC_CUDA(cudaStreamSynchronize(h->copy_out));
  if (first_err) return fail(first_err, err);
  return BBC_OK;
}

// ---------------------------------------------------------------------------
// Autotuner of the batched path: which size buckets run split products and how
// many persistent CTAs the launch uses, chosen by timing on this GPU.
// ---------------------------------------------------------------------------
namespace {
struct DevBuf {
  void* p = nullptr;
  ~DevBuf() { if (p) cudaFree(p); }
};

// Best of `reps` event-timed launches (after one warm-up) of the batched kernel.
int time_batch(bbc_handle h, const void* const* dA, void* const* dOut, const int64_t* dNs, int64_t count,
               const double* theta, int ctas, uint32_t mask, cudaStream_t st, int reps, float* best_ms,
               const BatchShapes* shapes = nullptr) {
  cudaEvent_t a = nullptr, b = nullptr;
  BBC_CUDA(cudaEventCreate(&a));
  BBC_CUDA(cudaEventCreate(&b));
  float best = 1e30f;
  cudaError_t e = cudaSuccess;
  for (int r = 0; r <= reps && e == cudaSuccess; ++r) {
    e = cudaEventRecord(a, st);
    if (e == cudaSuccess)
      e = batched_launch(dA, dOut, dNs, count, h->batch_nmax, BBC_DTYPE_F64, theta, h->batch_work, ctas, nullptr,
                         st, nullptr, true, mask, nullptr, nullptr, 0, nullptr, shapes);
    if (e == cudaSuccess) e = cudaEventRecord(b, st);
    if (e == cudaSuccess) e = cudaEventSynchronize(b);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, a, b);
    if (r > 0 && ms < best) best = ms;  // r = 0 is the warm-up
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  if (e != cudaSuccess) return cuda_fail(e, "autotuner launch");
  *best_ms = best;
  return BBC_OK;
}
}  // namespace

int bbc_batch_tune(bbc_handle h, int64_t max_n, double tol, void* stream, uint32_t* split_mask, int* ctas) {
  int rc = begin(h);
  if (rc) return rc;
  const double u = tol > 0 ? tol : std::ldexp(1.0, -53);
  if (!valid_u(u)) return fail(BBC_INVALID_ARG, "tol out of range [2^-60, 2^-5]");
  std::lock_guard<std::mutex> lk(h->mu);
  if (!h->batch_work || !h->batch_split) return fail(BBC_INVALID_ARG, "reserve with BBC_PREC_OZAKI first");
  if (max_n < 1 || max_n > h->batch_nmax) return fail(BBC_INVALID_ARG, "max_n beyond the reservation");
  cudaStream_t st = (cudaStream_t)stream;
  static const int deg[6] = {1, 2, 4, 8, 12, 18};
  double theta[6];
  for (int i = 0; i < 6; ++i) theta[i] = theta_cached(deg[i], u);
  const int64_t nlim = std::min<int64_t>(max_n, 256);  // split products serve N <= 256
  const int nb = (int)((nlim + 7) / 8);
  const int64_t per = 2 * (int64_t)h->batch_ctas;      // matrices per bucket: every CTA gets two
  // 1. per size bucket: split or FP64 products, whichever is faster here
  DevBuf buf, ptrs, ns;
  BBC_CUDA(cudaMalloc(&buf.p, (size_t)2 * per * nlim * nlim * sizeof(double)));
  BBC_CUDA(cudaMalloc(&ptrs.p, (size_t)2 * per * sizeof(void*)));
  BBC_CUDA(cudaMalloc(&ns.p, (size_t)per * sizeof(int64_t)));
  std::vector<void*> hp(2 * per);
  std::vector<int64_t> hn(per);
  uint32_t mask = 0;
  BatchShapes shapes;
  for (int b = 0; b < nb; ++b) {
    const int64_t N = std::min<int64_t>(8 * (b + 1), nlim);
    double* in = static_cast<double*>(buf.p);
    double* out = in + (size_t)per * N * N;
    BBC_CUDA(calibration_matrices(in, N, per, 0x5eed0000ull + (uint64_t)b, 5.0, st));
    for (int64_t i = 0; i < per; ++i) {
      hp[i] = in + (size_t)i * N * N;
      hp[per + i] = out + (size_t)i * N * N;
      hn[i] = N;
    }
    BBC_CUDA(cudaMemcpyAsync(ptrs.p, hp.data(), hp.size() * sizeof(void*), cudaMemcpyHostToDevice, st));
    BBC_CUDA(cudaMemcpyAsync(ns.p, hn.data(), hn.size() * sizeof(int64_t), cudaMemcpyHostToDevice, st));
    const void* const* dA = static_cast<const void* const*>(ptrs.p);
    void* const* dO = static_cast<void* const*>(ptrs.p) + per;
    // five candidates: split products in 32 x 16 or 16 x 16 warp tasks, FP64 products in
    // 64 x 64, 32 x 32 or 16 x 16 output tiles
    struct Cand { bool split; BatchShapes sh; };
    BatchShapes s16, t32, t16;
    s16.split_task16 = 1u << b;
    t32.f64_tile32 = 1u << b;
    t16.f64_tile16 = 1u << b;
    const Cand cands[5] = {{true, BatchShapes{}}, {true, s16}, {false, BatchShapes{}}, {false, t32}, {false, t16}};
    float best_t = 1e30f;
    int best_c = 0;
    for (int c = 0; c < 5; ++c) {
      float t = 0.f;
      if ((rc = time_batch(h, dA, dO, static_cast<const int64_t*>(ns.p), per, theta, h->batch_ctas,
                           cands[c].split ? (1u << b) : 0u, st, 3, &t, &cands[c].sh)))
        return rc;
      if (t < best_t) { best_t = t; best_c = c; }
    }
    if (cands[best_c].split) mask |= 1u << b;
    shapes.split_task16 |= cands[best_c].sh.split_task16;
    shapes.f64_tile32 |= cands[best_c].sh.f64_tile32;
    shapes.f64_tile16 |= cands[best_c].sh.f64_tile16;
  }
  for (int b = nb; b < 32; ++b) mask |= 1u << b;  // buckets not tuned keep the default
  // 2. the persistent grid: one or two CTAs per SM, on a mix of every bucket large
  //    enough (eight matrices per resident CTA) that the queue's tail does not decide
  const int64_t mix_per = std::max<int64_t>(16, (8 * (int64_t)h->batch_ctas + nb - 1) / nb);
  const int64_t mcount = mix_per * nb;
  DevBuf mbuf, mptrs, mns;
  size_t mdoubles = 0;
  for (int b = 0; b < nb; ++b) {
    const int64_t N = std::min<int64_t>(8 * (b + 1), nlim);
    mdoubles += (size_t)mix_per * N * N;
  }
  BBC_CUDA(cudaMalloc(&mbuf.p, 2 * mdoubles * sizeof(double)));
  BBC_CUDA(cudaMalloc(&mptrs.p, (size_t)2 * mcount * sizeof(void*)));
  BBC_CUDA(cudaMalloc(&mns.p, (size_t)mcount * sizeof(int64_t)));
  std::vector<void*> mp(2 * mcount);
  std::vector<int64_t> mn(mcount);
  {
    double* in = static_cast<double*>(mbuf.p);
    double* out = in + mdoubles;
    size_t off = 0;
    int64_t k = 0;
    for (int b = nb - 1; b >= 0; --b) {  // largest first, as bbc_batch_order would put them
      const int64_t N = std::min<int64_t>(8 * (b + 1), nlim);
      BBC_CUDA(calibration_matrices(in + off, N, mix_per, 0x5eed1000ull + (uint64_t)b, 5.0, st));
      for (int64_t i = 0; i < mix_per; ++i, ++k) {
        mp[k] = in + off + (size_t)i * N * N;
        mp[mcount + k] = out + off + (size_t)i * N * N;
        mn[k] = N;
      }
      off += (size_t)mix_per * N * N;
    }
  }
  BBC_CUDA(cudaMemcpyAsync(mptrs.p, mp.data(), mp.size() * sizeof(void*), cudaMemcpyHostToDevice, st));
  BBC_CUDA(cudaMemcpyAsync(mns.p, mn.data(), mn.size() * sizeof(int64_t), cudaMemcpyHostToDevice, st));
  const int grids[2] = {h->batch_ctas / 2, h->batch_ctas};
  float best = 1e30f;
  int best_grid = h->batch_ctas;
  for (int g : grids) {
    if (g < 1) continue;
    float t = 0.f;
    if ((rc = time_batch(h, static_cast<const void* const*>(mptrs.p), static_cast<void* const*>(mptrs.p) + mcount,
                         static_cast<const int64_t*>(mns.p), mcount, theta, g, mask, st, 3, &t, &shapes)))
      return rc;
    if (t < best) { best = t; best_grid = g; }
  }
  BBC_CUDA(cudaStreamSynchronize(st));
  h->batch_split_mask = mask;
  h->batch_grid = best_grid;
  h->batch_shapes = shapes;
  if (split_mask) *split_mask = mask;
  if (ctas) *ctas = best_grid;
  return BBC_OK;
}

int bbc_batch_get_shapes(bbc_handle h, uint32_t* masks) {
  int rc = begin(h);
  if (rc) return rc;
  if (!masks) return fail(BBC_INVALID_ARG, "null masks");
  std::lock_guard<std::mutex> lk(h->mu);
  masks[0] = h->batch_shapes.f64_tile16;
  masks[1] = h->batch_shapes.f64_tile32;
  masks[2] = h->batch_shapes.split_task16;
  return BBC_OK;
}

int bbc_batch_set_shapes(bbc_handle h, const uint32_t* masks) {
  int rc = begin(h);
  if (rc) return rc;
  std::lock_guard<std::mutex> lk(h->mu);
  h->batch_shapes = BatchShapes{};
  if (masks) {
    h->batch_shapes.f64_tile16 = masks[0];
    h->batch_shapes.f64_tile32 = masks[1];
    h->batch_shapes.split_task16 = masks[2];
  }
  return BBC_OK;
}

int bbc_batch_set_tuning(bbc_handle h, uint32_t split_mask, int ctas) {
  int rc = begin(h);
  if (rc) return rc;
  std::lock_guard<std::mutex> lk(h->mu);
  if (ctas < 0 || (h->batch_ctas > 0 && ctas > h->batch_ctas))
    return fail(BBC_INVALID_ARG, "CTA count beyond the reservation");
  h->batch_split_mask = split_mask;
  h->batch_grid = ctas;
  return BBC_OK;
}

int bbc_batch_launch_shape(bbc_handle h, int64_t count, int* csize, int* grid) {
  int rc = begin(h);
  if (rc) return rc;
  if (count < 1 || !csize || !grid) return fail(BBC_INVALID_ARG, "bad launch-shape query");
  std::lock_guard<std::mutex> lk(h->mu);
  if (!h->batch_work) return fail(BBC_INVALID_ARG, "call bbc_batch_reserve first");
  const int ctas = (h->batch_grid > 0 && h->batch_grid <= h->batch_ctas) ? h->batch_grid : h->batch_ctas;
  *csize = batched_cluster_size(&h->batch_cl, count, ctas, grid);
  return BBC_OK;
}

int bbc_mlp_sizes(int in, int hid, int out, int64_t B, int64_t* n_params, int64_t* ws_floats) {
  if (in < 1 || hid < 1 || out < 1 || B < 0 || !n_params || !ws_floats) return fail(BBC_INVALID_ARG, "bad MLP sizes");
  *n_params = mlp_param_count(in, hid, out);
  *ws_floats = mlp_workspace_floats(hid, out, B);
  return BBC_OK;
}

int bbc_mlp_forward(const float* dParams, int in, int hid, int out, const float* dX, int64_t B, float* dLogits,
                    float* dWs, void* stream) {
  g_err.clear();
  if (!dParams || !dX || !dLogits || !dWs || in < 1 || hid < 1 || out < 1 || B < 1)
    return fail(BBC_INVALID_ARG, "bad MLP forward arguments");
  const cudaError_t e = mlp_forward(dParams, in, hid, out, dX, B, dLogits, dWs, (cudaStream_t)stream);
  return e == cudaSuccess ? BBC_OK : cuda_fail(e, "mlp forward");
}

int bbc_mlp_grad(const float* dParams, int in, int hid, int out, const float* dX, const int* dLabels, int64_t B,
                 float* dGrad, float* dLoss, float* dWs, void* stream) {
  g_err.clear();
  if (!dParams || !dX || !dLabels || !dGrad || !dLoss || !dWs || in < 1 || hid < 1 || out < 1 || B < 1)
    return fail(BBC_INVALID_ARG, "bad MLP gradient arguments");
  const cudaError_t e = mlp_grad(dParams, in, hid, out, dX, dLabels, B, dGrad, dLoss, dWs, (cudaStream_t)stream);
  return e == cudaSuccess ? BBC_OK : cuda_fail(e, "mlp grad");
}

int bbc_mlp_adam(float* dParams, const float* dGrad, float* dM, float* dV, int64_t n, float lr, float beta1,
                 float beta2, float eps, int step, void* stream) {
  g_err.clear();
  if (!dParams || !dGrad || !dM || !dV || n < 1 || step < 1) return fail(BBC_INVALID_ARG, "bad Adam arguments");
  const cudaError_t e = mlp_adam(dParams, dGrad, dM, dV, n, lr, beta1, beta2, eps, step, (cudaStream_t)stream);
  return e == cudaSuccess ? BBC_OK : cuda_fail(e, "adam");
}

int bbc_batch_reserve(bbc_handle h, int64_t max_n, int flags) {
  int rc = begin(h);
  if (rc) return rc;
  if (max_n < 1 || max_n > 512) return fail(BBC_INVALID_ARG, "batched max_n must be in 1..512");
  if ((rc = check_flags(flags))) return rc;
  if ((rc = batch_flags_ok(flags))) return rc;
  const bool split = (flags & BBC_PREC_MASK) == BBC_PREC_OZAKI;
  std::lock_guard<std::mutex> lk(h->mu);
  if (max_n > h->batch_nmax || (split && !h->batch_split)) {
    if (h->batch_work) BBC_CUDA(cudaFree(h->batch_work));
    h->batch_work = nullptr;
    const int64_t nmax = std::max(max_n, h->batch_nmax);
    h->batch_nmax = 0;
    const bool want_split = split || h->batch_split;
    const int ctas = batched_ctas(h->device);
    BBC_CUDA(cudaMalloc(&h->batch_work, batched_workspace_bytes(nmax, ctas, want_split)));
    BBC_CUDA(batched_upload_programs());
    BBC_CUDA(batched_cluster_probe(h->device, &h->batch_cl));
    h->batch_ctas = ctas;
    h->batch_nmax = nmax;
    h->batch_split = want_split;
  }
  if (!h->one_dev) BBC_CUDA(cudaMalloc(&h->one_dev, ONE_DESC_BYTES));
  if (!h->one_host) BBC_CUDA(cudaMallocHost(&h->one_host, ONE_DESC_BYTES));
  return BBC_OK;
}

int bbc_select_certified(const double* norms3, double u, int scheme, int* m, int* s) {
  if (!norms3 || !m || !s || !valid_u(u)) return fail(BBC_INVALID_ARG, "bad certified selection query");
  if (scheme != BBC_SCHEME_NEW && scheme != BBC_SCHEME_PS) return fail(BBC_INVALID_ARG, "unknown scheme");
  for (int k = 0; k < 3; ++k)
    if (!std::isfinite(norms3[k]) || norms3[k] < 0) return fail(BBC_NONFINITE_INPUT, "norm not finite");
  const double alpha2 = std::fmax(std::sqrt(norms3[1]), std::cbrt(norms3[2]));
  const int *deg, *prod;
  const int cnt = scheme_degrees(scheme, &deg, &prod);
  int bm = -1, bs = 0, bc = 1 << 30;
  for (int i = 0; i < cnt; ++i) {
    const double th = theta_cached(deg[i], u);
    const int si = std::min(least_squarings(norms3[0], th), least_squarings(alpha2, th));
    const int cost = prod[i] + si;
    if (cost < bc || (cost == bc && si < bs)) { bc = cost; bm = deg[i]; bs = si; }
  }
  *m = bm;
  *s = bs;
  return BBC_OK;
}

int bbc_batch_set_selector(bbc_handle h, const float* dParams, int hid, int out, int S, const float* hMu,
                           const float* hSd) {
  int rc = begin(h);
  if (rc) return rc;
  if (!dParams || !hMu || !hSd || hid < 1 || hid > 256 || S < 1 || out != 6 * S || out > 256)
    return fail(BBC_INVALID_ARG, "bad selector network (hid <= 256, out = 6 S <= 256)");
  std::lock_guard<std::mutex> lk(h->mu);
  BatchSelector sel = {};
  sel.mode = 1;
  sel.params = dParams;
  sel.hid = hid;
  sel.out = out;
  sel.S = S;
  for (int i = 0; i < 5; ++i) { sel.mu[i] = hMu[i]; sel.sd[i] = hSd[i]; }
  h->selector = sel;
  return BBC_OK;
}

int bbc_selector_data_batched(bbc_handle h, const void* const* dA, const int64_t* dNs, int64_t count, int dtype,
                              float* dFeat, double* dNorms, void* stream, bbc_info* dInfo) {
  int rc = begin(h);
  if (rc) return rc;
  if (count < 0 || (count > 0 && (!dA || !dNs || !dFeat || !dNorms))) return fail(BBC_INVALID_ARG, "bad data arguments");
  if (dtype != BBC_DTYPE_F32 && dtype != BBC_DTYPE_F64) return fail(BBC_INVALID_ARG, "unknown dtype");
  if (count == 0) return BBC_OK;
  std::lock_guard<std::mutex> lk(h->mu);
  if (!h->batch_work) return fail(BBC_INVALID_ARG, "call bbc_batch_reserve first");
  static const int deg[6] = {1, 2, 4, 8, 12, 18};
  double theta[6];
  for (int i = 0; i < 6; ++i) theta[i] = theta_cached(deg[i], std::ldexp(1.0, -53));
  BatchSelector sel = {};
  sel.mode = 3;
  sel.feat_out = dFeat;
  sel.norms_out = dNorms;
  cudaStream_t st = (cudaStream_t)stream;
  LaunchScope scope(h, BBC_KERNEL_BATCHED, st);
  const cudaError_t e = batched_launch(dA, nullptr, dNs, count, h->batch_nmax, dtype, theta, h->batch_work,
                                       h->batch_ctas, dInfo, st, &sel, false, 0xFFFFFFFFu, &h->batch_cl);
  if (e != cudaSuccess) return cuda_fail(e, "selector data launch");
  return BBC_OK;
}

int bbc_batch_order(const int64_t* hNs, int64_t count, int64_t* hOrder) {
  if (count < 0 || (count > 0 && (!hNs || !hOrder))) return fail(BBC_INVALID_ARG, "bad batch order arguments");
  std::vector<int64_t> idx((size_t)count);
  for (int64_t i = 0; i < count; ++i) idx[(size_t)i] = i;
  std::stable_sort(idx.begin(), idx.end(), [&](int64_t a, int64_t b) { return hNs[a] > hNs[b]; });
  for (int64_t i = 0; i < count; ++i) hOrder[i] = idx[(size_t)i];
  return BBC_OK;
}

}  // extern "C"

namespace {
int expm_batched_impl(bbc_handle h, const void* const* dA, const void* const* dB, const int64_t* dNs, int64_t count,
                      void* const* dOut, int dtype, double tol, int flags, void* stream, bbc_info* dInfo) {
  int rc = begin(h);
  if (rc) return rc;
  if (count < 0 || (count > 0 && (!dA || !dNs || !dOut))) return fail(BBC_INVALID_ARG, "bad batched arguments");
  if (dtype != BBC_DTYPE_F32 && dtype != BBC_DTYPE_F64) return fail(BBC_INVALID_ARG, "unknown dtype");
  const double u = tol > 0 ? tol : std::ldexp(1.0, -53);
  if (!valid_u(u)) return fail(BBC_INVALID_ARG, "tol out of range [2^-60, 2^-5]");
  if ((rc = check_flags(flags))) return rc;
  if ((rc = batch_flags_ok(flags))) return rc;
  if (count == 0) return BBC_OK;
  std::lock_guard<std::mutex> lk(h->mu);
  return batched_locked(h, dA, dB, dNs, count, dOut, dtype, u, flags, (cudaStream_t)stream, dInfo);
}

// The launch of bbc_expm_batched / bbc_expm_apply_batched once the arguments are
// checked; the caller holds h->mu.
int batched_locked(bbc_handle h, const void* const* dA, const void* const* dB, const int64_t* dNs, int64_t count,
                   void* const* dOut, int dtype, double u, int flags, cudaStream_t st, bbc_info* dInfo) {
  const bool split = (flags & BBC_PREC_MASK) == BBC_PREC_OZAKI;
  if (!h->batch_work) return fail(BBC_INVALID_ARG, "call bbc_batch_reserve first");
  if (split && !h->batch_split) return fail(BBC_INVALID_ARG, "reserve with BBC_PREC_OZAKI first");
  static const int deg[6] = {1, 2, 4, 8, 12, 18};
  double theta[6];
  for (int i = 0; i < 6; ++i) theta[i] = theta_cached(deg[i], u);
  BatchSelector sel = {};
  const BatchSelector* psel = nullptr;
  if (flags & BBC_SELECT_LEARNED) {
    if (h->selector.mode != 1) return fail(BBC_INVALID_ARG, "no network installed (bbc_batch_set_selector)");
    sel = h->selector;
    psel = &sel;
  } else if (flags & BBC_SELECT_ALPHA) {
    sel.mode = 2;
    psel = &sel;
  }
  LaunchScope scope(h, BBC_KERNEL_BATCHED, st);
  const int ctas = (h->batch_grid > 0 && h->batch_grid <= h->batch_ctas) ? h->batch_grid : h->batch_ctas;
  const int scheme = flags & BBC_SCHEME_MASK;
  const int pade = scheme == BBC_SCHEME_PADE ? 1 : scheme == BBC_SCHEME_PADE26 ? 2 : 0;
  const double theta_pade[2] = {theta_cached(-10, u), theta_cached(-26, u)};
  const cudaError_t e = batched_launch(dA, dOut, dNs, count, h->batch_nmax, dtype, theta, h->batch_work,
                                       ctas, dInfo, st, psel, split, h->batch_split_mask, &h->batch_cl, dB,
                                       pade, theta_pade, &h->batch_shapes);
  if (e != cudaSuccess) return cuda_fail(e, "batched launch");
  return BBC_OK;
}
}  // namespace

extern "C" {

int bbc_expm_batched(bbc_handle h, const void* const* dA, const int64_t* dNs, int64_t count, void* const* dOut,
                     int dtype, double tol, int flags, void* stream, bbc_info* dInfo) {
  return expm_batched_impl(h, dA, nullptr, dNs, count, dOut, dtype, tol, flags, stream, dInfo);
}

int bbc_expm_apply_batched(bbc_handle h, const void* const* dA, const void* const* dB, const int64_t* dNs,
                           int64_t count, void* const* dOut, int dtype, double tol, int flags, void* stream,
                           bbc_info* dInfo) {
  if (count > 0 && !dB) return fail(BBC_INVALID_ARG, "bad batched arguments");
  return expm_batched_impl(h, dA, dB, dNs, count, dOut, dtype, tol, flags, stream, dInfo);
}

}  // extern "C"
