/*
 * expm_oracle.c -- plain, slow FP64 CPU oracle for scaling-and-squaring exp(A)
 * with the reduced-product Taylor scheme of Bader, Blanes and Casas,
 * "An improved algorithm to compute the exponential of a matrix"
 * (arXiv:1710.10989).
 *
 * TEST INFRASTRUCTURE. Only the test suite, the smoke entry point and the
 * benchmark's CPU-baseline leg load this library. The CUDA library shares no
 * code, header, table or generator with it, and neither calls the other.
 *
 * Conventions: every matrix is square, n x n, row-major, IEEE double. The file
 * is compiled with -ffp-contract=off, so every a*b+c rounds twice, in exactly
 * the order written. There is no blocking or fusion: a product is the triple
 * loop of its definition (the k sum runs in ascending k for every entry), a
 * linear combination is evaluated term by term in the order the paper writes.
 *
 * Parity status: every function here is pinned by the CPU test suite
 * (closed forms, exact-rational Taylor sums, symbolic coefficient checks,
 * invariants, an independent library). Nothing here is "parity unpinned".
 */
#include <math.h>
#ifdef _OPENMP
#include <omp.h>
#endif
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
  int m;          /* Taylor degree, or 2m for Pade */
  int s;          /* number of squarings */
  int products;   /* dense n x n products performed (LU/solve not counted) */
  int status;     /* 0 ok, 1 invalid argument, 2 non-finite input, 3 overflow */
  double norm1;   /* ||A||_1 of the input */
} orc_info;

enum { ORC_NEW = 0, ORC_PS = 1, ORC_PADE26 = 2, ORC_PADE = 3 };

/* ------------------------------------------------------------------------ */
/* Planted mistakes for the negative-control tests (0 = none). Each code     */
/* makes exactly one plausible error; the pins must catch every one.         */
/* ------------------------------------------------------------------------ */
static int g_mutation = 0;
void orc_set_mutation(int code) { g_mutation = code; }
int orc_get_mutation(void) { return g_mutation; }

/* threads the products run on (the CPU-baseline leg reports it) */
int orc_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

/* cap on those threads (n >= 1), for single-core and all-core timings */
void orc_set_num_threads(int n) {
#ifdef _OPENMP
  if (n >= 1) omp_set_num_threads(n);
#else
  (void)n;
#endif
}

static long long g_products = 0;
long long orc_product_count(void) { return g_products; }
void orc_reset_product_count(void) { g_products = 0; }

/* ------------------------------------------------------------------------ */
/* Dense building blocks                                                     */
/* ------------------------------------------------------------------------ */

/* C = A * B, c_ij = sum_k a_ik b_kj with k ascending. The i-k-j loop order
 * keeps that summation order per entry and streams rows of B. */
void orc_gemm(int64_t n, const double* A, const double* B, double* C) {
  g_products++;
  const int transposed = (g_mutation == 5);
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; ++i) {
    double* c = C + i * n;
    for (int64_t j = 0; j < n; ++j) c[j] = 0.0;
    for (int64_t k = 0; k < n; ++k) {
      const double a = A[i * n + k];
      if (!transposed) {
        const double* b = B + k * n;
        for (int64_t j = 0; j < n; ++j) c[j] += a * b[j];
      } else {
        for (int64_t j = 0; j < n; ++j) c[j] += a * B[j * n + k];
      }
    }
  }
}

/* ||A||_1 = max_j sum_i |a_ij| (maximum absolute column sum). */
double orc_norm1(int64_t n, const double* A) {
  double best = 0.0;
  for (int64_t j = 0; j < n; ++j) {
    double col = 0.0;
    for (int64_t i = 0; i < n; ++i)
      col += fabs(g_mutation == 9 ? A[j * n + i] : A[i * n + j]);
    if (col > best || isnan(col)) best = col;
    if (isnan(col)) break;
  }
  return best;
}

/* Y = c0*I + c1*M1 + ... + ck*Mk (terms added left to right). NULL matrices
 * with a zero coefficient are skipped. */
static void lincomb(int64_t n, double* Y, double c0, int k, const double* c,
                    const double* const* M) {
  const int64_t nn = n * n;
  for (int64_t e = 0; e < nn; ++e) Y[e] = 0.0;
  for (int64_t i = 0; i < n; ++i) Y[i * n + i] = c0;
  for (int t = 0; t < k; ++t) {
    if (M[t] == NULL) continue;
    for (int64_t e = 0; e < nn; ++e) Y[e] += c[t] * M[t][e];
  }
}

/* Y += M (elementwise) */
static void addto(int64_t n, double* Y, const double* M) {
  const int64_t nn = n * n;
  for (int64_t e = 0; e < nn; ++e) Y[e] += M[e];
}

static double* mat(int64_t n) { return (double*)malloc((size_t)(n * n) * sizeof(double)); }

/* ------------------------------------------------------------------------ */
/* Coefficients of the reduced-product scheme (Section 3)                    */
/* ------------------------------------------------------------------------ */

/* T8, eq. (Algorithm83eA): closed forms in sqrt(177) with x3 = 2/3. */
typedef struct { double x1, x2, x3, x4, x5, x6, x7, y0, y1, y2; } t8_coef;
static t8_coef t8_coefficients(void) {
  const double r = sqrt(177.0);
  t8_coef c;
  c.x3 = 2.0 / 3.0;
  c.x1 = c.x3 * (1.0 + r) / 88.0;
  c.x2 = (1.0 + r) / 352.0 * c.x3;
  c.x4 = (-271.0 + 29.0 * r) / (315.0 * c.x3);
  c.x5 = 11.0 * (-1.0 + r) / (1260.0 * c.x3);
  c.x6 = 11.0 * (-9.0 + r) / (5040.0 * c.x3);
  c.x7 = (89.0 - r) / (5040.0 * c.x3 * c.x3);
  c.y0 = 1.0;
  c.y1 = 1.0;
  c.y2 = (857.0 - 58.0 * r) / 630.0;
  if (g_mutation == 3) { double t = c.x5; c.x5 = c.x6; c.x6 = t; }
  return c;
}

/* T12, eq. (poly12): a[i][j-1] = a_{i,j}, i = power of A (0..3), j = 1..4.
 * Decimal strings as printed, converted to the nearest double. */
static const char* const T12_A[4][4] = {
    {"9.0198e-16", "5.31597895759871264183", "0.18188869982170434744", "-2.0861320e-13"},
    {"0.46932117595418237389", "1.19926790417132231573", "0.05502798439925399070", "-0.13181061013830184015"},
    {"-0.20099424927047284052", "0.01179296240992997031", "0.09351590770535414968", "-0.02027855540589259079"},
    {"-0.04623946134063071740", "0.01108844528519167989", "0.00610700528898058230", "-0.00675951846863086359"}};

/* T18, eq. (poly.18): a_{i,1} for i = 0..3, and b_{i,j} for i in {0,1,2,3,6},
 * j = 1..4 (row index 4 below holds i = 6). */
static const char* const T18_A1[4] = {"0", "-0.100365581030144620", "-0.0080292464824115696",
                                      "-0.0008921384980457299"};
static const char* const T18_B[5][4] = {
    {"0", "-10.967639605296206259", "-0.0904316832390810561", "0"},
    {"0.39784974949964507614", "1.68015813878906197182", "-0.0676404519071381907", "0"},
    {"1.36783778460411719922", "0.05717798464788655127", "0.06759613017704596460", "-0.0923364619367118592"},
    {"0.49828962252538267755", "-0.0069821012248805208", "0.02955525704293155274", "-0.0169364939002081717"},
    {"-0.0006378981945947233", "0.00003349750170860705", "-0.0000139180257516060", "-0.0000140086798182036"}};

static double dec(const char* s) { return strtod(s, NULL); }

static void t12_coefficients(double a[4][4]) {
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 4; ++j) a[i][j] = dec(T12_A[i][j]);
  if (g_mutation == 1) a[0][3] = 0.0;
}

static void t18_coefficients(double a1[4], double b[5][4]) {
  for (int i = 0; i < 4; ++i) a1[i] = dec(T18_A1[i]);
  for (int i = 0; i < 5; ++i)
    for (int j = 0; j < 4; ++j) b[i][j] = dec(T18_B[i][j]);
  if (g_mutation == 2) b[4][2] = -b[4][2];
}

/* Export the coefficient tables in the order documented per id:
 *   1: T8  -> x1..x7, y0, y1, y2                      (10 values)
 *   2: T12 -> a_{i,j}, i = 0..3 outer, j = 1..4 inner  (16 values)
 *   3: T18 -> a_{i,1} (i = 0..3), then b_{i,j}, i in {0,1,2,3,6} outer, j inner (4 + 20)
 *   4: Pade p_13 coefficients b_0..b_13               (14 values)
 *   5: Pade p_5 coefficients b_0..b_5                 (6 values)
 * Returns the number of values written. */
static void pade_coefficients(int m, double* b);
int orc_coeffs(int which, double* out) {
  if (which == 1) {
    t8_coef c = t8_coefficients();
    const double v[10] = {c.x1, c.x2, c.x3, c.x4, c.x5, c.x6, c.x7, c.y0, c.y1, c.y2};
    memcpy(out, v, sizeof v);
    return 10;
  }
  if (which == 2) {
    double a[4][4];
    t12_coefficients(a);
    for (int i = 0; i < 4; ++i)
      for (int j = 0; j < 4; ++j) out[i * 4 + j] = a[i][j];
    return 16;
  }
  if (which == 3) {
    double a1[4], b[5][4];
    t18_coefficients(a1, b);
    for (int i = 0; i < 4; ++i) out[i] = a1[i];
    for (int i = 0; i < 5; ++i)
      for (int j = 0; j < 4; ++j) out[4 + i * 4 + j] = b[i][j];
    return 24;
  }
  if (which == 4) { pade_coefficients(13, out); return 14; }
  if (which == 5) { pade_coefficients(5, out); return 6; }
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Taylor polynomial T_m(X), reduced-product scheme (Section 3)              */
/* Returns the number of products used, or -1 for an unsupported degree.     */
/* ------------------------------------------------------------------------ */
int orc_taylor_new(int64_t n, const double* X, int m, double* T) {
  const long long p0 = g_products;
  const int64_t nn = n * n;
  if (m == 1) { /* T1 = I + X */
    const double c[1] = {1.0};
    const double* M[1] = {X};
    lincomb(n, T, 1.0, 1, c, M);
  } else if (m == 2) { /* T2 = I + X + X^2/2 */
    double* A2 = mat(n);
    orc_gemm(n, X, X, A2);
    const double c[2] = {1.0, 0.5};
    const double* M[2] = {X, A2};
    lincomb(n, T, 1.0, 2, c, M);
    free(A2);
  } else if (m == 4) { /* T4 = I + X + A2 (I/2 + X/6 + A2/24) */
    double *A2 = mat(n), *P = mat(n), *Q = mat(n);
    orc_gemm(n, X, X, A2);
    const double cp[2] = {1.0 / 6.0, 1.0 / 24.0};
    const double* Mp[2] = {X, A2};
    lincomb(n, P, 0.5, 2, cp, Mp);
    orc_gemm(n, A2, P, Q);
    const double c[1] = {1.0};
    const double* M[1] = {X};
    lincomb(n, T, 1.0, 1, c, M);
    addto(n, T, Q);
    free(A2); free(P); free(Q);
  } else if (m == 8) { /* eq. (Algorithm83eA) */
    const t8_coef k = t8_coefficients();
    double *A2 = mat(n), *L = mat(n), *A4 = mat(n), *P = mat(n), *Q = mat(n), *A8 = mat(n);
    orc_gemm(n, X, X, A2);                         /* A2 = A^2 */
    { const double c[2] = {k.x1, k.x2}; const double* M[2] = {X, A2}; lincomb(n, L, 0.0, 2, c, M); }
    orc_gemm(n, A2, L, A4);                        /* A4 = A2 (x1 A + x2 A2) */
    { const double c[2] = {k.x3, 1.0}; const double* M[2] = {A2, A4}; lincomb(n, P, 0.0, 2, c, M); }
    { const double c[3] = {k.x5, k.x6, k.x7}; const double* M[3] = {X, A2, A4}; lincomb(n, Q, k.x4, 3, c, M); }
    orc_gemm(n, P, Q, A8);                         /* A8 = (x3 A2 + A4)(x4 I + x5 A + x6 A2 + x7 A4) */
    { const double c[2] = {k.y1, k.y2}; const double* M[2] = {X, A2}; lincomb(n, T, k.y0, 2, c, M); }
    addto(n, T, A8);                               /* T8 = y0 I + y1 A + y2 A2 + A8 */
    free(A2); free(L); free(A4); free(P); free(Q); free(A8);
  } else if (m == 12) { /* eq. (poly12) */
    double a[4][4];
    t12_coefficients(a);
    double *A2 = mat(n), *A3 = mat(n), *B[4], *A6 = mat(n), *P = mat(n), *Q = mat(n);
    orc_gemm(n, X, X, A2);
    orc_gemm(n, A2, X, A3);
    for (int j = 0; j < 4; ++j) {
      B[j] = mat(n);
      const double c[3] = {a[1][j], a[2][j], a[3][j]};
      const double* M[3] = {X, A2, A3};
      lincomb(n, B[j], a[0][j], 3, c, M);          /* B_j = a0j I + a1j A + a2j A2 + a3j A3 */
    }
    orc_gemm(n, B[3], B[3], A6);                   /* B4^2 */
    addto(n, A6, B[2]);                            /* A6 = B3 + B4^2 */
    memcpy(P, B[1], (size_t)nn * sizeof(double));
    addto(n, P, A6);                               /* B2 + A6 */
    orc_gemm(n, P, A6, Q);                         /* (B2 + A6) A6 */
    memcpy(T, B[0], (size_t)nn * sizeof(double));
    addto(n, T, Q);                                /* T12 = B1 + (B2 + A6) A6 */
    for (int j = 0; j < 4; ++j) free(B[j]);
    free(A2); free(A3); free(A6); free(P); free(Q);
  } else if (m == 18) { /* eq. (poly.18) */
    double a1[4], b[5][4];
    t18_coefficients(a1, b);
    double *A2 = mat(n), *A3 = mat(n), *A6 = mat(n), *B1 = mat(n), *Bj[4];
    double *A9 = mat(n), *P = mat(n), *Q = mat(n);
    orc_gemm(n, X, X, A2);
    orc_gemm(n, A2, X, A3);
    orc_gemm(n, A3, A3, A6);
    { const double c[3] = {a1[1], a1[2], a1[3]}; const double* M[3] = {X, A2, A3}; lincomb(n, B1, a1[0], 3, c, M); }
    for (int j = 0; j < 4; ++j) { /* B_{j+2} uses b_{.,j+1} */
      Bj[j] = mat(n);
      const double c[4] = {b[1][j], b[2][j], b[3][j], b[4][j]};
      const double* M[4] = {X, A2, A3, A6};
      lincomb(n, Bj[j], b[0][j], 4, c, M);
    }
    /* Bj[0] = B2, Bj[1] = B3, Bj[2] = B4, Bj[3] = B5 */
    orc_gemm(n, B1, Bj[3], A9);                    /* B1 B5 */
    if (g_mutation != 4) addto(n, A9, Bj[2]);      /* A9 = B1 B5 + B4 */
    memcpy(P, Bj[1], (size_t)nn * sizeof(double));
    addto(n, P, A9);                               /* B3 + A9 */
    orc_gemm(n, P, A9, Q);                         /* (B3 + A9) A9 */
    memcpy(T, Bj[0], (size_t)nn * sizeof(double));
    addto(n, T, Q);                                /* T18 = B2 + (B3 + A9) A9 */
    for (int j = 0; j < 4; ++j) free(Bj[j]);
    free(A2); free(A3); free(A6); free(B1); free(A9); free(P); free(Q);
  } else {
    return -1;
  }
  return (int)(g_products - p0);
}

/* ------------------------------------------------------------------------ */
/* Taylor polynomial T_m(X), Paterson-Stockmeyer (eq. poli9 and its         */
/* evident siblings). c_i = 1/i!.                                           */
/* ------------------------------------------------------------------------ */
static double inv_fact(int i) {
  double f = 1.0;
  for (int k = 2; k <= i; ++k) f *= (double)k;
  return 1.0 / f;
}

/* Horner in the block power Y = A_q: T = h_0 + (h_1 + (... + (h_{r-1} + c_top Y) Y ...) Y) Y,
 * h_i = sum_{k=0}^{q-1} c_{q i + k} A_k, with A_0 = I, A_1 = X and pw[k] = A_k. */
static void ps_horner(int64_t n, const double* const* pw, int q, int r, int top, double* T) {
  const int64_t nn = n * n;
  double *H = mat(n), *acc = mat(n), *tmp = mat(n);
  /* innermost: h_{r-1} + c_top Y */
  {
    double c[8]; const double* M[8]; int t = 0;
    for (int k = 1; k < q; ++k) { c[t] = inv_fact(q * (r - 1) + k); M[t] = pw[k]; ++t; }
    c[t] = (g_mutation == 6) ? 0.0 : inv_fact(top); M[t] = pw[q]; ++t;
    lincomb(n, acc, inv_fact(q * (r - 1)), t, c, M);
  }
  for (int i = r - 2; i >= 0; --i) {
    orc_gemm(n, acc, pw[q], tmp);                  /* (...) Y */
    double c[8]; const double* M[8]; int t = 0;
    for (int k = 1; k < q; ++k) { c[t] = inv_fact(q * i + k); M[t] = pw[k]; ++t; }
    lincomb(n, H, inv_fact(q * i), t, c, M);       /* h_i */
    for (int64_t e = 0; e < nn; ++e) acc[e] = H[e] + tmp[e];
  }
  memcpy(T, acc, (size_t)nn * sizeof(double));
  free(H); free(acc); free(tmp);
}

int orc_taylor_ps(int64_t n, const double* X, int m, double* T) {
  const long long p0 = g_products;
  if (m == 1 || m == 2) return orc_taylor_new(n, X, m, T); /* same forms, Table 3 */
  double *A2 = mat(n), *A3 = NULL, *A4 = NULL;
  orc_gemm(n, X, X, A2);
  if (m == 4) {          /* (c0 I + c1 A) + (c2 I + c3 A + c4 A2) A2 */
    const double* pw[3] = {NULL, X, A2};
    ps_horner(n, pw, 2, 2, 4, T);
  } else if (m == 6) {   /* g0 + (g1 + (g2 + c6 A2) A2) A2, g_i = c_{2i} I + c_{2i+1} A */
    const double* pw[3] = {NULL, X, A2};
    ps_horner(n, pw, 2, 3, 6, T);
  } else if (m == 9 || m == 12) { /* f0 + (f1 + (f2 + c9 A3) A3) A3, f_i = sum_k c_{3i+k} A_k */
    A3 = mat(n);
    orc_gemm(n, A2, X, A3);
    const double* pw[4] = {NULL, X, A2, A3};
    ps_horner(n, pw, 3, m / 3, m, T);
  } else if (m == 16) {  /* g0 + (g1 + (g2 + (g3 + c16 A4) A4) A4) A4 */
    A3 = mat(n); A4 = mat(n);
    orc_gemm(n, A2, X, A3);
    orc_gemm(n, A2, A2, A4);
    const double* pw[5] = {NULL, X, A2, A3, A4};
    ps_horner(n, pw, 4, 4, 16, T);
  } else {
    free(A2);
    return -1;
  }
  free(A2); free(A3); free(A4);
  return (int)(g_products - p0);
}

/* ------------------------------------------------------------------------ */
/* Diagonal Pade r_2m (eq. 24, eq. pade10, eq. pade26)                       */
/* ------------------------------------------------------------------------ */

/* p_m(x) = sum_j b_j x^j, b_j = (2m-j)! m! / ((2m)! (m-j)! j!), b_0 = 1. */
static void pade_coefficients(int m, double* b) {
  for (int j = 0; j <= m; ++j) {
    /* product form of the ratio of factorials, all in double */
    double v = 1.0;
    for (int k = 0; k < j; ++k) v *= (double)(m - k) / (double)(2 * m - k);
    v *= inv_fact(j);
    b[j] = v;
  }
}

/* Solve P R = Q in place for R (Q overwritten), by Gaussian elimination with
 * partial pivoting applied to all n right-hand sides. Returns 0, or 1 if P is
 * singular to working precision. */
static int lu_solve(int64_t n, double* P, double* Q, double* R) {
  for (int64_t k = 0; k < n; ++k) {
    int64_t piv = k;
    double best = fabs(P[k * n + k]);
    for (int64_t i = k + 1; i < n && g_mutation != 13; ++i)   /* planted (13): no row interchanges */
      if (fabs(P[i * n + k]) > best) { best = fabs(P[i * n + k]); piv = i; }
    if (best == 0.0) return 1;
    if (piv != k) {
      for (int64_t j = 0; j < n; ++j) {
        double t = P[k * n + j]; P[k * n + j] = P[piv * n + j]; P[piv * n + j] = t;
        t = Q[k * n + j]; Q[k * n + j] = Q[piv * n + j]; Q[piv * n + j] = t;
      }
    }
    const double d = P[k * n + k];
#pragma omp parallel for schedule(static)
    for (int64_t i = k + 1; i < n; ++i) {
      const double l = P[i * n + k] / d;
      P[i * n + k] = l;
      for (int64_t j = k + 1; j < n; ++j) P[i * n + j] -= l * P[k * n + j];
      for (int64_t j = 0; j < n; ++j) Q[i * n + j] -= l * Q[k * n + j];
    }
  }
  for (int64_t i = n - 1; i >= 0; --i) {
    double* r = R + i * n;
    for (int64_t j = 0; j < n; ++j) r[j] = Q[i * n + j];
    for (int64_t t = i + 1; t < n; ++t) {
      const double p = P[i * n + t];
      const double* rt = R + t * n;
      for (int64_t j = 0; j < n; ++j) r[j] -= p * rt[j];
    }
    const double d = P[i * n + i];
    for (int64_t j = 0; j < n; ++j) r[j] /= d;
  }
  return 0;
}

/* The same solve as a public entry (the comparator's solve, tested on its own):
 * R = P^-1 Q for n x n P and Q (both overwritten: P by its LU factors, Q by
 * the eliminated right-hand sides). Returns 0, or 1 if P is singular. */
int orc_solve(int64_t n, double* P, double* Q, double* R) { return lu_solve(n, P, Q, R); }

/* R = r_2m(X) for 2m in {10, 26}. Returns the number of products, -1 for an
 * unsupported order, -2 if the denominator is singular. */
int orc_pade(int64_t n, const double* X, int two_m, double* R) {
  const long long p0 = g_products;
  const int64_t nn = n * n;
  double b[14];
  double *U = mat(n), *V = mat(n), *A2 = mat(n), *A4 = mat(n), *W = mat(n);
  int rc = 0;
  if (two_m == 10) {
    pade_coefficients(5, b);
    orc_gemm(n, X, X, A2);
    orc_gemm(n, A2, A2, A4);
    { const double c[2] = {b[5], b[3]}; const double* M[2] = {A4, A2}; lincomb(n, W, b[1], 2, c, M); }
    orc_gemm(n, X, W, U);                                        /* u5 */
    { const double c[2] = {b[4], b[2]}; const double* M[2] = {A4, A2}; lincomb(n, V, b[0], 2, c, M); } /* v5 */
  } else if (two_m == 26) {
    pade_coefficients(13, b);
    double *A6 = mat(n), *Z = mat(n);
    orc_gemm(n, X, X, A2);
    orc_gemm(n, A2, A2, A4);
    orc_gemm(n, A2, A4, A6);
    { const double c[3] = {b[13], b[11], b[9]}; const double* M[3] = {A6, A4, A2}; lincomb(n, W, 0.0, 3, c, M); }
    orc_gemm(n, A6, W, Z);                                       /* A6 (b13 A6 + b11 A4 + b9 A2) */
    { const double c[3] = {b[7], b[5], b[3]}; const double* M[3] = {A6, A4, A2}; lincomb(n, W, b[1], 3, c, M); }
    addto(n, Z, W);
    orc_gemm(n, X, Z, U);                                        /* u13 */
    { const double c[3] = {b[12], b[10], b[8]}; const double* M[3] = {A6, A4, A2}; lincomb(n, W, 0.0, 3, c, M); }
    orc_gemm(n, A6, W, V);                                       /* A6 (b12 A6 + b10 A4 + b8 A2) */
    { const double c[3] = {b[6], b[4], b[2]}; const double* M[3] = {A6, A4, A2}; lincomb(n, W, b[0], 3, c, M); }
    addto(n, V, W);                                              /* v13 */
    free(A6); free(Z);
  } else {
    rc = -1;
  }
  if (rc == 0) {
    const int swap = (g_mutation == 7);
    for (int64_t e = 0; e < nn; ++e) {           /* W = -u + v, A2 = u + v */
      const double u = U[e], v = V[e];
      W[e] = swap ? (u + v) : (-u + v);
      A2[e] = swap ? (-u + v) : (u + v);
    }
    if (lu_solve(n, W, A2, R)) rc = -2;
  }
  free(U); free(V); free(A2); free(A4); free(W);
  return rc < 0 ? rc : (int)(g_products - p0);
}

/* ------------------------------------------------------------------------ */
/* Selection of (m, s) (eq. theta with Tables 1-3)                          */
/* theta[d] holds theta_d(u) for Taylor degree d (schemes NEW, PS) or for   */
/* Pade order d = 2m (scheme PADE26 reads theta[26], scheme PADE theta[10]  */
/* and theta[26]); length >= 27.                                            */
/* ------------------------------------------------------------------------ */
static const int NEW_DEG[6] = {1, 2, 4, 8, 12, 18};
static const int NEW_PI[6] = {0, 1, 2, 3, 4, 5};   /* Table 3, new decomposition */
static const int PS_DEG[7] = {1, 2, 4, 6, 9, 12, 16};
static const int PS_PI[7] = {0, 1, 2, 3, 4, 5, 6}; /* Table 3, Paterson-Stockmeyer */
/* r_10 and r_26 (eq. pade10, eq. pade26): 3 and 6 products, each plus one     */
/* solve, whose cost is the same for both and so cannot change the choice      */
static const int PADE_DEG[2] = {10, 26};
static const int PADE_PI[2] = {3, 6};

/* smallest s >= 0 with norm / 2^s <= th */
static int min_squarings(double norm, double th) {
  if (!(norm > th)) return 0;
  int s = (int)ceil(log2(norm / th));
  if (s < 0) s = 0;
  while (ldexp(norm, -s) > th) ++s;
  while (s > 0 && ldexp(norm, -(s - 1)) <= th) --s;
  return s;
}

int orc_select(double norm, int scheme, const double* theta, int* m_out, int* s_out) {
  if (!isfinite(norm) || norm < 0.0) return 2;
  if (scheme == ORC_PADE26) {
    *m_out = 26;
    *s_out = min_squarings(norm, theta[26]);
  } else {
    const int* deg = scheme == ORC_NEW ? NEW_DEG : scheme == ORC_PS ? PS_DEG : PADE_DEG;
    static const int PADE_PI_MUT[2] = {6, 6};  /* planted (12): r_10 charged as r_26 */
    const int* pi = scheme == ORC_NEW ? NEW_PI : scheme == ORC_PS ? PS_PI
                    : (g_mutation == 12 ? PADE_PI_MUT : PADE_PI);
    const int cnt = scheme == ORC_NEW ? 6 : scheme == ORC_PS ? 7 : 2;
    int best_m = -1, best_s = 0, best_cost = 1 << 30;
    for (int i = 0; i < cnt; ++i) {
      const int s = min_squarings(norm, theta[deg[i]]);
      const int cost = pi[i] + s;
      if (cost < best_cost || (cost == best_cost && s < best_s)) {
        best_cost = cost; best_m = deg[i]; best_s = s;
      }
    }
    *m_out = best_m;
    *s_out = best_s;
  }
  if (g_mutation == 8 && *s_out > 0) *s_out -= 1;
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Certified selection with power norms (an extension the paper does not    */
/* use; it cites the work it comes from). A choice (m, s) is certified when */
/* the paper's bound holds, ||A||_1 / 2^s <= theta_m, or when               */
/* alpha_2 / 2^s <= theta_m with alpha_2 = max(||A^2||^(1/2), ||A^3||^(1/3)), */
/* which bounds the same backward-error majorant because its Taylor series  */
/* starts at degree m + 1 >= 2.                                             */
/* ------------------------------------------------------------------------ */

/* out[0..3] = ||A||_1, ||A^2||_1, ||A^3||_1, ||A^4||_1 (oracle products). */
void orc_power_norms(int64_t n, const double* A, double* out) {
  double *A2 = mat(n), *A3 = mat(n), *A4 = mat(n);
  orc_gemm(n, A, A, A2);
  orc_gemm(n, A2, A, A3);
  orc_gemm(n, A2, A2, A4);
  out[0] = orc_norm1(n, A);
  out[1] = orc_norm1(n, A2);
  out[2] = orc_norm1(n, A3);
  out[3] = orc_norm1(n, A4);
  free(A2); free(A3); free(A4);
}

/* Minimal products + s over (m, s) certified by either bound; ties to the
 * smaller s. norms = {||A||, ||A^2||, ||A^3||}. */
int orc_select_certified(const double* norms, int scheme, const double* theta, int* m_out, int* s_out) {
  for (int k = 0; k < 3; ++k)
    if (!isfinite(norms[k]) || norms[k] < 0.0) return 2;
  const double alpha2 = fmax(sqrt(norms[1]), cbrt(norms[2]));
  const int* deg = scheme == ORC_NEW ? NEW_DEG : PS_DEG;
  const int* pi = scheme == ORC_NEW ? NEW_PI : PS_PI;
  const int cnt = scheme == ORC_NEW ? 6 : 7;
  int best_m = -1, best_s = 0, best_cost = 1 << 30;
  for (int i = 0; i < cnt; ++i) {
    const int s1 = min_squarings(norms[0], theta[deg[i]]);
    const int s2 = min_squarings(alpha2, theta[deg[i]]);
    const int s = s1 < s2 ? s1 : s2;
    const int cost = pi[i] + s;
    if (cost < best_cost || (cost == best_cost && s < best_s)) {
      best_cost = cost; best_m = deg[i]; best_s = s;
    }
  }
  *m_out = best_m;
  *s_out = best_s;
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Scaling and squaring, eq. (eses)                                          */
/* m_force > 0 together with s_force >= 0 bypasses the selection (for       */
/* comparing two implementations at the same (m, s)).                        */
/* ------------------------------------------------------------------------ */
int orc_expm(int64_t n, const double* A, double* out, int scheme, const double* theta,
             int m_force, int s_force, orc_info* info) {
  orc_info loc;
  if (info == NULL) info = &loc;
  memset(info, 0, sizeof *info);
  if (n <= 0 || A == NULL || out == NULL) { info->status = 1; return 1; }
  const int64_t nn = n * n;
  for (int64_t e = 0; e < nn; ++e)
    if (!isfinite(A[e])) { info->status = 2; return 2; }
  const long long p0 = g_products;
  info->norm1 = orc_norm1(n, A);
  int m, s;
  if (m_force > 0 && s_force >= 0) {
    m = m_force; s = s_force;
  } else {
    if (theta == NULL) { info->status = 1; return 1; }
    const int rc = orc_select(info->norm1, scheme, theta, &m, &s);
    if (rc) { info->status = rc; return rc; }
  }
  info->m = m;
  info->s = s;
  double* X = mat(n);
  for (int64_t e = 0; e < nn; ++e) X[e] = ldexp(A[e], -s);   /* X = A / 2^s */
  int rc;
  if (scheme == ORC_NEW) rc = orc_taylor_new(n, X, m, out);
  else if (scheme == ORC_PS) rc = orc_taylor_ps(n, X, m, out);
  else rc = orc_pade(n, X, m, out);
  free(X);
  if (rc < 0) { info->status = 1; return 1; }
  double* tmp = mat(n);
  for (int k = 0; k < s; ++k) {                                /* T <- T^2, s times */
    orc_gemm(n, out, out, tmp);
    memcpy(out, tmp, (size_t)nn * sizeof(double));
  }
  free(tmp);
  info->products = (int)(g_products - p0);
  for (int64_t e = 0; e < nn; ++e)
    if (!isfinite(out[e])) { info->status = 3; return 3; }
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Upper triangular A (Section 5, after Al-Mohy and Higham): the diagonal     */
/* and first superdiagonal of exp(2^-q A) are known in closed form, and the   */
/* computed ones are replaced by them before every squaring and in the        */
/* result. For the 2 x 2 block [[l1, t], [0, l2]] of 2^-q A,                  */
/*   exp = [[e^l1, t (e^l2 - e^l1)/(l2 - l1)], [0, e^l2]],                    */
/* the divided difference written as e^((l1+l2)/2) sinh(d)/d, d = (l2-l1)/2,  */
/* which has no cancellation (and is e^l1 when l1 = l2).                      */
/* ------------------------------------------------------------------------ */
static double exp_superdiag(double l1, double l2, double t) {
  const double d = 0.5 * (l2 - l1);
  const double sinhc = (d == 0.0) ? 1.0 : sinh(d) / d;
  if (g_mutation == 10) return t * exp(l1);                 /* planted: divided difference dropped */
  return t * exp(0.5 * (l1 + l2)) * sinhc;
}

/* Overwrite diag and first superdiagonal of T with those of exp(2^-q A). */
static void replace_exact(int64_t n, const double* A, int q, double* T) {
  for (int64_t i = 0; i < n; ++i) T[i * n + i] = exp(ldexp(A[i * n + i], -q));
  for (int64_t i = 0; i + 1 < n; ++i)
    T[i * n + i + 1] = exp_superdiag(ldexp(A[i * n + i], -q), ldexp(A[(i + 1) * n + i + 1], -q),
                                     ldexp(A[i * n + i + 1], -q));
}

/* 1 if every entry strictly below the diagonal is zero. */
int orc_is_upper(int64_t n, const double* A) {
  for (int64_t i = 1; i < n; ++i)
    for (int64_t j = 0; j < i; ++j)
      if (A[i * n + j] != 0.0) return 0;
  return 1;
}

/* As orc_expm for an upper triangular A (status 1 otherwise), with the exact
 * diagonal and superdiagonal put in after the polynomial and after every
 * squaring. The products are the plain ones: their lower triangles come out
 * exactly zero. */
int orc_expm_upper(int64_t n, const double* A, double* out, int scheme, const double* theta,
                   int m_force, int s_force, orc_info* info) {
  orc_info loc;
  if (info == NULL) info = &loc;
  memset(info, 0, sizeof *info);
  if (n <= 0 || A == NULL || out == NULL || !orc_is_upper(n, A)) { info->status = 1; return 1; }
  const int64_t nn = n * n;
  for (int64_t e = 0; e < nn; ++e)
    if (!isfinite(A[e])) { info->status = 2; return 2; }
  const long long p0 = g_products;
  info->norm1 = orc_norm1(n, A);
  int m, s;
  if (m_force > 0 && s_force >= 0) {
    m = m_force; s = s_force;
  } else {
    if (theta == NULL) { info->status = 1; return 1; }
    const int rc = orc_select(info->norm1, scheme, theta, &m, &s);
    if (rc) { info->status = rc; return rc; }
  }
  info->m = m;
  info->s = s;
  double* X = mat(n);
  for (int64_t e = 0; e < nn; ++e) X[e] = ldexp(A[e], -s);
  int rc;
  if (scheme == ORC_NEW) rc = orc_taylor_new(n, X, m, out);
  else if (scheme == ORC_PS) rc = orc_taylor_ps(n, X, m, out);
  else rc = orc_pade(n, X, m, out);
  free(X);
  if (rc < 0) { info->status = 1; return 1; }
  replace_exact(n, A, s, out);                                 /* T = exp(2^-s A) on the two diagonals */
  double* tmp = mat(n);
  for (int k = 1; k <= s; ++k) {                               /* T <- T^2, then exact diagonals of exp(2^(k-s) A) */
    orc_gemm(n, out, out, tmp);
    memcpy(out, tmp, (size_t)nn * sizeof(double));
    if (!(g_mutation == 11 && k == s)) replace_exact(n, A, s - k, out);   /* planted (11): last one skipped */
  }
  free(tmp);
  info->products = (int)(g_products - p0);
  for (int64_t e = 0; e < nn; ++e)
    if (!isfinite(out[e])) { info->status = 3; return 3; }
  return 0;
}
