// schemes.cu -- coefficient tables and evaluation programs of the Taylor schemes.
//
// Reduced-product scheme, Section 3 of Bader, Blanes, Casas (arXiv:1710.10989):
//   T8  in 3 products, eq. (Algorithm83eA), closed forms in sqrt(177), x3 = 2/3;
//   T12 in 4 products, eq. (poly12), 16 numeric coefficients a_{i,j};
//   T18 in 5 products, eq. (poly.18), coefficients a_{i,1} and b_{i,j};
//   T1, T2, T4 in 0, 1, 2 products (Horner-like, as Paterson-Stockmeyer).
// Paterson-Stockmeyer comparator, eq. (poli9): T9, T16 as printed, and the
// analogous T4, T6 (blocks in A2) and T12 (blocks in A3).
#include <cmath>

#include "bbcexpm.h"
#include "schemes.h"

namespace bbc {
namespace {

// eq. (poly12): T12A[i][j-1] = a_{i,j}, i = power of A (0..3), j = 1..4.
const double T12A[4][4] = {
    {9.0198e-16, 5.31597895759871264183, 0.18188869982170434744, -2.0861320e-13},
    {0.46932117595418237389, 1.19926790417132231573, 0.05502798439925399070, -0.13181061013830184015},
    {-0.20099424927047284052, 0.01179296240992997031, 0.09351590770535414968, -0.02027855540589259079},
    {-0.04623946134063071740, 0.01108844528519167989, 0.00610700528898058230, -0.00675951846863086359}};

// eq. (poly.18): a_{i,1}, i = 0..3.
const double T18A1[4] = {0.0, -0.100365581030144620, -0.0080292464824115696, -0.0008921384980457299};
// eq. (poly.18): T18B[r][j-1] = b_{i,j} with i = {0, 1, 2, 3, 6}[r], j = 1..4.
const double T18B[5][4] = {
    {0.0, -10.967639605296206259, -0.0904316832390810561, 0.0},
    {0.39784974949964507614, 1.68015813878906197182, -0.0676404519071381907, 0.0},
    {1.36783778460411719922, 0.05717798464788655127, 0.06759613017704596460, -0.0923364619367118592},
    {0.49828962252538267755, -0.0069821012248805208, 0.02955525704293155274, -0.0169364939002081717},
    {-0.0006378981945947233, 0.00003349750170860705, -0.0000139180257516060, -0.0000140086798182036}};

const int NEW_DEG[6] = {1, 2, 4, 8, 12, 18};
const int NEW_PROD[6] = {0, 1, 2, 3, 4, 5};
const int PS_DEG[7] = {1, 2, 4, 6, 9, 12, 16};
const int PS_PROD[7] = {0, 1, 2, 3, 4, 5, 6};
const int PADE_DEG[2] = {10, 26};
const int PADE_PROD[2] = {3, 6};

double inv_factorial(int k) {
  double f = 1.0;
  for (int i = 2; i <= k; ++i) f *= i;
  return 1.0 / f;
}

// Small builder so that programs read like the paper's sequences.
struct Out {
  OutS o{};
  Out(int dst, double cv, double cI = 0.0) { o.dst = dst; o.cv = cv; o.cI = cI; o.nt = 0; }
  Out& t(int slot, double c) {
    if (c != 0.0) o.t[o.nt++] = TermS{slot, c};
    return *this;
  }
};
struct Step {
  StepS s{};
  Step(int P, int Q, double alpha) { s.P = P; s.Q = Q; s.alpha = alpha; s.nout = 0; }
  Step& out(const Out& o) { s.o[s.nout++] = o.o; return *this; }
};

void add(Program* p, const Step& st) {
  p->steps.push_back(st.s);
  if (st.s.P >= 0) p->products++;
}

enum { W0 = 0, W1, W2, W3, W4, W5, W6, W7, W8 };

// Paterson-Stockmeyer Horner tail: given block power Y = A_q in slot `ys`,
// powers A (scaled by sig), A2 in W0 and A3 in W1 (if q > 3), and the innermost
// block already in slot `acc`, emit the remaining r - 1 Horner products.
void ps_tail(Program* p, int q, int r, int ys, int acc, int spare, double sig) {
  for (int i = r - 2; i >= 0; --i) {
    const int dst = (i == 0) ? SL_T : spare;
    Out o(dst, 1.0, inv_factorial(q * i));
    o.t(SL_A, inv_factorial(q * i + 1) * sig);
    if (q >= 3) o.t(W0, inv_factorial(q * i + 2));
    if (q >= 4) o.t(W1, inv_factorial(q * i + 3));
    add(p, Step(acc, ys, 1.0).out(o));
    const int t = acc; acc = spare; spare = t;
  }
}

}  // namespace

bool make_prefilled_program(int m, Program* p, int* a2_slot, int* a3_slot) {
  p->m = m;
  p->products = 0;
  p->steps.clear();
  auto term = [](Out& o, int slot, double c, int sp) -> Out& {
    if (c != 0.0) { o.o.t[o.o.nt] = TermS{slot, c}; o.o.t[o.o.nt].sp = sp; o.o.nt++; }
    return o;
  };
  auto zero_powers = [](Step& st) {
    for (int o = 0; o < st.s.nout; ++o)
      for (int t = 0; t < st.s.o[o].nt; ++t) st.s.o[o].t[t].sp = 0;
    st.s.ap = 0;
  };
  if (m == 18) {  // A^2 in W0, A^3 in W1
    *a2_slot = W0;
    *a3_slot = W1;
    Step st(W1, W1, 1.0);  // v = (2^-3s A^3)^2 = X6
    st.s.ap = 6;
    Out b1(W2, 0.0, T18A1[0]);
    term(b1, SL_A, T18A1[1], 1); term(b1, W0, T18A1[2], 2); term(b1, W1, T18A1[3], 3);
    st.out(b1);
    for (int j = 0; j < 4; ++j) {
      Out b(W3 + j, T18B[4][j], T18B[0][j]);
      term(b, SL_A, T18B[1][j], 1); term(b, W0, T18B[2][j], 2); term(b, W1, T18B[3][j], 3);
      st.out(b);
    }
    add(p, st);
    Step s4 = Step(W2, W6, 1.0).out(Out(W7, 1.0).t(W5, 1.0)).out(Out(W8, 1.0).t(W5, 1.0).t(W4, 1.0));
    zero_powers(s4);
    add(p, s4);
    Step s5 = Step(W8, W7, 1.0).out(Out(SL_T, 1.0).t(W3, 1.0));
    zero_powers(s5);
    add(p, s5);
    return true;
  }
  if (m == 12) {  // A^2 in W0, A^3 in W1; B_1..B_4 -> W2..W5
    *a2_slot = W0;
    *a3_slot = W1;
    Step st(-1, -1, 0.0);  // B_j = a0j I + a1j X + a2j X2 + a3j X3, no product
    st.s.ap = 0;
    for (int j = 0; j < 4; ++j) {
      Out b(W2 + j, 0.0, T12A[0][j]);
      term(b, SL_A, T12A[1][j], 1); term(b, W0, T12A[2][j], 2); term(b, W1, T12A[3][j], 3);
      st.out(b);
    }
    add(p, st);
    // A6 = B3 + B4^2 -> W6;  B2 + A6 -> W7;  T12 = B1 + (B2 + A6) A6
    Step s3 = Step(W5, W5, 1.0).out(Out(W6, 1.0).t(W4, 1.0)).out(Out(W7, 1.0).t(W4, 1.0).t(W3, 1.0));
    zero_powers(s3);
    add(p, s3);
    Step s4 = Step(W7, W6, 1.0).out(Out(SL_T, 1.0).t(W2, 1.0));
    zero_powers(s4);
    add(p, s4);
    return true;
  }
  return false;
}

int scheme_degrees(int scheme, const int** deg, const int** products) {
  if (scheme == BBC_SCHEME_PS) { *deg = PS_DEG; *products = PS_PROD; return 7; }
  if (scheme == BBC_SCHEME_PADE26) { *deg = PADE_DEG + 1; *products = PADE_PROD + 1; return 1; }
  if (scheme == BBC_SCHEME_PADE) { *deg = PADE_DEG; *products = PADE_PROD; return 2; }
  *deg = NEW_DEG; *products = NEW_PROD; return 6;
}

bool make_program(int scheme, int m, int s, Program* p) {
  p->m = m;
  p->products = 0;
  p->steps.clear();
  const double sig = std::ldexp(1.0, -s);     // X = sig * A
  const double sig2 = sig * sig;
  if ((scheme == BBC_SCHEME_PADE26 || scheme == BBC_SCHEME_PADE) && m == 10) {  // eq. (pade10)
    double b[6];                               // p_5(x) = sum b_j x^j, eq. (24), b_0 = 1
    for (int j = 0; j <= 5; ++j) {
      double v = inv_factorial(j);
      for (int t = 0; t < j; ++t) v *= (double)(5 - t) / (double)(10 - t);
      b[j] = v;
    }
    add(p, Step(SL_A, SL_A, sig2).out(Out(W0, 1.0)));                             // A2
    add(p, Step(W0, W0, 1.0)                                                       // A4, and
               .out(Out(W1, b[5], b[1]).t(W0, b[3]))                               // b5 A4 + b3 A2 + b1 I
               .out(Out(W2, b[4], b[0]).t(W0, b[2])));                             // v5 = b4 A4 + b2 A2 + b0 I
    add(p, Step(SL_A, W1, sig)                                                     // u5 = A (...), and
               .out(Out(W8, -1.0).t(W2, 1.0))                                      // -u5 + v5
               .out(Out(SL_T, 1.0).t(W2, 1.0)));                                   // u5 + v5
    return true;                                                                   // then (-u + v) r = u + v
  }
  if (scheme == BBC_SCHEME_PADE26 || scheme == BBC_SCHEME_PADE) {  // eq. (pade26): r_26
    if (m != 26) return false;
    double b[14];                              // p_13(x) = sum b_j x^j, eq. (24), b_0 = 1
    for (int j = 0; j <= 13; ++j) {
      double v = inv_factorial(j);
      for (int t = 0; t < j; ++t) v *= (double)(13 - t) / (double)(26 - t);
      b[j] = v;
    }
    add(p, Step(SL_A, SL_A, sig2).out(Out(W0, 1.0)));                             // A2
    add(p, Step(W0, W0, 1.0).out(Out(W1, 1.0)));                                  // A4
    add(p, Step(W0, W1, 1.0)                                                       // A6, and
               .out(Out(W2, 1.0))
               .out(Out(W3, b[13]).t(W1, b[11]).t(W0, b[9]))                       // b13 A6 + b11 A4 + b9 A2
               .out(Out(W4, b[12]).t(W1, b[10]).t(W0, b[8])));                     // b12 A6 + b10 A4 + b8 A2
    add(p, Step(W2, W3, 1.0).out(Out(W5, 1.0, b[1]).t(W2, b[7]).t(W1, b[5]).t(W0, b[3])));
    add(p, Step(SL_A, W5, sig).out(Out(W6, 1.0)));                                // u13 = A (...)
    add(p, Step(W2, W4, 1.0).out(Out(W7, 1.0, b[0]).t(W2, b[6]).t(W1, b[4]).t(W0, b[2])));  // v13
    add(p, Step(-1, -1, 0.0).out(Out(W8, 0.0).t(W6, -1.0).t(W7, 1.0))             // -u + v
               .out(Out(SL_T, 0.0).t(W6, 1.0).t(W7, 1.0)));                       // u + v
    return true;                                                                   // then (-u + v) r = u + v
  }
  if (m == 1) {                                // T1 = I + X
    add(p, Step(-1, -1, 0.0).out(Out(SL_T, 0.0, 1.0).t(SL_A, sig)));
    return true;
  }
  if (m == 2) {                                // T2 = I + X + X^2/2
    add(p, Step(SL_A, SL_A, sig2).out(Out(SL_T, 0.5, 1.0).t(SL_A, sig)));
    return true;
  }
  if (scheme == BBC_SCHEME_NEW) {
    if (m == 4) {                              // T4 = I + X + A2 (I/2 + X/6 + A2/24)
      add(p, Step(SL_A, SL_A, sig2).out(Out(W0, 1.0)).out(Out(W1, 1.0 / 24, 0.5).t(SL_A, sig / 6)));
      add(p, Step(W0, W1, 1.0).out(Out(SL_T, 1.0, 1.0).t(SL_A, sig)));
      return true;
    }
    if (m == 8) {                              // eq. (Algorithm83eA)
      const double r = std::sqrt(177.0);
      const double x3 = 2.0 / 3.0;
      const double x1 = x3 * (1.0 + r) / 88.0, x2 = x3 * (1.0 + r) / 352.0;
      const double x4 = (-271.0 + 29.0 * r) / (315.0 * x3);
      const double x5 = 11.0 * (-1.0 + r) / (1260.0 * x3);
      const double x6 = 11.0 * (-9.0 + r) / (5040.0 * x3);
      const double x7 = (89.0 - r) / (5040.0 * x3 * x3);
      const double y0 = 1.0, y1 = 1.0, y2 = (857.0 - 58.0 * r) / 630.0;
      // A2 = X^2; also x1 X + x2 A2
      add(p, Step(SL_A, SL_A, sig2).out(Out(W0, 1.0)).out(Out(W1, x2).t(SL_A, x1 * sig)));
      // A4 = A2 (x1 X + x2 A2); emits x3 A2 + A4 and x4 I + x5 X + x6 A2 + x7 A4
      add(p, Step(W0, W1, 1.0)
                 .out(Out(W2, 1.0).t(W0, x3))
                 .out(Out(W3, x7, x4).t(SL_A, x5 * sig).t(W0, x6)));
      // A8 = (x3 A2 + A4)(x4 I + ...); T8 = y0 I + y1 X + y2 A2 + A8
      add(p, Step(W2, W3, 1.0).out(Out(SL_T, 1.0, y0).t(SL_A, y1 * sig).t(W0, y2)));
      return true;
    }
    if (m == 12) {                             // eq. (poly12)
      add(p, Step(SL_A, SL_A, sig2).out(Out(W0, 1.0)));           // A2
      Step st(W0, SL_A, sig);                                       // v = A3; B_j -> W1..W4
      for (int j = 0; j < 4; ++j)
        st.out(Out(W1 + j, T12A[3][j], T12A[0][j]).t(SL_A, T12A[1][j] * sig).t(W0, T12A[2][j]));
      add(p, st);
      // A6 = B3 + B4^2 -> W5;  B2 + A6 -> W6
      add(p, Step(W4, W4, 1.0).out(Out(W5, 1.0).t(W3, 1.0)).out(Out(W6, 1.0).t(W3, 1.0).t(W2, 1.0)));
      // T12 = B1 + (B2 + A6) A6
      add(p, Step(W6, W5, 1.0).out(Out(SL_T, 1.0).t(W1, 1.0)));
      return true;
    }
    if (m == 18) {                             // eq. (poly.18)
      add(p, Step(SL_A, SL_A, sig2).out(Out(W0, 1.0)));           // A2
      add(p, Step(W0, SL_A, sig).out(Out(W1, 1.0)));              // A3
      // v = A6 = A3^2; B1 -> W2, B2..B5 -> W3..W6
      Step st(W1, W1, 1.0);
      st.out(Out(W2, 0.0, T18A1[0]).t(SL_A, T18A1[1] * sig).t(W0, T18A1[2]).t(W1, T18A1[3]));
      for (int j = 0; j < 4; ++j)
        st.out(Out(W3 + j, T18B[4][j], T18B[0][j]).t(SL_A, T18B[1][j] * sig).t(W0, T18B[2][j]).t(W1, T18B[3][j]));
      add(p, st);
      // A9 = B1 B5 + B4 -> W7;  B3 + A9 -> W8
      add(p, Step(W2, W6, 1.0).out(Out(W7, 1.0).t(W5, 1.0)).out(Out(W8, 1.0).t(W5, 1.0).t(W4, 1.0)));
      // T18 = B2 + (B3 + A9) A9
      add(p, Step(W8, W7, 1.0).out(Out(SL_T, 1.0).t(W3, 1.0)));
      return true;
    }
    return false;
  }
  if (scheme == BBC_SCHEME_PS) {
    auto c = inv_factorial;
    if (m == 4 || m == 6) {                    // blocks in A2: g_i = c_{2i} I + c_{2i+1} X
      const int r = m / 2;
      add(p, Step(SL_A, SL_A, sig2)
                 .out(Out(W0, 1.0))
                 .out(Out(W1, c(m), c(m - 2)).t(SL_A, c(m - 1) * sig)));
      ps_tail(p, 2, r, W0, W1, W2, sig);
      return true;
    }
    if (m == 9 || m == 12) {                   // blocks in A3: f_i = sum_{k<3} c_{3i+k} A_k
      const int r = m / 3;
      add(p, Step(SL_A, SL_A, sig2).out(Out(W0, 1.0)));           // A2
      add(p, Step(W0, SL_A, sig)
                 .out(Out(W1, 1.0))                                   // A3
                 .out(Out(W2, c(m), c(m - 3)).t(SL_A, c(m - 2) * sig).t(W0, c(m - 1))));
      ps_tail(p, 3, r, W1, W2, W3, sig);
      return true;
    }
    if (m == 16) {                             // blocks in A4: g_i = sum_{k<4} c_{4i+k} A_k
      add(p, Step(SL_A, SL_A, sig2).out(Out(W0, 1.0)));           // A2
      add(p, Step(W0, SL_A, sig).out(Out(W1, 1.0)));              // A3
      add(p, Step(W0, W0, 1.0)
                 .out(Out(W2, 1.0))                                   // A4
                 .out(Out(W3, c(16), c(12)).t(SL_A, c(13) * sig).t(W0, c(14)).t(W1, c(15))));
      ps_tail(p, 4, 4, W2, W3, W4, sig);
      return true;
    }
    return false;
  }
  return false;
}

}  // namespace bbc
