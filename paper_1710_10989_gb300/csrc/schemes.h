// schemes.h -- Taylor-polynomial evaluation programs (host side).
//
// A program is a short list of steps; each step is one dense product
// v = alpha * (P Q) followed by the fused epilogue outputs (internal.h), or a
// product-free linear combination. The programs encode the paper's
// evaluation sequences with X = 2^-s A folded in: a term "c X" is stored as
// the term "(c 2^-s) A", and the first products carry alpha = 2^-2s / 2^-s, so
// no scaled copy of A is ever formed (scaling by a power of two is exact).
#pragma once
#include <vector>

#include "internal.h"

namespace bbc {

constexpr int SL_A = 100;  // the input A
constexpr int SL_T = 101;  // the polynomial's result
constexpr int NUM_WORK_SLOTS = 10;  // W0..W9 (W9 is the squaring ping-pong buffer)
constexpr int SL_SQ = 9;

struct TermS {
  int slot;
  double c;
  int sp = -1;   // batched path: power of 2^-s the coefficient carries (-1: derive from the slot)
};
struct OutS {
  int dst;
  double cv, cI;
  int nt;
  TermS t[MAX_TERMS];
};
struct StepS {
  int P, Q;        // operand slots; P < 0 means no product (v = 0)
  double alpha;
  int ap = -1;     // batched path: alpha = (2^-s)^ap (-1: derive from the operands)
  int nout;
  OutS o[MAX_OUT];
};
struct Program {
  int m;
  int products;
  std::vector<StepS> steps;
};

// scheme: BBC_SCHEME_NEW, BBC_SCHEME_PS (Taylor degree m) or BBC_SCHEME_PADE26
// (m = 26: the numerator / denominator products of eq. pade26, leaving -u + v in
// W8 and u + v in the result slot for the solve); false for a degree the scheme
// does not have.
bool make_program(int scheme, int m, int s, Program* out);

// T12 / T18 of the reduced-product scheme for a caller that already holds the
// UNSCALED powers A^2 and A^3 (computed to certify the choice of (m, s)): the
// programs start after those two products and carry 2^-s powers explicitly
// (X^2 = 2^-2s A^2, X^3 = 2^-3s A^3). *a2_slot / *a3_slot tell where the
// powers must be. Returns false for other degrees.
bool make_prefilled_program(int m, Program* out, int* a2_slot, int* a3_slot);

// Degrees and product counts (Table 3) of a scheme.
int scheme_degrees(int scheme, const int** deg, const int** products);

}  // namespace bbc
