// slices.h -- the split-precision workspace shared by slices.cu (which fills it)
// and gemm_ozaki.cu (whose product kernel reads it).
#pragma once
#include <stdint.h>

namespace bbc {
namespace slices {

constexpr int PAD = 128;                      // planes are padded to a multiple of 128 rows / columns
constexpr unsigned int STATUS_NONFINITE = 1u;  // bit of the handle's status word

inline int64_t padded(int64_t N) { return (N + PAD - 1) / PAD * PAD; }

// Layout of the workspace: 256 reserved bytes, erow[Rp], fcol[Rp], fexp[Rp], the
// deflated diagonals pdiag[Rp], qdiag[Rp], then the P planes and the Q^T planes,
// each k x Rp x Rp BF16.
struct OzLayout {
  int64_t Rp;
  int* erow;       // row scale exponents of P
  int* fcol;       // column scale exponents of Q
  int* fexp;       // column maxima of Q's biased exponents (scratch)
  double* pdiag;   // P's diagonal, taken out before slicing
  double* qdiag;   // Q's diagonal
  uint16_t* Ps;    // [k][Rp][Rp] digits of P's rows
  uint16_t* Qs;    // [k][Rp][Rp] digits of Q's columns (Q^T rows)
};
inline OzLayout layout(void* work, int64_t N, int slices) {
  OzLayout L;
  L.Rp = padded(N);
  uint8_t* w = static_cast<uint8_t*>(work);
  L.erow = reinterpret_cast<int*>(w + 256);
  L.fcol = L.erow + L.Rp;
  L.fexp = L.fcol + L.Rp;
  size_t off = 256 + 3 * (size_t)L.Rp * sizeof(int);
  off = (off + 255) / 256 * 256;
  L.pdiag = reinterpret_cast<double*>(w + off);
  L.qdiag = L.pdiag + L.Rp;
  off += 2 * (size_t)L.Rp * sizeof(double);
  off = (off + 255) / 256 * 256;
  L.Ps = reinterpret_cast<uint16_t*>(w + off);
  L.Qs = L.Ps + (size_t)slices * L.Rp * L.Rp;
  return L;
}

}  // namespace slices
}  // namespace bbc
