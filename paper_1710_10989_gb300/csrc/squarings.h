// squarings.h -- the squaring count of the selection rule, shared by the host
// selection (api.cu) and the persistent batched kernel (batched.cu).
#pragma once
#include <cuda_runtime.h>

#include <math.h>

namespace bbc {

// Squarings a bound needs (eq. theta): the least s >= 0 with norm / 2^s <= th, for
// a finite th > 0. With 2^a <= norm < 2^(a+1) and 2^b <= th < 2^(b+1), that s is
// a - b or a - b + 1, so it is found from the exponents in at most two exact
// halvings, whatever the magnitudes. A norm that is not finite (an overflowed
// power norm) certifies nothing: it gets a count larger than any selection takes.
constexpr int SQUARINGS_NONE = 1 << 20;
__host__ __device__ inline int least_squarings(double norm, double th) {
  if (!(norm <= 1.7976931348623157e308)) return SQUARINGS_NONE;  // +inf or NaN
  if (!(norm > th)) return 0;
  int s = ilogb(norm) - ilogb(th) - 1;
  if (s < 0) s = 0;
  for (int k = 0; k < 4 && ldexp(norm, -s) > th; ++k) ++s;
  return s;
}

}  // namespace bbc
