// gemm_ozaki.cu -- placeholder until the tcgen05 split-precision product lands.
#include "internal.h"

namespace bbc {
size_t ozaki_workspace_bytes(int64_t, int) { return 0; }
bool ozaki_supported(int64_t) { return false; }
cudaError_t gemm_ozaki(const double*, const double*, int64_t, double, const Epilogue&, int, void*,
                       cudaStream_t) {
  return cudaErrorNotSupported;
}
}  // namespace bbc
