// Placeholder until the tensor-core filter lands: the mixed mode reports
// CHASE_ERR_INVALID_ARG.
#include "mixed.cuh"

namespace chase {
cudaError_t mixed_alloc(MixedWork& w, int64_t N, int64_t ne) {
  w.N = N;
  w.ne = ne;
  return cudaErrorNotSupported;
}
void mixed_free(MixedWork& w) { (void)w; }
int mixed_filter(cudaStream_t, int64_t, const double2*, int64_t, double2*, int64_t, int64_t,
                 const int32_t*, double, const double*, const double*, double2*, int64_t,
                 MixedWork&) {
  return CHASE_ERR_INVALID_ARG;
}
}  // namespace chase
