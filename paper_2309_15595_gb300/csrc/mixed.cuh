// Reduced-precision filter on the tensor cores (split-BF16 x3, FP32
// accumulation in tensor memory). Declarations used by the host driver.
#pragma once

#include "common.cuh"

namespace chase {

struct MixedWork {
  void* Ahi = nullptr;   // planar BF16 hi/lo copies of A (see mixed.cu)
  void* Alo = nullptr;
  void* Yhi = nullptr;   // planar BF16 hi/lo copies of the filter operand (2 buffers)
  void* Ylo = nullptr;
  void* maps = nullptr;  // TMA tensor maps of the planes (pinned host)
  int* err = nullptr;    // device: nonzero when a pipeline wait expired
  void* S32 = nullptr;   // two FP32 recurrence-state buffers, N x ne complex each
  int64_t N = 0, ne = 0;
};

cudaError_t mixed_alloc(MixedWork& w, int64_t N, int64_t ne);
void mixed_free(MixedWork& w);
// Filter of Eq. 1 with coefficients al[i], be[i] (i = 1..degs[ncols-1]) on
// V[:, 0:ncols]; W (ld ldw) is the ping-pong buffer. Returns a chase_status.
int mixed_filter(cudaStream_t s, int64_t N, const double2* A, int64_t lda, double2* V,
                 int64_t ldv, int64_t ncols, const int32_t* degs, double c, const double* al,
                 const double* be, double2* W, int64_t ldw, MixedWork& w);

}  // namespace chase
