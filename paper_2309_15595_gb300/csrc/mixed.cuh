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
// V[:, 0:ncols]; W (ld ldw) is the ping-pong buffer. autotune: pick the raster
// order of the tensor-core kernel by timing on the first call for a shape.
// Returns a chase_status.
int mixed_filter(cudaStream_t s, int64_t N, const double2* A, int64_t lda, double2* V,
                 int64_t ldv, int64_t ncols, const int32_t* degs, double c, const double* al,
                 const double* be, double2* W, int64_t ldw, MixedWork& w, bool autotune = true);

// One problem of a grouped filter (several problems' filters in the same
// kernel launches, one launch per degree step): the arguments of mixed_filter.
struct MixedGroupItem {
  int64_t N;
  const double2* A;
  int64_t lda;
  double2* V;
  int64_t ldv;
  int64_t ncols;
  const int32_t* degs;  // host, even, ascending
  double c;
  const double* al;     // host, dmax + 1 coefficients
  const double* be;
  MixedWork* w;
};
// Table of per-step, per-problem launch entries (device + pinned host).
struct MixedGroupTable {
  void* dev = nullptr;
  void* host = nullptr;
  size_t capacity = 0;  // entries
};
// Entries a grouped filter of these items needs (sum of their largest degrees).
size_t mixed_group_entries(int count, const MixedGroupItem* items);
cudaError_t mixed_group_reserve(MixedGroupTable& t, size_t entries);
void mixed_group_free(MixedGroupTable& t);
// All items' filters on stream s: their degree steps as one CUDA graph of
// grouped launches (step i covers every problem whose largest degree is >= i).
// Each problem's result equals mixed_filter on it alone. Synchronises s.
// *launches (may be null) receives the number of grouped launches.
int mixed_filter_grouped(cudaStream_t s, int count, const MixedGroupItem* items,
                         MixedGroupTable& t, int* launches);

}  // namespace chase
