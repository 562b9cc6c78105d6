// Householder QR on the device (the fallback of Alg. 4), see householder.cu.
#pragma once

#include "common.cuh"

namespace chase {

constexpr int kHouseholderNB = 64;  // panel width

struct HouseholderWork {
  double2* Vp = nullptr;     // N x NB explicit reflectors of one panel
  double2* T = nullptr;      // one NB x NB block-reflector factor per panel
  double2* S = nullptr;      // NB x NB: V^H V of the panel
  double2* W = nullptr;      // NB x ne: V^H C
  double2* W2 = nullptr;     // NB x ne: op(T) V^H C
  double2* dots = nullptr;   // per-block partial dot products
  double* norms = nullptr;   // per-block partial squared norms
  double* beta = nullptr;    // diagonal of R (real)
  double2* tau = nullptr;    // reflector coefficients
  double2* scale = nullptr;  // 1 / (alpha - beta) of the current column
  int* bad = nullptr;        // a non-finite reflector was met
  double2* gws = nullptr;    // split-K workspace of the NB-row Gram products
  size_t gws_elems = 0;
  int64_t N = 0, ne = 0;
};

cudaError_t householder_alloc(HouseholderWork& w, int64_t N, int64_t ne);
void householder_free(HouseholderWork& w);
// X (m x n, ldx; m >= n) is overwritten by the reflectors and R; Q (m x n, ldq,
// not aliasing X) receives the orthonormal factor with diag(R) real positive.
// Synchronises; CHASE_ERR_QR_BREAKDOWN if the input held non-finite values.
int householder_qr(cudaStream_t s, int64_t m, int64_t n, double2* X, int64_t ldx, double2* Q,
                   int64_t ldq, HouseholderWork& w);

}  // namespace chase
