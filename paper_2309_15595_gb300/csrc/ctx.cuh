// Internal: the solver context shared by the C ABI translation units.
#pragma once

#include <vector>

#include "common.cuh"
#include "householder.cuh"
#include "mixed.cuh"
#include "ozaki.cuh"
#include "../../include/chase.h"

struct chase_ctx {
  chase_params p;
  cudaStream_t stream;
  int device = 0;               // current device at chase_create
  int64_t N, ne;
  double2* V2 = nullptr;        // N x ne, ld N  (C2 of Alg. 2)
  double2* W = nullptr;         // N x ne, ld N  (B of Alg. 2, filter ping-pong)
  double2* G = nullptr;         // ne x ne, ld ne
  double2* Yeig = nullptr;      // ne x ne, ld ne
  double2* gram_ws = nullptr;
  size_t gram_ws_elems = 0;
  double2* dinv = nullptr;
  int* info = nullptr;
  double* resid_partial = nullptr;
  double* dscal = nullptr;
  int* perm_d = nullptr;
  double* host = nullptr;       // pinned: 2 ne + 16 doubles
  chase::JacobiWork jw{};
  chase::LanczosWork lw{};
  chase::MixedWork mw{};
  chase::OzakiWork ow{};
  chase::HouseholderWork hw{};  // Householder QR fallback of Alg. 4
  double* oz_partial = nullptr;  // residual partials of the tensor-core path (32-row tiles)
  bool oz_a_valid = false;       // digits of the current solve's A are prepared
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  double2* gw = nullptr;         // gradient workspace (grown on first use)
  size_t gw_elems = 0;
  double* gd = nullptr;          // gradient per-column scalars
  size_t gd_elems = 0;
};

namespace chase {
// Digits of A for the tensor-core FP64 products (no-op without fp64_tensor or
// while a solve holds valid digits).
int ctx_prepare_a(chase_ctx* c, const double2* A, int64_t lda);
// Eq. 1 coefficients alpha_i, beta_i (i = 1..dmax, gamma_i = c) of the scaled
// or unscaled recurrence; al and be get dmax + 1 entries.
void cheb_coefficients(int dmax, double c, double e, double mu1, bool scaled,
                       std::vector<double>& al, std::vector<double>& be);
}  // namespace chase
