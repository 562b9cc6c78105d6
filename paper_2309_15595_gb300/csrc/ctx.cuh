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
  double2* QRt = nullptr;        // N x ne: iterate of the tensor-core triangular solve
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

// One solve of Alg. 2 as resumable phases, so that a batch of problems can
// advance in lockstep and share the filter launches (chase_solve_batch);
// chase_solve runs the same phases in a loop.
struct SolveState {
  chase_ctx* c = nullptr;
  const double2* A = nullptr;
  int64_t lda = 0;
  double2* C = nullptr;
  int64_t ldv = 0;
  double* ritz = nullptr;
  double* resid = nullptr;
  chase_stats st{};
  cudaEvent_t t_start = nullptr, t_end = nullptr;
  long long launches = 0;  // kernels launched by this solve's phases (on any thread)
  double b_sup = 0, mu_1 = 0, mu_ne = 0, norm_est = 0, tol_abs = 0, cc = 0, ee = 0;
  double rmax_prev = 1e300, cond = 0;
  std::vector<int32_t> degs;
  std::vector<double> rz, rs;
  int64_t locked = 0;
  int iter = 1;
  bool mixed = false;
  SolveState() = default;
  SolveState(const SolveState&) = delete;
  SolveState& operator=(const SolveState&) = delete;
  ~SolveState();
};
// Validation, digits of A, Lanczos bounds (Alg. 2 first line).
int solve_begin(SolveState& S, chase_ctx* c, const double2* A, int64_t lda, double2* C,
                int64_t ldv, const double2* Q0, int64_t ldq, double* ritz, double* resid);
// locked < nev and iter <= max_iter (Alg. 2 loop test)
bool solve_active(const SolveState& S);
// Bounds update, degreeOpt and sort of the active columns, CondEst.
int solve_prepare(SolveState& S);
// The filter of the active columns with this problem's own launches.
int solve_filter(SolveState& S);
// MatVec accounting of one filter phase (solve_filter calls it).
void solve_count_filter(SolveState& S);
// QR, restore of the locked columns, Rayleigh-Ritz, residuals, locking,
// precision switch; advances the iteration.
int solve_complete(SolveState& S);
// Output order (Alg. 2 "Return") and statistics; returns the solve's status.
int solve_end(SolveState& S, chase_stats* stats);
}  // namespace chase
