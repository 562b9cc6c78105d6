// C ABI and host driver of the single-GPU ChASE solver (Alg. 2 on one GPU).
//
// The host code only makes the scalar decisions the paper leaves to the
// driver (degrees, sort order, QR variant, locking, precision switch) on
// arrays of nev + nex doubles; every vector and matrix operation runs in the
// kernels of this library on the context's stream.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <numeric>
#include <vector>

#include "ctx.cuh"

using namespace chase;

namespace chase {
int report_cuda_failure(const char* file, int line) {
  const cudaError_t e = cudaGetLastError();
  const char* base = std::strrchr(file, '/');
  fprintf(stderr, "[chase] CUDA failure at %s:%d (%s)\n", base ? base + 1 : file, line,
          cudaGetErrorString(e));
  return CHASE_ERR_CUDA;
}
// per host thread, so concurrent solves on different threads count their own launches
static thread_local long long g_launches = 0;
void count_launch() { ++g_launches; }
long long launch_count() { return g_launches; }
}  // namespace chase

namespace {

const double kU = 1.1102230246251565e-16;  // 2^-53

int cuda_fail(cudaError_t e, const char* what) {
  if (e != cudaSuccess) {
    fprintf(stderr, "[chase] CUDA error in %s: %s\n", what, cudaGetErrorString(e));
    return CHASE_ERR_CUDA;
  }
  return CHASE_OK;
}
#define CK(call)                                              \
  do {                                                        \
    int _rc = cuda_fail((call), #call);                       \
    if (_rc != CHASE_OK) return _rc;                          \
  } while (0)
#define RC(call)                                              \
  do {                                                        \
    int _rc = (call);                                         \
    if (_rc != CHASE_OK) return _rc;                          \
  } while (0)

double rho_of(double t) {
  // max{|t - sqrt(t^2-1)|, |t + sqrt(t^2-1)|}: |t| + sqrt(t^2-1) outside
  // [-1, 1], exactly 1 inside (complex conjugate roots on the unit circle).
  const double d = t * t - 1.0;
  if (d < 0.0) return 1.0;
  const double s = std::sqrt(d);
  return std::max(std::fabs(t - s), std::fabs(t + s));
}

struct PhaseTimer {
  cudaStream_t s;
  cudaEvent_t a, b;
  double* acc;
  PhaseTimer(chase_ctx* c, double* acc_) : s(c->stream), a(c->ev0), b(c->ev1), acc(acc_) {
    if (acc) cudaEventRecord(a, s);
  }
  void stop() {
    if (!acc) return;
    cudaEventRecord(b, s);
    cudaEventSynchronize(b);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, a, b);
    *acc += ms;
    acc = nullptr;
  }
  ~PhaseTimer() { stop(); }
};

void free_ctx(chase_ctx* c) {
  if (!c) return;
  void* bufs[] = {c->V2, c->W, c->G, c->Yeig, c->gram_ws, c->dinv, c->info, c->resid_partial,
                  c->dscal, c->perm_d, c->jw.Gw, c->jw.Gw2, c->jw.Zw, c->jw.Zw2, c->jw.T,
                  c->jw.G32a, c->jw.G32b, c->jw.Z32, c->jw.params, c->jw.red,
                  c->jw.pairs, c->jw.npairs, c->jw.cl_idx, c->jw.cl_off, c->jw.Rb,
                  c->lw.Q, c->lw.ws, c->lw.red, c->lw.ab, c->lw.T, c->lw.theta, c->lw.Z,
                  c->lw.out4, c->lw.status};
  for (void* b : bufs)
    if (b) cudaFree(b);
  mixed_free(c->mw);
  ozaki_free(c->ow);
  householder_free(c->hw);
  if (c->oz_partial) cudaFree(c->oz_partial);
  if (c->QRt) cudaFree(c->QRt);
  if (c->gw) cudaFree(c->gw);
  if (c->gd) cudaFree(c->gd);
  if (c->host) cudaFreeHost(c->host);
  if (c->ev0) cudaEventDestroy(c->ev0);
  if (c->ev1) cudaEventDestroy(c->ev1);
  delete c;
}

int validate_params(const chase_params* p) {
  if (!p) return CHASE_ERR_INVALID_ARG;
  if (p->N < 2 || p->nev < 1 || p->nex < 0 || p->nev + p->nex > p->N) return CHASE_ERR_INVALID_ARG;
  // the Jacobi kernel keeps two FP64 columns of the (nev+nex)^2 Rayleigh-Ritz
  // matrix and one round's rotations in shared memory: 64 (nev+nex) + 32 bytes <= 223 KB
  if (p->nev + p->nex > 3500) return CHASE_ERR_INVALID_ARG;
  if (p->deg_init < 2 || (p->deg_init & 1) || p->deg_max < 2 || p->deg_extra < 0)
    return CHASE_ERR_INVALID_ARG;
  if (p->max_iter < 1 || !(p->tol > 0.0) || !(p->switch_tol > 0.0)) return CHASE_ERR_INVALID_ARG;
  if (p->lanczos_steps < 1 || p->lanczos_steps > 64 || p->lanczos_steps > p->N)
    return CHASE_ERR_INVALID_ARG;
  if (p->lanczos_vecs < 1 || p->lanczos_vecs > 8) return CHASE_ERR_INVALID_ARG;
  if (p->precision != CHASE_FP64 && p->precision != CHASE_MIXED_BF16X3) return CHASE_ERR_INVALID_ARG;
  if (p->fp64_tensor != 0 && p->fp64_tensor != 1) return CHASE_ERR_INVALID_ARG;
  if (p->heev_max_sweeps < 0 || p->reserved != 0) return CHASE_ERR_INVALID_ARG;
  return CHASE_OK;
}

template <typename T>
cudaError_t dalloc(T** p, size_t n) {
  return cudaMalloc(reinterpret_cast<void**>(p), std::max<size_t>(n, 1) * sizeof(T));
}

// Digits of A for the tensor-core FP64 products (once per solve, else per call).
int prepare_a(chase_ctx* c, const double2* A, int64_t lda) {
  if (!c->p.fp64_tensor || c->oz_a_valid) return CHASE_OK;
  CK(ozaki_prepare_a(c->stream, A, lda, c->ow));
  return CHASE_OK;
}

}  // namespace

namespace chase {
int ctx_prepare_a(chase_ctx* c, const double2* A, int64_t lda) { return prepare_a(c, A, lda); }

void cheb_coefficients(int dmax, double cc, double e, double mu1, bool scaled,
                       std::vector<double>& al, std::vector<double>& be) {
  al.assign(dmax + 1, 0.0);
  be.assign(dmax + 1, 0.0);
  if (dmax < 1) return;
  if (scaled) {
    const double sigma1 = e / (mu1 - cc);
    al[1] = sigma1 / e;
    double sig = sigma1;
    for (int i = 2; i <= dmax; ++i) {
      const double sn = 1.0 / (2.0 / sigma1 - sig);
      al[i] = 2.0 * sn / e;
      be[i] = -sig * sn;
      sig = sn;
    }
  } else {
    al[1] = 1.0 / e;
    for (int i = 2; i <= dmax; ++i) {
      al[i] = 2.0 / e;
      be[i] = -1.0;
    }
  }
}
}  // namespace chase

namespace {
// ------------------------------------------------------------------ filter
int filter_impl(chase_ctx* c, const double2* A, int64_t lda, double2* V, int64_t ldv,
                int64_t ncols, const int32_t* degs, double cc, double e, double mu1, int prec,
                double* ms) {
  if (ncols == 0) return CHASE_OK;
  const int dmax = degs[ncols - 1];
  // Eq. 1 coefficients (gamma_i = c), see chase_filter in chase.h
  std::vector<double> al, be;
  cheb_coefficients(dmax, cc, e, mu1, c->p.scaled_filter != 0, al, be);
  PhaseTimer tm(c, ms);
  if (prec == CHASE_MIXED_BF16X3)
    return mixed_filter(c->stream, c->N, A, lda, V, ldv, ncols, degs, cc, al.data(), be.data(),
                        c->W, c->N, c->mw);
  double2* buf[2] = {V, c->W};
  const int64_t ld[2] = {ldv, c->N};
  if (c->p.fp64_tensor) {
    RC(prepare_a(c, A, lda));
    for (int i = 1; i <= dmax; ++i) {
      const int64_t j0 = std::lower_bound(degs, degs + ncols, i) - degs;
      const int s = (i - 1) & 1, d = i & 1;
      Epilogue ep{};
      ep.mode = EPI_FILTER;
      ep.alpha = al[i];
      ep.beta = (i == 1) ? 0.0 : be[i];
      ep.gamma = cc;
      ep.X = buf[s];
      ep.ldx = ld[s];
      ep.Y = buf[d];
      ep.ldy = ld[d];
      CK(ozaki_gemm(c->stream, ncols, j0, buf[s], ld[s], ep, c->ow));
    }
    return ozaki_check(c->stream, c->ow);
  }
  for (int i = 1; i <= dmax; ++i) {
    const int64_t j0 = std::lower_bound(degs, degs + ncols, i) - degs;
    const int64_t nact = ncols - j0;
    const int s = (i - 1) & 1, d = i & 1;
    Epilogue ep{};
    ep.mode = EPI_FILTER;
    ep.alpha = al[i];
    ep.beta = (i == 1) ? 0.0 : be[i];
    ep.gamma = cc;
    ep.X = buf[s] + j0 * ld[s];
    ep.ldx = ld[s];
    ep.Y = buf[d] + j0 * ld[d];
    ep.ldy = ld[d];
    CK(zgemm_nn(c->stream, c->N, nact, c->N, A, lda, buf[s] + j0 * ld[s], ld[s], ep));
  }
  return CHASE_OK;
}

int check_degs(const int32_t* degs, int64_t n, int deg_cap) {
  for (int64_t j = 0; j < n; ++j) {
    if (degs[j] < 2 || (degs[j] & 1) || degs[j] > deg_cap) return CHASE_ERR_INVALID_ARG;
    if (j > 0 && degs[j] < degs[j - 1]) return CHASE_ERR_INVALID_ARG;
  }
  return CHASE_OK;
}

// ---------------------------------------------------------------------- QR
// One CholeskyQR pass (Alg. 3 body): G = X^H X (+ s I), G = U^H U, X = X U^-1.
// Returns the POTRF info through *info_h (0 = success; X untouched otherwise).
//
// With the tensor-core FP64 products (fp64_tensor):
//  * Gram matrix. A digit-sliced X^H X carries an error of about
//    sqrt(2N) 2^-50 2^(e_i + e_j) from the dropped digit pairs, where 2^e_i
//    (between 2 and 4 times the largest entry of column i) is the column's
//    digit scale, plus the rounding of the digits themselves, about
//    2^(e_i - 48) ||x_j|| + 2^(e_j - 48) ||x_i||. FP64 gives about sqrt(N)
//    2^-53 of the column norms' product. The orthogonality a pass delivers is
//    the Gram error times kappa(X)^2. Every pass keeps the level-8 digit pairs
//    too, which lowers the first term to sqrt(2N) 2^-58 2^(e_i + e_j): with
//    the plain product a first pass over a block of localised columns (Gram
//    error near 1e-12) left kappa(X1) large enough for the second pass to
//    square it into its orthogonality (2e-11 at N = 40000, n = 3000). The last
//    pass of CholeskyQR2 / shifted CholeskyQR2 (input orthonormal to about the
//    previous pass's kappa^2 times its Gram error) uses the tensor cores when
//    2^(emax - 46) + sqrt(2N) 2^(2 emax - 56), with the largest column scale,
//    stays below 1e-13 (the orthogonality target is 1e-12): true for any
//    nearly orthonormal block (its entries are at most 1, emax <= 2), flat or
//    localised. CholeskyQR1's single pass (kappa up to 20) keeps the FP64
//    Gram.
//  * X U^-1. When max |U - I| <= 1e-4 (the input is orthonormal to about 1e-4),
//    X U^-1 = X + X D with D = U^-1 - I, |D| <= ~1e-4: the digit-sliced product
//    X D carries an error of about sqrt(2n) 2^-44 max|X_i.| max|D_.j|, below
//    1e-15 absolute, so it runs on the tensor cores (U^-1 by a recursive blocked
//    inversion with FP64 GEMMs). Otherwise the solve is a digit-sliced product
//    with iterative refinement (tensor_trsm below).
constexpr double kNearIdentity = 1e-4;

constexpr double kGramTol = 1e-13;

// Refinement of T = X U^-1 on the tensor cores. A digit-sliced product with a
// general U^-1 is accurate to about sqrt(n) 2^-48 of max|X_i.| max|U^-1_.j|,
// which for a filtered block is kappa(X) times the size of the result: the
// first product T0 = X U^-1 leaves a relative backward error
// eta0 = max_j ||X_j - (T0 U)_j|| / ||X_j|| of about sqrt(n) 2^-48 kappa. Each
// step rounds T to its own digits (so the next product takes it exactly),
// forms R = X - T U (extended product: the result cancels to eta of X, so the
// level-8 pairs are kept) and T <- T + R U^-1 in the FP64 epilogue; this
// multiplies the backward error by about eta0, down to the dropped pairs'
// sqrt(n) 2^-58 of the scales (the triangular solve in FP64 leaves about
// sqrt(n) 2^-53). Steps continue
// while eta_k eta0 > 1e-14 (at most kMaxRefine). The input must stay readable
// for every step: Xsaved holds a copy of X (the block the QR was given, for
// the first pass); without it one step is taken, overwriting X with R (passes
// after the first, whose input is already well conditioned). If the steps
// do not converge the FP64 triangular solve runs on the saved input.
constexpr int kMaxRefine = 6;
constexpr double kRefineTarget = 1e-14;

int tensor_trsm(chase_ctx* c, double2* X, int64_t ldx, int64_t n, const double2* Xsaved) {
  const int64_t N = c->N;
  double2* T = c->QRt;
  double* eta_h = c->host + 2 * c->ne + 9;
  // U^-1 into Yeig (free during the QR); U itself as a dense operand
  CK(triangular_inverse(c->stream, n, c->G, c->ne, c->dinv, c->Yeig, c->ne, c->jw.T));
  CK(zero_lower(c->stream, n, c->G, c->ne));
  {
    Epilogue ep{};  // T = X U^-1
    ep.mode = EPI_STORE;
    ep.Y = T;
    ep.ldy = N;
    CK(ozaki_gemm_general(c->stream, N, n, X, ldx, false, n, c->Yeig, c->ne, ep, c->ow));
  }
  const double2* Xin = Xsaved ? Xsaved : X;
  const int64_t ldin = Xsaved ? N : ldx;
  double eta0 = -1.0;
  for (int k = 0;; ++k) {
    // T to the value its digits represent, so that T U below takes it exactly:
    // R then carries only the dropped pairs' error, not T's digit rounding
    // (which would leave a backward error of a few 2^-48 of the rows' scales)
    CK(ozaki_round_left(c->stream, N, n, T, N, c->ow));
    {
      Epilogue ep{};  // R = Xin - T U, into X (X's content is Xin's copy or used last here)
      ep.mode = EPI_FILTER;
      ep.alpha = -1.0;
      ep.gamma = 1.0;
      ep.beta = 0.0;
      ep.X = Xin;
      ep.ldx = ldin;
      ep.Y = X;
      ep.ldy = ldx;
      CK(ozaki_gemm_general(c->stream, N, n, T, N, false, n, c->G, c->ne, ep, c->ow, true));
    }
    bool last = Xsaved == nullptr;
    if (!last) {
      CK(max_col_ratio(c->stream, N, n, X, ldx, Xin, ldin, c->dscal + 2));
      CK(cudaMemcpyAsync(eta_h, c->dscal + 2, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
      CK(cudaStreamSynchronize(c->stream));
      RC(ozaki_check(c->stream, c->ow));
      const double eta = *eta_h;
      if (eta0 < 0.0) eta0 = eta;
      // steps still needed at the rate eta0 per step: eta0^(k + 2) <= target
      const bool hopeless =
          eta0 > 1e-300 && std::log(kRefineTarget) / std::log(eta0) - 2.0 > kMaxRefine - 1;
      if (!(eta <= 0.5) || hopeless || (k + 1 >= kMaxRefine && eta * eta0 > kRefineTarget)) {
        // no convergence (or non-finite values): the FP64 solve on the input
        CK(copy_cols(c->stream, N, n, Xsaved, N, X, ldx));
        CK(trsm_right_upper(c->stream, N, n, X, ldx, c->G, c->ne, c->dinv, c->info));
        return CHASE_OK;
      }
      last = eta * eta0 <= kRefineTarget;
    }
    Epilogue ep{};
    ep.mode = EPI_FILTER;
    ep.alpha = 1.0;
    if (last) {  // X = T + R U^-1 (R's digits are taken before X is written)
      ep.gamma = -1.0;
      ep.beta = 0.0;
      ep.X = T;
      ep.ldx = N;
      ep.Y = X;
      ep.ldy = ldx;
    } else {     // T <- T + R U^-1
      ep.gamma = 0.0;
      ep.beta = 1.0;
      ep.X = T;
      ep.ldx = N;
      ep.Y = T;
      ep.ldy = N;
    }
    CK(ozaki_gemm_general(c->stream, N, n, X, ldx, false, n, c->Yeig, c->ne, ep, c->ow));
    if (last) return ozaki_check(c->stream, c->ow);
  }
}

int cholqr_pass(chase_ctx* c, double2* X, int64_t ldx, int64_t n, double shift_factor,
                bool last, bool single, const double2* Xsaved, int* info_h) {
  const bool tensor = c->p.fp64_tensor != 0;
  bool tc = tensor && !single;
  double* dev_h = c->host + 2 * c->ne + 10;
  {
    if (tc) {
      Epilogue ep{};
      ep.mode = EPI_STORE;
      ep.Y = c->G;
      ep.ldy = c->ne;
      CK(ozaki_gemm_general(c->stream, n, c->N, X, ldx, true, n, X, ldx, ep, c->ow, true));
      CK(hermitian_part(c->stream, n, c->G, c->ne));
      if (last) {  // keep it only if its error bound allows (see above)
        int* emax_h = reinterpret_cast<int*>(c->host + 2 * c->ne + 11);
        CK(ozaki_left_exp_max(c->stream, n, c->ow, c->info + 1));
        CK(cudaMemcpyAsync(emax_h, c->info + 1, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
        CK(cudaStreamSynchronize(c->stream));
        RC(ozaki_check(c->stream, c->ow));
        const double bound = std::ldexp(1.0, *emax_h - 46) +
                             std::sqrt(2.0 * (double)c->N) * std::ldexp(1.0, 2 * *emax_h - 56);
        tc = bound <= kGramTol;
      }
    }
    if (!tc) {
      CK(zgram(c->stream, c->N, n, n, X, ldx, X, ldx, c->G, c->ne, true, c->gram_ws,
               c->gram_ws_elems));
    }
    if (shift_factor > 0.0) CK(add_trace_shift(c->stream, n, c->G, c->ne, shift_factor, c->dscal));
    CK(potrf_upper(c->stream, n, c->G, c->ne, c->dinv, c->info));
    if (tensor) CK(max_dev_identity(c->stream, n, c->G, c->ne, c->dscal + 1));
    CK(cudaMemcpyAsync(info_h, c->info, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    if (tensor)
      CK(cudaMemcpyAsync(dev_h, c->dscal + 1, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    if (tc) RC(ozaki_check(c->stream, c->ow));
    if (*info_h != 0) return CHASE_OK;
  }
  if (tensor && *dev_h <= kNearIdentity) {
    // X <- X + X (U^-1 - I) on the tensor cores; U^-1 (recursive blocked
    // inverse, FP64 GEMMs) into Yeig, which is free during the QR
    CK(triangular_inverse(c->stream, n, c->G, c->ne, c->dinv, c->Yeig, c->ne, c->jw.T));
    CK(set_identity(c->stream, n, c->Yeig, c->ne, true));
    Epilogue ep{};
    ep.mode = EPI_FILTER;  // X = (X D) + X, in place: the product reads X's digit planes
    ep.alpha = 1.0;
    ep.beta = 1.0;
    ep.gamma = 0.0;
    ep.X = X;
    ep.ldx = ldx;
    ep.Y = X;
    ep.ldy = ldx;
    CK(ozaki_gemm_general(c->stream, c->N, n, X, ldx, false, n, c->Yeig, c->ne, ep, c->ow));
    return ozaki_check(c->stream, c->ow);
  }
  if (tensor) return tensor_trsm(c, X, ldx, n, Xsaved);
  CK(trsm_right_upper(c->stream, c->N, n, X, ldx, c->G, c->ne, c->dinv, c->info));
  return CHASE_OK;
}

int qr_impl(chase_ctx* c, double2* X, int64_t ldx, int64_t n, double cond, int32_t* variant) {
  int* info_h = reinterpret_cast<int*>(c->host + 2 * c->ne + 8);
  // the input block is kept in W (free while the QR runs) for the Householder
  // fallback, which factors the block the caller passed in
  CK(copy_cols(c->stream, c->N, n, X, ldx, c->W, c->N));
  int v = cond > 1e8 ? CHASE_QR_SHIFTED : (cond < 20 ? CHASE_QR_CHOLQR1 : CHASE_QR_CHOLQR2);
  if (v != CHASE_QR_SHIFTED) {
    const int passes = v == CHASE_QR_CHOLQR1 ? 1 : 2;
    bool ok = true;
    for (int k = 0; k < passes && ok; ++k) {
      RC(cholqr_pass(c, X, ldx, n, 0.0, k == passes - 1, passes == 1, k == 0 ? c->W : nullptr,
                     info_h));
      ok = (*info_h == 0);
    }
    if (ok) {
      if (variant) *variant = v;
      return CHASE_OK;
    }
    // reading: Alg. 4 names no fallback for CholeskyQR1/2; a failed POTRF there
    // (the estimate was too low) re-runs the shifted branch on the input block
    CK(copy_cols(c->stream, c->N, n, c->W, c->N, X, ldx));
  }
  // Alg. 4 shifted branch: s = 11 (m n + n (n + 1)) u ||X||_F^2, then CholeskyQR2
  const double factor = 11.0 * ((double)c->N * (double)n + (double)n * (double)(n + 1)) * kU;
  RC(cholqr_pass(c, X, ldx, n, factor, false, false, c->W, info_h));
  if (*info_h == 0) RC(cholqr_pass(c, X, ldx, n, 0.0, false, false, nullptr, info_h));
  if (*info_h == 0) RC(cholqr_pass(c, X, ldx, n, 0.0, true, false, nullptr, info_h));
  if (*info_h == 0) {
    if (variant) *variant = CHASE_QR_SHIFTED;
    return CHASE_OK;
  }
  // Alg. 4: a POTRF of the shifted branch failed -> Householder QR of the input
  // (reading: also when the failure is in the CholeskyQR2 after the shift)
  RC(householder_qr(c->stream, c->N, n, c->W, c->N, X, ldx, c->hw));
  if (variant) *variant = CHASE_QR_HOUSEHOLDER;
  return CHASE_OK;
}

// ----------------------------------------------------------- Rayleigh-Ritz
// Q (N x n, ldq) orthonormal, not aliasing V. V[:, 0:n] = Q Y, ritz = eigenvalues.
int rr_impl(chase_ctx* c, const double2* A, int64_t lda, const double2* Q, int64_t ldq,
            double2* V, int64_t ldv, int64_t n, double* ritz, chase_stats* st = nullptr) {
  Epilogue ep{};
  ep.mode = EPI_STORE;
  ep.Y = c->W;
  ep.ldy = c->N;
  if (c->p.fp64_tensor) {                                                        // W = A Q
    RC(prepare_a(c, A, lda));
    CK(ozaki_gemm(c->stream, n, 0, Q, ldq, ep, c->ow));
  } else {
    CK(zgemm_nn(c->stream, c->N, n, c->N, A, lda, Q, ldq, ep));
  }
  if (c->p.fp64_tensor) {                                                        // G = Q^H W
    Epilogue eg{};
    eg.mode = EPI_STORE;
    eg.Y = c->G;
    eg.ldy = c->ne;
    // extended: the off-diagonal of Q^H A Q cancels to the size of the residuals
    CK(ozaki_gemm_general(c->stream, n, c->N, Q, ldq, true, n, c->W, c->N, eg, c->ow, true));
  } else {
    CK(zgram(c->stream, c->N, n, n, Q, ldq, c->W, c->N, c->G, c->ne, false, c->gram_ws,
             c->gram_ws_elems));
  }
  CK(hermitian_part(c->stream, n, c->G, c->ne));
  int sweeps = 0;
  {
    cudaEvent_t h0 = nullptr, h1 = nullptr;
    if (st) {
      cudaEventCreate(&h0);
      cudaEventCreate(&h1);
      cudaEventRecord(h0, c->stream);
    }
    int sweeps64 = 0, cl[3] = {0, 0, 0};
    const int rc = jacobi_heev(c->stream, n, c->G, c->ne, ritz, c->Yeig, c->ne, c->jw, &sweeps,
                               &sweeps64, cl);
    if (st) {
      cudaEventRecord(h1, c->stream);
      cudaEventSynchronize(h1);
      float ms = 0.f;
      cudaEventElapsedTime(&ms, h0, h1);
      st->ms_heev += ms;
      st->heev_sweeps += sweeps;
      st->heev_fp64_sweeps += sweeps64;
      st->heev_cluster_solves += cl[0];
      st->heev_cluster_max = std::max(st->heev_cluster_max, cl[1]);
      cudaEventDestroy(h0);
      cudaEventDestroy(h1);
    }
    RC(rc);
  }
  Epilogue e2{};
  e2.mode = EPI_STORE;
  e2.Y = V;
  e2.ldy = ldv;
  if (c->p.fp64_tensor) {                                                        // V = Q Y
    CK(ozaki_gemm_general(c->stream, c->N, n, Q, ldq, false, n, c->Yeig, c->ne, e2, c->ow));
    return ozaki_check(c->stream, c->ow);
  }
  CK(zgemm_nn(c->stream, c->N, n, n, Q, ldq, c->Yeig, c->ne, e2));
  return CHASE_OK;
}

int resid_impl(chase_ctx* c, const double2* A, int64_t lda, const double2* V, int64_t ldv,
               const double* ritz, int64_t n, double* resid) {
  if (n == 0) return CHASE_OK;
  Epilogue ep{};
  ep.mode = EPI_RESID;
  ep.X = V;
  ep.ldx = ldv;
  ep.theta = ritz;
  if (c->p.fp64_tensor) {
    RC(prepare_a(c, A, lda));
    ep.partial = c->oz_partial;
    CK(ozaki_gemm(c->stream, n, 0, V, ldv, ep, c->ow));
    CK(resid_reduce(c->stream, c->oz_partial, cdiv(c->N, 32), n, resid));
    return ozaki_check(c->stream, c->ow);
  }
  ep.partial = c->resid_partial;
  CK(zgemm_nn(c->stream, c->N, n, c->N, A, lda, V, ldv, ep));
  CK(resid_reduce(c->stream, c->resid_partial, zgemm_row_tiles(c->N), n, resid));
  return CHASE_OK;
}

// Lanczos block product on the tensor cores (digits of A prepared by the caller).
cudaError_t heev_tensor_gemm(void* vc, int64_t M, int64_t K, const double2* X, int64_t ldx,
                             bool conj_trans, int64_t ncols, const double2* B, int64_t ldb,
                             const Epilogue& ep, bool extended) {
  chase_ctx* c = static_cast<chase_ctx*>(vc);
  return ozaki_gemm_general(c->stream, M, K, X, ldx, conj_trans, ncols, B, ldb, ep, c->ow,
                            extended);
}

cudaError_t lanczos_tensor_matmul(void* vc, const double2* Q, int64_t ldq, int nvec, double2* W,
                                  int64_t ldw) {
  chase_ctx* c = static_cast<chase_ctx*>(vc);
  Epilogue ep{};
  ep.mode = EPI_STORE;
  ep.Y = W;
  ep.ldy = ldw;
  return ozaki_gemm(c->stream, nvec, 0, Q, ldq, ep, c->ow);
}

int lanczos_impl(chase_ctx* c, const double2* A, int64_t lda, const double2* Q0, int64_t ldq,
                 int nvec, double* out4_h) {
  if (c->p.fp64_tensor) {
    RC(prepare_a(c, A, lda));
    c->lw.matmul = lanczos_tensor_matmul;
    c->lw.matmul_ctx = c;
  } else {
    c->lw.matmul = nullptr;
  }
  CK(lanczos_bounds(c->stream, c->N, A, lda, Q0, ldq, nvec, c->p.lanczos_steps, c->ne, c->lw));
  if (c->p.fp64_tensor) RC(ozaki_check(c->stream, c->ow));
  CK(cudaMemcpyAsync(out4_h, c->lw.out4, 4 * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  int st = 0;
  CK(cudaMemcpyAsync(&st, c->lw.status, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  return st ? CHASE_ERR_HEEV_NOCONV : CHASE_OK;
}

}  // namespace

// ============================================================ solve phases
namespace chase {
namespace {
// adds the kernels launched on this thread while it lives to S.launches
struct LaunchTally {
  SolveState& S;
  long long l0;
  explicit LaunchTally(SolveState& s) : S(s), l0(launch_count()) {}
  ~LaunchTally() { S.launches += launch_count() - l0; }
};
}  // namespace

SolveState::~SolveState() {
  if (t_start) cudaEventDestroy(t_start);
  if (t_end) cudaEventDestroy(t_end);
  if (c) c->oz_a_valid = false;
}

int solve_begin(SolveState& S, chase_ctx* c, const double2* A, int64_t lda, double2* C,
                int64_t ldv, const double2* Q0, int64_t ldq, double* ritz, double* resid) {
  if (!c || !A || !C || !ritz || !resid || lda < c->N || ldv < c->N)
    return CHASE_ERR_INVALID_ARG;
  if (Q0 && ldq < c->N) return CHASE_ERR_INVALID_ARG;
  if (!Q0 && c->p.lanczos_vecs > c->ne) return CHASE_ERR_INVALID_ARG;
  const chase_params& P = c->p;
  const int64_t ne = c->ne;
  S.c = c;
  S.A = A;
  S.lda = lda;
  S.C = C;
  S.ldv = ldv;
  S.ritz = ritz;
  S.resid = resid;
  std::memset(&S.st, 0, sizeof(S.st));
  CK(cudaEventCreate(&S.t_start));
  CK(cudaEventCreate(&S.t_end));
  CK(cudaEventRecord(S.t_start, c->stream));
  S.launches = 0;
  LaunchTally tally(S);
  if (P.fp64_tensor) {  // digits of A once for every tensor-core FP64 product of this solve
    c->oz_a_valid = false;
    RC(prepare_a(c, A, lda));
    c->oz_a_valid = true;
  }
  double b4[4];
  {
    PhaseTimer tm(c, &S.st.ms_lanczos);
    RC(lanczos_impl(c, A, lda, Q0 ? Q0 : C, Q0 ? ldq : ldv, P.lanczos_vecs, b4));
  }
  S.b_sup = b4[0];
  S.mu_1 = b4[1];
  S.mu_ne = b4[2];
  S.norm_est = b4[3];
  S.st.b_sup = S.b_sup;
  S.st.mu_1 = S.mu_1;
  S.st.mu_ne = S.mu_ne;
  S.st.norm_est = S.norm_est;
  S.tol_abs = P.tol * S.norm_est;
  S.degs.assign(ne, P.deg_init);
  S.rz.assign(ne, 0.0);
  S.rs.assign(ne, 0.0);
  S.locked = 0;
  S.iter = 1;
  S.cc = (S.b_sup + S.mu_ne) / 2.0;
  S.ee = (S.b_sup - S.mu_ne) / 2.0;
  S.mixed = P.precision == CHASE_MIXED_BF16X3;
  S.rmax_prev = 1e300;
  S.st.switch_iter = S.mixed ? -1 : 0;
  return CHASE_OK;
}

bool solve_active(const SolveState& S) {
  return S.locked < S.c->p.nev && S.iter <= S.c->p.max_iter;
}

int solve_prepare(SolveState& S) {
  LaunchTally tally(S);
  chase_ctx* c = S.c;
  const chase_params& P = c->p;
  const int64_t N = c->N, ne = c->ne, locked = S.locked, nact = ne - locked;
  double2* C = S.C;
  const int64_t ldv = S.ldv;
  std::vector<int32_t>& degs = S.degs;
  std::vector<double>& rz = S.rz;
  std::vector<double>& rs = S.rs;
  if (S.iter != 1) {
    S.mu_1 = *std::min_element(rz.begin(), rz.end());
    S.mu_ne = *std::max_element(rz.begin(), rz.end());
    S.cc = (S.b_sup + S.mu_ne) / 2.0;
    S.ee = (S.b_sup - S.mu_ne) / 2.0;
    if (P.deg_opt) {
      chase_degree_opt(rs.data() + locked, rz.data() + locked, nact, S.cc, S.ee, S.tol_abs,
                       P.deg_max, P.deg_extra, degs.data() + locked);
      std::vector<int> ord(nact);
      std::iota(ord.begin(), ord.end(), 0);
      std::stable_sort(ord.begin(), ord.end(), [&](int a, int b) {
        const int32_t da = degs[locked + a], db = degs[locked + b];
        if (da != db) return da < db;
        return rz[locked + a] < rz[locked + b];
      });
      bool ident = true;
      for (int64_t k = 0; k < nact; ++k) ident = ident && ord[k] == k;
      if (!ident) {
        std::vector<int32_t> d2(nact);
        std::vector<double> z2(nact), s2(nact);
        for (int64_t k = 0; k < nact; ++k) {
          d2[k] = degs[locked + ord[k]];
          z2[k] = rz[locked + ord[k]];
          s2[k] = rs[locked + ord[k]];
        }
        std::copy(d2.begin(), d2.end(), degs.begin() + locked);
        std::copy(z2.begin(), z2.end(), rz.begin() + locked);
        std::copy(s2.begin(), s2.end(), rs.begin() + locked);
        CK(cudaMemcpyAsync(c->perm_d, ord.data(), nact * sizeof(int), cudaMemcpyHostToDevice,
                           c->stream));
        CK(copy_cols(c->stream, N, nact, C + locked * ldv, ldv, c->W, N));
        CK(gather_cols(c->stream, N, nact, c->W, N, c->perm_d, C + locked * ldv, ldv));
        CK(cudaStreamSynchronize(c->stream));  // ord is a stack buffer
      }
    }
  }
  if (S.iter == 1) {
    std::vector<double> lam(ne, S.mu_1);
    S.cond = chase_cond_est(lam.data(), degs.data(), ne, locked, S.cc, S.ee);
  } else {
    S.cond = chase_cond_est(rz.data(), degs.data(), ne, locked, S.cc, S.ee);
  }
  return CHASE_OK;
}

void solve_count_filter(SolveState& S) {
  int64_t mv = 0;
  for (int64_t j = S.locked; j < S.c->ne; ++j) mv += S.degs[j];
  S.st.matvecs += mv;
  if (S.mixed) S.st.matvecs_mixed += mv;
}

int solve_filter(SolveState& S) {
  LaunchTally tally(S);
  chase_ctx* c = S.c;
  const int prec = S.mixed ? CHASE_MIXED_BF16X3 : CHASE_FP64;
  RC(filter_impl(c, S.A, S.lda, S.C + S.locked * S.ldv, S.ldv, c->ne - S.locked,
                 S.degs.data() + S.locked, S.cc, S.ee, S.mu_1, prec, &S.st.ms_filter));
  solve_count_filter(S);
  return CHASE_OK;
}

int solve_complete(SolveState& S) {
  LaunchTally tally(S);
  chase_ctx* c = S.c;
  const chase_params& P = c->p;
  const int64_t N = c->N, ne = c->ne, nev = P.nev, locked = S.locked, nact = ne - locked;
  double2* C = S.C;
  const int64_t ldv = S.ldv;
  int32_t variant = 0;
  {
    PhaseTimer tm(c, &S.st.ms_qr);
    RC(qr_impl(c, C, ldv, ne, S.cond, &variant));
    CK(copy_cols(c->stream, N, locked, c->V2, N, C, ldv));                       // C[:, :locked] = C2
    CK(copy_cols(c->stream, N, nact, C + locked * ldv, ldv, c->V2 + locked * N, N));
  }
  if (variant >= 1 && variant <= 4) S.st.qr_variant_count[variant]++;
  {
    PhaseTimer tm(c, &S.st.ms_rr);
    RC(rr_impl(c, S.A, S.lda, c->V2 + locked * N, N, C + locked * ldv, ldv, nact,
               S.ritz + locked, &S.st));
    CK(copy_cols(c->stream, N, nact, C + locked * ldv, ldv, c->V2 + locked * N, N));
  }
  {
    PhaseTimer tm(c, &S.st.ms_resid);
    RC(resid_impl(c, S.A, S.lda, C + locked * ldv, ldv, S.ritz + locked, nact,
                  S.resid + locked));
  }
  double* rz_pin = c->host;
  double* rs_pin = c->host + ne;
  CK(cudaMemcpyAsync(rz_pin, S.ritz + locked, nact * sizeof(double), cudaMemcpyDeviceToHost,
                     c->stream));
  CK(cudaMemcpyAsync(rs_pin, S.resid + locked, nact * sizeof(double), cudaMemcpyDeviceToHost,
                     c->stream));
  CK(cudaStreamSynchronize(c->stream));
  std::copy(rz_pin, rz_pin + nact, S.rz.begin() + locked);
  std::copy(rs_pin, rs_pin + nact, S.rs.begin() + locked);
  int64_t nc = 0;
  while (locked + nc < ne && S.rs[locked + nc] <= S.tol_abs) ++nc;
  // precision switch (reading of the mixed-precision policy): leave the
  // reduced-precision filter once the largest residual among the wanted active
  // pairs reaches switch_tol, or stops falling by at least 3x per iteration.
  if (S.mixed) {
    double rmax = 0.0;
    for (int64_t j = locked + nc; j < nev; ++j) rmax = std::max(rmax, S.rs[j] / S.norm_est);
    if (rmax <= P.switch_tol || rmax > S.rmax_prev / 3.0) {
      S.mixed = false;
      S.st.switch_iter = S.iter;
    }
    S.rmax_prev = rmax;
  }
  S.locked += nc;
  ++S.iter;
  return CHASE_OK;
}

int solve_end(SolveState& S, chase_stats* stats) {
  chase_ctx* c = S.c;
  const long long l0 = launch_count();
  const int64_t N = c->N, nev = c->p.nev, locked = S.locked;
  double2* C = S.C;
  const int64_t ldv = S.ldv;
  // Output: the first nev Ritz pairs in ascending order (Alg. 2 "Return").
  const int64_t nsort = std::max<int64_t>(locked, nev);
  std::vector<int> ord(nsort);
  std::iota(ord.begin(), ord.end(), 0);
  std::stable_sort(ord.begin(), ord.end(), [&](int a, int b) { return S.rz[a] < S.rz[b]; });
  bool ident = true;
  for (int64_t k = 0; k < nev; ++k) ident = ident && ord[k] == k;
  if (!ident) {
    std::vector<double> z2(nev), s2(nev);
    for (int64_t k = 0; k < nev; ++k) {
      z2[k] = S.rz[ord[k]];
      s2[k] = S.rs[ord[k]];
    }
    CK(cudaMemcpyAsync(c->perm_d, ord.data(), nev * sizeof(int), cudaMemcpyHostToDevice,
                       c->stream));
    CK(copy_cols(c->stream, N, nsort, C, ldv, c->W, N));
    CK(gather_cols(c->stream, N, nev, c->W, N, c->perm_d, C, ldv));
    CK(cudaMemcpyAsync(S.ritz, z2.data(), nev * sizeof(double), cudaMemcpyHostToDevice,
                       c->stream));
    CK(cudaMemcpyAsync(S.resid, s2.data(), nev * sizeof(double), cudaMemcpyHostToDevice,
                       c->stream));
  }
  S.launches += launch_count() - l0;
  CK(cudaEventRecord(S.t_end, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  float ms = 0.f;
  cudaEventElapsedTime(&ms, S.t_start, S.t_end);
  S.st.ms_total = ms;
  S.st.iters = S.iter - 1;
  S.st.locked = (int32_t)locked;
  S.st.filter_flops = 8.0 * (double)N * (double)N * (double)S.st.matvecs;
  S.st.kernel_launches = S.launches;
  if (stats) *stats = S.st;
  return locked >= nev ? CHASE_OK : CHASE_ERR_NOT_CONVERGED;
}

}  // namespace chase

// ======================================================================= ABI
extern "C" {

void chase_default_params(chase_params* p, int64_t N, int64_t nev, int64_t nex) {
  if (!p) return;
  std::memset(p, 0, sizeof(*p));
  p->N = N;
  p->nev = nev;
  p->nex = nex;
  p->deg_init = 20;
  p->deg_max = 36;
  p->deg_extra = 2;
  p->deg_opt = 1;
  p->max_iter = 30;
  p->lanczos_steps = (int32_t)std::min<int64_t>(25, N);
  p->lanczos_vecs = 4;
  p->precision = CHASE_FP64;
  p->scaled_filter = 1;
  p->tol = 1e-10;
  p->switch_tol = 1e-5;
}

const char* chase_status_string(int s) {
  switch (s) {
    case CHASE_OK: return "CHASE_OK";
    case CHASE_ERR_INVALID_ARG: return "CHASE_ERR_INVALID_ARG";
    case CHASE_ERR_CUDA: return "CHASE_ERR_CUDA";
    case CHASE_ERR_OOM: return "CHASE_ERR_OOM";
    case CHASE_ERR_QR_BREAKDOWN: return "CHASE_ERR_QR_BREAKDOWN";
    case CHASE_ERR_HEEV_NOCONV: return "CHASE_ERR_HEEV_NOCONV";
    case CHASE_ERR_NOT_CONVERGED: return "CHASE_ERR_NOT_CONVERGED";
    default: return "CHASE_UNKNOWN_STATUS";
  }
}

double chase_cond_est(const double* ritz, const int32_t* degs, int64_t n, int64_t locked,
                      double c, double e) {
  if (!ritz || !degs || n <= 0 || locked < 0 || locked >= n || !(e > 0.0)) return NAN;
  const double tp = (ritz[0] - c) / e;
  const double t = (ritz[locked] - c) / e;
  const double rho = rho_of(t), rhop = rho_of(tp);
  const int d = degs[locked];
  int dmax = d;
  for (int64_t j = locked; j < n; ++j) dmax = std::max<int>(dmax, degs[j]);
  return std::pow(rho, (double)d) * std::pow(rhop, (double)(dmax - d));
}

void chase_degree_opt(const double* resid, const double* ritz, int64_t n, double c, double e,
                      double tol_abs, int32_t deg_max, int32_t deg_extra, int32_t* degs) {
  const int dm = deg_max - (deg_max % 2);
  for (int64_t j = 0; j < n; ++j) {
    const double t = (ritz[j] - c) / e;
    const double rho = rho_of(t);
    int d;
    if (rho <= 1.0) {
      d = dm;
    } else if (resid[j] <= tol_abs) {
      d = 2;
    } else {
      const double x = (std::log(resid[j]) - std::log(tol_abs)) / std::log(rho);
      d = x >= dm ? dm : (int)std::ceil(x) + deg_extra;
    }
    d = std::max(2, std::min(d, dm));
    d += d % 2;
    degs[j] = std::min(d, dm);
  }
}

int chase_create(const chase_params* p, void* stream, chase_ctx** out) {
  if (!out) return CHASE_ERR_INVALID_ARG;
  *out = nullptr;
  RC(validate_params(p));
  chase_ctx* c = new (std::nothrow) chase_ctx();
  if (!c) return CHASE_ERR_OOM;
  c->p = *p;
  c->stream = reinterpret_cast<cudaStream_t>(stream);
  if (cudaGetDevice(&c->device) != cudaSuccess) c->device = 0;
  c->N = p->N;
  c->ne = p->nev + p->nex;
  const int64_t N = c->N, ne = c->ne;
  bool ok = true;
  auto A = [&](cudaError_t e) { ok = ok && (e == cudaSuccess); };
  A(dalloc(&c->V2, (size_t)N * ne));
  A(dalloc(&c->W, (size_t)N * ne));
  A(dalloc(&c->G, (size_t)ne * ne));
  A(dalloc(&c->Yeig, (size_t)ne * ne));
  c->gram_ws_elems = gram_workspace_elems(ne, ne);
  A(dalloc(&c->gram_ws, c->gram_ws_elems));
  A(dalloc(&c->dinv, (size_t)cdiv(ne, kNB) * kNB * kNB));
  A(dalloc(&c->info, 4));
  A(dalloc(&c->resid_partial, (size_t)zgemm_row_tiles(N) * ne));
  A(dalloc(&c->dscal, 16));
  A(dalloc(&c->perm_d, (size_t)ne));
  A(dalloc(&c->jw.Gw, (size_t)ne * ne));
  A(dalloc(&c->jw.Gw2, (size_t)ne * ne));
  A(dalloc(&c->jw.Zw, (size_t)ne * ne));
  A(dalloc(&c->jw.Zw2, (size_t)ne * ne));
  A(dalloc(&c->jw.T, (size_t)ne * ne));
  A(dalloc(&c->jw.G32a, (size_t)ne * ne));
  A(dalloc(&c->jw.G32b, (size_t)ne * ne));
  A(dalloc(&c->jw.Z32, (size_t)ne * ne));
  A(dalloc(&c->jw.params, jacobi_params_elems(ne)));
  A(dalloc(&c->jw.red, std::max<size_t>(1024, jacobi_red_elems())));
  c->jw.rb_elems = jacobi_rot_elems(ne);
  A(dalloc(&c->jw.Rb, c->jw.rb_elems));
  A(dalloc(&c->jw.pairs, (size_t)2 * kMaxClusterPairs));
  A(dalloc(&c->jw.npairs, 1));
  A(dalloc(&c->jw.cl_idx, (size_t)ne));
  A(dalloc(&c->jw.cl_off, (size_t)ne + 1));
  c->jw.nmax = ne;
  c->jw.max_sweeps = p->heev_max_sweeps;
  A(dalloc(&c->lw.Q, (size_t)3 * N * 8));
  A(dalloc(&c->lw.ws, skinny_workspace_elems(N, 8)));
  A(dalloc(&c->lw.red, 2048));
  A(dalloc(&c->lw.ab, 24 * 64));
  A(dalloc(&c->lw.T, (size_t)8 * 64 * 64));
  A(dalloc(&c->lw.theta, 8 * 64));
  A(dalloc(&c->lw.Z, (size_t)8 * 64 * 64));
  A(dalloc(&c->lw.out4, 4));
  A(dalloc(&c->lw.status, 4));
  if (ok) A(householder_alloc(c->hw, N, ne));
  if (ok && p->precision == CHASE_MIXED_BF16X3) A(mixed_alloc(c->mw, N, ne));
  if (ok && p->fp64_tensor) {
    A(ozaki_alloc(c->ow, N, ne));
    if (ok) A(dalloc(&c->oz_partial, (size_t)cdiv(N, 32) * ne));
    if (ok) A(dalloc(&c->QRt, (size_t)N * ne));
  }
  if (ok) A(cudaMallocHost(reinterpret_cast<void**>(&c->host), (2 * ne + 16 + 512) * sizeof(double)));
  if (ok) A(cudaEventCreate(&c->ev0));
  if (ok) A(cudaEventCreate(&c->ev1));
  if (ok) A(cudaMemsetAsync(c->lw.status, 0, sizeof(int), c->stream));
  if (ok) {
    c->jw.host_red = c->host + 2 * ne + 12;
    c->jw.host_part = c->host + 2 * ne + 16;
    c->jw.gram_ws = c->gram_ws;
    c->jw.gram_ws_elems = c->gram_ws_elems;
    c->jw.dinv = c->dinv;
    c->jw.info = c->info;
    if (p->fp64_tensor) {  // the heev's FP64 refinement products on the tensor cores
      c->jw.gemm = heev_tensor_gemm;
      c->jw.gemm_ctx = c;
    }
  }
  if (!ok) {
    cudaGetLastError();
    free_ctx(c);
    return CHASE_ERR_OOM;
  }
  *out = c;
  return CHASE_OK;
}

int chase_destroy(chase_ctx* ctx) {
  if (ctx) {
    cudaStreamSynchronize(ctx->stream);
    free_ctx(ctx);
  }
  return CHASE_OK;
}

int chase_lanczos(chase_ctx* c, const chase_c128* A, int64_t lda, const chase_c128* Q0,
                  int64_t ldq, int64_t nvec, double* bounds) {
  if (!c || !A || !Q0 || !bounds || lda < c->N || ldq < c->N || nvec < 1 ||
      nvec > c->p.lanczos_vecs)
    return CHASE_ERR_INVALID_ARG;
  return lanczos_impl(c, reinterpret_cast<const double2*>(A), lda,
                      reinterpret_cast<const double2*>(Q0), ldq, (int)nvec, bounds);
}

int chase_filter(chase_ctx* c, const chase_c128* A, int64_t lda, chase_c128* V, int64_t ldv,
                 int64_t ncols, const int32_t* degs, double cc, double e, double mu_1,
                 int32_t precision) {
  if (!c || !A || !V || lda < c->N || ldv < c->N || ncols < 0 || ncols > c->ne)
    return CHASE_ERR_INVALID_ARG;
  if (ncols > 0 && !degs) return CHASE_ERR_INVALID_ARG;
  if (!(e > 0.0) || (c->p.scaled_filter && !(mu_1 <= cc - e))) return CHASE_ERR_INVALID_ARG;
  if (precision != CHASE_FP64 && precision != CHASE_MIXED_BF16X3) return CHASE_ERR_INVALID_ARG;
  if (precision == CHASE_MIXED_BF16X3 && c->p.precision != CHASE_MIXED_BF16X3)
    return CHASE_ERR_INVALID_ARG;
  RC(check_degs(degs, ncols, 1 << 20));
  return filter_impl(c, reinterpret_cast<const double2*>(A), lda, reinterpret_cast<double2*>(V),
                     ldv, ncols, degs, cc, e, mu_1, precision, nullptr);
}

int chase_qr(chase_ctx* c, chase_c128* V, int64_t ldv, int64_t ncols, double cond_est,
             int32_t* variant_used) {
  if (!c || !V || ldv < c->N || ncols < 1 || ncols > c->ne || std::isnan(cond_est))
    return CHASE_ERR_INVALID_ARG;
  return qr_impl(c, reinterpret_cast<double2*>(V), ldv, ncols, cond_est, variant_used);
}

int chase_rayleigh_ritz(chase_ctx* c, const chase_c128* A, int64_t lda, chase_c128* V,
                        int64_t ldv, int64_t ncols, double* ritz) {
  if (!c || !A || !V || !ritz || lda < c->N || ldv < c->N || ncols < 1 || ncols > c->ne)
    return CHASE_ERR_INVALID_ARG;
  double2* Vd = reinterpret_cast<double2*>(V);
  CK(copy_cols(c->stream, c->N, ncols, Vd, ldv, c->V2, c->N));
  RC(rr_impl(c, reinterpret_cast<const double2*>(A), lda, c->V2, c->N, Vd, ldv, ncols, ritz));
  CK(cudaStreamSynchronize(c->stream));
  return CHASE_OK;
}

int chase_residuals(chase_ctx* c, const chase_c128* A, int64_t lda, const chase_c128* V,
                    int64_t ldv, const double* ritz, int64_t ncols, double* resid) {
  if (!c || !A || !V || !ritz || !resid || lda < c->N || ldv < c->N || ncols < 0 ||
      ncols > c->ne)
    return CHASE_ERR_INVALID_ARG;
  return resid_impl(c, reinterpret_cast<const double2*>(A), lda,
                    reinterpret_cast<const double2*>(V), ldv, ritz, ncols, resid);
}

int chase_solve(chase_ctx* c, const chase_c128* Ac, int64_t lda, chase_c128* Vc, int64_t ldv,
                const chase_c128* lanczos_start, int64_t ldl, double* ritz, double* resid,
                chase_stats* stats) {
  SolveState S;
  RC(solve_begin(S, c, reinterpret_cast<const double2*>(Ac), lda, reinterpret_cast<double2*>(Vc),
                 ldv, reinterpret_cast<const double2*>(lanczos_start), ldl, ritz, resid));
  while (solve_active(S)) {
    RC(solve_prepare(S));
    RC(solve_filter(S));
    RC(solve_complete(S));
  }
  return solve_end(S, stats);
}

}  // extern "C"
