/*
 * chase.h -- C ABI of a single-GPU (sm_103a) Chebyshev-filtered subspace
 * eigensolver for the lowest eigenpairs of a dense complex Hermitian matrix,
 * after Wu & Di Napoli, "Advancing the distributed Multi-GPU ChASE library
 * through algorithm optimization and NCCL library" (arXiv 2309.15595).
 *
 * Problem (Section 1): A x = lambda x with A^H = A in C^{N x N}; the nev lowest
 * eigenpairs are wanted and nex extra vectors widen the search space
 * (Alg. 2 "Require"/"Ensure").
 *
 * Conventions shared by every entry point
 *   - Matrices are complex128, interleaved (re, im), COLUMN-MAJOR (LAPACK):
 *     element (i, j) of A lives at A[i + j * lda]. Leading dimensions must be
 *     >= the number of rows. A must hold the full Hermitian matrix (both
 *     triangles); a row-major Hermitian buffer read column-major is conj(A).
 *   - Pointers named A, V, ritz, resid are DEVICE pointers owned by the caller.
 *     Pointers documented as host arrays are host memory.
 *   - All work is enqueued on the stream given to chase_create, in order.
 *     Calls that need a host decision (chase_qr, chase_solve, chase_lanczos,
 *     chase_rayleigh_ritz) synchronise that stream before returning; the others
 *     return after enqueueing.
 *   - The library allocates all of its workspace in chase_create and frees it in
 *     chase_destroy; apart from chase_solve_batch's small launch table and the
 *     gradient calls' workspace (documented below), no other call allocates
 *     device memory.
 *   - Every call returns a chase_status. On CHASE_ERR_INVALID_ARG nothing was
 *     enqueued. On CHASE_ERR_CUDA the context should be destroyed.
 *   - A context is not thread-safe; use one context per host thread.
 */
#ifndef CHASE_GB300_H
#define CHASE_GB300_H

#include <stdint.h>

#if defined(__GNUC__)
#define CHASE_API __attribute__((visibility("default")))
#else
#define CHASE_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum chase_status {
  CHASE_OK = 0,
  CHASE_ERR_INVALID_ARG = 1,   /* bad size, pointer, degree or parameter */
  CHASE_ERR_CUDA = 2,          /* a CUDA runtime call or kernel launch failed */
  CHASE_ERR_OOM = 3,           /* workspace allocation failed in chase_create */
  CHASE_ERR_QR_BREAKDOWN = 4,  /* the QR met non-finite values (the Householder
                                  fallback of Alg. 4 does not break down otherwise) */
  CHASE_ERR_HEEV_NOCONV = 5,   /* Jacobi sweep cap reached before convergence */
  CHASE_ERR_NOT_CONVERGED = 6  /* max_iter reached; outputs hold the best pairs */
} chase_status;

/* Filter arithmetic (the QR, Rayleigh-Ritz, residual and Lanczos steps are
 * always FP64). */
enum {
  CHASE_FP64 = 0,          /* filter HEMM in FP64 (DFMA) */
  CHASE_MIXED_BF16X3 = 1   /* filter in split-BF16 x3 on tensor cores (FP32
                              accumulation) while the residuals are above
                              switch_tol, FP64 afterwards */
};

/* QR variant codes (Alg. 4). */
enum {
  CHASE_QR_CHOLQR1 = 1,
  CHASE_QR_CHOLQR2 = 2,
  CHASE_QR_SHIFTED = 3,   /* shifted CholeskyQR pass + CholeskyQR2 */
  CHASE_QR_HOUSEHOLDER = 4, /* a POTRF of the shifted branch failed: Householder QR
                               of the input block (Alg. 4 fallback) */
  CHASE_QR_FALLBACK = CHASE_QR_HOUSEHOLDER  /* former name of the same code */
};

typedef struct chase_c128 { double re, im; } chase_c128;

typedef struct chase_params {
  int64_t N;              /* matrix order, >= 2 */
  int64_t nev;            /* wanted eigenpairs, >= 1 */
  int64_t nex;            /* extra search vectors, >= 0; nev + nex <= min(N, 3500) */
  int32_t deg_init;       /* first-iteration filter degree (20, Section 4.2), even */
  int32_t deg_max;        /* degree cap (36, Section 4.2) */
  int32_t deg_extra;      /* safety margin added by degreeOpt (2) */
  int32_t deg_opt;        /* 1: per-vector degree optimisation (Alg. 2 "opt") */
  int32_t max_iter;       /* MaxIter of Alg. 2 */
  int32_t lanczos_steps;  /* Lanczos steps per run (25), <= N */
  int32_t lanczos_vecs;   /* Lanczos runs (4), 1..8 */
  int32_t precision;      /* CHASE_FP64 or CHASE_MIXED_BF16X3 */
  int32_t scaled_filter;  /* 1: filter normalised at mu_1 (default); 0: plain
                             T_m((A - cI)/e) recurrence */
  int32_t fp64_tensor;    /* 1: the FP64 N x N products (filter in FP64, Rayleigh-Ritz
                             A Q, residual A V) run on the BF16 tensor cores with
                             exact digit slicing (FP64-class accuracy); 0: DFMA */
  double tol;             /* residual tolerance relative to ||A|| (1e-10, Section 4) */
  double switch_tol;      /* mixed -> FP64 switch, relative residual (1e-5) */
  int32_t heev_max_sweeps;  /* cap on each stage of the Rayleigh-Ritz Jacobi eigensolver
                               (sweeps, refinement steps); 0: library defaults (30 FP32
                               sweeps, 8 FP64 refinement steps, 40 FP64 sweeps). A cap
                               reached before convergence returns CHASE_ERR_HEEV_NOCONV */
  int32_t reserved;       /* must be 0 */
} chase_params;

typedef struct chase_stats {
  int32_t iters;          /* outer iterations done */
  int32_t locked;         /* converged (locked) pairs */
  int64_t matvecs;        /* sum of filter degrees over filtered columns */
  int64_t matvecs_mixed;  /* of which filtered in reduced precision */
  double b_sup, mu_1, mu_ne, norm_est;   /* Lanczos bounds and ||A|| estimate */
  double ms_lanczos, ms_filter, ms_qr, ms_rr, ms_resid, ms_total;
  double filter_flops;    /* 8 N^2 per MatVec */
  int32_t qr_variant_count[5];  /* index = CHASE_QR_* */
  int32_t switch_iter;    /* iteration at which the filter became FP64 (0: never mixed) */
  int64_t kernel_launches;  /* kernels this library launched during the solve */
  int32_t heev_sweeps;    /* heev iterations summed over the solve: FP32 Jacobi sweeps, FP64
                             refinement steps and FP64 Jacobi sweeps */
  int32_t heev_fp64_sweeps;  /* Jacobi heev: FP64 sweeps run for pairs the refinement could not separate */
  double ms_heev;         /* part of ms_rr spent in the Jacobi eigensolver */
  int32_t heev_cluster_solves;  /* Rayleigh-Ritz eigensolves whose near-degenerate pairs were
                                   finished cluster by cluster (no full FP64 sweep) */
  int32_t heev_cluster_max;     /* largest such cluster over the solve */
} chase_stats;

/* Fills *p with the defaults above for the given sizes. Host only. */
CHASE_API void chase_default_params(chase_params* p, int64_t N, int64_t nev, int64_t nex);

/* Creates a context: validates *p and allocates every workspace buffer for
 * order N and nev + nex vectors on the current CUDA device. stream may be NULL
 * (legacy default stream). Returns CHASE_ERR_OOM if allocation fails. */
CHASE_API int chase_create(const chase_params* p, void* stream, struct chase_ctx** out);

/* Frees the workspace and the context. Safe on NULL. */
CHASE_API int chase_destroy(struct chase_ctx* ctx);

/* Full solve, Alg. 2 on one GPU (the 2D grid collapses to one block):
 * Lanczos bounds, then {degreeOpt + sort, Filter, CondEst, 1D-CAQR, restore
 * locked, Rayleigh-Ritz, Residual, Locking} until nev pairs are locked or
 * max_iter is reached.
 *   A      device, N x N, lda >= N, read only.
 *   V      device, N x (nev+nex), ldv >= N: in = start block (need not be
 *          orthonormal), out = Ritz vectors; columns 0..nev-1 are the answer,
 *          ascending.
 *   lanczos_start  device, N x lanczos_vecs, ld = ldl; may be NULL, then the
 *          first lanczos_vecs columns of the input V start the Lanczos runs.
 *   ritz, resid  device, nev+nex doubles: Ritz values (ascending in 0..nev-1)
 *          and absolute residual norms ||A v - theta v||_2.
 *   stats  host, may be NULL.
 * Returns CHASE_ERR_NOT_CONVERGED if max_iter was reached (outputs are then the
 * current best pairs). */
CHASE_API int chase_solve(struct chase_ctx* ctx, const chase_c128* A, int64_t lda,
                chase_c128* V, int64_t ldv, const chase_c128* lanczos_start,
                int64_t ldl, double* ritz, double* resid, chase_stats* stats);

/* Spectral bounds by Lanczos (Alg. 1 "Lanczos", Alg. 2 first line): runs
 * nvec (<= lanczos_vecs) Lanczos recurrences of lanczos_steps steps from the
 * columns of Q0 (device, N x nvec, ldq >= N) and writes, to the HOST array
 * bounds[4]: b_sup, mu_1, mu_ne, norm_est (see the design notes for the DoS
 * reading). Synchronises. */
CHASE_API int chase_lanczos(struct chase_ctx* ctx, const chase_c128* A, int64_t lda,
                  const chase_c128* Q0, int64_t ldq, int64_t nvec, double* bounds);

/* Chebyshev filter, Eq. 1 with gamma_i = c, in place on V[:, 0:ncols]:
 * column j becomes p_{degs[j]}(A) v_j with p_m normalised at mu_1 (or plain
 * T_m((A-cI)/e) if scaled_filter = 0). degs is a HOST array of ncols EVEN
 * degrees >= 2, sorted ascending (Section 3.1 even-degree rule; Alg. 1 sort).
 * precision: CHASE_FP64 or CHASE_MIXED_BF16X3 (the latter needs a context
 * created with that precision; its first call for a given N and column count
 * on a device times the tensor-core kernel's raster orders once and keeps the
 * fastest, which never changes a result). Requires e > 0 and mu_1 <= c - e, so
 * that the normalisation T_m((mu_1 - c)/e) never vanishes. */
CHASE_API int chase_filter(struct chase_ctx* ctx, const chase_c128* A, int64_t lda,
                 chase_c128* V, int64_t ldv, int64_t ncols, const int32_t* degs,
                 double c, double e, double mu_1, int32_t precision);

/* 1D-CAQR of Alg. 4 on V[:, 0:ncols] (ncols <= nev+nex), in place: V becomes
 * Q with V_in = Q R, R upper triangular with positive real diagonal. The
 * variant follows cond_est (> 1e8 shifted, < 20 CholeskyQR1, else
 * CholeskyQR2); a CholeskyQR1/2 whose POTRF fails re-runs the shifted branch,
 * and a shifted branch whose POTRF fails (or that of the CholeskyQR2 after it)
 * reverts to Householder QR of the input block (Alg. 4). *variant_used (host,
 * may be NULL) receives a CHASE_QR_* code. Synchronises (POTRF info is a host
 * decision). Unlike Alg. 2, which runs the QR on all nev + nex columns and then
 * restores the locked ones from C2, this call factors exactly the columns it is
 * given: chase_solve does the restore itself, and a caller that wants it passes
 * the full block and copies its locked columns back. */
CHASE_API int chase_qr(struct chase_ctx* ctx, chase_c128* V, int64_t ldv, int64_t ncols,
             double cond_est, int32_t* variant_used);

/* Rayleigh-Ritz (Alg. 2 RR lines): with Q = V[:, 0:ncols] orthonormal, forms
 * G = Q^H A Q, diagonalises it with a two-sided Jacobi method and overwrites V
 * with the Ritz vectors Q Y; ritz (device, ncols doubles) receives the Ritz
 * values ascending. Synchronises. */
CHASE_API int chase_rayleigh_ritz(struct chase_ctx* ctx, const chase_c128* A, int64_t lda,
                        chase_c128* V, int64_t ldv, int64_t ncols, double* ritz);

/* Residual norms (Alg. 2 residual lines): resid[j] = ||A v_j - ritz[j] v_j||_2
 * for j < ncols. V, ritz, resid are device arrays. */
CHASE_API int chase_residuals(struct chase_ctx* ctx, const chase_c128* A, int64_t lda,
                    const chase_c128* V, int64_t ldv, const double* ritz,
                    int64_t ncols, double* resid);

/* Residual norms exactly like chase_residuals (same kernels, same results), for
 * callers that cannot allocate device memory and so cannot create a context:
 * code that lives inside another framework's memory budget (a caching allocator
 * or pool that owns the device memory) or that must not trigger the
 * device-wide synchronisation that cudaMalloc/cudaFree can imply. It needs no
 * chase_ctx and calls no allocating routine. The paper has no counterpart to
 * this entry point.
 *   A (N x N, lda >= N), V (N x ncols, ldv >= N), ritz, resid: device pointers
 *   owned by the caller, as for chase_residuals; stream: a cudaStream_t or NULL.
 * Scratch: a fixed 4 MiB array of doubles in the library's device memory
 * (every GPU that loads the library holds it until the process exits); the
 * call needs ceil(N/64) * ncols doubles of it and returns CHASE_ERR_INVALID_ARG
 * (with a message on stderr) above that, e.g. ncols > 1675 at N = 20000.
 * The first call on each device looks up the array's device address with that
 * device current and caches it for the life of the process; make that first
 * call before any stream capture. The cache assumes the device's primary
 * context (the CUDA runtime's, which torch uses) and no cudaDeviceReset in the
 * process: a reset reloads the library's device code elsewhere. All calls
 * share the one array: calls whose kernels overlap on the GPU (different
 * streams or host threads) race and give wrong results. Nothing in the array
 * needs to start at zero; each call writes every partial it reads. Returns
 * after enqueueing on `stream`. */
CHASE_API int chase_residuals_noalloc(const chase_c128* A, int64_t lda, const chase_c128* V,
                                      int64_t ldv, const double* ritz, int64_t N, int64_t ncols,
                                      double* resid, void* stream);

/* Many independent solves at once: problem k is chase_solve(ctxs[k], A[k],
 * lda[k], V[k], ldv[k], Q0 ? Q0[k] : NULL, ldq ? ldq[k] : 0, ritz[k],
 * resid[k], stats ? &stats[k] : NULL), and each problem's results are exactly
 * those of chase_solve on it alone. The problems advance through Alg. 2 in
 * lockstep, phase by phase. `threads` host threads (<= 0: 8) run every
 * problem's Lanczos start, degree/sort/CondEst step and QR / Rayleigh-Ritz /
 * residual / locking step on the problem's own context and stream (largest
 * N^2 (nev + nex) first), so that small problems overlap on the GPU. The
 * filter phase of all problems in the reduced-precision mode on one device
 * runs as one CUDA graph of grouped tensor-core launches, one launch per
 * degree step covering every such problem's tiles; so does the filter phase of
 * all problems in the FP64 mode with the tensor-core products (fp64_tensor),
 * per degree step one grouped digit-slicing launch and one grouped product
 * launch. Problems with the CUDA-core FP64 products filter with their own
 * launches. The split-BF16x3 filter's raster order is
 * chosen per shape by timing on its first use (see chase_filter). Warm starts
 * (a sequence of related matrices, Section 1) pass the previous Ritz vectors
 * as V. The contexts must be distinct. This call creates one extra stream per
 * device that holds grouped problems and small tables of launch parameters
 * (device and pinned host memory, under 1 KB per problem and degree step),
 * and frees them before returning. In stats, the grouped filter's time
 * and launches are charged to every problem of the group. status[k] receives
 * each return code; the call returns CHASE_OK if all are CHASE_OK, else the
 * first non-OK status in problem order. The paper solves one problem at a
 * time; this batching has no counterpart there. */
CHASE_API int chase_solve_batch(int64_t count, struct chase_ctx* const* ctxs,
                                const chase_c128* const* A, const int64_t* lda,
                                chase_c128* const* V, const int64_t* ldv,
                                const chase_c128* const* Q0, const int64_t* ldq,
                                double* const* ritz, double* const* resid, chase_stats* stats,
                                int32_t* status, int32_t threads);

/* ---------------------------------------------------------------- gradients
 * Adjoints for differentiating through the filter and the converged lowest
 * eigenpairs. The paper states the forward method only (Section 2); these are
 * its derivatives. Convention for a real loss L: the adjoint of a complex array
 * Z is Zbar = 2 dL/d conj(Z), so dL = Re sum(conj(Zbar) dZ) (the convention
 * torch uses). A is Hermitian, so the adjoint written for A is the Hermitian
 * part of the unconstrained one. Both calls use the context's product path
 * (FP64 CUDA-core or, with fp64_tensor, tensor-core FP64 for the products with
 * A), allocate their workspace on first use (kept until chase_destroy), and
 * synchronise the context's stream before returning. */

/* Adjoint of Y = p(A) V, the Eq. 1 recurrence with the same degree `deg` for
 * all ncols columns (Y_1 = alpha_1 (A - cI) V, Y_i = alpha_i (A - cI) Y_{i-1}
 * + beta_i Y_{i-2}, scaled or not as the context's scaled_filter says):
 * given Ybar (N x ncols), writes Abar (N x N) = herm(sum_i alpha_i Z_i Y_{i-1}^H)
 * and Vbar (N x ncols) = Z_0, where Z_deg = Ybar, Z_{deg+1} = 0 and
 * Z_{i-1} = alpha_i (A - cI) Z_i + beta_{i+1} Z_{i+1}. The states Y_i are
 * recomputed segment by segment from checkpoints taken every `checkpoint`
 * steps (<= 0: ceil(sqrt(deg))), so the workspace holds
 * 2 ceil(deg/s) + 3 s + 2 blocks of N x ncols instead of deg + 1.
 * All matrices column-major device arrays owned by the caller; Abar and Vbar
 * are overwritten and must not alias A, V or Ybar. 1 <= deg <= 64,
 * ncols <= nev + nex, e > 0 (and mu_1 <= c - e when scaled); else
 * CHASE_ERR_INVALID_ARG. */
CHASE_API int chase_filter_vjp(struct chase_ctx* ctx, const chase_c128* A, int64_t lda,
                               const chase_c128* V, int64_t ldv, int64_t ncols, int32_t deg,
                               double c, double e, double mu_1, const chase_c128* Ybar,
                               int64_t ldyb, chase_c128* Abar, int64_t ldab, chase_c128* Vbar,
                               int64_t ldvb, int32_t checkpoint);

/* Adjoint of the nev lowest eigenpairs (lambda_i, x_i) of A, computed from a
 * converged Ritz basis X (N x ne, nev <= ne <= nev + nex, columns 0..nev-1 the
 * wanted pairs converged to the solver's tolerance, e.g. the V and ritz that
 * chase_solve returns) and its Ritz values ritz (device, ne doubles, ascending).
 * Given lam_bar (device, nev doubles, or NULL for 0) and X_bar (N x nev, or
 * NULL for 0), writes
 *   Abar = herm( sum_i (lam_bar_i x_i + y_i) x_i^H ),
 *   y_i = sum_{j < nev, j != i} x_j (x_j^H xbar_i) / (ritz_i - ritz_j) - z_i,
 * where z_i solves (A - ritz_i I) z_i = (I - Xw Xw^H) xbar_i on the orthogonal
 * complement of the wanted block Xw = X[:, 0:nev] (conjugate gradients with the
 * operator projected onto that complement, per column, to ||r|| <= cg_tol ||b||,
 * at most cg_max_iter iterations, *cg_iters receives the count). The extra
 * Ritz pairs nev..ne-1 give the initial guess (the Galerkin solution in their
 * span). The first term is the Hellmann-Feynman derivative d lambda_i / dA =
 * x_i x_i^H; the rest is first-order perturbation theory of x_i split into the
 * wanted block and its complement, on which A - ritz_i I is positive definite
 * when ritz_{nev-1} lies below the rest of the spectrum. The loss must not
 * depend on the phase of each x_i, and the wanted eigenvalues must be simple.
 * Returns CHASE_ERR_NOT_CONVERGED (Abar still written) if the solves did not
 * reach cg_tol. */
CHASE_API int chase_eig_vjp(struct chase_ctx* ctx, const chase_c128* A, int64_t lda,
                            const chase_c128* X, int64_t ldx, const double* ritz, int64_t ne,
                            int64_t nev, const double* lam_bar, const chase_c128* X_bar,
                            int64_t ldxb, chase_c128* Abar, int64_t ldab, double cg_tol,
                            int32_t cg_max_iter, int32_t* cg_iters);

/* Alg. 5 condition estimate, host arithmetic on host arrays in the solver's
 * current column order: t' = (ritz[0]-c)/e, t = (ritz[locked]-c)/e,
 * cond = |rho(t)|^d |rho(t')|^(d_M - d), d = degs[locked],
 * d_M = max(degs[locked:n]). */
CHASE_API double chase_cond_est(const double* ritz, const int32_t* degs, int64_t n,
                      int64_t locked, double c, double e);

/* degreeOpt (host arithmetic, host arrays): for j < n,
 * degs[j] = even clamp of ceil(ln(resid[j]/tol_abs)/ln rho_j) + deg_extra
 * with rho_j = |t_j| + sqrt(t_j^2 - 1), t_j = (ritz[j]-c)/e. */
CHASE_API void chase_degree_opt(const double* resid, const double* ritz, int64_t n,
                      double c, double e, double tol_abs, int32_t deg_max,
                      int32_t deg_extra, int32_t* degs);

/* Human-readable name of a chase_status. */
CHASE_API const char* chase_status_string(int status);

#ifdef __cplusplus
}
#endif

#endif /* CHASE_GB300_H */
