"""Plain CPU FP64 oracle of the ChASE hot path (Wu & Di Napoli, arXiv 2309.15595).

TEST INFRASTRUCTURE ONLY. Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / reference legs of ``bench.py`` may import this module. The
product path (the CUDA library and its Python binding) never calls it.

Every function states the passage of the paper it follows. Library primitives
(numpy matmul, LAPACK Cholesky / eigh / Householder QR, a triangular solve) serve
as single steps; there is no blocking or fusion beyond what the paper states.
Readings of passages the paper leaves open are marked READING and listed in the
design notes; they are the same readings the CUDA path implements.

Parity status: every function here is pinned by ``tests/test_oracle_pins.py``
(closed forms, known spectra, textbook routines, invariants). Iteration and
MatVec counts of a full solve are "parity unpinned" (a degree rounded by
``ceil`` can flip on the last bit), see ``solve``.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np
import scipy.linalg
import scipy.linalg.lapack

U_ROUNDOFF = 2.0 ** -53  # unit round-off u of IEEE double (Alg. 4, shift s)

QR_CHOLQR1 = 1
QR_CHOLQR2 = 2
QR_SHIFTED = 3
QR_HOUSEHOLDER = 4


# --------------------------------------------------------------------- Lanczos
@dataclasses.dataclass
class LanczosResult:
    b_sup: float
    mu_1: float
    mu_ne: float
    norm_est: float
    ritz: list  # per run: (theta, tau, beta_k)


def lanczos_run(A: np.ndarray, q0: np.ndarray, k: int):
    """k steps of Hermitian Lanczos from q0 without re-orthogonalisation
    (Alg. 1 line "Lanczos"; READING: the paper defers the details, Section 2.1).
    Returns the tridiagonal T_k's eigenvalues theta (ascending), the DoS weights
    tau_i = |z_{1i}|^2 and the last off-diagonal beta_k."""
    q = q0 / np.linalg.norm(q0)
    q_prev = np.zeros_like(q)
    beta_prev = 0.0
    alphas, betas = [], []
    for j in range(k):
        w = A @ q - beta_prev * q_prev
        a = float(np.real(np.vdot(q, w)))
        w = w - a * q
        b = float(np.linalg.norm(w))
        alphas.append(a)
        betas.append(b)
        if j + 1 < k:
            q_prev, q, beta_prev = q, w / b, b
    T = np.diag(alphas) + np.diag(betas[:-1], 1) + np.diag(betas[:-1], -1)
    theta, Z = np.linalg.eigh(T)
    tau = np.abs(Z[0, :]) ** 2
    return theta, tau, betas[-1]


def lanczos_bounds(A: np.ndarray, Q0: np.ndarray, k: int, ne: int) -> LanczosResult:
    """Spectral bounds (b_sup, mu_1, mu_ne) from n_L Lanczos runs (Alg. 1
    "Lanczos", Alg. 2 first statement; READING of the unspecified DoS step):
      b_sup  = max over runs of (theta_max + |beta_k|)
      mu_1   = min over runs of theta_min
      mu_ne  = smallest pooled theta whose run-averaged cumulative weight reaches
               ne/N, clamped to [mu_1, b_sup)
      norm_est = max over runs of max(|theta_min|, |theta_max|)  (a lower bound
               of ||A||_2, used to make the residual tolerance relative)."""
    N = A.shape[0]
    nruns = Q0.shape[1]
    runs = [lanczos_run(A, Q0[:, r], k) for r in range(nruns)]
    b_sup = max(th[-1] + abs(bk) for th, _, bk in runs)
    mu_1 = min(th[0] for th, _, _ in runs)
    norm_est = max(max(abs(th[0]), abs(th[-1])) for th, _, _ in runs)
    thetas = np.concatenate([th for th, _, _ in runs])
    weights = np.concatenate([tau for _, tau, _ in runs]) / nruns
    order = np.argsort(thetas, kind="stable")
    cum = np.cumsum(weights[order])
    target = ne / N
    idx = int(np.searchsorted(cum, target, side="left"))
    idx = min(idx, len(order) - 1)
    mu_ne = float(thetas[order[idx]])
    mu_ne = min(max(mu_ne, mu_1), b_sup)
    return LanczosResult(float(b_sup), float(mu_1), mu_ne, float(norm_est), runs)


# ---------------------------------------------------------------------- Filter
def chebyshev_coefficients(dmax: int, c: float, e: float, mu_1: float, scaled: bool = True):
    """alpha_i, beta_i of Eq. 1 with gamma_i = c for i = 1..dmax.

    scaled (READING of Eq. 1, default): sigma_1 = e/(mu_1 - c),
    sigma_{i} = 1/(2/sigma_1 - sigma_{i-1});  Y_1 = (sigma_1/e)(A - cI)Y_0,
    Y_i = (2 sigma_i/e)(A - cI)Y_{i-1} - sigma_{i-1} sigma_i Y_{i-2}, which
    yields T_m((A-cI)/e) Y_0 / T_m((mu_1-c)/e).
    unscaled: Y_1 = (A-cI)Y_0/e, Y_i = 2(A-cI)Y_{i-1}/e - Y_{i-2}, which yields
    T_m((A-cI)/e) Y_0."""
    alpha = np.zeros(dmax + 1)
    beta = np.zeros(dmax + 1)
    if scaled:
        sigma1 = e / (mu_1 - c)
        alpha[1] = sigma1 / e
        sig = sigma1
        for i in range(2, dmax + 1):
            sig_new = 1.0 / (2.0 / sigma1 - sig)
            alpha[i] = 2.0 * sig_new / e
            beta[i] = -sig * sig_new
            sig = sig_new
    else:
        alpha[1] = 1.0 / e
        for i in range(2, dmax + 1):
            alpha[i] = 2.0 / e
            beta[i] = -1.0
    return alpha, beta


def chebyshev_filter(A, V, degs, c, e, mu_1, scaled=True):
    """Eq. 1 three-term recurrence with a degree per column (Alg. 1 "Filter",
    Alg. 2 filter line; Section 3.1: even degrees keep results in C).
    Column j of the result is p_{degs[j]}(A) V[:, j]."""
    V = np.array(V, dtype=np.complex128)
    degs = np.asarray(degs, dtype=np.int64)
    if V.shape[1] == 0:
        return V
    if np.any(degs < 1):
        raise ValueError("filter degrees must be >= 1")
    dmax = int(degs.max())
    alpha, beta = chebyshev_coefficients(dmax, c, e, mu_1, scaled)
    out = V.copy()
    Y_prev = V.copy()                      # Y_0
    Y = alpha[1] * (A @ V - c * V)         # Y_1
    out[:, degs == 1] = Y[:, degs == 1]
    for i in range(2, dmax + 1):
        act = degs >= i
        Y_new = alpha[i] * (A @ Y[:, act] - c * Y[:, act]) + beta[i] * Y_prev[:, act]
        Y_prev[:, act] = Y[:, act]
        Y[:, act] = Y_new
        done = degs == i
        out[:, done] = Y[:, done]
    return out


# ------------------------------------------------------------------- CondEst
def _rho(t: float) -> float:
    """|rho| = max{|t - sqrt(t^2-1)|, |t + sqrt(t^2-1)|} (Alg. 5). For |t| < 1
    the square root is imaginary and both roots t +- i sqrt(1-t^2) have
    modulus exactly 1."""
    d = t * t - 1.0
    if d < 0.0:
        return 1.0
    s = math.sqrt(d)
    return max(abs(t - s), abs(t + s))


def cond_est(ritz, c, e, degs, locked):
    """Alg. 5: estimate of kappa_2 of the filtered block.
    ritz and degs are in the solver's current column order (Lambda[1] is the
    first entry, Lambda[locked+1] the first active one)."""
    t_p = (ritz[0] - c) / e
    t = (ritz[locked] - c) / e
    rho = _rho(t)
    rho_p = _rho(t_p)
    d = int(degs[locked])
    d_max = int(np.max(degs[locked:]))
    return rho ** d * rho_p ** (d_max - d)


# ------------------------------------------------------------------------ CAQR
def cholesky_upper(R: np.ndarray):
    """POTRF: R = U^H U with U upper triangular; info = 0 on success, else the
    1-based index of the first non-positive pivot (LAPACK zpotrf)."""
    U, info = scipy.linalg.lapack.zpotrf(np.asfortranarray(R), lower=0, clean=1)
    return np.triu(U), int(info)


def trsm_right_upper(X: np.ndarray, U: np.ndarray) -> np.ndarray:
    """TRSM: X U^{-1} for upper-triangular U."""
    return scipy.linalg.solve_triangular(U, X.T, trans="T", lower=False).T


def cholesky_qr(X: np.ndarray, chol_degree: int):
    """Alg. 3: repeat {R = X^H X (SYRK/HERK); U = POTRF(R); X = X U^{-1}}."""
    X = np.array(X, dtype=np.complex128)
    for _ in range(chol_degree):
        R = X.conj().T @ X
        U, info = cholesky_upper(R)
        if info != 0:
            return X, info
        X = trsm_right_upper(X, U)
    return X, 0


def shift_value(m: int, n: int, fro2: float) -> float:
    """Alg. 4 shift s = 11 (m n + n (n + 1)) u ||X||_F^2."""
    return 11.0 * (m * n + n * (n + 1)) * U_ROUNDOFF * fro2


def householder_qr(X: np.ndarray) -> np.ndarray:
    """Textbook Householder QR (LAPACK zgeqrf) with diag(R) made real positive,
    the fallback of Alg. 4 when POTRF of the shifted Gram matrix fails."""
    Q, R = np.linalg.qr(X)
    d = np.diag(R)
    ph = np.where(np.abs(d) > 0, d / np.maximum(np.abs(d), 1e-300), 1.0)
    return Q * ph[None, :]


def select_qr_variant(est_cond: float) -> int:
    """Alg. 4 variant choice: > 1e8 shifted CholeskyQR2, < 20 CholeskyQR1,
    otherwise CholeskyQR2."""
    if est_cond > 1e8:
        return QR_SHIFTED
    if est_cond < 20:
        return QR_CHOLQR1
    return QR_CHOLQR2


def caqr(X: np.ndarray, est_cond: float):
    """Alg. 4 (1D-CAQR) on one process. Returns (Q, variant_used, info)."""
    X = np.array(X, dtype=np.complex128)
    m, n = X.shape
    variant = select_qr_variant(est_cond)
    if variant == QR_SHIFTED:
        R = X.conj().T @ X
        fro2 = float(np.real(np.trace(R)))
        s = shift_value(m, n, fro2)
        U, info = cholesky_upper(R + s * np.eye(n))
        if info == 0:
            Q, info = cholesky_qr(trsm_right_upper(X, U), 2)
            if info == 0:
                return Q, QR_SHIFTED, 0
        # Alg. 4 reverts to Householder QR when POTRF fails (READING: also when
        # the CholeskyQR2 that follows the shifted pass fails).
        return householder_qr(X), QR_HOUSEHOLDER, info
    passes = 1 if variant == QR_CHOLQR1 else 2
    Q, info = cholesky_qr(X, passes)
    if info != 0:
        # READING: Alg. 4 names no fallback for CholeskyQR1/2; a failed POTRF
        # there (the estimate was too low) re-runs the shifted branch.
        return caqr(X, np.inf)
    return Q, variant, 0


# -------------------------------------------------------------- Rayleigh-Ritz
def rayleigh_ritz(A: np.ndarray, Q: np.ndarray):
    """Alg. 2 RR block: W = A Q, G = Q^H W (made exactly Hermitian), heev(G) =
    (theta ascending, Y), back-transform V = Q Y. The small dense eigensolver is
    LAPACK's (Section 2.1 names a standard dense solver)."""
    W = A @ Q
    G = Q.conj().T @ W
    G = 0.5 * (G + G.conj().T)
    theta, Y = np.linalg.eigh(G)
    return theta, Q @ Y


def residuals(A: np.ndarray, V: np.ndarray, theta: np.ndarray) -> np.ndarray:
    """Alg. 2 residual block: r_j = || A v_j - theta_j v_j ||_2."""
    W = A @ V
    return np.linalg.norm(W - V * theta[None, :], axis=0)


# ------------------------------------------------- degreeOpt, locking, bounds
def degree_opt(resid, ritz, c, e, tol_abs, deg_max, deg_extra=2):
    """Alg. 1/2 degreeOpt (READING, the paper defers the formula): for each
    active column t = (theta - c)/e, rho = |t| + sqrt(t^2 - 1);
    d = ceil(ln(r / tol_abs) / ln rho) + deg_extra, clamped to [2, deg_max] and
    rounded up to even (Section 3.1); rho <= 1 gives deg_max."""
    dm_even = deg_max - (deg_max % 2)
    out = np.empty(len(resid), dtype=np.int64)
    for j, (r, th) in enumerate(zip(resid, ritz)):
        t = (th - c) / e
        rho = _rho(t)
        if rho <= 1.0:
            d = dm_even
        elif r <= tol_abs:
            d = 2
        else:
            x = (math.log(r) - math.log(tol_abs)) / math.log(rho)
            d = dm_even if x >= dm_even else math.ceil(x) + deg_extra
        d = max(2, min(d, dm_even))
        d += d % 2
        out[j] = min(d, dm_even)
    return out


def sort_active(degs, ritz):
    """Alg. 1 sort step: order of the active columns by (degree, Ritz value),
    stable."""
    return np.lexsort((np.arange(len(degs)), np.asarray(ritz), np.asarray(degs)))


def count_converged(resid, tol_abs) -> int:
    """Locking (Alg. 2): the contiguous prefix of the (ascending) active Ritz
    pairs with r_j <= tol_abs (READING: prefix only, so the locked set is always
    the lowest part)."""
    n = 0
    for r in resid:
        if r <= tol_abs:
            n += 1
        else:
            break
    return n


# ------------------------------------------------------------------ full solve
@dataclasses.dataclass
class SolveResult:
    ritz: np.ndarray
    V: np.ndarray
    resid: np.ndarray
    iters: int
    matvecs: int
    locked: int
    converged: bool
    qr_variants: list
    bounds: LanczosResult


def solve(A, V0, nev, nex, *, lanczos_start, lanczos_steps=25, deg_init=20,
          deg_max=36, deg_extra=2, tol=1e-10, max_iter=30, opt=True, scaled=True,
          trace=None):
    """Alg. 2 on one process (all blocks of the 2D grid are one block; Bcast and
    AllReduce are identities). Lowest end of the spectrum (Alg. 2 "Ensure").
    ``trace`` (optional) is called once per iteration with a dict holding the
    iteration number, the condition estimate and the filtered block."""
    A = np.asarray(A)
    N = A.shape[0]
    ne = nev + nex
    lz = lanczos_bounds(A, lanczos_start, lanczos_steps, ne)
    b_sup, mu_1, mu_ne = lz.b_sup, lz.mu_1, lz.mu_ne
    tol_abs = tol * lz.norm_est
    C = np.array(V0, dtype=np.complex128)
    C2 = C.copy()
    degs = np.full(ne, deg_init, dtype=np.int64)
    ritz = np.zeros(ne)
    resid = np.zeros(ne)
    locked, it, matvecs = 0, 1, 0
    c = (b_sup + mu_ne) / 2.0
    e = (b_sup - mu_ne) / 2.0
    variants = []
    while locked < nev and it <= max_iter:
        if it != 1:
            mu_1 = float(ritz.min())
            mu_ne = float(ritz.max())
            c = (b_sup + mu_ne) / 2.0
            e = (b_sup - mu_ne) / 2.0
            if opt:
                degs[locked:] = degree_opt(resid[locked:], ritz[locked:], c, e, tol_abs,
                                           deg_max, deg_extra)
                p = locked + sort_active(degs[locked:], ritz[locked:])
                C[:, locked:] = C[:, p]
                C2[:, locked:] = C2[:, p]
                ritz[locked:] = ritz[p]
                resid[locked:] = resid[p]
                degs[locked:] = degs[p]
        if it == 1:
            cond = cond_est(np.full(ne, mu_1), c, e, degs, locked)
        else:
            cond = cond_est(ritz, c, e, degs, locked)
        C[:, locked:] = chebyshev_filter(A, C[:, locked:], degs[locked:], c, e, mu_1, scaled)
        matvecs += int(np.sum(degs[locked:]))
        if trace is not None:
            trace(dict(iter=it, cond=cond, X=C.copy(), locked=locked, c=c, e=e,
                       degs=degs.copy()))
        Q, variant, info = caqr(C, cond)
        variants.append(variant)
        C = Q
        C[:, :locked] = C2[:, :locked]
        C2[:, locked:] = C[:, locked:]
        theta, Vr = rayleigh_ritz(A, C2[:, locked:])
        C[:, locked:] = Vr
        C2[:, locked:] = Vr
        ritz[locked:] = theta
        resid[locked:] = residuals(A, C[:, locked:], theta)
        locked += count_converged(resid[locked:], tol_abs)
        it += 1
    order = np.argsort(ritz[:max(locked, nev)], kind="stable")[:nev]
    return SolveResult(ritz[order].copy(), C[:, order].copy(), resid[order].copy(),
                       it - 1, matvecs, locked, locked >= nev, variants, lz)
