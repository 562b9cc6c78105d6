"""Pins of the CPU oracle against facts fixed by the paper and by mathematics.

Nothing here calls the CUDA path. Each test checks the oracle against something
other than itself: closed forms of Chebyshev polynomials, matrices with exactly
known spectra, textbook routines, brute-force Jacobi on tiny inputs, invariants
(Courant-Fischer, QR uniqueness) and the paper's stated bound property of the
condition estimate (Section 4.2).
"""
import math

import numpy as np
import pytest

from oracle import chase_oracle as O
from synth import Problem, complex_normal, config_problem, uniform01


# ----------------------------------------------------------------- helpers
def cheb_T(m, t):
    """T_m(t) from its closed forms: cos(m acos t) on [-1, 1],
    sign(t)^m cosh(m acosh |t|) outside."""
    t = np.asarray(t, dtype=np.float64)
    out = np.empty_like(t)
    inside = np.abs(t) <= 1
    out[inside] = np.cos(m * np.arccos(t[inside]))
    ti = t[~inside]
    out[~inside] = np.sign(ti) ** m * np.cosh(m * np.arccosh(np.abs(ti)))
    return out


def random_unitary(n, seed):
    z = complex_normal(seed, 77, n * n).reshape(n, n)
    q, r = np.linalg.qr(z)
    return q * (np.diag(r) / np.abs(np.diag(r)))[None, :]


def matrix_with_cond(m, n, kappa, seed):
    U = np.linalg.qr(complex_normal(seed, 78, m * n).reshape(n, m).T)[0]
    W = random_unitary(n, seed + 1)
    s = np.logspace(0, -np.log10(kappa), n)
    return np.asfortranarray((U * s[None, :]) @ W.conj().T)


def brute_jacobi_eigvals(H, sweeps=60):
    """Cyclic two-sided Jacobi on a tiny Hermitian matrix, pure Python loops."""
    A = np.array(H, dtype=np.complex128)
    n = A.shape[0]
    for _ in range(sweeps):
        off = math.sqrt(sum(abs(A[i, j]) ** 2 for i in range(n) for j in range(n) if i != j))
        if off < 1e-15 * np.linalg.norm(A):
            break
        for p in range(n - 1):
            for q in range(p + 1, n):
                apq = A[p, q]
                if abs(apq) < 1e-300:
                    continue
                phase = apq / abs(apq)
                tau = (A[q, q].real - A[p, p].real) / (2 * abs(apq))
                t = math.copysign(1.0, tau) / (abs(tau) + math.sqrt(1 + tau * tau))
                c = 1 / math.sqrt(1 + t * t)
                s = t * c
                J = np.eye(n, dtype=np.complex128)
                J[p, p] = c
                J[q, q] = c
                J[p, q] = s * phase
                J[q, p] = -s * np.conj(phase)
                A = J.conj().T @ A @ J
    return np.sort(np.diag(A).real)


# ----------------------------------------------------------- generator pins
def test_generator_known_spectrum():
    p = Problem(N=96, nev=4, nex=4, spectrum="uniform", lo=-1.0, hi=3.0, reflectors=5, seed=9)
    A = p.matrix()
    lam = p.eigenvalues()
    X = p.eigenvectors(np.arange(p.N))
    assert np.allclose(A, A.conj().T, atol=0, rtol=0)
    assert A.flags.f_contiguous
    assert np.abs(X.conj().T @ X - np.eye(p.N)).max() < 1e-13
    assert np.abs(A @ X - X * lam[None, :]).max() < 1e-13 * p.norm2()


def test_generator_torch_build_matches_numpy():
    torch = pytest.importorskip("torch")
    p = Problem(N=80, nev=4, nex=4, reflectors=6, seed=3)
    A = p.matrix()
    At = p.matrix_torch("cpu")
    assert At.stride(0) == 1
    assert np.abs(At.numpy() - A).max() < 1e-13 * p.norm2()


def test_rng_counter_addressing():
    full = uniform01(5, 2, 100)
    assert np.array_equal(full[40:60], uniform01(5, 2, 20, offset=40))
    z = complex_normal(5, 3, 200000)
    assert abs(np.mean(np.abs(z) ** 2) - 1.0) < 0.01
    assert abs(np.mean(z.real)) < 0.01 and abs(np.var(z.real) - 0.5) < 0.01


@pytest.mark.parametrize("name", ["C1", "C3"])
def test_config_spectra(name):
    over = {} if name == "C1" else dict(N=400, nev=45, nex=15, n_low=60)
    p = config_problem(name, **over)
    lam = p.eigenvalues()
    assert np.all(np.diff(lam) >= 0)
    if name == "C1":
        k = np.arange(1, p.N + 1)
        assert np.allclose(lam, 10 * (1e-4 + (k - 1) * (1 - 1e-4) / (p.N - 1)), rtol=1e-15)
    else:
        low = lam[:p.n_low]
        assert low.min() >= -2.0 and low.max() < 0
        # every clustered value has a partner 1e-3 away (clusters may overlap)
        dist = np.abs(np.abs(low[:, None] - low[None, :]) - 1e-3)
        assert np.all(dist.min(axis=1) < 1e-12)
        assert lam[p.n_low:].min() >= 0 and lam.max() <= 50


# -------------------------------------------------------------- filter pins
@pytest.mark.parametrize("scaled", [True, False])
def test_filter_closed_form_diagonal(scaled):
    N = 64
    lam = np.linspace(-1.0, 3.0, N)
    A = np.diag(lam).astype(np.complex128)
    V = complex_normal(1, 11, N * 6).reshape(6, N).T
    degs = np.array([2, 2, 4, 10, 20, 36])
    c, e, mu1 = 1.75, 1.25, -1.0
    Y = O.chebyshev_filter(A, V, degs, c, e, mu1, scaled=scaled)
    for j, m in enumerate(degs):
        p = cheb_T(m, (lam - c) / e)
        if scaled:
            p = p / cheb_T(m, np.array([(mu1 - c) / e]))[0]
        np.testing.assert_allclose(Y[:, j], p * V[:, j], rtol=1e-11, atol=1e-11 * np.abs(p).max())


def test_filter_closed_form_dense_known_spectrum():
    p = Problem(N=72, nev=6, nex=4, spectrum="uniform", lo=0.0, hi=5.0, reflectors=4, seed=4)
    A = p.matrix()
    lam = p.eigenvalues()
    X = p.eigenvectors(np.arange(p.N))
    V = p.start_block()
    degs = np.array([2] * 3 + [8] * 4 + [16] * 3)
    c, e, mu1 = 3.0, 2.0, 0.0
    Y = O.chebyshev_filter(A, V, degs, c, e, mu1)
    for j, m in enumerate(degs):
        pm = cheb_T(m, (lam - c) / e) / cheb_T(m, np.array([(mu1 - c) / e]))[0]
        ref = X @ (pm * (X.conj().T @ V[:, j]))
        assert np.linalg.norm(Y[:, j] - ref) <= 1e-12 * np.linalg.norm(ref)


def test_filter_degree_one_and_empty():
    A = np.diag([1.0, 2.0]).astype(np.complex128)
    V = np.eye(2, dtype=np.complex128)
    Y = O.chebyshev_filter(A, V, [1, 1], 0.0, 1.0, -1.0, scaled=False)
    assert np.allclose(Y, A)
    assert O.chebyshev_filter(A, V[:, :0], [], 0.0, 1.0, -1.0).shape == (2, 0)


# ------------------------------------------------------------- CondEst pins
def _rho_acosh(t):
    return math.exp(math.acosh(abs(t))) if abs(t) > 1 else 1.0


def test_cond_est_closed_form():
    c, e = 1.0, 2.0
    ritz = np.array([-5.0, -3.0, -2.0, 0.5, 2.0])  # t' = -3, t(locked=1) = -2
    degs = np.array([0, 6, 8, 10, 14])
    got = O.cond_est(ritz, c, e, degs, 1)
    ref = _rho_acosh(-2.0) ** 6 * _rho_acosh(-3.0) ** (14 - 6)
    assert got == pytest.approx(ref, rel=1e-12)
    # |t| <= 1 gives |rho| = 1 (complex roots on the unit circle)
    assert O.cond_est(np.array([1.5, 1.5]), c, e, np.array([4, 4]), 0) == pytest.approx(1.0)


@pytest.mark.parametrize("prob", [
    config_problem("C1"),
    Problem(N=500, nev=50, nex=20, spectrum="clusters", lo=-2, hi=50, n_low=70,
            spacing=1e-3, reflectors=6, seed=3)])
def test_cond_est_bounds_condition_number(prob):
    """Section 4.2: kappa_est bounds kappa_2 of the filtered (active) block from
    above at every iteration (iteration 1 may miss by the last digit). Alg. 5's
    formula is the ratio of the largest filtered column, (rho/rho')^d, to the
    smallest, rho'^(-d_M), of the filter normalised at mu_1."""
    A = prob.matrix()
    V0 = np.linalg.qr(prob.start_block())[0]
    seen = []

    def trace(d):
        s = np.linalg.svd(d["X"][:, d["locked"]:], compute_uv=False)
        seen.append((d["iter"], d["cond"], s[0] / s[-1]))

    O.solve(A, V0, prob.nev, prob.nex, lanczos_start=prob.lanczos_start(), trace=trace)
    assert len(seen) >= 3
    for it, est, com in seen:
        slack = 0.9 if it == 1 else 1.0
        assert est >= slack * com, (it, est, com)


# ---------------------------------------------------------------- QR pins
def test_shift_value_hand():
    assert O.shift_value(4, 2, 3.0) == pytest.approx(11 * (4 * 2 + 2 * 3) * 2.0 ** -53 * 3.0)


@pytest.mark.parametrize("kappa,variant,orth_tol", [
    (5.0, O.QR_CHOLQR1, 1e-13), (1e4, O.QR_CHOLQR2, 1e-13), (1e7, O.QR_CHOLQR2, 1e-13),
    (1e12, O.QR_SHIFTED, 1e-12), (1e13, O.QR_SHIFTED, 1e-12),
    (1e15, O.QR_HOUSEHOLDER, 1e-12)])
def test_caqr_variants(kappa, variant, orth_tol):
    X = matrix_with_cond(300, 24, kappa, 3)
    Q, used, info = O.caqr(X, kappa)
    # kappa = 1e15 exceeds what one shift plus CholeskyQR2 handles at this m, n
    # (kappa * sqrt(11 (mn + n(n+1)) u) > u^-1/2), so a later POTRF fails and
    # Alg. 4 reverts to Householder QR.
    assert used == variant
    assert np.abs(Q.conj().T @ Q - np.eye(24)).max() < orth_tol
    R = Q.conj().T @ X
    assert np.abs(np.tril(R, -1)).max() <= 1e-12 * np.linalg.norm(X, 2) * (1 if kappa < 1e10 else kappa * 1e-4)
    assert np.all(np.diag(R).real > 0)
    assert np.linalg.norm(Q @ R - X) <= 1e-13 * np.linalg.norm(X)
    if kappa <= 1e4:  # QR with positive diagonal is unique: equals Householder's
        Qh = O.householder_qr(X)
        assert np.abs(Q - Qh).max() < 1e-11 * kappa


def test_caqr_selection_thresholds():
    assert O.select_qr_variant(19.9) == O.QR_CHOLQR1
    assert O.select_qr_variant(20.0) == O.QR_CHOLQR2
    assert O.select_qr_variant(1e8) == O.QR_CHOLQR2
    assert O.select_qr_variant(1.0001e8) == O.QR_SHIFTED


def test_potrf_info_and_householder_fallback(monkeypatch):
    _, info = O.cholesky_upper(np.diag([1.0, -1.0, 2.0]).astype(np.complex128))
    assert info == 2
    X = matrix_with_cond(100, 8, 10.0, 5)
    real = O.cholesky_upper
    monkeypatch.setattr(O, "cholesky_upper", lambda R: (R, 1))
    Q, used, info = O.caqr(X, 1e12)
    monkeypatch.setattr(O, "cholesky_upper", real)
    assert used == O.QR_HOUSEHOLDER and info == 1
    assert np.abs(Q.conj().T @ Q - np.eye(8)).max() < 1e-13


# ---------------------------------------------------- Rayleigh-Ritz, residual
def test_rayleigh_ritz_invariant_subspace():
    p = Problem(N=120, nev=6, nex=4, spectrum="uniform", lo=0.5, hi=9.0, reflectors=6, seed=8)
    A = p.matrix()
    lam = p.eigenvalues()
    X = p.eigenvectors(np.arange(10))
    Q = X @ random_unitary(10, 2)
    theta, V = O.rayleigh_ritz(A, Q)
    assert np.abs(theta - lam[:10]).max() < 1e-13 * p.norm2()
    assert np.abs(np.abs(np.sum(V.conj() * X, axis=0)) - 1).max() < 1e-12


def test_rayleigh_ritz_courant_fischer():
    p = Problem(N=150, nev=6, nex=4, reflectors=6, seed=10)
    A = p.matrix()
    lam = p.eigenvalues()
    Q = np.linalg.qr(p.start_block())[0]
    theta, _ = O.rayleigh_ritz(A, Q)
    assert np.all(theta >= lam[:10] - 1e-12) and np.all(theta <= lam[-10:] + 1e-12)


def test_residuals_closed_form():
    p = Problem(N=60, nev=3, nex=3, reflectors=3, seed=6)
    A = p.matrix()
    lam = p.eigenvalues()
    X = p.eigenvectors([0, 1, 2])
    delta = np.array([0.0, 1e-3, -0.25])
    r = O.residuals(A, X, lam[:3] + delta)
    np.testing.assert_allclose(r, np.abs(delta), atol=1e-13 * p.norm2())


# ------------------------------------------------------------ Lanczos pins
def test_lanczos_exact_on_diagonal():
    """N Lanczos steps on a diagonal matrix reproduce the spectrum exactly, and the
    Gauss weights tau_i equal |q_0,i|^2 (the DoS of the start vector)."""
    lam = np.array([0.5, 1.0, 1.5, 2.0, 4.0, 5.0, 7.5, 9.0])
    w = np.array([0.05, 0.1, 0.2, 0.15, 0.1, 0.1, 0.2, 0.1])
    A = np.diag(lam).astype(np.complex128)
    q = (np.sqrt(w) * np.exp(1j * np.arange(8)))[:, None]
    lz = O.lanczos_bounds(A, q, 8, 3)      # target weight 3/8 = 0.375
    th, tau, bk = lz.ritz[0]
    np.testing.assert_allclose(th, lam, atol=1e-12)
    np.testing.assert_allclose(tau, w, atol=1e-12)
    # cumulative weights 0.05, 0.15, 0.35, 0.50: first reaching 0.375 is lam_4
    assert lz.mu_1 == pytest.approx(0.5) and lz.mu_ne == pytest.approx(2.0)
    assert lz.b_sup == pytest.approx(9.0, abs=1e-10) and lz.norm_est == pytest.approx(9.0)


def test_lanczos_bounds_enclose_spectrum():
    p = config_problem("C1")
    lz = O.lanczos_bounds(p.matrix(), p.lanczos_start(), 25, p.ne)
    lam = p.eigenvalues()
    assert lz.b_sup >= lam[-1]
    assert lz.mu_1 >= lam[0] - 1e-12
    assert lz.norm_est <= p.norm2() + 1e-12
    assert lz.mu_1 <= lz.mu_ne < lz.b_sup


# ------------------------------------------------- degreeOpt / locking pins
def test_degree_opt_closed_form():
    c, e, tol_abs = 0.0, 1.0, 1e-10
    t = -1.25                      # rho = 2
    rho = _rho_acosh(t)
    assert rho == pytest.approx(2.0)
    r = np.array([tol_abs * rho ** 9.5, tol_abs * rho ** 10.5, tol_abs * 0.5, 1e300, 1.0])
    th = np.array([t, t, t, t, -0.5])
    d = O.degree_opt(r, th, c, e, tol_abs, 36, 2)
    # ceil(9.5)+2 = 12; ceil(10.5)+2 = 13 -> 14; converged -> minimum 2; cap 36;
    # |t| <= 1 -> maximum degree
    assert list(d) == [12, 14, 2, 36, 36]


def test_count_converged_prefix_only():
    assert O.count_converged([1e-12, 2e-11, 5e-10, 1e-12], 1e-10) == 2
    assert O.count_converged([1e-9, 1e-12], 1e-10) == 0


def test_sort_active_by_degree_then_value():
    p = O.sort_active(np.array([6, 4, 6, 4]), np.array([0.3, 0.9, 0.1, 0.2]))
    assert list(p) == [3, 1, 2, 0]


# ------------------------------------------------------------ full solve
def principal_sines(U, X):
    Qu = np.linalg.qr(U)[0]
    s = np.linalg.svd(X.conj().T @ Qu, compute_uv=False)
    return np.sqrt(np.clip(1 - s ** 2, 0, None))


def test_solve_c1_against_exact_spectrum():
    p = config_problem("C1")
    A = p.matrix()
    lam = p.eigenvalues()
    r = O.solve(A, p.start_block(), p.nev, p.nex, lanczos_start=p.lanczos_start())
    nA = p.norm2()
    assert r.converged
    assert np.abs(r.ritz - lam[:p.nev]).max() <= 1e-10 * nA
    res = np.linalg.norm(A @ r.V - r.V * r.ritz[None, :], axis=0)
    assert res.max() <= 1e-10 * nA
    assert np.abs(r.V.conj().T @ r.V - np.eye(p.nev)).max() <= 1e-12
    gap = lam[p.nev] - lam[p.nev - 1]
    sines = principal_sines(r.V, p.eigenvectors(np.arange(p.nev)))
    assert sines.max() <= max(1e-8, 2 * res.max() / gap)
    # conjugation guard: conj(A) = A^T has the same spectrum
    rc = O.solve(A.conj(), p.start_block().conj(), p.nev, p.nex,
                 lanczos_start=p.lanczos_start().conj())
    assert np.abs(rc.ritz - lam[:p.nev]).max() <= 1e-10 * nA


def test_solve_tiny_against_brute_force_jacobi():
    z = complex_normal(21, 5, 16 * 16).reshape(16, 16)
    H = np.asfortranarray(0.5 * (z + z.conj().T))
    ref = brute_jacobi_eigvals(H)
    V0 = np.asfortranarray(complex_normal(21, 6, 16 * 6).reshape(6, 16).T)
    Q0 = np.asfortranarray(complex_normal(21, 7, 16 * 2).reshape(2, 16).T)
    r = O.solve(H, V0, 3, 3, lanczos_start=Q0, lanczos_steps=8, max_iter=60)
    assert r.converged
    np.testing.assert_allclose(r.ritz, ref[:3], atol=1e-10 * np.abs(ref).max())


def test_solve_gap_spectrum_matches_scipy_eigh():
    scipy_linalg = pytest.importorskip("scipy.linalg")
    p = Problem(N=300, nev=12, nex=8, spectrum="gap", lo=0.0, hi=10.0, n_low=12,
                spacing=0.05, reflectors=6, seed=12)
    A = p.matrix()
    r = O.solve(A, p.start_block(), p.nev, p.nex, lanczos_start=p.lanczos_start())
    w = scipy_linalg.eigh(A, eigvals_only=True, subset_by_index=[0, p.nev - 1])
    assert r.converged
    np.testing.assert_allclose(r.ritz, w, atol=1e-10 * p.norm2())
