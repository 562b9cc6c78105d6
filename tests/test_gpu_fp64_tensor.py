"""FP64-accurate products on the BF16 tensor cores (fp64_tensor = 1) against the
FP64 oracle.

Each real operand is scaled per row/column to |x| < 1/2 (the diagonal of A is
left out and applied exactly in FP64) and cut into six signed 8-bit digits
(exact in BF16), leaving a truncation error below 2^-49 of the row or column
maximum; the 21 kept digit pairs are accumulated exactly (levels 2-5) or in
FP32 at weights <= 2^-32 of the leading level (levels 6-7), and the dropped
pairs weigh below 2^-56. The truncation errors of the K = 2N terms of a
product add with random signs, about sqrt(K) 2^-48 of max|a| max|y| per entry
(FP64 itself: about sqrt(K) 2^-53). Bounds used: filter columns
degs[j] * 2^-42 of the column's largest entry (sqrt(K) 2^-48 per degree at
K <= 1400, with a factor 4 of margin for the max/typical ratio of the scaled
rows; one lost digit level would exceed it), Ritz values 1e-12 ||A||,
residual norms 1e-9 relative, full solves the paper's 1e-10.
"""
import numpy as np
import pytest

from oracle import chase_oracle as O
from synth import Problem, complex_normal, config_problem

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def dev(x, lib):
    return lib.colmajor(torch.from_numpy(np.asfortranarray(x)).cuda())


def params(lib, p, **kw):
    return lib.default_params(p.N, p.nev, p.nex, fp64_tensor=1, **kw)


@pytest.mark.parametrize("N,ncols,dmax", [(512, 60, 20), (333, 37, 36), (700, 150, 36),
                                          (130, 1, 2)])
def test_tensor_fp64_filter_against_oracle(lib, N, ncols, dmax):
    p = Problem(N=N, nev=ncols - ncols // 4, nex=ncols // 4, spectrum="uniform", lo=-1.0,
                hi=4.0, reflectors=5, seed=N + 2)
    A, V = p.matrix(), p.start_block()
    rng = np.random.default_rng(N)
    degs = np.sort(2 * rng.integers(1, dmax // 2 + 1, ncols)).astype(np.int32)
    lam = p.eigenvalues()
    b_sup = lam[-1] * 1.01
    c, e, mu1 = (b_sup + lam[p.ne - 1]) / 2, (b_sup - lam[p.ne - 1]) / 2, lam[0]
    ref = O.chebyshev_filter(A, V, degs, c, e, mu1)
    with lib.Context(params(lib, p)) as ctx:
        Vd = dev(V, lib)
        ctx.chase_filter(dev(A, lib), Vd, ncols, degs, c, e, mu1)
        got = Vd.cpu().numpy()
    rel = np.abs(got - ref).max(axis=0) / np.abs(ref).max(axis=0)
    print(f"N={N} ncols={ncols}: max rel err {rel.max():.3e}")
    assert np.all(rel <= degs * 2.0 ** -42)


def matrix_with_cond(m, n, kappa, seed):
    U = np.linalg.qr(complex_normal(seed, 78, m * n).reshape(n, m).T)[0]
    W = np.linalg.qr(complex_normal(seed + 1, 77, n * n).reshape(n, n))[0]
    s = np.logspace(0, -np.log10(kappa), n)
    return np.asfortranarray((U * s[None, :]) @ W.conj().T)


@pytest.mark.parametrize("m,n,kappa,graded", [
    (400, 24, 5.0, 0), (333, 37, 1e4, 0), (700, 150, 1e6, 0), (500, 40, 1e11, 0),
    (300, 20, 1e15, 0), (129, 129, 10.0, 0), (600, 60, 1e10, 1), (400, 48, 1e6, 1)])
def test_tensor_fp64_qr(lib, m, n, kappa, graded):
    # Gram matrix X^H X as a digit-sliced product: error about sqrt(m) 2^-47 of
    # the column maxima instead of sqrt(m) 2^-53, so the unique (positive
    # diag R) Q matches the oracle to 1e-12 kappa instead of 1e-13 kappa; the
    # orthogonality bar stays 1e-12. graded: columns scaled over `kappa` like a
    # filtered block (column norms from T_d of the Ritz values).
    if graded:
        X = matrix_with_cond(m, n, 10.0, 7) * np.logspace(0, np.log10(kappa), n)[None, :]
        X = np.asfortranarray(X)
    else:
        X = matrix_with_cond(m, n, kappa, 7)
    Qo, vo, _ = O.caqr(X, kappa)
    with lib.Context(lib.default_params(m, n, 0, fp64_tensor=1)) as ctx:
        Xd = dev(X, lib)
        v = ctx.chase_qr(Xd, n, kappa)
        Q = Xd.cpu().numpy()
    orth = np.abs(Q.conj().T @ Q - np.eye(n)).max()
    print(f"m={m} n={n} kappa={kappa:.0e}: variant {v} (oracle {vo}), orth {orth:.2e}, "
          f"vs oracle {np.abs(Q - Qo).max():.2e}")
    if kappa <= 1e6:
        assert v == vo
        assert np.abs(Q - Qo).max() <= 1e-12 * kappa * 10
    else:
        assert v in (3, 4)
    assert orth <= 1e-12
    R = Q.conj().T @ X
    assert np.abs(np.tril(R, -1)).max() <= 1e-12 * max(1.0, kappa * 1e-3) * np.abs(R).max()
    assert np.all(np.diag(R).real > 0)


@pytest.mark.parametrize("N,n", [(400, 30), (300, 65), (600, 129)])
def test_tensor_fp64_rayleigh_ritz_and_residuals(lib, N, n):
    p = Problem(N=N, nev=n - n // 4, nex=n // 4, spectrum="uniform", lo=0.5, hi=9.0,
                reflectors=6, seed=N + n)
    A = p.matrix()
    Q = np.asfortranarray(np.linalg.qr(p.start_block())[0])
    th_o, V_o = O.rayleigh_ritz(A, Q)
    r_o = O.residuals(A, V_o, th_o)
    with lib.Context(params(lib, p)) as ctx:
        Vd = dev(Q, lib)
        Ad = dev(A, lib)
        ritz = torch.zeros(n, dtype=torch.float64, device="cuda")
        ctx.chase_rayleigh_ritz(Ad, Vd, n, ritz)
        th = ritz.cpu().numpy()
        resid = torch.zeros(n, dtype=torch.float64, device="cuda")
        ctx.chase_residuals(Ad, Vd, ritz, n, resid)
        r = resid.cpu().numpy()
    assert np.abs(th - th_o).max() <= 1e-12 * p.norm2()
    np.testing.assert_allclose(r, r_o, rtol=1e-9)
    V = Vd.cpu().numpy()
    assert np.abs(V.conj().T @ V - np.eye(n)).max() <= 1e-12


@pytest.mark.parametrize("precision", [0, 1])
def test_tensor_fp64_solve_c1(lib, precision):
    p = config_problem("C1")
    A = p.matrix()
    V0, Q0 = p.start_block(), p.lanczos_start()
    with lib.Context(params(lib, p, precision=precision)) as ctx:
        Vd = dev(V0, lib)
        ritz = torch.zeros(p.ne, dtype=torch.float64, device="cuda")
        resid = torch.zeros_like(ritz)
        st = ctx.chase_solve(dev(A, lib), Vd, ritz, resid, lanczos_start=dev(Q0, lib))
    assert st["status"] == 0
    lam = p.eigenvalues()
    nA = p.norm2()
    r = ritz.cpu().numpy()[:p.nev]
    V = Vd.cpu().numpy()[:, :p.nev]
    assert np.abs(r - lam[:p.nev]).max() <= 1e-10 * nA
    res = np.linalg.norm(A @ V - V * r[None, :], axis=0)
    assert res.max() <= 1e-10 * nA
    assert np.abs(V.conj().T @ V - np.eye(p.nev)).max() <= 1e-12


def localized_orthonormal(m, n, seed):
    """Orthonormal columns that each hold one entry near 1 (a nearly converged
    block of localised eigenvectors): the digit scale of every column is the
    largest possible, which is the worst case for the digit-sliced products."""
    rng = np.random.default_rng(seed)
    E = np.zeros((m, n), dtype=np.complex128)
    E[rng.permutation(m)[:n], np.arange(n)] = 1.0
    Z = complex_normal(seed, 96, m * n).reshape(n, m).T
    Q, R = np.linalg.qr(E + 0.02 * Z)
    return Q * (np.diag(R) / np.abs(np.diag(R)))[None, :]


@pytest.mark.parametrize("m,n,kappa,kind", [
    (2037, 200, 1e3, "collinear"), (2037, 200, 1e6, "collinear"), (700, 130, 1e5, "graded"),
    (2037, 200, 1e7, "graded"), (1500, 300, 3e7, "collinear")])
@pytest.mark.parametrize("tensor", [0, 1])
def test_qr_triangular_solve_is_backward_stable(lib, m, n, kappa, kind, tensor):
    """X = Q0 T with Q0 localised and orthonormal and T upper triangular with a
    positive diagonal, so Q0 is the exact Q factor. kind = collinear: T =
    diag(s) (I + U) (every column dominated by the first: a filtered block's
    true ill-conditioning, kappa(X) ~ kappa); graded: T = (I + U) diag(s)
    (columns scaled over kappa: equilibrated, X is well conditioned).

    The span test holds at any kappa: with P the orthogonal projector onto
    span(Q) (from an exactly orthonormalised copy of Q, so that Q's own
    orthogonality error does not enter), a QR whose span is that of X + dX
    gives ||X_j - P X_j|| <= ||dX_j|| for every column, and the bound
    2e-14 ||X_j|| is the backward error the triangular solves may leave (the
    oracle's FP64 CholeskyQR2 gives about 1e-15 here, LAPACK's Householder QR
    the same). The forward error ||Q - Q0|| is that backward error times the
    conditioning of the columns' directions: at most 1e-12 for the graded
    block, and 2e-15 kappa for the collinear one (the oracle's FP64
    CholeskyQR2 gives |Q - Q0| of about 6e-18 kappa on the collinear ones)."""
    Q0 = localized_orthonormal(m, n, int(kappa) % 1000 + n)
    s = np.logspace(0, -np.log10(kappa), n)
    U = np.triu(complex_normal(n, 97, n * n).reshape(n, n), 1) * (0.3 / np.sqrt(n))
    T = (s[:, None] * (np.eye(n) + U)) if kind == "collinear" else ((np.eye(n) + U) * s[None, :])
    X = np.asfortranarray(Q0 @ T)
    with lib.Context(lib.default_params(m, n, 0, fp64_tensor=tensor)) as ctx:
        Xd = dev(X, lib)
        v = ctx.chase_qr(Xd, n, kappa)
        Q = Xd.cpu().numpy()
    orth = np.abs(Q.conj().T @ Q - np.eye(n)).max()
    P = np.linalg.qr(Q)[0]
    span = (np.linalg.norm(X - P @ (P.conj().T @ X), axis=0) / np.linalg.norm(X, axis=0)).max()
    fwd = np.abs(Q - Q0).max()
    print(f"{kind} m={m} n={n} kappa={kappa:.0e} tensor={tensor}: variant {v}, orth {orth:.2e}, "
          f"span residual {span:.2e}, |Q - Q0| {fwd:.2e}")
    assert orth <= 1e-12
    assert span <= 2e-14
    assert fwd <= (1e-12 if kind == "graded" else 2e-15 * kappa)
    R = Q.conj().T @ X
    assert np.all(np.diag(R).real > 0)
