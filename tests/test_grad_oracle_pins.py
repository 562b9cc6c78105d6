"""Pins of the gradient oracle (filter adjoint and eigenpair adjoint) against
facts fixed by mathematics, without the CUDA path.

- Polynomial of a diagonal matrix: the Frechet derivative is the
  Daleckii-Krein divided-difference matrix, p[a_j, a_k] off the diagonal and
  p'(a_j) on it, with p and p' from the Chebyshev closed forms
  (T_m = cos(m acos), T_m' = m U_{m-1}, U_{m-1}(cos t) = sin(m t) / sin t).
- Eigenpairs of a diagonal matrix with L = tr(X^H B X): second-order
  perturbation theory gives the gradient in closed form.
- Central finite differences on small random Hermitian problems.
"""
import numpy as np
import pytest

from oracle import chase_oracle as O
from oracle import grad_oracle as G
from synth import complex_normal, uniform01


def cheb_T(m, x):
    x = np.asarray(x, dtype=np.float64)
    out = np.empty_like(x)
    inside = np.abs(x) <= 1
    out[inside] = np.cos(m * np.arccos(x[inside]))
    xo = x[~inside]
    out[~inside] = np.sign(xo) ** m * np.cosh(m * np.arccosh(np.abs(xo)))
    return out


def cheb_dT(m, x):
    """T_m'(x) = m U_{m-1}(x)."""
    x = np.asarray(x, dtype=np.float64)
    out = np.empty_like(x)
    inside = np.abs(x) < 1
    th = np.arccos(x[inside])
    out[inside] = m * np.sin(m * th) / np.sin(th)
    xo = x[~inside]
    ph = np.arccosh(np.abs(xo))
    out[~inside] = m * np.sign(xo) ** (m - 1) * np.sinh(m * ph) / np.sinh(ph)
    return out


def rand_herm(n, seed, stream=90):
    Z = complex_normal(seed, stream, n * n).reshape(n, n)
    return 0.5 * (Z + Z.conj().T)


def rand_c(shape, seed, stream=91):
    return complex_normal(seed, stream, int(np.prod(shape))).reshape(shape)


@pytest.mark.parametrize("scaled", [True, False])
@pytest.mark.parametrize("deg", [1, 2, 7, 20])
def test_filter_vjp_daleckii_krein(scaled, deg):
    # distinct eigenvalues inside and outside the damped interval [c - e, c + e]
    N = 14
    c, e = 3.0, 2.0
    a = np.sort(np.concatenate([-1.5 + 2.4 * uniform01(5, 1, 4), 1.1 + 3.8 * uniform01(5, 2, 10)]))
    mu_1 = -1.5
    A = np.diag(a).astype(np.complex128)
    Ybar = rand_c((N, N), deg)
    x, x0 = (a - c) / e, (mu_1 - c) / e
    scale = 1.0 / cheb_T(deg, np.array([x0]))[0] if scaled else 1.0
    p = cheb_T(deg, x) * scale
    dp = cheb_dT(deg, x) / e * scale
    P = np.empty((N, N))
    for j in range(N):
        for k in range(N):
            P[j, k] = dp[j] if j == k else (p[j] - p[k]) / (a[j] - a[k])
    Abar, Vbar = G.filter_vjp(A, np.eye(N), deg, c, e, mu_1, Ybar, scaled)
    want = G.hermitian_part(Ybar * P)
    assert np.abs(Abar - want).max() <= 1e-11 * np.abs(want).max()
    np.testing.assert_allclose(Vbar, p[:, None] * Ybar, rtol=0, atol=1e-11 * np.abs(p).max())


def test_filter_vjp_finite_differences():
    N, n, deg = 10, 3, 6
    A = rand_herm(N, 3) + 2.0 * np.eye(N)
    V = rand_c((N, n), 4)
    W = rand_c((N, n), 5)
    lam = np.linalg.eigvalsh(A)
    c, e, mu_1 = (lam[-1] + lam[3]) / 2, (lam[-1] - lam[3]) / 2, lam[0]

    def loss(Am, Vm):
        Y = O.chebyshev_filter(Am, Vm, [deg] * n, c, e, mu_1)
        return float(np.real(np.sum(W.conj() * Y)))

    Abar, Vbar = G.filter_vjp(A, V, deg, c, e, mu_1, W)
    h = 1e-5
    for k in range(6):
        E = rand_herm(N, 100 + k)
        dV = rand_c((N, n), 200 + k)
        fd = (loss(A + h * E, V + h * dV) - loss(A - h * E, V - h * dV)) / (2 * h)
        an = float(np.real(np.sum(Abar.conj() * E) + np.sum(Vbar.conj() * dV)))
        assert abs(fd - an) <= 1e-7 * max(1.0, abs(an)), (k, fd, an)


def test_eig_vjp_diagonal_closed_form():
    # A = diag(a), L = sum w_i lambda_i + tr(X^H B X): the trace term's gradient
    # is 2 B_ji / (a_i - a_j) at (j, i) for i < nev <= j, Hermitian part
    N, nev = 9, 3
    a = np.array([-2.0, -1.3, -0.4, 0.5, 0.9, 1.7, 2.2, 3.1, 4.0])
    A = np.diag(a).astype(np.complex128)
    B = rand_herm(N, 7)
    w = np.array([0.3, -1.1, 0.7])
    lam, X = G.lowest_eigenpairs(A, nev)
    Abar = G.eig_vjp(A, nev, w, 2.0 * (B @ X))
    want = np.zeros((N, N), dtype=np.complex128)
    for i in range(nev):
        want[i, i] += w[i]
        for j in range(nev, N):
            want[j, i] += 2.0 * B[j, i] / (a[i] - a[j])
    want = G.hermitian_part(want)
    assert np.abs(Abar - want).max() <= 1e-13 * np.abs(want).max()


@pytest.mark.parametrize("N,nev,seed", [(12, 3, 1), (20, 6, 2)])
def test_eig_vjp_finite_differences(N, nev, seed):
    A = rand_herm(N, seed)
    B = rand_herm(N, seed + 50)
    w = uniform01(seed, 3, nev) - 0.5

    def loss(Am):
        lam, X = G.lowest_eigenpairs(Am, nev)
        return G.c4_loss(lam, X, w, B)

    lam, X = G.lowest_eigenpairs(A, nev)
    lb, xb = G.c4_loss_adjoints(lam, X, w, B)
    Abar = G.eig_vjp(A, nev, lb, xb)
    h = 1e-6
    for k in range(8):
        E = rand_herm(N, 300 + k)
        fd = (loss(A + h * E) - loss(A - h * E)) / (2 * h)
        an = float(np.real(np.sum(Abar.conj() * E)))
        assert abs(fd - an) <= 1e-6 * max(1.0, abs(an)), (k, fd, an)


def test_c4_loss_adjoints_finite_differences():
    N, nev = 10, 4
    X = rand_c((N, nev), 9)
    B = rand_herm(N, 10)
    w = uniform01(2, 2, nev)
    lam = uniform01(3, 3, nev)
    lb, xb = G.c4_loss_adjoints(lam, X, w, B)
    h = 1e-6
    for k in range(5):
        dX = rand_c((N, nev), 400 + k)
        dl = uniform01(5, 400 + k, nev)
        fd = (G.c4_loss(lam + h * dl, X + h * dX, w, B)
              - G.c4_loss(lam - h * dl, X - h * dX, w, B)) / (2 * h)
        an = float(np.dot(lb, dl) + np.real(np.sum(xb.conj() * dX)))
        assert abs(fd - an) <= 1e-7 * max(1.0, abs(an))
