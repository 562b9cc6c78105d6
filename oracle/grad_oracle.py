"""Plain CPU FP64 oracle of the gradients through the ChASE filter and through
the wanted eigenpairs (differentiation of the Section 2 method).

TEST INFRASTRUCTURE ONLY. Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / reference legs of ``bench.py`` may import this module. The
product path never calls it.

Convention (the one torch uses for complex tensors and a real loss L): the
adjoint of a complex array Z is Zbar = 2 dL/d conj(Z), so that
dL = Re sum(conj(Zbar) * dZ). A is constrained to be Hermitian, so the adjoint
returned for A is the Hermitian part of the unconstrained one: for every
Hermitian direction E, dL = Re sum(conj(Abar) * E).

Pins (``tests/test_grad_oracle_pins.py``): the Daleckii-Krein divided-difference
formula for a polynomial of a diagonal matrix, Chebyshev derivative closed forms
T_m' = m U_{m-1}, and central finite differences on small random problems.
"""
from __future__ import annotations

import numpy as np

from .chase_oracle import chebyshev_coefficients


def hermitian_part(G: np.ndarray) -> np.ndarray:
    return 0.5 * (G + G.conj().T)


# ---------------------------------------------------------------- filter VJP
def filter_forward_states(A, V, deg, c, e, mu_1, scaled=True):
    """All states Y_0 .. Y_deg of the Eq. 1 recurrence with one degree for every
    column (Y_1 = alpha_1 (A - cI) Y_0, Y_i = alpha_i (A - cI) Y_{i-1} + beta_i Y_{i-2})."""
    alpha, beta = chebyshev_coefficients(deg, c, e, mu_1, scaled)
    Ys = [np.array(V, dtype=np.complex128)]
    Ys.append(alpha[1] * (A @ Ys[0] - c * Ys[0]))
    for i in range(2, deg + 1):
        Ys.append(alpha[i] * (A @ Ys[i - 1] - c * Ys[i - 1]) + beta[i] * Ys[i - 2])
    return Ys, alpha, beta


def filter_vjp(A, V, deg, c, e, mu_1, Ybar, scaled=True):
    """Adjoint of Y_deg = p(A) V (Eq. 1 with a common degree): returns (Abar, Vbar).

    Reverse sweep of the recurrence, step i = deg .. 1, with accumulators
    Ybar_i: the step Y_i = alpha_i (A - cI) Y_{i-1} + beta_i Y_{i-2} sends
    alpha_i (A - cI)^H Ybar_i to Ybar_{i-1}, beta_i Ybar_i to Ybar_{i-2} and
    alpha_i Ybar_i Y_{i-1}^H to Abar. Every state is kept (no checkpointing)."""
    Ys, alpha, beta = filter_forward_states(A, V, deg, c, e, mu_1, scaled)
    n = deg
    bars = [np.zeros_like(Ys[0]) for _ in range(n + 1)]
    bars[n] = np.array(Ybar, dtype=np.complex128)
    Abar = np.zeros_like(A, dtype=np.complex128)
    AcH = (A - c * np.eye(A.shape[0])).conj().T
    for i in range(n, 0, -1):
        Abar += alpha[i] * bars[i] @ Ys[i - 1].conj().T
        bars[i - 1] += alpha[i] * (AcH @ bars[i])
        if i >= 2:
            bars[i - 2] += beta[i] * bars[i]
    return hermitian_part(Abar), bars[0]


# ------------------------------------------------------------ eigenpair VJP
def lowest_eigenpairs(A, nev):
    """The nev lowest eigenpairs of Hermitian A (the converged output of the
    method, Section 2: Alg. 2 returns the lowest nev Ritz pairs)."""
    lam, X = np.linalg.eigh(A)
    return lam[:nev], X[:, :nev]


def eig_vjp(A, nev, lam_bar, X_bar):
    """Adjoint of (lambda_1..nev, x_1..nev) = lowest eigenpairs of Hermitian A,
    for a loss that is invariant under the phase of each x_i.

    First-order perturbation theory on the full eigendecomposition:
    d lambda_i = x_i^H dA x_i (Hellmann-Feynman) and
    d x_i = sum_{j != i} x_j (x_j^H dA x_i) / (lambda_i - lambda_j), so
    Abar = sum_i lambda_bar_i x_i x_i^H + sum_i y_i x_i^H with
    y_i = sum_{j != i} x_j (x_j^H xbar_i) / (lambda_i - lambda_j) over all N
    eigenpairs; Hermitian part. Requires simple eigenvalues lambda_1..nev."""
    lam, X = np.linalg.eigh(A)
    N = A.shape[0]
    Xw = X[:, :nev]
    C = X.conj().T @ np.asarray(X_bar, dtype=np.complex128)  # N x nev: x_j^H xbar_i
    F = np.zeros((N, nev))
    for i in range(nev):
        for j in range(N):
            if j != i:
                F[j, i] = 1.0 / (lam[i] - lam[j])
    Y = X @ (F * C)
    M = Xw * np.asarray(lam_bar, dtype=np.float64)[None, :] + Y
    return hermitian_part(M @ Xw.conj().T)


# --------------------------------------------------------------- test loss
def c4_loss(lam, X, w, B):
    """L = sum_i w_i lambda_i + ||X^H B X||_F^2 (the differentiation workload)."""
    M = X.conj().T @ B @ X
    return float(np.dot(w, lam) + np.sum(np.abs(M) ** 2))


def c4_loss_adjoints(lam, X, w, B):
    """(lambda_bar, X_bar) of c4_loss: lambda_bar = w; with M = X^H B X
    (Hermitian for Hermitian B), dL = 2 Re tr(M^H dM) = Re <4 B X M, dX>."""
    M = X.conj().T @ B @ X
    return np.asarray(w, dtype=np.float64), 4.0 * (B @ X @ M)
