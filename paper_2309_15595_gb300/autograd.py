"""torch.autograd Functions over the C ABI (argument marshalling only).

``chase_eigh(A, V0, nev, nex, ...)`` returns the nev lowest eigenvalues and
eigenvectors of the Hermitian complex128 CUDA tensor A, computed by
``chase_solve``; its backward calls ``chase_eig_vjp`` (Hellmann-Feynman for the
eigenvalues, first-order perturbation theory for the eigenvectors: the part
inside the nev + nex Ritz basis directly, the complement by projected conjugate
gradients).

``chebyshev_filter(A, V, deg, c, e, mu_1)`` is the Eq. 1 filter with one even
degree for all columns (``chase_filter``); its backward runs the recurrence in
reverse from checkpoints (``chase_filter_vjp``).

Gradients follow torch's convention for complex tensors (grad = 2 dL/d conj(z)
for a real loss); the gradient of A is Hermitian. A loss through
``chase_eigh`` must not depend on the phase of each eigenvector.
"""
from __future__ import annotations

import torch

from . import Context, colmajor, default_params


def _colmajor_empty(n, m, like):
    return torch.empty((m, n), dtype=like.dtype, device=like.device).mT


class ChaseEigh(torch.autograd.Function):
    @staticmethod
    def forward(ctx, A, V0, nev, nex, lanczos_start, cg_tol, params):
        N = int(A.shape[0])
        Ad = colmajor(A.detach())
        V = colmajor(V0.detach().clone())
        ne = nev + nex
        ritz = torch.zeros(ne, dtype=torch.float64, device=A.device)
        resid = torch.zeros_like(ritz)
        prm = default_params(N, nev, nex, **(params or {}))
        with Context(prm) as c:
            c.chase_solve(Ad, V, ritz, resid, lanczos_start=lanczos_start)
        ctx.save_for_backward(Ad, V, ritz)
        ctx.nev, ctx.nex, ctx.cg_tol, ctx.params = nev, nex, cg_tol, params
        lam_out, x_out, r_out = ritz[:nev].clone(), V[:, :nev].clone(), resid[:nev].clone()
        ctx.mark_non_differentiable(r_out)
        return lam_out, x_out, r_out

    @staticmethod
    def backward(ctx, lam_bar, X_bar, _resid_bar):
        Ad, V, ritz = ctx.saved_tensors
        N, nev, ne = Ad.shape[0], ctx.nev, ctx.nev + ctx.nex
        lb = lam_bar.contiguous() if lam_bar is not None else None
        xb = colmajor(X_bar) if X_bar is not None else None
        Abar = _colmajor_empty(N, N, Ad)
        prm = default_params(N, ctx.nev, ctx.nex, **(ctx.params or {}))
        with Context(prm) as c:
            c.chase_eig_vjp(Ad, V, ritz, ne, nev, lb, xb, Abar, cg_tol=ctx.cg_tol)
        return Abar, None, None, None, None, None, None


def chase_eigh(A, V0, nev, nex, lanczos_start=None, cg_tol=1e-10, **params):
    """(eigenvalues[nev], eigenvectors[N, nev], residual norms[nev]) of Hermitian A."""
    return ChaseEigh.apply(A, V0, nev, nex, lanczos_start, cg_tol, params)


class ChebyshevFilter(torch.autograd.Function):
    @staticmethod
    def forward(ctx, A, V, deg, c, e, mu_1, checkpoint, params):
        N, n = int(A.shape[0]), int(V.shape[1])
        Ad = colmajor(A.detach())
        Vd = colmajor(V.detach())
        Y = colmajor(V.detach().clone())
        prm = default_params(N, n, 0, **(params or {}))
        with Context(prm) as cx:
            cx.chase_filter(Ad, Y, n, [deg] * n, c, e, mu_1)
        ctx.save_for_backward(Ad, Vd)
        ctx.args = (deg, c, e, mu_1, checkpoint, params)
        return Y

    @staticmethod
    def backward(ctx, Ybar):
        Ad, Vd = ctx.saved_tensors
        deg, c, e, mu_1, checkpoint, params = ctx.args
        N, n = Ad.shape[0], Vd.shape[1]
        Abar = _colmajor_empty(N, N, Ad)
        Vbar = _colmajor_empty(N, n, Ad)
        prm = default_params(N, n, 0, **(params or {}))
        with Context(prm) as cx:
            cx.chase_filter_vjp(Ad, Vd, n, deg, c, e, mu_1, colmajor(Ybar), Abar, Vbar,
                                checkpoint=checkpoint)
        return Abar, Vbar, None, None, None, None, None, None


def chebyshev_filter(A, V, deg, c, e, mu_1, checkpoint=0, **params):
    """p(A) V for the Eq. 1 recurrence of even degree ``deg`` (scaled by default)."""
    return ChebyshevFilter.apply(A, V, deg, c, e, mu_1, checkpoint, params)
