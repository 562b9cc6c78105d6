"""Single-GPU (sm_103a) ChASE: Chebyshev-filtered subspace iteration for the
lowest eigenpairs of a dense complex Hermitian matrix (Wu & Di Napoli,
arXiv 2309.15595), exposed through the C ABI of ``include/chase.h``.

The functions here carry the ABI's names and only marshal arguments: torch
tensors supply device memory and the stream, every computation runs in the
library's CUDA kernels. Matrices must be complex128 CUDA tensors with
column-major strides (``stride(0) == 1``); ``colmajor(t)`` makes one.
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import _lib
from ._lib import (  # noqa: F401
    CHASE_FP64,
    CHASE_MIXED_BF16X3,
    CHASE_QR_CHOLQR1,
    CHASE_QR_CHOLQR2,
    CHASE_QR_FALLBACK,
    CHASE_QR_HOUSEHOLDER,
    CHASE_QR_SHIFTED,
    ChaseParams,
    ChaseStats,
    LIB,
)

__all__ = ["Context", "ChaseError", "colmajor", "default_params", "solve", "solve_batch",
           "chase_cond_est",
           "chase_degree_opt", "chase_status_string", "LIB"]


class ChaseError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        super().__init__(f"{where}: {chase_status_string(status)} ({status})")


def chase_status_string(status: int) -> str:
    return LIB.chase_status_string(int(status)).decode()


def _check(rc: int, where: str, allow=()):
    if rc != 0 and rc not in allow:
        raise ChaseError(rc, where)
    return rc


def default_params(N: int, nev: int, nex: int, **over) -> ChaseParams:
    p = ChaseParams()
    LIB.chase_default_params(ctypes.byref(p), int(N), int(nev), int(nex))
    for k, v in over.items():
        if not hasattr(p, k):
            raise KeyError(k)
        setattr(p, k, v)
    return p


def colmajor(t):
    """Same matrix, column-major strides (copies if needed)."""
    return t if t.dim() == 2 and t.stride(0) == 1 else t.mT.contiguous().mT


def _mat(t, rows: int, cols: int, name: str):
    import torch

    if not isinstance(t, torch.Tensor) or t.dtype != torch.complex128 or not t.is_cuda:
        raise TypeError(f"{name} must be a complex128 CUDA tensor")
    if t.dim() != 2 or t.shape[0] != rows or t.shape[1] < cols:
        raise ValueError(f"{name} must have shape ({rows}, >= {cols}), got {tuple(t.shape)}")
    if t.stride(0) != 1 or (t.shape[1] > 1 and t.stride(1) < rows):
        raise ValueError(f"{name} must be column-major (stride(0) == 1); use colmajor()")
    ld = t.stride(1) if t.shape[1] > 1 else rows
    return ctypes.c_void_p(t.data_ptr()), int(ld)


def _vec(t, n: int, name: str):
    import torch

    if not isinstance(t, torch.Tensor) or t.dtype != torch.float64 or not t.is_cuda:
        raise TypeError(f"{name} must be a float64 CUDA tensor")
    if t.dim() != 1 or t.numel() < n or t.stride(0) != 1:
        raise ValueError(f"{name} must be a contiguous 1-D tensor of >= {n} elements")
    return ctypes.c_void_p(t.data_ptr())


class Context:
    """A chase_ctx: workspace for order N and nev + nex vectors, bound to a
    CUDA stream (the current torch stream by default)."""

    def __init__(self, params: ChaseParams, stream=None):
        import torch

        self.params = params
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self._h = ctypes.c_void_p()
        _check(LIB.chase_create(ctypes.byref(params), ctypes.c_void_p(self.stream.cuda_stream),
                                ctypes.byref(self._h)), "chase_create")
        self.N = int(params.N)
        self.ne = int(params.nev + params.nex)

    def close(self):
        if self._h:
            LIB.chase_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ------------------------------------------------------------ entry points
    def chase_solve(self, A, V, ritz, resid, lanczos_start=None, allow_not_converged=False):
        a, lda = _mat(A, self.N, self.N, "A")
        v, ldv = _mat(V, self.N, self.ne, "V")
        if lanczos_start is not None:
            q, ldq = _mat(lanczos_start, self.N, int(self.params.lanczos_vecs), "lanczos_start")
        else:
            q, ldq = ctypes.c_void_p(), 0
        st = ChaseStats()
        rc = LIB.chase_solve(self._h, a, lda, v, ldv, q, ldq, _vec(ritz, self.ne, "ritz"),
                             _vec(resid, self.ne, "resid"), ctypes.byref(st))
        _check(rc, "chase_solve", allow=(_lib.CHASE_ERR_NOT_CONVERGED,) if allow_not_converged else ())
        d = st.as_dict()
        d["status"] = rc
        return d

    def chase_lanczos(self, A, Q0):
        a, lda = _mat(A, self.N, self.N, "A")
        nvec = int(Q0.shape[1])
        q, ldq = _mat(Q0, self.N, nvec, "Q0")
        out = (ctypes.c_double * 4)()
        _check(LIB.chase_lanczos(self._h, a, lda, q, ldq, nvec, out), "chase_lanczos")
        return tuple(out)

    def chase_filter(self, A, V, ncols, degs, c, e, mu_1, precision=CHASE_FP64):
        a, lda = _mat(A, self.N, self.N, "A")
        v, ldv = _mat(V, self.N, ncols, "V")
        d = np.ascontiguousarray(np.asarray(degs, dtype=np.int32))
        if d.size != ncols:
            raise ValueError("degs must have ncols entries")
        _check(LIB.chase_filter(self._h, a, lda, v, ldv, int(ncols),
                                d.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                                float(c), float(e), float(mu_1), int(precision)), "chase_filter")

    def chase_qr(self, V, ncols, cond_est):
        v, ldv = _mat(V, self.N, ncols, "V")
        var = ctypes.c_int32(0)
        _check(LIB.chase_qr(self._h, v, ldv, int(ncols), float(cond_est), ctypes.byref(var)),
               "chase_qr")
        return int(var.value)

    def chase_rayleigh_ritz(self, A, V, ncols, ritz):
        a, lda = _mat(A, self.N, self.N, "A")
        v, ldv = _mat(V, self.N, ncols, "V")
        _check(LIB.chase_rayleigh_ritz(self._h, a, lda, v, ldv, int(ncols),
                                       _vec(ritz, ncols, "ritz")), "chase_rayleigh_ritz")

    def chase_residuals(self, A, V, ritz, ncols, resid):
        a, lda = _mat(A, self.N, self.N, "A")
        v, ldv = _mat(V, self.N, ncols, "V")
        _check(LIB.chase_residuals(self._h, a, lda, v, ldv, _vec(ritz, ncols, "ritz"), int(ncols),
                                   _vec(resid, ncols, "resid")), "chase_residuals")


    def chase_filter_vjp(self, A, V, ncols, deg, c, e, mu_1, Ybar, Abar, Vbar, checkpoint=0):
        a, lda = _mat(A, self.N, self.N, "A")
        v, ldv = _mat(V, self.N, ncols, "V")
        yb, ldyb = _mat(Ybar, self.N, ncols, "Ybar")
        ab, ldab = _mat(Abar, self.N, self.N, "Abar")
        vb, ldvb = _mat(Vbar, self.N, ncols, "Vbar")
        _check(LIB.chase_filter_vjp(self._h, a, lda, v, ldv, int(ncols), int(deg), float(c),
                                    float(e), float(mu_1), yb, ldyb, ab, ldab, vb, ldvb,
                                    int(checkpoint)), "chase_filter_vjp")

    def chase_eig_vjp(self, A, X, ritz, ne, nev, lam_bar, X_bar, Abar, cg_tol=1e-10,
                      cg_max_iter=2000, allow_not_converged=False):
        a, lda = _mat(A, self.N, self.N, "A")
        x, ldx = _mat(X, self.N, ne, "X")
        ab, ldab = _mat(Abar, self.N, self.N, "Abar")
        lb = _vec(lam_bar, nev, "lam_bar") if lam_bar is not None else ctypes.c_void_p()
        if X_bar is not None:
            xb, ldxb = _mat(X_bar, self.N, nev, "X_bar")
        else:
            xb, ldxb = ctypes.c_void_p(), 0
        it = ctypes.c_int32(0)
        rc = LIB.chase_eig_vjp(self._h, a, lda, x, ldx, _vec(ritz, ne, "ritz"), int(ne), int(nev),
                               lb, xb, ldxb, ab, ldab, float(cg_tol), int(cg_max_iter),
                               ctypes.byref(it))
        _check(rc, "chase_eig_vjp",
               allow=(_lib.CHASE_ERR_NOT_CONVERGED,) if allow_not_converged else ())
        return int(it.value)


# ------------------------------------------------------------ host helpers
def chase_cond_est(ritz, degs, locked: int, c: float, e: float) -> float:
    r = np.ascontiguousarray(np.asarray(ritz, dtype=np.float64))
    d = np.ascontiguousarray(np.asarray(degs, dtype=np.int32))
    return float(LIB.chase_cond_est(r.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                    d.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                                    r.size, int(locked), float(c), float(e)))


def chase_degree_opt(resid, ritz, c, e, tol_abs, deg_max, deg_extra):
    rs = np.ascontiguousarray(np.asarray(resid, dtype=np.float64))
    rz = np.ascontiguousarray(np.asarray(ritz, dtype=np.float64))
    out = np.zeros(rs.size, dtype=np.int32)
    LIB.chase_degree_opt(rs.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                         rz.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), rs.size, float(c),
                         float(e), float(tol_abs), int(deg_max), int(deg_extra),
                         out.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)))
    return out


def solve_batch(contexts, As, Vs, ritzs, resids, lanczos_starts=None, threads=0,
                allow_not_converged=False):
    """chase_solve_batch: problem k solved on contexts[k] (its own stream) with
    A = As[k], start block / result Vs[k], outputs ritzs[k], resids[k].
    Returns (list of per-problem stats dicts, list of status codes)."""
    n = len(contexts)
    if not (len(As) == len(Vs) == len(ritzs) == len(resids) == n):
        raise ValueError("one A, V, ritz and resid per context")
    P = ctypes.c_void_p * n
    I = ctypes.c_int64 * n
    a, lda, v, ldv, q, ldq, rz, rs = P(), I(), P(), I(), P(), I(), P(), P()
    for k, cx in enumerate(contexts):
        a[k], lda[k] = _mat(As[k], cx.N, cx.N, "A")
        v[k], ldv[k] = _mat(Vs[k], cx.N, cx.ne, "V")
        rz[k] = _vec(ritzs[k], cx.ne, "ritz")
        rs[k] = _vec(resids[k], cx.ne, "resid")
        if lanczos_starts is not None:
            q[k], ldq[k] = _mat(lanczos_starts[k], cx.N, int(cx.params.lanczos_vecs),
                                "lanczos_start")
    handles = P(*[cx._h.value for cx in contexts])
    stats = (ChaseStats * n)()
    status = (ctypes.c_int32 * n)()
    rc = LIB.chase_solve_batch(n, handles, a, lda, v, ldv, q if lanczos_starts is not None else None,
                               ldq if lanczos_starts is not None else None, rz, rs, stats, status,
                               int(threads))
    allow = (_lib.CHASE_ERR_NOT_CONVERGED,) if allow_not_converged else ()
    for k in range(n):
        _check(status[k], f"chase_solve_batch[{k}]", allow=allow)
    if rc != 0 and rc not in allow:
        _check(rc, "chase_solve_batch")
    out = []
    for k in range(n):
        d = stats[k].as_dict()
        d["status"] = int(status[k])
        out.append(d)
    return out, [int(x) for x in status]


def solve(A, nev: int, nex: int, V0=None, lanczos_start=None, allow_not_converged=False, **params):
    """Lowest ``nev`` eigenpairs of the Hermitian complex128 CUDA tensor A.
    Returns (ritz[nev], V[:, :nev], resid[nev], stats)."""
    import torch

    N = int(A.shape[0])
    A = colmajor(A)
    p = default_params(N, nev, nex, **params)
    if V0 is None:
        raise ValueError("a start block V0 (N x (nev+nex)) is required")
    V = colmajor(V0.clone())
    ritz = torch.zeros(nev + nex, dtype=torch.float64, device=A.device)
    resid = torch.zeros_like(ritz)
    with Context(p) as ctx:
        st = ctx.chase_solve(A, V, ritz, resid, lanczos_start=lanczos_start,
                             allow_not_converged=allow_not_converged)
    return ritz[:nev], V[:, :nev], resid[:nev], st
