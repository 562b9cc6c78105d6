"""Seeded synthetic Hermitian eigenproblems with exactly known spectra.

Random numbers come from a counter-based generator: SplitMix64 (Steele, Lea and
Flood, "Fast splittable pseudorandom number generators", OOPSLA 2014) applied to
``key + (i + 1) * golden``; a uniform in (0, 1) takes the top 53 bits plus half
an ulp; a complex Gaussian with Re, Im ~ N(0, 1/2) is Box-Muller in polar form,
``sqrt(-ln u1) * exp(2 pi i u2)``. Every value is addressed by (seed, stream,
counter), so any sub-block can be regenerated alone.

Test matrices follow the paper's "Uniform" artificial matrices (Section 4.1.2):
a diagonal D holds the prescribed eigenvalues and A = H D H^H with a unitary H.
The paper takes H from the QR factorisation of a random matrix; here H is a
product of r complex Householder reflectors H_i = I - 2 v_i v_i^H / (v_i^H v_i)
with Gaussian v_i, which is unitary as well and costs O(r N^2) to apply, so the
eigenvectors H e_k stay known exactly. Matrices are returned column-major
(LAPACK layout), which is what the C ABI reads.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)

# stream identifiers (any distinct constants)
STREAM_SPECTRUM = 1
STREAM_REFLECTORS = 2
STREAM_START = 3
STREAM_LANCZOS = 4
STREAM_EXTRA = 5


def _mix64(z: np.ndarray) -> np.ndarray:
    z = (z ^ (z >> np.uint64(30))) * _M1
    z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def uniform01(seed: int, stream: int, count: int, offset: int = 0) -> np.ndarray:
    """``count`` uniforms in (0, 1) at counters offset .. offset+count-1."""
    with np.errstate(over="ignore"):
        key = _mix64(np.array([(seed * 0x100000001B3 + stream * 0x5851F42D4C957F2D)
                               & 0xFFFFFFFFFFFFFFFF], dtype=np.uint64))[0]
        ctr = np.arange(offset + 1, offset + count + 1, dtype=np.uint64)
        bits = _mix64(key + ctr * _GOLDEN)
    return ((bits >> np.uint64(11)).astype(np.float64) + 0.5) * (2.0 ** -53)


def complex_normal(seed: int, stream: int, count: int, offset: int = 0) -> np.ndarray:
    """``count`` complex Gaussians with E|z|^2 = 1 (Re, Im ~ N(0, 1/2))."""
    u = uniform01(seed, stream, 2 * count, 2 * offset)
    r = np.sqrt(-np.log(u[0::2]))
    ang = 2.0 * math.pi * u[1::2]
    return r * np.cos(ang) + 1j * (r * np.sin(ang))


@dataclasses.dataclass(frozen=True)
class Problem:
    """A Hermitian test problem A = H D H^H with prescribed eigenvalues D.

    spectrum kinds:
      * ``"uniform"``   lambda_k = lo + (k-1)(hi-lo)/(N-1)
      * ``"geometric"`` lambda_k = 10**(a + (b-a)(k-1)/(N-1))
      * ``"clusters"``  the lowest ``n_low`` eigenvalues come in clusters of 4
        spaced by ``spacing`` with cluster starts U[lo, -3*spacing]; the rest are
        U[0, hi]
      * ``"gap"``       uniform in [lo, hi] with an extra gap ``spacing`` after
        index ``n_low``
    """

    N: int
    nev: int
    nex: int
    spectrum: str = "uniform"
    lo: float = 1e-3
    hi: float = 10.0
    n_low: int = 0
    spacing: float = 1e-3
    reflectors: int = 8
    seed: int = 1

    @property
    def ne(self) -> int:
        return self.nev + self.nex

    # ------------------------------------------------------------------ spectrum
    def eigenvalues(self) -> np.ndarray:
        N = self.N
        k = np.arange(N, dtype=np.float64)
        if self.spectrum == "uniform":
            lam = self.lo + k * (self.hi - self.lo) / (N - 1)
        elif self.spectrum == "geometric":
            a, b = math.log10(self.lo), math.log10(self.hi)
            lam = 10.0 ** (a + (b - a) * k / (N - 1))
        elif self.spectrum == "clusters":
            ncl = (self.n_low + 3) // 4
            u = uniform01(self.seed, STREAM_SPECTRUM, ncl + (N - 4 * ncl))
            starts = self.lo + u[:ncl] * (-3.0 * self.spacing - self.lo)
            low = (starts[:, None] + self.spacing * np.arange(4)[None, :]).ravel()
            high = u[ncl:] * self.hi
            lam = np.concatenate([low, high])
        elif self.spectrum == "gap":
            lam = self.lo + k * (self.hi - self.lo) / (N - 1)
            lam[self.n_low:] += self.spacing
        else:
            raise ValueError(f"unknown spectrum {self.spectrum!r}")
        return np.sort(lam)

    def norm2(self) -> float:
        lam = self.eigenvalues()
        return float(max(abs(lam[0]), abs(lam[-1])))

    # ---------------------------------------------------------------- reflectors
    def reflector_vectors(self) -> np.ndarray:
        """(r, N) complex array; row i is v_{i+1}."""
        z = complex_normal(self.seed, STREAM_REFLECTORS, self.reflectors * self.N)
        return z.reshape(self.reflectors, self.N)

    def start_block(self, ncols: int | None = None) -> np.ndarray:
        """N x ncols complex Gaussian start block, column-major counters."""
        n = self.ne if ncols is None else ncols
        z = complex_normal(self.seed, STREAM_START, self.N * n)
        return np.asfortranarray(z.reshape(n, self.N).T)

    def lanczos_start(self, nvec: int = 4) -> np.ndarray:
        z = complex_normal(self.seed, STREAM_LANCZOS, self.N * nvec)
        return np.asfortranarray(z.reshape(nvec, self.N).T)

    # ------------------------------------------------------------------- matrix
    def matrix(self) -> np.ndarray:
        """A = H D H^H as a column-major (Fortran-ordered) complex128 array."""
        lam = self.eigenvalues()
        A = np.asfortranarray(np.diag(lam.astype(np.complex128)))
        for v in self.reflector_vectors()[::-1]:
            tau = 2.0 / np.real(np.vdot(v, v))
            w = A @ v
            alpha = np.real(np.vdot(v, w))
            u = w - (0.5 * tau * alpha) * v
            A -= tau * (np.outer(v, u.conj()) + np.outer(u, v.conj()))
        A = 0.5 * (A + A.conj().T)
        A[np.diag_indices(self.N)] = A.diagonal().real
        return np.asfortranarray(A)

    def matrix_torch(self, device):
        """The same A built on ``device`` with torch; returns a tensor equal to A
        whose strides are column-major (stride(0) == 1), so its buffer is in the
        layout the C ABI reads. Used where N is too large to build on the host."""
        import torch

        lam = torch.as_tensor(self.eigenvalues(), device=device)
        # M holds conj(A) row-major; M.mT is A with column-major strides.
        M = torch.diag(lam.to(torch.complex128))
        for v_np in self.reflector_vectors()[::-1]:
            v = torch.as_tensor(np.conj(v_np), device=device)
            tau = 2.0 / float(torch.real(torch.vdot(v, v)))
            w = M @ v
            alpha = float(torch.real(torch.vdot(v, w)))
            u = w - (0.5 * tau * alpha) * v
            M.sub_(tau * torch.outer(v, u.conj()))
            M.sub_(tau * torch.outer(u, v.conj()))
        T = M.mH.contiguous()
        M.add_(T).mul_(0.5)
        del T
        M.diagonal().imag.zero_()
        return M.mT

    def eigenvectors(self, cols) -> np.ndarray:
        """Exact eigenvectors H e_k for the given column indices (N x len(cols))."""
        cols = np.atleast_1d(np.asarray(cols))
        X = np.zeros((self.N, len(cols)), dtype=np.complex128)
        X[cols, np.arange(len(cols))] = 1.0
        for v in self.reflector_vectors()[::-1]:
            tau = 2.0 / np.real(np.vdot(v, v))
            X -= tau * np.outer(v, v.conj() @ X)
        return X


def config_problem(name: str, **over) -> Problem:
    """The named workloads. C1: N=512 parity case; C2: N=20000 geometric
    spectrum; C3: N=40000 DFT-like clustered spectrum; C4: N=4096 with a gap."""
    table = {
        "C1": dict(N=512, nev=40, nex=20, spectrum="uniform", lo=10 * 1e-4, hi=10.0,
                   reflectors=8, seed=1),
        "C2": dict(N=20000, nev=1000, nex=300, spectrum="geometric", lo=1e-4, hi=1.0,
                   reflectors=16, seed=2),
        "C3": dict(N=40000, nev=2250, nex=750, spectrum="clusters", lo=-2.0, hi=50.0,
                   n_low=3000, spacing=1e-3, reflectors=16, seed=3),
        "C4": dict(N=4096, nev=64, nex=32, spectrum="gap", lo=0.0, hi=10.0, n_low=64,
                   spacing=0.05, reflectors=8, seed=4),
    }
    d = dict(table[name])
    d.update(over)
    return Problem(**d)
