"""Tensor-core (tcgen05, split-BF16 x3) filter against the FP64 oracle.

The mixed filter computes every HEMM of Eq. 1 as hi*hi + hi*lo + lo*hi BF16
products, accumulated in FP32 tensor memory over K chunks of 256 and across
chunks in FP32 registers. Splitting x = hi + lo leaves |x - hi - lo| <= 2^-17 |x|
and the dropped lo*lo term is <= 2^-16 |a||y|, so one step carries a relative
error of about 2^-16 of the operands' magnitudes; the recurrence adds these step
errors, which the normalised filter does not amplify in the columns' dominant
directions. A CPU emulation of the split products (FP64 accumulation) gives
1.1e-5 per degree on a geometric spectrum and 3e-6 on a uniform one. Bound used:
per column j, max |Y_mixed - Y_oracle| <= degs[j] * 2^-16 * max |Y_oracle|
(measured values are printed).
"""
import numpy as np
import pytest

from oracle import chase_oracle as O
from synth import Problem, config_problem

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def dev(x, pkg):
    return pkg.colmajor(torch.from_numpy(np.asfortranarray(x)).cuda())


@pytest.mark.parametrize("N,ncols,dmax", [(512, 60, 20), (333, 37, 36), (700, 300, 36),
                                          (130, 1, 2)])
def test_mixed_filter_against_oracle(lib, N, ncols, dmax):
    p = Problem(N=N, nev=ncols - ncols // 4, nex=ncols // 4, spectrum="uniform", lo=-1.0,
                hi=4.0, reflectors=5, seed=N + 1)
    A = p.matrix()
    V = p.start_block()
    rng = np.random.default_rng(N)
    degs = np.sort(2 * rng.integers(1, dmax // 2 + 1, ncols)).astype(np.int32)
    lam = p.eigenvalues()
    b_sup = lam[-1] * 1.01
    c, e, mu1 = (b_sup + lam[p.ne - 1]) / 2, (b_sup - lam[p.ne - 1]) / 2, lam[0]
    ref = O.chebyshev_filter(A, V, degs, c, e, mu1)
    prm = lib.default_params(N, p.nev, p.nex, precision=lib.CHASE_MIXED_BF16X3)
    with lib.Context(prm) as ctx:
        Vd = dev(V, lib)
        ctx.chase_filter(dev(A, lib), Vd, ncols, degs, c, e, mu1,
                         precision=lib.CHASE_MIXED_BF16X3)
        got = Vd.cpu().numpy()
    rel = np.abs(got - ref).max(axis=0) / np.abs(ref).max(axis=0)
    print(f"N={N} ncols={ncols}: max rel err {rel.max():.3e} median {np.median(rel):.3e}")
    assert np.all(np.isfinite(got))
    assert np.all(rel <= degs * 2.0 ** -16)


def test_mixed_solve_c1_reaches_fp64_accuracy(lib):
    p = config_problem("C1")
    A = p.matrix()
    V0, Q0 = p.start_block(), p.lanczos_start()
    prm = lib.default_params(p.N, p.nev, p.nex, precision=lib.CHASE_MIXED_BF16X3)
    with lib.Context(prm) as ctx:
        Vd = dev(V0, lib)
        ritz = torch.zeros(p.ne, dtype=torch.float64, device="cuda")
        resid = torch.zeros_like(ritz)
        st = ctx.chase_solve(dev(A, lib), Vd, ritz, resid, lanczos_start=dev(Q0, lib))
    assert st["status"] == 0 and st["matvecs_mixed"] > 0
    lam = p.eigenvalues()
    nA = p.norm2()
    r = ritz.cpu().numpy()[:p.nev]
    V = Vd.cpu().numpy()[:, :p.nev]
    assert np.abs(r - lam[:p.nev]).max() <= 1e-10 * nA
    res = np.linalg.norm(A @ V - V * r[None, :], axis=0)
    assert res.max() <= 1e-10 * nA
    assert np.abs(V.conj().T @ V - np.eye(p.nev)).max() <= 1e-12
