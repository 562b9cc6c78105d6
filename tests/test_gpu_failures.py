"""Failure paths of the C ABI, forced from the host (no GPU fault is involved).

The Rayleigh-Ritz eigensolver is a Jacobi method whose stages each stop at a
sweep cap; the context parameter heev_max_sweeps lowers that cap, so a cap of
one sweep makes the eigensolver stop before convergence. The solve must then
end with CHASE_ERR_HEEV_NOCONV (Alg. 2's loop cannot continue without the
Ritz pairs) and leave finite values behind, for the single-CTA path (n <= 64)
and for the cooperative large-n path.
"""
import numpy as np
import pytest

from synth import Problem, config_problem

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

HEEV_NOCONV = 5


def dev(x, lib):
    return lib.colmajor(torch.from_numpy(np.asfortranarray(x)).cuda())


def test_solve_reports_heev_sweep_cap(lib):
    p = config_problem("C1")  # nev + nex = 60: the single-CTA Jacobi kernel
    A, V0, Q0 = p.matrix(), p.start_block(), p.lanczos_start()
    with lib.Context(lib.default_params(p.N, p.nev, p.nex, heev_max_sweeps=1)) as ctx:
        ritz = torch.zeros(p.ne, dtype=torch.float64, device="cuda")
        resid = torch.zeros_like(ritz)
        with pytest.raises(lib.ChaseError) as ei:
            ctx.chase_solve(dev(A, lib), dev(V0, lib), ritz, resid, lanczos_start=dev(Q0, lib))
        assert ei.value.status == HEEV_NOCONV
        assert np.all(np.isfinite(ritz.cpu().numpy()))


@pytest.mark.parametrize("N,n", [(400, 100), (333, 65)])
def test_rayleigh_ritz_reports_heev_sweep_cap(lib, N, n):
    p = Problem(N=N, nev=n - n // 4, nex=n // 4, spectrum="uniform", lo=0.5, hi=9.0,
                reflectors=6, seed=N + n)
    A = p.matrix()
    Q = np.asfortranarray(np.linalg.qr(p.start_block())[0])
    with lib.Context(lib.default_params(N, p.nev, p.nex, heev_max_sweeps=1)) as ctx:
        ritz = torch.zeros(n, dtype=torch.float64, device="cuda")
        with pytest.raises(lib.ChaseError) as ei:
            ctx.chase_rayleigh_ritz(dev(A, lib), dev(Q, lib), n, ritz)
        assert ei.value.status == HEEV_NOCONV
        assert np.all(np.isfinite(ritz.cpu().numpy()))
    # the default caps converge on the same input
    with lib.Context(lib.default_params(N, p.nev, p.nex)) as ctx:
        ritz = torch.zeros(n, dtype=torch.float64, device="cuda")
        ctx.chase_rayleigh_ritz(dev(A, lib), dev(Q, lib), n, ritz)


def test_create_rejects_negative_sweep_cap(lib):
    import ctypes

    h = ctypes.c_void_p()
    bad = lib.default_params(64, 8, 4, heev_max_sweeps=-1)
    assert lib.LIB.chase_create(ctypes.byref(bad), None, ctypes.byref(h)) == 1
