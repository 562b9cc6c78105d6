"""The allocation-free residual entry point, chase_residuals_noalloc.

It serves callers that cannot allocate device memory (and so cannot create a
chase context): its scratch is a fixed array inside the library. This test
calls it through the C ABI twice in a row, with different sizes, so the second
call runs over the first call's leftover scratch contents, and checks each
output against the context-based chase_residuals on the same inputs and against
the CPU oracle's residual norms, within the residual tolerance the other GPU
tests use (1e-11 relative). It also checks that a size beyond the fixed scratch
is rejected before any launch.
Collected last so that a failure here leaves every other test already run.
"""
import ctypes

import numpy as np
import pytest

from oracle import chase_oracle as O
from synth import Problem

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _dev(x, lib):
    return lib.colmajor(torch.from_numpy(np.asfortranarray(x)).cuda())


def _noalloc(lib, Ad, Vd, theta_d, ncols, out_d):
    N = Ad.shape[0]
    stream = torch.cuda.current_stream()
    return lib.LIB.chase_residuals_noalloc(
        ctypes.c_void_p(Ad.data_ptr()), Ad.stride(1), ctypes.c_void_p(Vd.data_ptr()),
        Vd.stride(1), ctypes.c_void_p(theta_d.data_ptr()), N, ncols,
        ctypes.c_void_p(out_d.data_ptr()), ctypes.c_void_p(stream.cuda_stream))


def test_residuals_noalloc_matches_context_entry_point(lib):
    for N, ncols, seed in [(512, 60, 11), (333, 37, 12)]:
        p = Problem(N=N, nev=ncols, nex=0, reflectors=4, seed=seed)
        A, V = p.matrix(), p.start_block()
        Ad = _dev(A, lib)
        Vd = _dev(V, lib)
        theta_h = np.linspace(0.1, 7.0, ncols)
        theta = torch.from_numpy(theta_h).cuda()
        ref = torch.zeros(ncols, dtype=torch.float64, device="cuda")
        with lib.Context(lib.default_params(N, ncols, 0)) as ctx:
            ctx.chase_residuals(Ad, Vd, theta, ncols, ref)
        got = torch.full((ncols,), -1.0, dtype=torch.float64, device="cuda")
        assert _noalloc(lib, Ad, Vd, theta, ncols, got) == 0
        torch.cuda.synchronize()
        np.testing.assert_allclose(got.cpu().numpy(), ref.cpu().numpy(), rtol=1e-11)
        np.testing.assert_allclose(got.cpu().numpy(), O.residuals(A, V, theta_h), rtol=1e-11)


def test_residuals_noalloc_rejects_oversize(lib):
    N = 64 * 40000  # ceil(N/64) * 14 > 524288 doubles; never launched
    Ad = torch.zeros((1, 1), dtype=torch.complex128, device="cuda")
    out = torch.zeros(14, dtype=torch.float64, device="cuda")
    rc = lib.LIB.chase_residuals_noalloc(
        ctypes.c_void_p(Ad.data_ptr()), N, ctypes.c_void_p(Ad.data_ptr()), N,
        ctypes.c_void_p(out.data_ptr()), N, 14, ctypes.c_void_p(out.data_ptr()), None)
    assert rc == 1
