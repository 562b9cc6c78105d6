"""The constants the paper prints for its method (tests/golden/paper_constants.txt,
each line citing its passage) against the oracle and the library defaults."""
import os

import numpy as np
import pytest

from oracle import chase_oracle as O

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden",
                      "paper_constants.txt")


def constants():
    out = {}
    for line in open(GOLDEN):
        line = line.strip()
        if line and not line.startswith("#"):
            name, value, _cite = line.split(" ", 2)
            out[name] = float(value)
    return out


def test_oracle_qr_variant_thresholds():
    c = constants()
    hi, lo = c["qr_shifted_above"], c["qr_cholqr1_below"]
    assert O.select_qr_variant(np.nextafter(hi, np.inf)) == O.QR_SHIFTED
    assert O.select_qr_variant(hi) == O.QR_CHOLQR2
    assert O.select_qr_variant(np.nextafter(lo, -np.inf)) == O.QR_CHOLQR1
    assert O.select_qr_variant(lo) == O.QR_CHOLQR2


def test_oracle_shift_constant():
    c = constants()
    m, n, fro2 = 1000, 30, 7.5
    assert O.shift_value(m, n, fro2) == pytest.approx(
        c["shift_constant"] * (m * n + n * (n + 1)) * 2.0 ** -53 * fro2, rel=1e-15)


def test_library_defaults_follow_the_paper():
    # the library's host-side defaults (no GPU call); skipped on a checkout
    # where the shared library has not been built yet
    lib_path = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                            "paper_2309_15595_gb300", "libchase_gb300.so")
    if not os.path.exists(lib_path):
        pytest.skip("libchase_gb300.so not built")
    import paper_2309_15595_gb300 as lib

    c = constants()
    p = lib.default_params(512, 40, 20)
    assert p.deg_init == c["deg_init"] and p.deg_max == c["deg_max"]
    assert p.tol == c["tol"]
    import inspect
    sig = inspect.signature(O.solve)
    assert sig.parameters["deg_init"].default == c["deg_init"]
    assert sig.parameters["deg_max"].default == c["deg_max"]
    assert sig.parameters["tol"].default == c["tol"]


@pytest.mark.gpu
def test_library_qr_variant_thresholds():
    """The library's own Alg. 4 choice at the thresholds the paper states:
    cond > 1e8 shifted, cond < 20 CholeskyQR1, otherwise CholeskyQR2."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2309_15595_gb300 as lib
    from synth import Problem

    c = constants()
    hi, lo = c["qr_shifted_above"], c["qr_cholqr1_below"]
    X = Problem(N=300, nev=24, nex=0, seed=9).start_block()
    cases = [(np.nextafter(lo, -np.inf), lib.CHASE_QR_CHOLQR1), (lo, lib.CHASE_QR_CHOLQR2),
             (hi, lib.CHASE_QR_CHOLQR2), (np.nextafter(hi, np.inf), lib.CHASE_QR_SHIFTED)]
    with lib.Context(lib.default_params(300, 24, 0)) as ctx:
        for cond, want in cases:
            Xd = lib.colmajor(torch.from_numpy(X).cuda())
            assert ctx.chase_qr(Xd, 24, float(cond)) == want, cond
            assert O.select_qr_variant(float(cond)) == want

