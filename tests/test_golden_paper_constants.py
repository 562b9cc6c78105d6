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
