"""The Householder QR fallback of Alg. 4 on the GPU against the oracle.

Alg. 4 reverts to Householder QR when a POTRF of the shifted CholeskyQR branch
fails. The inputs here make that happen on both sides: the first `nwell`
columns are well conditioned (kappa ~ 2), the remaining ones are combinations
of them plus new directions of relative size 1e-18, so kappa(X) ~ 1e16 - 1e17
cannot be reduced by column scaling; after the shift the CholeskyQR2 Gram
matrix has eigenvalues far below its rounding and POTRF meets a non-positive
pivot. Both sides then take Householder QR of the input block.

Checks: the same Alg. 4 branch (variant 4) as the oracle; orthonormality
||Q^H Q - I|| <= 1e-12; backward error ||X - Q Q^H X|| <= 1e-13 ||X||
(Householder QR is backward stable); the leading `nwell` columns element by
element against the oracle's Householder Q (the QR factor with positive real
diag(R) is unique there: those columns have kappa ~ 2, so both sides agree to
a few units of rounding, bound 1e-12); and diag(R) real positive.
"""
import numpy as np
import pytest

from oracle import chase_oracle as O
from synth import complex_normal

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def nearly_dependent(m, n, nwell, seed, eps=1e-18):
    Z = complex_normal(seed, 91, m * n).reshape(n, m).T
    Q0 = np.linalg.qr(Z)[0]
    R0 = np.eye(n, dtype=np.complex128) + np.triu(
        complex_normal(seed, 92, n * n).reshape(n, n), 1) * (0.3 / np.sqrt(n))
    R0[nwell:, nwell:] *= eps
    return np.asfortranarray(Q0 @ R0)


@pytest.mark.parametrize("m,n,nwell,seed", [(2037, 200, 150, 1), (700, 130, 100, 2)])
@pytest.mark.parametrize("tensor", [0, 1])
def test_householder_fallback_matches_oracle(lib, m, n, nwell, seed, tensor):
    X = nearly_dependent(m, n, nwell, seed)
    Qo, vo, info = O.caqr(X, 1e20)
    assert vo == O.QR_HOUSEHOLDER and info != 0  # the input takes the fallback
    with lib.Context(lib.default_params(m, n, 0, fp64_tensor=tensor)) as ctx:
        Xd = lib.colmajor(torch.from_numpy(X).cuda())
        v = ctx.chase_qr(Xd, n, 1e20)
        Q = Xd.cpu().numpy()
    assert v == lib.CHASE_QR_HOUSEHOLDER == vo
    orth = np.abs(Q.conj().T @ Q - np.eye(n)).max()
    back = np.linalg.norm(X - Q @ (Q.conj().T @ X)) / np.linalg.norm(X)
    lead = np.abs(Q[:, :nwell] - Qo[:, :nwell]).max()
    print(f"m={m} n={n}: orth {orth:.2e} backward {back:.2e} leading vs oracle {lead:.2e}")
    assert orth <= 1e-12
    assert back <= 1e-13
    assert lead <= 1e-12
    R = Q.conj().T @ X
    d = np.diag(R)
    assert np.all(d[:nwell].real > 0) and np.abs(d[:nwell].imag).max() <= 1e-13


def test_householder_solve_step_keeps_locked_columns(lib):
    """The fallback inside chase_qr factors exactly the columns it is given and
    leaves the rest of the caller's buffer alone."""
    m, n, nwell = 700, 130, 100
    X = nearly_dependent(m, n, nwell, 2)
    extra = np.asfortranarray(complex_normal(7, 93, m * 5).reshape(5, m).T)
    full = np.asfortranarray(np.concatenate([X, extra], axis=1))
    with lib.Context(lib.default_params(m, n + 5, 0)) as ctx:
        Xd = lib.colmajor(torch.from_numpy(full).cuda())
        v = ctx.chase_qr(Xd, n, 1e20)
        out = Xd.cpu().numpy()
    assert v == lib.CHASE_QR_HOUSEHOLDER
    assert np.array_equal(out[:, n:], extra)
