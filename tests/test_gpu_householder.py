"""The Householder QR fallback of Alg. 4 on the GPU against the oracle.

Alg. 4 reverts to Householder QR when a POTRF of the shifted CholeskyQR branch
fails. Two kinds of input:

* Deterministic: well-conditioned columns (kappa ~ 2) and one exactly zero
  last column. The shifted pass keeps the zero column zero (its Gram row is
  exactly zero and the shift only touches the diagonal), so the next POTRF
  meets an exactly zero pivot on both sides and both take Householder QR; the
  block without the zero column is well conditioned, so its n - 1 columns of Q
  agree element by element (bound 1e-12). The last column of Q completes the
  orthonormal basis; any unit vector orthogonal to the others is valid there,
  so it is checked only through orthonormality.
* Nearly dependent: the first `nwell` columns well conditioned, the others
  combinations of them plus new directions of relative size 1e-18
  (kappa ~ 1e16). Whether a POTRF after the shift meets a non-positive pivot
  then depends on rounding (the oracle takes either branch depending on the
  machine's BLAS), so the test does not compare branches: whichever branch the
  GPU takes must give an orthonormal, backward-stable Q whose leading `nwell`
  columns (unique there) match the oracle's element by element.

Checks on every case: orthonormality ||Q^H Q - I|| <= 1e-12; backward error
||X - Q Q^H X|| <= 1e-13 ||X|| (Householder QR is backward stable); diag(R)
real positive where X has full column rank.
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


def zero_last_column(m, n, seed):
    Z = complex_normal(seed, 91, m * n).reshape(n, m).T
    R0 = np.eye(n, dtype=np.complex128) + np.triu(
        complex_normal(seed, 92, n * n).reshape(n, n), 1) * (0.3 / np.sqrt(n))
    X = np.linalg.qr(Z)[0] @ R0
    X[:, -1] = 0.0
    return np.asfortranarray(X)


def _run(lib, X, n, cond, tensor):
    with lib.Context(lib.default_params(X.shape[0], n, 0, fp64_tensor=tensor)) as ctx:
        Xd = lib.colmajor(torch.from_numpy(X).cuda())
        v = ctx.chase_qr(Xd, n, cond)
        return v, Xd.cpu().numpy()


def _common_checks(X, Q, n, nfull):
    orth = np.abs(Q.conj().T @ Q - np.eye(n)).max()
    back = np.linalg.norm(X - Q @ (Q.conj().T @ X)) / np.linalg.norm(X)
    assert orth <= 1e-12
    assert back <= 1e-13
    d = np.diag(Q.conj().T @ X)[:nfull]
    assert np.all(d.real > 0) and np.abs(d.imag).max() <= 1e-13 * np.abs(d).max()
    return orth, back


@pytest.mark.parametrize("m,n", [(2037, 200), (700, 130), (300, 20)])
@pytest.mark.parametrize("cond", [1e20, 1e4])
@pytest.mark.parametrize("tensor", [0, 1])
def test_householder_fallback_zero_column(lib, m, n, cond, tensor):
    X = zero_last_column(m, n, m + n)
    Qo, vo, info = O.caqr(X, cond)
    assert vo == O.QR_HOUSEHOLDER and info == n  # the zero pivot, last column
    v, Q = _run(lib, X, n, cond, tensor)
    assert v == lib.CHASE_QR_HOUSEHOLDER == vo
    orth, back = _common_checks(X, Q, n, n - 1)
    err = np.abs(Q[:, :n - 1] - Qo[:, :n - 1]).max()
    print(f"zero column m={m} n={n} cond={cond:.0e} tensor={tensor}: orth {orth:.2e} "
          f"backward {back:.2e} vs oracle {err:.2e}")
    assert err <= 1e-12


@pytest.mark.parametrize("m,n,nwell,seed", [(2037, 200, 150, 1), (700, 130, 100, 2)])
@pytest.mark.parametrize("tensor", [0, 1])
def test_householder_fallback_nearly_dependent(lib, m, n, nwell, seed, tensor):
    X = nearly_dependent(m, n, nwell, seed)
    Qo, vo, info = O.caqr(X, 1e20)
    v, Q = _run(lib, X, n, 1e20, tensor)
    assert v in (lib.CHASE_QR_SHIFTED, lib.CHASE_QR_HOUSEHOLDER)
    orth, back = _common_checks(X, Q, n, nwell)
    lead = np.abs(Q[:, :nwell] - Qo[:, :nwell]).max()
    print(f"nearly dependent m={m} n={n}: variant {v} orth {orth:.2e} backward {back:.2e} "
          f"leading vs oracle {lead:.2e}")
    assert lead <= 1e-12


def test_householder_solve_step_keeps_locked_columns(lib):
    """The fallback inside chase_qr factors exactly the columns it is given and
    leaves the rest of the caller's buffer alone."""
    m, n = 700, 130
    X = zero_last_column(m, n, 4)
    extra = np.asfortranarray(complex_normal(7, 93, m * 5).reshape(5, m).T)
    full = np.asfortranarray(np.concatenate([X, extra], axis=1))
    with lib.Context(lib.default_params(m, n + 5, 0)) as ctx:
        Xd = lib.colmajor(torch.from_numpy(full).cuda())
        v = ctx.chase_qr(Xd, n, 1e20)
        out = Xd.cpu().numpy()
    assert v == lib.CHASE_QR_HOUSEHOLDER
    assert np.array_equal(out[:, n:], extra)
