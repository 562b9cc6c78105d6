"""CPU model of the digit-sliced FP64 product the tensor-core kernels compute
(error-free splitting in the manner of Ozaki, Ogita, Oishi and Rump, Numer.
Algorithms 59, 2012), checked in exact integer arithmetic. It pins the error
analysis the FP64-accurate products rest on; the kernels themselves are
checked against the FP64 oracle in the -m gpu tests.

The model, per real entry x of an operand already scaled by a power of two
to |x| < 1/2:
  * X = rint(x 2^48) (round half to even), written in balanced base 256:
    six integer digits d_1..d_6, the low five in [-128, 127] and the leading
    one in [-128, 128], with sum_s d_s 2^(48 - 8s) = X; so x = sum_s d_s 2^-8s
    + r with |r| <= 2^-49;
  * a product of two digit expansions keeps the digit pairs (s, t) with
    s + t <= 7 (21 pairs) or, in the extended variant, s + t <= 8 (26 pairs).
Bounds per term x*y (|x|, |y| < 1/2): the operand roundings contribute at most
2^-50 each; the pairs of level L weigh at most (number of pairs) 2^14 2^-8L,
so the dropped levels 8..12 (21 pairs) sum to below 5.1 2^-50 and the dropped
levels 9..12 (26 pairs) to below 4.1 2^-58.
"""
import numpy as np
import pytest


def digits(x):
    """Six balanced base-256 digits of rint(x 2^48), most significant first."""
    X = np.rint(np.asarray(x, dtype=np.float64) * 2.0 ** 48).astype(np.int64)
    d = np.empty(X.shape + (6,), dtype=np.int64)
    for s in range(5, 0, -1):
        low = ((X + 128) & 255) - 128
        d[..., s] = low
        X = (X - low) >> 8
    d[..., 0] = X
    return d


def test_digits_reconstruct_the_rounded_value():
    rng = np.random.default_rng(11)
    x = np.concatenate([
        rng.uniform(-0.5, 0.5, 200000) * 2.0 ** -rng.integers(0, 60, 200000),
        0.5 - np.arange(1, 2000) * 2.0 ** -60, -0.5 + np.arange(1, 2000) * 2.0 ** -60,
        (np.arange(-3000, 3000) + 0.5) * 2.0 ** -48,   # ties of the rounding to 2^-48
        (np.arange(-3000, 3000) + 0.5) * 2.0 ** -40,   # ties at a digit boundary
        np.array([0.0, -0.0, 1e-300, -1e-300, 2.0 ** -1074]),
    ])
    x = x[np.abs(x) < 0.5]
    d = digits(x)
    assert np.abs(d).max() <= 128
    assert np.abs(d[:, 1:]).max() <= 128 and d[:, 1:].min() >= -128 and d[:, 1:].max() <= 127
    X = np.zeros(len(x), dtype=np.int64)
    for s in range(6):
        X = X * 256 + d[:, s]
    # the digits represent rint(x 2^48) exactly, within half a unit of x 2^48
    assert np.array_equal(X, np.rint(x * 2.0 ** 48).astype(np.int64))
    assert np.abs(x * 2.0 ** 48 - X.astype(np.float64)).max() <= 0.5


def _exact_units(v, p):
    """v (float64 array, multiples of 2^-p) as Python integers in units of 2^-p."""
    return np.array([int(t) for t in np.round(v * 2.0 ** p).ravel()], dtype=object)


@pytest.mark.parametrize("levels,bound", [(7, 7.2 * 2.0 ** -50), (8, 2.02 * 2.0 ** -50)])
def test_truncated_digit_product_error_bound(levels, bound):
    """sum_k x_ik y_kj from the kept digit pairs against the exact sum, for
    operands with more bits than the digits hold (x = m 2^-54, |m| <= 2^52):
    error <= K * (2 * 2^-50 + dropped pairs) per entry in the worst case."""
    rng = np.random.default_rng(levels)
    M, K, n = 6, 300, 5
    xa = rng.integers(-2 ** 52, 2 ** 52, size=(M, K)).astype(np.float64) * 2.0 ** -54
    yb = rng.integers(-2 ** 52, 2 ** 52, size=(K, n)).astype(np.float64) * 2.0 ** -54
    da, db = digits(xa), digits(yb)
    # level sums are exact integers: |d_s e_t| <= 2^14, K terms
    model = np.zeros((M, n), dtype=object)
    for s in range(6):
        for t in range(6):
            if (s + 1) + (t + 1) > levels:
                continue
            lev = da[:, :, s] @ db[:, :, t]          # int64, exact
            model = model + lev.astype(object) * (2 ** (8 * (12 - (s + 1) - (t + 1))))
    # model in units of 2^-96, exact product in units of 2^-108
    exact = _exact_units(xa, 54).reshape(M, K).dot(_exact_units(yb, 54).reshape(K, n))
    err = np.array([[abs(model[i, j] * 2 ** 12 - exact[i, j]) for j in range(n)]
                    for i in range(M)], dtype=object)
    worst = max(float(e) for e in err.ravel()) * 2.0 ** -108
    print(f"levels <= {levels}: worst error {worst:.3e} = {worst / K:.3e} per term "
          f"(bound {bound:.3e} per term)")
    assert worst <= K * bound


def test_extended_variant_is_exact_on_digit_representable_operands():
    """Operands that the six digits hold exactly (the library rounds the
    triangular solve's iterate to its own digits so its products take it
    exactly): only the dropped pairs remain, below 5.1 2^-50 (21 pairs) and
    4.1 2^-58 (26 pairs) per term."""
    rng = np.random.default_rng(3)
    M, K, n = 5, 257, 4
    xa = rng.integers(-2 ** 46, 2 ** 46, size=(M, K)).astype(np.float64) * 2.0 ** -48
    yb = rng.integers(-2 ** 46, 2 ** 46, size=(K, n)).astype(np.float64) * 2.0 ** -48
    da, db = digits(xa), digits(yb)
    exact = _exact_units(xa, 48).reshape(M, K).dot(_exact_units(yb, 48).reshape(K, n))
    for levels, per_term in [(7, 5.1 * 2.0 ** -50), (8, 4.1 * 2.0 ** -58)]:
        model = np.zeros((M, n), dtype=object)
        for s in range(6):
            for t in range(6):
                if s + t + 2 <= levels:
                    lev = da[:, :, s] @ db[:, :, t]
                    model = model + lev.astype(object) * (2 ** (8 * (12 - s - t - 2)))
        worst = max(abs(float(model[i, j] - exact[i, j])) for i in range(M) for j in range(n))
        worst *= 2.0 ** -96
        assert worst <= K * per_term, (levels, worst)
