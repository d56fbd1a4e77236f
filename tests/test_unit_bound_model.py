"""The bound behind the data-driven accumulator units, checked by brute force (CPU).

The tensor-core leaf may let one FP32 accumulator run over a K range as long
as every partial sum of Σ_k x_k·z_k stays an integer of magnitude ≤ 2^24.
The library bounds that from per-block maxima of row sums of squares: with
T_x[b] = max over rows of Σ_{k in block b} x_k² (blocks of 256 columns), a
range touching blocks B has, for every row pair and every partial sum in any
order, |Σ x_k·z_k| ≤ Σ |x_k|·|z_k| ≤ sqrt(Σ_B T_x[b] · Σ_B T_z[b])
(Cauchy–Schwarz on each row pair, then the maxima).  These tests model that
bound in numpy and compare it with the exact worst partial sums of small
random and adversarial digit matrices, and check it never exceeds the
worst-case bound K·max|x|·max|z| it replaces (the library takes the smaller).
"""
import numpy as np
import pytest

BLOCK = 256


def block_maxima(X):
    """T[b] = max over rows of the sum of squares of X's entries in block b."""
    n, k = X.shape
    nb = (k + BLOCK - 1) // BLOCK
    sq = X.astype(np.int64) ** 2
    return np.array([sq[:, b * BLOCK:(b + 1) * BLOCK].sum(axis=1).max() for b in range(nb)])


def data_bound(TX, TZ, k0, k1):
    """The library's bound for columns [k0, k1): the blocks the range touches."""
    b0, b1 = k0 // BLOCK, (k1 - 1) // BLOCK
    return np.sqrt(float(TX[b0:b1 + 1].sum()) * float(TZ[b0:b1 + 1].sum()))


def worst_partial(X, Z, k0, k1):
    """Largest |partial sum| over every row pair, every prefix and any order:
    the sum of |x_k|·|z_k| over the range bounds all of them and is attained."""
    A = np.abs(X[:, k0:k1]).astype(np.int64)
    B = np.abs(Z[:, k0:k1]).astype(np.int64)
    return int((A @ B.T).max())


@pytest.mark.parametrize("seed", range(6))
@pytest.mark.parametrize("lo,hi", [(-128, 128), (-256, 256), (-64, 64)])
def test_bound_holds_on_random_digits(seed, lo, hi):
    rng = np.random.default_rng(seed)
    X = rng.integers(lo, hi + 1, size=(48, 1024))
    Z = rng.integers(lo, hi + 1, size=(40, 1024))
    TX, TZ = block_maxima(X), block_maxima(Z)
    for k0, k1 in [(0, 256), (0, 1024), (64, 700), (256, 512), (300, 301), (0, 320)]:
        assert worst_partial(X, Z, k0, k1) <= data_bound(TX, TZ, k0, k1) + 1e-6


def test_bound_is_attained_at_the_digit_bounds():
    """Every digit at its bound: the data bound equals the worst-case bound."""
    X = np.full((8, 1024), -128)
    Z = np.full((8, 1024), 128)
    TX, TZ = block_maxima(X), block_maxima(Z)
    for k0, k1 in [(0, 256), (0, 1024)]:
        worst_case = (k1 - k0) * 128 * 128
        assert worst_partial(X, Z, k0, k1) == worst_case
        assert data_bound(TX, TZ, k0, k1) == worst_case


def test_bound_never_exceeds_the_worst_case_on_whole_blocks():
    rng = np.random.default_rng(7)
    X = rng.integers(-128, 129, size=(32, 1024))
    TX = block_maxima(X)
    for nblocks in range(1, 5):
        k1 = nblocks * BLOCK
        assert data_bound(TX, TX, 0, k1) <= k1 * 128 * 128


def test_uniform_digits_let_a_digit_sum_span_sixteen_k_blocks():
    """Uniform byte digits: a Karatsuba sum plane (|x0 + x1| ≤ 256) fits one exact
    unit over 1024 columns with the data bound, where the worst case needs four."""
    rng = np.random.default_rng(11)
    d0 = rng.integers(-128, 128, size=(2048, 1024))
    d1 = rng.integers(-128, 128, size=(2048, 1024))
    S = d0 + d1
    TS = block_maxima(S)
    assert data_bound(TS, TS, 0, 1024) <= 2 ** 24
    assert 1024 * 256 * 256 > 2 ** 24  # the worst-case bound splits the range
    assert worst_partial(S, S, 0, 1024) <= data_bound(TS, TS, 0, 1024)
