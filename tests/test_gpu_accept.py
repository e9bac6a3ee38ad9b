"""The warp engine's acceptance decision (R7): a <= fl(delta T[idx]) for an
integer penalty a, decided on the device in FP32 where that is provably
exact and by the IEEE double product near the boundary, against the plain
definition evaluated here in float64 with the oracle's -ln(u) table, on
random inputs and on penalties placed around the product itself (where the
double test must be the one that decides)."""
import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu


def _expected(a, delta, idx):
    T = oracle.neglog_table()
    return a.astype(np.float64) <= delta * T[idx]  # IEEE double product, exact float64(a)


def test_accept_random_inputs():
    from paper_2205_13399_gb300 import moda
    rng = np.random.default_rng(7)
    n = 200000
    delta = 10.0 ** rng.uniform(0, 10, n)
    idx = rng.integers(0, 65536, n).astype(np.uint32)
    prod = delta * oracle.neglog_table()[idx]
    # penalties spread over the product's scale, some far beyond 2^32
    a = np.floor(prod * rng.uniform(0.0, 2.0, n)).astype(np.int64)
    a[:1000] = rng.integers(2 ** 32, 2 ** 40, 1000)
    acc, path = moda.check_accept(a, delta, idx)
    assert np.array_equal(acc, _expected(a, delta, idx))
    assert (path >= 0).mean() > 0.99  # FP32 decides almost every bit


def test_accept_at_the_boundary():
    """a = floor(fl(delta T)) + k for k in [-8, 8]: accepted exactly for
    k <= 0; these lie within 2^-20 of the product, so the double test
    decides them."""
    from paper_2205_13399_gb300 import moda
    rng = np.random.default_rng(11)
    m = 20000
    delta = 10.0 ** rng.uniform(7, 10, m)
    idx = rng.integers(0, 65536, m).astype(np.uint32)
    prod = delta * oracle.neglog_table()[idx]
    base = np.floor(prod).astype(np.int64)
    k = rng.integers(-8, 9, m)
    a = np.maximum(base + k, 0)
    keep = prod > 2.0 ** 24  # the band 2^-20 prod holds more than 8 integers
    a, delta, idx, k = a[keep], delta[keep], idx[keep], k[keep]
    acc, path = moda.check_accept(a, delta, idx)
    exp = _expected(a, delta, idx)
    assert np.array_equal(acc, exp)
    assert np.array_equal(exp, k <= 0)
    assert (path == -1).all()

