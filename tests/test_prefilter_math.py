"""The FP32 acceptance test's error argument, checked on the host with
IEEE float32 arithmetic (numpy rounds every float32 product and conversion
to nearest, as the device's __fmul_rn and __uint2float_rn do): whenever the
float test decides (af <= fl32(pf (1 - 2^-20)) accepts, af >=
fl32(pf (1 + 2^-20)) rejects, pf = fl32(fl32(delta) fl32(T))), the decision
equals the double test a <= fl(delta T) of R7.  Random inputs over the
schedule's range and penalties placed at the product itself; the device
code is checked against the same definition in tests/test_gpu_accept.py."""
import numpy as np

import oracle

LO = np.float32(1.0 - 2.0 ** -20)
HI = np.float32(1.0 + 2.0 ** -20)


def _decide(a, delta, T):
    pf = np.float32(delta.astype(np.float32) * T.astype(np.float32))
    af = a.astype(np.float32)
    acc = af <= np.float32(pf * LO)
    rej = af >= np.float32(pf * HI)
    exact = a.astype(np.float64) <= delta * T
    return acc, rej, exact


def test_float_decisions_agree_with_the_double_test():
    rng = np.random.default_rng(17)
    T = oracle.neglog_table()
    n = 1_000_000
    delta = 10.0 ** rng.uniform(0.0, 10.5, n)
    idx = rng.integers(0, 65536, n)
    prod = delta * T[idx]
    a = np.floor(prod * rng.uniform(0.0, 2.0, n)).astype(np.int64)
    acc, rej, exact = _decide(a, delta, T[idx])
    assert not np.any(acc & rej)
    assert np.all(exact[acc])
    assert not np.any(exact[rej])
    assert (acc | rej).mean() > 0.999  # the double test is rarely needed


def test_penalties_at_the_product_never_decided_wrongly():
    rng = np.random.default_rng(23)
    T = oracle.neglog_table()
    n = 400_000
    delta = 10.0 ** rng.uniform(0.0, 10.5, n)
    idx = rng.integers(0, 65536, n)
    prod = delta * T[idx]
    a = np.maximum(np.floor(prod).astype(np.int64) + rng.integers(-40, 41, n), 0)
    acc, rej, exact = _decide(a, delta, T[idx])
    assert np.all(exact[acc])
    assert not np.any(exact[rej])
    # penalties within a few units of a large product are left to the
    # double test
    big = prod > 2.0 ** 26
    near = np.abs(a - prod) < 8
    assert not np.any((acc | rej)[big & near])
