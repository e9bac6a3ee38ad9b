"""Pins of the oracle's QUBO normalisation (Sec. 4.2: the largest coefficient
of each objective QUBO set to 2^23), applied as a per-objective scale
inside the acceptance test: the scale against the closed form of the
largest coefficient, exact invariance under power-of-two scaling of an
objective, and equality with the integer path when the scale is 1."""
import numpy as np
import pytest

import oracle
from paper_2205_13399_gb300 import inputs

FAST = dict(delta0=2e6, deltaf=3e3, xi=0.02)


def test_scale_is_two_to_the_23_over_the_largest_coefficient():
    qi = inputs.uniform_instance(6, index=4, workload="P8")
    inst = oracle.Instance(qi.F1, qi.F2, qi.D)
    for k, F in enumerate((qi.F1, qi.F2)):
        F = np.asarray(F, dtype=np.int64)
        Fs = F + F.T
        cmax = int(Fs.max()) * int(np.asarray(qi.D).max())  # C_pq = Fs_ij d_uv, p < q
        assert int(inst.matrix("R" if k == 0 else "S").max()) == cmax
        assert inst.norm_scale(k) == 8388608.0 / cmax


@pytest.mark.parametrize("acc,esc", [("strict", "archive"), ("lenient", "archive"),
                                     ("strict", "offset")])
def test_power_of_two_scaling_leaves_the_run_unchanged(acc, esc):
    """Doubling F1 halves s_1 exactly and doubles every Delta E_1 exactly, so
    the normalised run follows the same trajectory with E_1 doubled."""
    qi = inputs.uniform_instance(6, index=7, workload="P8")
    a = oracle.Instance(qi.F1, qi.F2, qi.D)
    b = oracle.Instance(2 * np.asarray(qi.F1), qi.F2, qi.D)
    kw = dict(I_max=2000, replicas=3, seed=8, accept=acc, escape=esc, beta=700,
              normalize=True, trace=True, **FAST)
    ra, rb = oracle.run(a, **kw), oracle.run(b, **kw)
    assert np.array_equal(ra["trace"][:, :, 2], rb["trace"][:, :, 2])
    assert np.array_equal(2 * ra["trace"][:, :, 0], rb["trace"][:, :, 0])
    assert np.array_equal(ra["trace"][:, :, 1], rb["trace"][:, :, 1])
    assert np.array_equal(ra["count"], rb["count"])
    assert np.array_equal(ra["bits"], rb["bits"])


def test_unit_scale_equals_the_integer_path():
    """When both largest coefficients are exactly 2^23 the scales are 1 and
    the normalised run is the plain one."""
    n = 5
    rng = np.random.default_rng(3)
    F1 = rng.integers(0, 4096, (n, n))
    F2 = rng.integers(0, 4096, (n, n))
    for F in (F1, F2):
        np.fill_diagonal(F, 0)
        F[0, 1] = F[1, 0] = 4096          # largest Fs entry 8192
    D = np.triu(rng.integers(1, 1024, (n, n)), 1)
    D[0, 2] = 1024                        # largest distance 1024
    D = D + D.T
    inst = oracle.Instance(F1, F2, D)
    assert inst.norm_scale(0) == 1.0 and inst.norm_scale(1) == 1.0
    kw = dict(I_max=1500, replicas=3, seed=2, trace=True, delta0=2e9, deltaf=3e6, xi=0.02)
    r0 = oracle.run(inst, **kw)
    r1 = oracle.run(inst, normalize=True, **kw)
    for key in ("trace", "count", "E", "bits", "x", "E_final", "stats"):
        assert np.array_equal(r0[key], r1[key]), key


def test_normalisation_changes_generic_runs():
    qi = inputs.uniform_instance(7, index=2, workload="P8")
    inst = oracle.Instance(qi.F1, qi.F2, qi.D)
    kw = dict(I_max=3000, replicas=2, seed=1, trace=True, **FAST)
    assert not np.array_equal(oracle.run(inst, **kw)["trace"],
                              oracle.run(inst, normalize=True, **kw)["trace"])
