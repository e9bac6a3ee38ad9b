"""Pins of the oracle's K-objective explicit-QUBO loop (Alg. 3 on stored
matrices): on the QAP's own Y and Z it must follow the pinned QAP loop
step for step (energies shifted by the constant alpha_k p_g), energies
equal full recomputation every iteration, and K = 1 / K = 3 runs keep a
mutually consistent archive."""
import numpy as np
import pytest

import oracle
from paper_2205_13399_gb300 import inputs

FAST = dict(delta0=2e6, deltaf=3e3, xi=0.02)


@pytest.mark.parametrize("acc,arc,esc", [("strict", "explore", "archive"),
                                         ("lenient", "exploit", "archive"),
                                         ("strict", "explore", "offset")])
def test_kqubo_on_qap_matrices_equals_qap_loop(acc, arc, esc):
    qi = inputs.uniform_instance(5, index=2, workload="P8")
    inst = oracle.Instance(qi.F1, qi.F2, qi.D)
    Y, Z = inst.matrix("Y"), inst.matrix("Z")
    q = oracle.KQubo(np.stack([Y, Z]))
    kw = dict(I_max=1500, replicas=3, seed=6, accept=acc, archive=arc, escape=esc, beta=700,
              trace=True, **FAST)
    ref = oracle.run(inst, **kw)
    got = oracle.kqubo_run(q, **kw)
    # E_k(QAP) = x^T Y_k x + alpha_k p_g: same trajectory, energies shifted
    x0 = np.zeros(25, dtype=np.uint8)
    off = np.array([inst.energy(0, x0), inst.energy(1, x0)])
    assert np.array_equal(got["trace"][:, :, 2], ref["trace"][:, :, 2])
    assert np.array_equal(got["trace"][:, :, :2] + off, ref["trace"][:, :, :2])
    assert np.array_equal(got["count"], ref["count"])
    assert np.array_equal(got["bits"], ref["bits"])
    assert np.array_equal(got["x"], ref["x"])
    assert np.array_equal(got["stats"], ref["stats"])


@pytest.mark.parametrize("K", [1, 3])
def test_kqubo_energies_checked_and_archive_consistent(K):
    rng = np.random.default_rng(K)
    m = 24
    Q = rng.integers(-50, 50, (K, m, m))
    q = oracle.KQubo(Q)
    out = oracle.kqubo_run(q, I_max=1500, replicas=3, seed=2, check=True, beta=30,
                           delta0=3e3, deltaf=5.0, xi=0.02)
    for r in range(3):
        c = int(out["count"][r])
        assert 0 < c <= m
        for y in range(c):
            for k in range(K):
                assert out["E"][r, y, k] == q.energy(k, out["bits"][r, y])
        for k in range(K):
            assert out["E_final"][r, k] == q.energy(k, out["x"][r])
