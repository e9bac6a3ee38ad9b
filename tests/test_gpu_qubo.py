"""Explicit QUBOs with K objectives (Alg. 3 on stored matrices): the CUDA
path against the oracle's K-objective loop, bit for bit -- traces, archives,
final states and counters -- and, on a QAP instance's own Y and Z, against
the dedicated bQAP kernel."""
import numpy as np
import pytest

import oracle
from paper_2205_13399_gb300 import inputs

pytestmark = pytest.mark.gpu

FAST = dict(delta0=3e3, deltaf=5.0, xi=0.02)


def _bits(words, m):
    from paper_2205_13399_gb300.moda import unpack_bits
    return unpack_bits(words, m)


def _compare(res, orc, m):
    for r in range(len(res["count"])):
        c = int(res["count"][r])
        assert c == int(orc["count"][r]), f"replica {r}: archive size"
        assert np.array_equal(res["E"][r, :c], orc["E"][r, :c]), f"replica {r}: energies"
        assert np.array_equal(_bits(res["bits"][r, :c], m), orc["bits"][r, :c])
    assert np.array_equal(_bits(res["x"], m), orc["x"])
    assert np.array_equal(res["E_final"], orc["E_final"])
    assert np.array_equal(res["stats"], orc["stats"])


@pytest.mark.parametrize("K,m", [(1, 20), (2, 37), (3, 64), (2, 200)])
@pytest.mark.parametrize("acc,arc,esc", [("strict", "explore", "archive"),
                                         ("lenient", "exploit", "archive"),
                                         ("strict", "explore", "offset")])
def test_qubo_matches_oracle(K, m, acc, arc, esc):
    from paper_2205_13399_gb300 import moda
    rng = np.random.default_rng(10 * K + m)
    Q = rng.integers(-60, 60, (K, m, m)).astype(np.int32)
    kw = dict(replicas=3, I_max=1200, seed=K + m, accept=acc, archive=arc, escape=esc,
              beta=25, **FAST)
    run = moda.Qubo(Q).anneal(trace=True, **kw).wait()
    res = run.read(trace=True)
    orc = oracle.kqubo_run(oracle.KQubo(Q), trace=True, **kw)
    assert np.array_equal(res["trace"], orc["trace"])
    _compare(res, orc, m)


def test_qubo_records_off_equals_on():
    from paper_2205_13399_gb300 import moda
    rng = np.random.default_rng(3)
    Q = rng.integers(-40, 40, (2, 50, 50)).astype(np.int32)
    q = moda.Qubo(Q)
    kw = dict(replicas=4, I_max=1500, seed=1, beta=20, **FAST)
    a = q.anneal(**kw).wait().read()
    b = q.anneal(field_cache="off", **kw).wait().read()
    for key in a:
        assert np.array_equal(a[key], b[key]), key


def test_qubo_on_qap_matrices_equals_qap_kernel():
    """Y and Z of a bQAP instance as explicit QUBOs: the same trajectory as
    the bQAP kernel, energies shifted by the constant alpha_k p_g."""
    from paper_2205_13399_gb300 import moda
    qi = inputs.uniform_instance(6, index=4, workload="P8")
    oi = oracle.Instance(qi.F1, qi.F2, qi.D)
    Y, Z = oi.matrix("Y"), oi.matrix("Z")
    off = np.array([oi.energy(0, np.zeros(36, np.uint8)), oi.energy(1, np.zeros(36, np.uint8))])
    kw = dict(replicas=3, I_max=1500, seed=4, delta0=2e6, deltaf=3e3, xi=0.02)
    res = moda.Qubo(np.stack([Y, Z]).astype(np.int32)).anneal(trace=True, **kw).wait() \
        .read(trace=True)
    g = moda.Instance(qi.F1, qi.F2, qi.D)
    ref = moda.anneal(g, trace=True, **kw).wait()
    for r in range(3):
        tr = ref.read_trace(r)
        assert np.array_equal(res["trace"][r, :, 2], tr[:, 2])
        assert np.array_equal(res["trace"][r, :, :2] + off, tr[:, :2])
    rr = ref.read()
    assert np.array_equal(res["count"], rr.count)
