"""SB-DA (Sec. 3.2, Alg. 2) on the GPU against the oracle's literal Alg. 1 /
Alg. 2: per weight and replica the best solution found, its energy, the
final state and the counters, then the merged non-dominated front, bit for
bit."""
import numpy as np
import pytest

import oracle
from paper_2205_13399_gb300 import inputs

pytestmark = pytest.mark.gpu

FAST = dict(delta0=2e6, deltaf=3e3, xi=0.02)


def _best(run, m):
    from paper_2205_13399_gb300.moda import unpack_bits
    res = run.read()
    bx = np.where(res.count[:, None] > 0, unpack_bits(res.bits[:, 0], m),
                  unpack_bits(res.x, m))
    return res, bx


@pytest.mark.parametrize("n,index,bt", [(6, 1, 0), (9, 2, 0), (12, 3, 64), (25, 4, 0)])
def test_sbda_matches_oracle(n, index, bt):
    from paper_2205_13399_gb300 import moda
    qi = inputs.uniform_instance(n, index=index, workload="P8") if n < 20 else \
        inputs.batch_instances(1, n_lo=n, n_hi=n)[0]
    kw = dict(replicas=3, I_max=1500 if n < 20 else 1000, seed=40 + n, beta=800, **FAST)
    inst = moda.Instance(qi.F1, qi.F2, qi.D)
    runs, front = moda.sbda(inst, block_threads=bt, **kw)
    oi = oracle.Instance(qi.F1, qi.F2, qi.D)
    orc = oracle.sbda(oi, **kw)
    m = n * n
    for g, (run, o) in enumerate(zip(runs, orc["runs"])):
        assert run.inst.w[0] == o["w"] and run.inst.w[1] == 0
        res, bx = _best(run, m)
        assert np.array_equal(bx, o["best_x"]), f"weight {g}: best states"
        best_E = np.where(res.count > 0, res.E[:, 0, 0], res.E_final[:, 0])
        assert np.array_equal(best_E, o["best_E"]), f"weight {g}: best energies"
        assert np.array_equal(moda.unpack_bits(res.x, m), o["x"]), f"weight {g}: final states"
        assert np.array_equal(res.E_final[:, 0], o["E_final"])
        assert np.all(res.E_final[:, 1] == 0)
        assert np.array_equal(res.stats[:, 0], o["stats"][:, 0]), f"weight {g}: flips"
        assert np.array_equal(res.stats[:, 3], o["stats"][:, 1]), f"weight {g}: offset raises"
    got = [(p["c1"], p["c2"], p["weight"], p["replica"]) for p in front]
    assert got == [tuple(int(v) for v in c) for c in orc["front"]]
    for p in front:
        assert p["c1"] == oracle.qap_cost(qi.F1, qi.D, p["perm"])
        assert p["c2"] == oracle.qap_cost(qi.F2, qi.D, p["perm"])


@pytest.mark.parametrize("n,index,bt", [(7, 5, 0), (12, 6, 64), (25, 7, 0)])
def test_normalised_sbda_matches_oracle(n, index, bt):
    """SB-DA on normalised QUBOs (Sec. 4.2): each weight's acceptance test
    sees s Delta E - E_off in IEEE double; per weight and replica the best
    state, its energy, the final state and the counters, then the merged
    front, against the oracle bit for bit."""
    from paper_2205_13399_gb300 import moda
    qi = inputs.uniform_instance(n, index=index, workload="P8") if n < 20 else \
        inputs.batch_instances(1, n_lo=n, n_hi=n)[0]
    # the paper's temperatures for normalised QUBOs, on a fast schedule
    kw = dict(replicas=3, I_max=1500 if n < 20 else 1000, seed=60 + n, delta0=1e9,
              deltaf=1e4, xi=0.02)
    inst = moda.Instance(qi.F1, qi.F2, qi.D)
    runs, front = moda.sbda(inst, block_threads=bt, normalize=True, **kw)
    oi = oracle.Instance(qi.F1, qi.F2, qi.D)
    orc = oracle.sbda(oi, normalize=True, **kw)
    m = n * n
    flips = raises = 0
    for g, (run, o) in enumerate(zip(runs, orc["runs"])):
        res, bx = _best(run, m)
        assert np.array_equal(bx, o["best_x"]), f"weight {g}: best states"
        best_E = np.where(res.count > 0, res.E[:, 0, 0], res.E_final[:, 0])
        assert np.array_equal(best_E, o["best_E"]), f"weight {g}: best energies"
        assert np.array_equal(moda.unpack_bits(res.x, m), o["x"]), f"weight {g}: final states"
        assert np.array_equal(res.E_final[:, 0], o["E_final"])
        assert np.array_equal(res.stats[:, 0], o["stats"][:, 0]), f"weight {g}: flips"
        assert np.array_equal(res.stats[:, 3], o["stats"][:, 1]), f"weight {g}: offset raises"
        flips += int(o["stats"][:, 0].sum())
        raises += int(o["stats"][:, 1].sum())
    assert flips > 0 and raises > 0
    got = [(p["c1"], p["c2"], p["weight"], p["replica"]) for p in front]
    assert got == [tuple(int(v) for v in c) for c in orc["front"]]


def test_scalarize_overflow_and_bad_weight():
    from paper_2205_13399_gb300 import moda
    n = 30
    F = np.full((n, n), 20000, dtype=np.int16)
    np.fill_diagonal(F, 0)
    D = np.full((n, n), 3, dtype=np.int16)
    np.fill_diagonal(D, 0)
    inst = moda.Instance(F, F, D)
    with pytest.raises(moda.MODAError, match="MODA_EOVERFLOW"):
        inst.scalarize(5, 1000)
    with pytest.raises(moda.MODAError, match="MODA_EINVAL"):
        inst.scalarize(11, 10)
