"""Pins of the oracle's SB-DA (Sec. 3.2, Alg. 2) and the DA it calls
(Sec. 3.1, Alg. 1), each against something other than the DA loop itself:
the closed form of the scalarised penalty, the MDA loop (already pinned)
on a single-objective instance, recomputed energies, and brute-force
Pareto fronts."""
import numpy as np
import pytest

import oracle
from paper_2205_13399_gb300 import inputs

FAST = dict(delta0=2e6, deltaf=3e3, xi=0.02)


def _inst(n, index=0):
    qi = inputs.uniform_instance(n, index=index, workload="P8")
    return qi, oracle.Instance(qi.F1, qi.F2, qi.D)


@pytest.mark.parametrize("g", [0, 3, 7, 10])
def test_scalarised_penalty_closed_form(g):
    """w of C = g R + (10 - g) S (Eq. vermap on the symmetric P, reading
    R1) equals max_i sum_j (g Fs1 + (10 - g) Fs2)_ij * max_u sum_v d_uv."""
    qi, inst = _inst(6, index=g)
    F1, F2, D = (np.asarray(a, dtype=np.int64) for a in (qi.F1, qi.F2, qi.D))
    Fs = g * (F1 + F1.T) + (10 - g) * (F2 + F2.T)
    w = int(Fs.sum(1).max() * D.sum(1).max())
    r = oracle.da_run(inst, g, 10, I_max=1, replicas=1, **FAST)
    assert r["w"] == w
    if g == 10:
        assert r["w"] == 10 * oracle.Instance(qi.F1, qi.F2, qi.D).w[0]


def test_da_equals_mda_on_one_objective():
    """DA on C = R (gamma = 1/1) is MDA with a zero second objective, the
    offset escape and an explorative archive of one slot: the archive keeps
    exactly the lowest-energy state reached by a flip, so DA's best solution
    and MDA's single member must coincide, replica by replica."""
    qi, inst = _inst(7, index=2)
    zero = np.zeros_like(qi.F2)
    inst1 = oracle.Instance(qi.F1, zero, qi.D)
    kw = dict(I_max=2500, replicas=6, seed=77, beta=900, **FAST)
    da = oracle.da_run(inst, 1, 1, **kw)
    mda = oracle.run(inst1, escape="offset", archive_size=1, **kw)
    assert np.all(mda["E_final"][:, 1] == 0)
    for r in range(6):
        assert mda["count"][r] == 1
        assert np.array_equal(da["best_x"][r], mda["bits"][r, 0])
        assert da["best_E"][r] == mda["E"][r, 0, 0]
        assert np.array_equal(da["x"][r], mda["x"][r])
        assert da["stats"][r, 0] == mda["stats"][r, 0]
        assert da["stats"][r, 1] == mda["stats"][r, 3]


def test_da_energies_recomputed():
    qi, inst = _inst(6, index=5)
    r = oracle.da_run(inst, 4, 10, I_max=2000, replicas=2, seed=3, beta=500, **FAST)
    assert r["energy_check"] == list(r["best_E"][:2])
    assert np.all(r["best_E"] <= r["E_final"])


def test_sbda_front_against_brute_force():
    """Every SB-DA front point is a permutation whose (c1, c2) is its QAP
    cost (Sec. 2.1), weakly dominated by the exact front (5! states)."""
    qi, inst = _inst(5, index=9)
    out = oracle.sbda(inst, I_max=3000, replicas=4, seed=5, beta=800, **FAST)
    exact = oracle.pareto_front_bruteforce(qi.F1, qi.F2, qi.D)
    ex = [(int(p[0]), int(p[1])) for p in exact]
    assert out["front"]
    for c1, c2, gi, rep in out["front"]:
        x = out["runs"][gi]["best_x"][rep]
        perm = oracle.decode_permutation(x.reshape(5, 5))
        assert perm is not None
        assert c1 == oracle.qap_cost(qi.F1, qi.D, perm)
        assert c2 == oracle.qap_cost(qi.F2, qi.D, perm)
        assert any(e1 <= c1 and e2 <= c2 for e1, e2 in ex)
    pts = [(c[0], c[1]) for c in out["front"]]
    assert len(oracle.nondominated(pts)) == len(pts)
