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


# --- SB-DA on normalised QUBOs (Sec. 4.2 applied to Alg. 2's scalarised QUBO)

@pytest.mark.parametrize("g", [0, 4, 10])
def test_normalised_scale_closed_form(g):
    """scale = 2^23 / max_{p<=q} C_pq with C = g R + (10 - g) S, whose
    largest entry is max_ij (g Fs1 + (10 - g) Fs2)_ij * max_uv d_uv."""
    qi, inst = _inst(6, index=20 + g)
    F1, F2, D = (np.asarray(a, dtype=np.int64) for a in (qi.F1, qi.F2, qi.D))
    Fs = g * (F1 + F1.T) + (10 - g) * (F2 + F2.T)
    r = oracle.da_run(inst, g, 10, I_max=1, replicas=1, normalize=True, **FAST)
    assert r["scale"] == 8388608.0 / (int(Fs.max()) * int(D.max()))


def test_normalised_da_invariant_to_the_weight_denominator():
    """gamma = 3/10 and 6/20 give C and 2C: the scale halves exactly, so
    scale * Delta E is the same double and the normalised runs coincide
    (temperatures and offset are in the normalised QUBO's units, not scaled
    by gden); the unnormalised energies double."""
    qi, inst = _inst(7, index=31)
    kw = dict(I_max=2500, replicas=4, seed=12, beta=700, normalize=True, **FAST)
    a = oracle.da_run(inst, 3, 10, **kw)
    b = oracle.da_run(inst, 6, 20, **kw)
    assert b["scale"] * 2 == a["scale"]
    assert np.array_equal(a["best_x"], b["best_x"])
    assert np.array_equal(a["x"], b["x"])
    assert np.array_equal(2 * a["best_E"], b["best_E"])
    assert np.array_equal(a["stats"], b["stats"])
    assert a["stats"][:, 0].min() > 0 and a["stats"][:, 1].max() > 0


def test_normalised_da_power_of_two_flows():
    """Doubling both flow matrices doubles C and every Delta E exactly and
    halves the scale: the normalised run is the same trajectory."""
    qi, inst = _inst(6, index=33)
    inst2 = oracle.Instance(2 * np.asarray(qi.F1), 2 * np.asarray(qi.F2), qi.D)
    kw = dict(I_max=2000, replicas=3, seed=4, beta=900, normalize=True, **FAST)
    a = oracle.da_run(inst, 7, 10, **kw)
    b = oracle.da_run(inst2, 7, 10, **kw)
    assert np.array_equal(a["best_x"], b["best_x"])
    assert np.array_equal(a["x"], b["x"])
    assert np.array_equal(a["stats"], b["stats"])


def test_normalised_da_unit_scale_equals_integer_path():
    """With gamma = 1/1 and max Fs1 * max d = 2^23 the scale is 1 and the
    normalised DA is the plain one (same temperatures, gden = 1)."""
    n = 5
    rng = np.random.default_rng(5)
    F1 = rng.integers(0, 4096, (n, n))
    F2 = rng.integers(0, 4096, (n, n))
    for F in (F1, F2):
        np.fill_diagonal(F, 0)
    F1[0, 1] = F1[1, 0] = 4096            # largest Fs1 entry 8192
    D = np.triu(rng.integers(1, 1024, (n, n)), 1)
    D[0, 2] = 1024                        # largest distance 1024
    D = D + D.T
    inst = oracle.Instance(F1, F2, D)
    kw = dict(I_max=1500, replicas=3, seed=9, beta=400000, delta0=2e9, deltaf=3e6, xi=0.02)
    a = oracle.da_run(inst, 1, 1, normalize=True, **kw)
    b = oracle.da_run(inst, 1, 1, **kw)
    assert a["scale"] == 1.0
    for key in ("best_x", "best_E", "x", "E_final", "stats"):
        assert np.array_equal(a[key], b[key]), key
    assert a["stats"][:, 0].min() > 0


def test_normalised_da_equals_normalised_mda_on_one_objective():
    """The normalised DA on C = R is the normalised MDA loop (pinned in
    test_oracle_normalize.py) with a zero second objective, the offset
    escape and a one-slot archive."""
    qi, inst = _inst(7, index=35)
    inst1 = oracle.Instance(qi.F1, np.zeros_like(qi.F2), qi.D)
    assert inst1.norm_scale(1) == 1.0
    kw = dict(I_max=2500, replicas=5, seed=21, beta=900, **FAST)
    da = oracle.da_run(inst, 1, 1, normalize=True, **kw)
    assert da["scale"] == inst1.norm_scale(0)
    mda = oracle.run(inst1, escape="offset", archive_size=1, normalize=True, **kw)
    for r in range(5):
        assert mda["count"][r] == 1
        assert np.array_equal(da["best_x"][r], mda["bits"][r, 0])
        assert da["best_E"][r] == mda["E"][r, 0, 0]
        assert np.array_equal(da["x"][r], mda["x"][r])
        assert da["stats"][r, 0] == mda["stats"][r, 0]
        assert da["stats"][r, 1] == mda["stats"][r, 3]
