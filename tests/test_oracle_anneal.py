"""Pins of the oracle's annealing loop (Sec. 3.3, Alg. 3-5) and its random
draws against closed forms, invariants, hand-made archive sequences and, for
n = 8, the exact Pareto front by enumeration of all 8! permutations."""
import math

import numpy as np
import pytest

import oracle
from paper_2205_13399_gb300 import inputs


# --------------------------------------------------------------------------
# cooling schedule and the -ln(u) table
# --------------------------------------------------------------------------

def test_schedule_closed_form():
    d0, df, xi = 1e9, 1e4, 1e-3
    sch = oracle.schedule(d0, df, xi, 20000)
    # cooling happens before the first Delta E (Alg. 3): delta_1 = d0 (1 - xi)
    assert sch[0] == d0 * (1.0 - xi)
    # the first delta at or below df: ln(df/d0) / ln(1 - xi) = 11507.2...
    t_freeze = math.ceil(math.log(df / d0) / math.log(1 - xi))
    first_low = int(np.argmax(sch <= df)) + 1
    assert first_low == t_freeze
    assert np.all(np.diff(sch[:first_low]) < 0)
    assert np.all(sch[first_low - 1:] == sch[first_low - 1])
    assert sch[first_low - 1] <= df < sch[first_low - 2]
    # each value within the rounding bound of the closed form d0 (1-xi)^t
    t = np.arange(1, first_low + 1, dtype=np.float64)
    closed = d0 * np.exp(t * math.log1p(-xi))
    rel = np.abs(sch[:first_low] - closed) / closed
    assert np.all(rel <= (t + 2) * 2.0 ** -52 * 4)


def test_neglog_table():
    T = oracle.neglog_table()
    assert T.shape == (65536,)
    assert np.all(np.diff(T) < 0)
    idx = np.arange(65536, dtype=np.float64)
    assert np.allclose(T, -np.log((idx + 0.5) / 65536.0), rtol=4.5e-16, atol=0)  # within 2 ulp of numpy's log
    # midpoint rule for int_0^1 -ln u du = 1, error below 1e-4
    assert abs(T.mean() - 1.0) < 1e-4
    # T[idx] - T[j] = ln((j + .5)/(idx + .5))
    assert math.isclose(T[0] - T[65535], math.log(65535.5 / 0.5), rel_tol=1e-14)


# --------------------------------------------------------------------------
# Philox4x32-10: properties fixed by its construction
# --------------------------------------------------------------------------

def test_philox_bijective_and_key_sensitive():
    outs = set()
    for c in range(4096):
        o = oracle.philox([c, 7, 3, 1], [11, 22])
        outs.add(tuple(int(v) for v in o))
    assert len(outs) == 4096  # each round is a bijection of the counter
    a = oracle.philox([5, 6, 7, 8], [1, 2])
    b = oracle.philox([5, 6, 7, 8], [1, 3])
    assert not np.array_equal(a, b)


def test_philox_avalanche_and_uniformity():
    rng = np.random.default_rng(0)
    flips = []
    top = []
    for _ in range(400):
        ctr = rng.integers(0, 2 ** 32, size=4, dtype=np.uint64).astype(np.uint32)
        key = rng.integers(0, 2 ** 32, size=2, dtype=np.uint64).astype(np.uint32)
        o = oracle.philox(ctr, key)
        top.extend(int(v) >> 24 for v in o)
        bit = int(rng.integers(0, 128))
        c2 = ctr.copy()
        c2[bit // 32] ^= np.uint32(1 << (bit % 32))
        o2 = oracle.philox(c2, key)
        flips.append(sum(bin(int(x) ^ int(y)).count("1") for x, y in zip(o, o2)))
    assert 60 < np.mean(flips) < 68  # about half of 128 output bits change
    counts = np.bincount(np.array(top), minlength=256)
    chi2 = ((counts - len(top) / 256) ** 2 / (len(top) / 256)).sum()
    assert chi2 < 256 + 6 * math.sqrt(2 * 256)


# --------------------------------------------------------------------------
# acceptance rule (Eq. pacceptms / pacceptml with the 16-bit variate)
# --------------------------------------------------------------------------

@pytest.mark.parametrize("ratio", [0.0, 0.1, 0.5, 1.0, 2.0, 5.0])
def test_acceptance_frequency(ratio):
    delta = 12345.678
    a = int(ratio * delta)
    groups = 50000
    n = 4 * groups
    acc = oracle.accept_count(a, delta, seed=9, step=17, replica=3, groups=groups)
    T = oracle.neglog_table()
    p_quant = float(np.mean(a <= delta * T))  # exact probability of the rule
    assert abs(p_quant - math.exp(-a / delta)) < 2e-4 + 1e-4 * a / delta
    sd = math.sqrt(max(p_quant * (1 - p_quant), 1e-12) / n)
    assert abs(acc / n - p_quant) <= 5 * sd + 1e-9
    if a == 0:
        assert acc == n


# --------------------------------------------------------------------------
# archive updates replayed on hand-made sequences
# --------------------------------------------------------------------------

def test_explorative_update_sequence():
    A = []
    A = oracle.archive_update("explore", 3, A, (5, 5))
    assert A == [(5, 5)]
    A = oracle.archive_update("explore", 3, A, (6, 4))   # non-dominated: added
    assert A == [(5, 5), (6, 4)]
    A = oracle.archive_update("explore", 3, A, (7, 7))   # dominated, not full: added
    assert A == [(5, 5), (6, 4), (7, 7)]
    A = oracle.archive_update("explore", 3, A, (4, 4))   # replaces the first it dominates
    assert A == [(4, 4), (6, 4), (7, 7)]
    A = oracle.archive_update("explore", 3, A, (8, 8))   # full, dominates nothing
    assert A == [(4, 4), (6, 4), (7, 7)]
    A = oracle.archive_update("explore", 3, A, (4, 4))   # equal to slot 0, dominates slot 1
    assert A == [(4, 4), (4, 4), (7, 7)]
    A = oracle.archive_update("explore", 3, A, (1, 9))   # full, dominates nothing
    assert A == [(4, 4), (4, 4), (7, 7)]


def test_exploitative_update_sequence():
    A = oracle.archive_update("exploit", 3, [], (5, 5))
    assert A == [(5, 5)]
    A = oracle.archive_update("exploit", 3, A, (7, 7))   # dominated: ignored
    assert A == [(5, 5)]
    A = oracle.archive_update("exploit", 3, A, (6, 4))
    assert A == [(5, 5), (6, 4)]
    # (4, 3) dominates both; the draw picks B[floor(u |B| / 2^32)]
    assert oracle.archive_update("exploit", 3, A, (4, 3), u=0) == [(4, 3), (6, 4)]
    assert oracle.archive_update("exploit", 3, A, (4, 3), u=2 ** 31) == [(5, 5), (4, 3)]
    assert oracle.archive_update("exploit", 3, A, (4, 3), u=2 ** 32 - 1) == [(5, 5), (4, 3)]
    A = [(4, 3), (6, 4)]
    # an equivalent member does not block: (4, 3) dominates (6, 4) only
    assert oracle.archive_update("exploit", 3, A, (4, 3), u=123) == [(4, 3), (4, 3)]
    # non-dominated, B empty, not full: appended
    assert oracle.archive_update("exploit", 3, A, (10, 1)) == [(4, 3), (6, 4), (10, 1)]
    # full: a non-dominated point that dominates nothing is dropped
    full = [(4, 3), (6, 4), (10, 1)]
    assert oracle.archive_update("exploit", 3, full, (2, 20)) == full


# --------------------------------------------------------------------------
# the loop itself
# --------------------------------------------------------------------------

VARIANTS = [(acc, arc, esc) for acc in ("strict", "lenient")
            for arc in ("explore", "exploit") for esc in ("archive", "offset")]


@pytest.mark.parametrize("acc,arc,esc", VARIANTS)
def test_loop_checked_every_iteration(acc, arc, esc):
    """check=True recomputes both energies and all fields from scratch after
    every iteration and fails on a mismatch (Eq. cale: E(y) = E(x) + dE)."""
    for n in (3, 5):
        I = inputs.uniform_instance(n, index=n, workload="P8")
        inst = oracle.Instance(I.F1, I.F2, I.D)
        out = oracle.run(inst, I_max=400, replicas=[0, 1], seed=5, accept=acc, archive=arc,
                         escape=esc, delta0=1e4, deltaf=10.0, xi=0.02, beta=50, check=True,
                         trace=True)
        _check_result(inst, out, 400)


def _check_result(inst, out, I_max):
    s = out["E"].shape[1]
    for r in range(out["count"].shape[0]):
        c = int(out["count"][r])
        assert 0 <= c <= s
        for slot in range(c):
            bits = out["bits"][r, slot]
            assert out["E"][r, slot, 0] == inst.energy(0, bits)
            assert out["E"][r, slot, 1] == inst.energy(1, bits)
        x = out["x"][r]
        assert out["E_final"][r, 0] == inst.energy(0, x)
        assert out["E_final"][r, 1] == inst.energy(1, x)
        st = out["stats"][r]
        assert st.sum() == I_max
        if "trace" in out:
            assert tuple(out["trace"][r, -1, :2]) == tuple(out["E_final"][r])
            ev = out["trace"][r, :, 2]
            assert (ev >= 0).sum() == st[0]


def test_determinism_and_replica_independence():
    I = inputs.uniform_instance(6, index=1, workload="P8")
    inst = oracle.Instance(I.F1, I.F2, I.D)
    a = oracle.run(inst, I_max=3000, replicas=[0, 1, 2], seed=42)
    b = oracle.run(inst, I_max=3000, replicas=[2, 0], seed=42)
    assert np.array_equal(a["E"][2], b["E"][0]) and np.array_equal(a["bits"][0], b["bits"][1])
    assert not np.array_equal(a["x"][0], a["x"][1])
    c = oracle.run(inst, I_max=3000, replicas=[0], seed=43)
    assert not np.array_equal(a["E"][0], c["E"][0])


def test_prefix_property():
    """The schedule does not depend on I_max, so a shorter run is a prefix."""
    I = inputs.uniform_instance(5, index=2, workload="P8")
    inst = oracle.Instance(I.F1, I.F2, I.D)
    a = oracle.run(inst, I_max=2000, replicas=[3], seed=1, trace=True)
    b = oracle.run(inst, I_max=1200, replicas=[3], seed=1, trace=True)
    assert np.array_equal(a["trace"][0, :1200], b["trace"][0])


def test_front_quality_n8():
    """n = 8 workload: every feasible archive point is an exact QAP cost pair
    of its decoded permutation and is weakly dominated by the exact front
    (brute force over 8! permutations); HV(output) <= HV(exact)."""
    I = inputs.workload_instance("P8")
    run = inputs.WORKLOAD_RUN["P8"]
    inst = oracle.Instance(I.F1, I.F2, I.D)
    out = oracle.run(inst, I_max=run["I_max"], replicas=range(run["replicas"]), seed=run["seed"])
    _check_result(inst, out, run["I_max"])
    front = oracle.pareto_front_bruteforce(I.F1, I.F2, I.D)
    pts = []
    for r in range(out["count"].shape[0]):
        for slot in range(int(out["count"][r])):
            bits = out["bits"][r, slot]
            perm = oracle.decode_permutation(bits)
            if perm is None:
                continue
            f1 = oracle.qap_cost(I.F1, I.D, perm)
            f2 = oracle.qap_cost(I.F2, I.D, perm)
            assert (f1, f2) == tuple(int(v) for v in out["E"][r, slot])
            assert any(a <= f1 and b <= f2 for a, b in front)
            pts.append((f1, f2))
    assert len(pts) > 0
    lo = (min(a for a, _ in front), min(b for _, b in front))
    hi = (max(a for a, _ in front + pts), max(b for _, b in front + pts))
    from oracle.front import normalised_hypervolume
    hv_out = normalised_hypervolume([pts[i] for i in oracle.nondominated(pts)], lo, hi)
    hv_exact = normalised_hypervolume(front, lo, hi)
    assert 0 < hv_out <= hv_exact + 1e-12 <= 1.21 + 1e-12


# --------------------------------------------------------------------------
# hypervolume and the dominance filter
# --------------------------------------------------------------------------

def test_hypervolume_hand_cases():
    assert math.isclose(oracle.hypervolume_2d([(1, 1)], (2.1, 2.1)), 1.21)
    assert math.isclose(oracle.hypervolume_2d([(1, 2), (2, 1)], (2.1, 2.1)), 0.21)
    # a dominated point adds nothing; a point outside the box adds nothing
    assert math.isclose(oracle.hypervolume_2d([(1, 2), (2, 1), (2, 2), (3, 0)], (2.1, 2.1)), 0.21)
    assert oracle.hypervolume_2d([], (2.1, 2.1)) == 0.0


def test_nondominated_filter():
    pts = [(5, 5), (4, 6), (5, 5), (6, 6), (3, 9), (4, 6)]
    keep = oracle.nondominated(pts)
    assert keep == [0, 1, 4]


# --------------------------------------------------------------------------
# selection: "choose one flip at random" among the accepted bits (Alg. 3)
# --------------------------------------------------------------------------

def test_selection_uniform():
    """With delta so large that every bit is accepted at iteration 1, the
    flipped bit is the rank floor(u * m / 2^32) of the tag-1 word u of
    (0, 1, replica, 1) in ascending bit order, and over many replicas every
    bit is chosen equally often (chi-square, m - 1 degrees of freedom)."""
    n, m, R = 4, 16, 4000
    rng = np.random.default_rng(5)
    F = rng.integers(0, 9, (n, n))
    np.fill_diagonal(F, 0)
    D = np.triu(rng.integers(1, 9, (n, n)), 1)
    D = D + D.T
    inst = oracle.Instance(F, F.T.copy(), D)
    seed = 0x1234_5678_9ABC
    out = oracle.run(inst, I_max=1, replicas=R, seed=seed, delta0=1e12, deltaf=1.0,
                     xi=1e-3, trace=True, threads=4)
    flipped = out["trace"][:, 0, 2]
    key = [seed & 0xFFFFFFFF, seed >> 32]
    for r in range(0, R, 97):
        u = int(oracle.philox([0, 1, r, 1], key)[0])
        assert flipped[r] == (u * m) >> 32
    counts = np.bincount(flipped, minlength=m)
    exp = R / m
    chi2 = float(((counts - exp) ** 2 / exp).sum())
    assert chi2 < (m - 1) + 6 * math.sqrt(2 * (m - 1))


# --------------------------------------------------------------------------
# archive snapshots (the per-iteration archive behind Fig. mdasl)
# --------------------------------------------------------------------------

def test_snapshots_are_prefix_archives():
    """Snapshot j of a run is the final archive of the same run stopped after
    (j + 1) K iterations (every iteration depends only on earlier ones)."""
    qi = inputs.uniform_instance(6, index=3, workload="P8")
    inst = oracle.Instance(qi.F1, qi.F2, qi.D)
    kw = dict(replicas=3, seed=4, delta0=2e6, deltaf=3e3, xi=0.02)
    K = 400
    full = oracle.run(inst, I_max=2000, snapshot_every=K, **kw)
    snap = full["snapshots"]
    assert snap["count"].shape == (3, 5)
    for j in (0, 2, 4):
        part = oracle.run(inst, I_max=(j + 1) * K, **kw)
        assert np.array_equal(snap["count"][:, j], part["count"])
        for r in range(3):
            c = int(part["count"][r])
            assert np.array_equal(snap["E"][r, j, :c], part["E"][r, :c])
            assert np.array_equal(snap["bits"][r, j, :c], part["bits"][r, :c])


def test_settled_runs_end_on_the_last_restart_draw():
    """The premise of the kernel's fast-forward, on the oracle alone.
    hi_t = floor(delta_t T_max) never rises (the schedule only cools), so an
    archive member none of whose bits has a strict penalty
    a = max(0, dE_1) + max(0, dE_2) <= hi_t never accepts again.  Every jump
    of Alg. 3 goes to pick(restart draw of t, |A|); once the archive stops
    changing and all its members are so, the run ends on the member that
    iteration I_max's draw picks."""
    FAST = dict(delta0=2e6, deltaf=3e3, xi=0.02)
    I_max, seed, R = 4000, 18, 3
    sched = oracle.schedule(FAST["delta0"], FAST["deltaf"], FAST["xi"], I_max)
    hi = np.floor(sched * oracle.neglog_table()[0])
    assert np.all(np.diff(hi) <= 0)
    inst = inputs.uniform_instance(7, index=7, workload="P8")
    n, m = 7, 49
    oi = oracle.Instance(inst.F1, inst.F2, inst.D)
    out = oracle.run(oi, I_max=I_max, replicas=R, seed=seed, trace=True, **FAST)
    w1, w2 = oi.w
    F1, F2, D = (np.asarray(a, dtype=np.int64) for a in (inst.F1, inst.F2, inst.D))
    Fs1, Fs2 = F1 + F1.T, F2 + F2.T

    def min_penalty(bits):
        X = np.asarray(bits, dtype=np.int64).reshape(n, n)
        r, c, sg = X.sum(1), X.sum(0), 1 - 2 * X
        h = sg * (-1 + (r[:, None] - X) + (c[None, :] - X))
        e1 = np.maximum(sg * (Fs1 @ X @ D) + w1 * h, 0)
        e2 = np.maximum(sg * (Fs2 @ X @ D) + w2 * h, 0)
        return int((e1 + e2).min())

    def restart_pick(t, rep, count):
        u = int(oracle.philox([0, t, rep, 2], [seed, 0])[0])
        return (u * count) >> 32

    settled = 0
    for rep in range(R):
        tr = out["trace"][rep]
        archive = []
        for t in range(1, I_max + 1):
            ev = int(tr[t - 1, 2])
            if ev >= 0:
                archive = oracle.archive_update("explore", m, archive, (int(tr[t - 1, 0]), int(tr[t - 1, 1])))
            elif ev != np.iinfo(np.int64).min:
                assert -1 - ev == restart_pick(t, rep, len(archive)), (rep, t)
        count = int(out["count"][rep])
        assert len(archive) == count
        flips = np.nonzero(tr[:, 2] >= 0)[0]
        t_last = int(flips[-1]) + 1 if len(flips) else 0
        pens = [min_penalty(out["bits"][rep, y]) for y in range(count)]
        none = np.iinfo(np.int64).min
        # iterations whose trial is at a member (the previous one jumped)
        # while every member's smallest penalty exceeds hi_t
        dead_from = [t for t in range(max(t_last, 1) + 1, I_max + 1)
                     if min(pens, default=0) > hi[t - 1] and none != tr[t - 2, 2] < 0]
        if count and dead_from:
            settled += 1
            y = restart_pick(I_max, rep, count)
            assert np.array_equal(out["E_final"][rep], out["E"][rep, y])
            assert np.array_equal(out["x"][rep], out["bits"][rep, y])
    assert settled >= 2
