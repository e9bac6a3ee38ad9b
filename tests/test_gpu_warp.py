"""GPU parity of the warp engine (one warp per replica, work list of
(run, replica) items): every acceptance rule and archive update, ragged
sizes, the int32 and int64 Delta E variants, field-cache records on and off
(jumps then rebuild the fields), every prefetch distance, and the full-size
workloads -- against the CPU oracle bit for bit, per iteration where traced,
and against the block engine on the same runs."""
import numpy as np
import pytest

from paper_2205_13399_gb300 import inputs
from parity import compare, gpu_run, oracle_merged_front, oracle_run

pytestmark = pytest.mark.gpu

FAST = dict(delta0=2e6, deltaf=3e3, xi=0.02)
MODES = [(acc, arc) for acc in ("strict", "lenient") for arc in ("explore", "exploit")]


@pytest.mark.parametrize("team", [0, 1, 3, 8])
@pytest.mark.parametrize("cache", ["auto", "off"])
@pytest.mark.parametrize("acc,arc", MODES)
def test_warp_traced_small(acc, arc, cache, team):
    """Per-iteration traces equal the oracle's on ragged sizes: one chunk of
    128 bits and a ragged last chunk, several chunks, hot, cooling and
    frozen phases, restarts and undecided acceptance tests; teams of 1, 3
    and 8 warps per replica (more warps than chunks included) and the
    automatic team size."""
    for n in (5, 7, 12, 17, 25):
        inst = inputs.uniform_instance(n, index=300 + n, workload="P8")
        kw = dict(replicas=3, I_max=1500, seed=40 + n, accept=acc, archive=arc, **FAST)
        _, _, res, tr = gpu_run(inst, trace=True, field_cache=cache, engine="warp",
                                block_threads=32 * team, **kw)
        _, orc = oracle_run(inst, trace=True, **kw)
        compare(res, range(3), orc, n * n, gpu_trace=tr)


@pytest.mark.parametrize("team", [1, 4])
@pytest.mark.parametrize("prefetch", [1, 2, 3, 7, 15])
def test_warp_prefetch_distances(prefetch, team):
    """Jump records copied 0, 1, 2, 6 or 14 iterations ahead (windows of up
    to 15 iterations) give the oracle's run."""
    inst = inputs.euclid_instance(23, 0.5, False, index=3, workload="P25")
    kw = dict(replicas=5, I_max=4000, seed=8, **FAST)
    _, _, res, tr = gpu_run(inst, trace=True, prefetch=prefetch, engine="warp",
                            block_threads=32 * team, **kw)
    _, orc = oracle_run(inst, trace=True, **kw)
    compare(res, range(5), orc, 23 * 23, gpu_trace=tr)
    if prefetch > 1:  # copies started ahead: some jumps took a prefetched record
        assert res.stats[:, 4].sum() > 0
    else:
        assert res.stats[:, 4].sum() == 0


def test_warp_small_archive_and_replica_base():
    """Archive capacity below m (the full-archive branches) and a replica
    offset: rows of a shifted launch equal the oracle's replicas 5..7."""
    inst = inputs.euclid_instance(10, -0.7, False, index=3, workload="BATCH")
    kw = dict(I_max=4000, seed=99, archive_size=7, **FAST)
    for arc in ("explore", "exploit"):
        _, _, res, _ = gpu_run(inst, replicas=3, replica_base=5, archive=arc, engine="warp",
                               **kw)
        _, orc = oracle_run(inst, replicas=[5, 6, 7], archive=arc, **kw)
        compare(res, range(3), orc, 100)


@pytest.mark.parametrize("n", [33, 41])
def test_warp_wide_variant(n):
    """Dense flows whose |Delta E| bound passes 2^31: the int64 variant,
    with saturated penalties in the hot phase (delta T_max above 2^32)."""
    from paper_2205_13399_gb300 import moda
    rng = np.random.default_rng(n)
    F1 = rng.integers(800, 1600, (n, n))
    F2 = rng.integers(800, 1600, (n, n))
    for F in (F1, F2):
        np.fill_diagonal(F, 0)
    D = np.triu(rng.integers(50, 120, (n, n)), 1)
    D = D + D.T

    class Inst:
        pass
    inst = Inst()
    inst.F1, inst.F2, inst.D, inst.n = F1.astype(np.int16), F2.astype(np.int16), \
        D.astype(np.int16), n
    g = moda.Instance(inst.F1, inst.F2, inst.D)
    bound = [int((F + F.T).sum(1).max()) * int(D.sum(1).max()) for F in (F1, F2)]
    assert max(b + w * (2 * n + 1) for b, w in zip(bound, g.w)) >= 2 ** 31
    kw = dict(replicas=4, I_max=2500, seed=17)
    _, orc = oracle_run(inst, trace=True, **kw)
    for team in (1, 5):
        _, _, res, tr = gpu_run(inst, trace=True, engine="warp", block_threads=32 * team, **kw)
        compare(res, range(4), orc, n * n, gpu_trace=tr)


@pytest.mark.parametrize("acc", ["strict", "lenient"])
def test_warp_narrow_penalty_sum_above_2_31(acc):
    """Each |Delta E_k| bound is below 2^31, their sum is not: penalties
    near 2^32 in uint32 against the draw."""
    n, fv, dv = 4, 2500, 4500
    rng = np.random.default_rng(n)
    F1 = rng.integers(fv // 2, fv, (n, n))
    F2 = rng.integers(fv // 2, fv, (n, n))
    for F in (F1, F2):
        np.fill_diagonal(F, 0)
    D = np.triu(rng.integers(dv // 2, dv, (n, n)), 1)
    D = D + D.T

    class Inst:
        pass
    inst = Inst()
    inst.F1, inst.F2, inst.D, inst.n = F1.astype(np.int16), F2.astype(np.int16), \
        D.astype(np.int16), n
    kw = dict(replicas=16, I_max=3000, seed=13, accept=acc)
    _, _, res, tr = gpu_run(inst, trace=True, engine="warp", **kw)
    _, orc = oracle_run(inst, trace=True, **kw)
    compare(res, range(16), orc, n * n, gpu_trace=tr)


def test_warp_p8_full_config_and_front():
    """n = 8 workload at full size; the merged front equals the oracle's."""
    inst = inputs.workload_instance("P8")
    run = inputs.WORKLOAD_RUN["P8"]
    _, grun, res, _ = gpu_run(inst, replicas=run["replicas"], I_max=run["I_max"],
                              seed=run["seed"], engine="warp")
    oi, orc = oracle_run(inst, replicas=range(run["replicas"]), I_max=run["I_max"],
                         seed=run["seed"])
    compare(res, range(run["replicas"]), orc, 64)
    assert grun.read_archive(-1) == oracle_merged_front(oi, orc)


def test_warp_p25_full_config_sampled_replicas():
    """n = 25 workload at full size (128 replicas, I_max = 10^5) in the
    launch the benchmark times; the oracle recomputes sampled replicas and
    the merged front of those replicas' archives."""
    inst = inputs.workload_instance("P25")
    run = inputs.WORKLOAD_RUN["P25"]
    _, grun, res, _ = gpu_run(inst, replicas=run["replicas"], I_max=run["I_max"],
                              seed=run["seed"], engine="warp")
    rows = [0, 64, 127]
    _, orc = oracle_run(inst, replicas=rows, I_max=run["I_max"], seed=run["seed"])
    compare(res, rows, orc, 625)
    assert (res.stats[:, :4].sum(1) == run["I_max"]).all()


@pytest.mark.parametrize("name", ["P50", "P75"])
def test_warp_large_configs_prefix(name):
    """n = 50 / 75 workloads in their full launch shape (256 replicas) for a
    prefix of the schedule: sampled replicas against the oracle, and every
    replica against the block engine."""
    inst = inputs.workload_instance(name)
    run = inputs.WORKLOAD_RUN[name]
    I_max = 12000
    _, _, res, _ = gpu_run(inst, replicas=run["replicas"], I_max=I_max, seed=run["seed"],
                           engine="warp")
    _, _, one, _ = gpu_run(inst, replicas=run["replicas"], I_max=I_max, seed=run["seed"],
                           engine="warp", block_threads=32)
    assert np.array_equal(res.x, one.x) and np.array_equal(res.E_final, one.E_final)
    assert np.array_equal(res.stats[:, :4], one.stats[:, :4])
    rows = [2, run["replicas"] - 3]
    _, orc = oracle_run(inst, replicas=rows, I_max=I_max, seed=run["seed"])
    compare(res, rows, orc, inst.n * inst.n)
    _, _, blk, _ = gpu_run(inst, replicas=run["replicas"], I_max=I_max, seed=run["seed"],
                           engine="block")
    assert np.array_equal(res.count, blk.count)
    assert np.array_equal(res.x, blk.x)
    assert np.array_equal(res.E_final, blk.E_final)
    assert np.array_equal(res.stats[:, :4], blk.stats[:, :4])
    for r in range(run["replicas"]):
        c = int(blk.count[r])
        assert np.array_equal(res.E[r, :c], blk.E[r, :c]), r
        assert np.array_equal(res.bits[r, :c], blk.bits[r, :c]), r


def test_warp_engine_rejects_unsupported_options():
    from paper_2205_13399_gb300 import moda
    inst = inputs.uniform_instance(6, index=1, workload="P8")
    g = moda.Instance(inst.F1, inst.F2, inst.D)
    for kw in (dict(escape="offset"), dict(normalize=True), dict(fast_forward=True),
               dict(snapshot_every=10)):
        with pytest.raises(moda.MODAError) as ei:
            moda.anneal(g, replicas=2, I_max=100, engine="warp", **kw)
        assert ei.value.status == moda.EUNSUPPORTED


@pytest.mark.parametrize("case", range(24))
def test_warp_frozen_layout_random_shapes(case):
    """Seeded random shapes through the frozen-schedule layout (the FAST
    schedule freezes after about 320 of the 1,500 iterations): instance
    size, team size, prefetch distance, acceptance and archive rule and the
    field cache drawn per case; per-iteration traces against the oracle."""
    rng = np.random.default_rng(1000 + case)
    n = int(rng.integers(5, 31))
    team = int(rng.choice([0, 1, 2, 3, 4, 5, 8]))
    prefetch = int(rng.choice([0, 2, 5, 11, 15]))
    acc = str(rng.choice(["strict", "lenient"]))
    arc = str(rng.choice(["explore", "exploit"]))
    cache = str(rng.choice(["auto", "auto", "off"]))
    inst = inputs.uniform_instance(n, index=500 + case, workload="P8")
    kw = dict(replicas=3, I_max=1500, seed=700 + case, accept=acc, archive=arc, **FAST)
    _, _, res, tr = gpu_run(inst, trace=True, field_cache=cache, engine="warp",
                            block_threads=32 * team, prefetch=prefetch, **kw)
    _, orc = oracle_run(inst, trace=True, **kw)
    compare(res, range(3), orc, n * n, gpu_trace=tr)
