"""Fast-forward (moda_params.fast_forward).  A trial at an archive member in
which no bit has an acceptance penalty a <= hi_t marks the member; hi_t
never rises (the schedule only cools), so no later trial there accepts.
Once every member is marked and the replica is about to try one of them,
every remaining iteration of Alg. 3 is a jump to a uniformly drawn member,
and the kernel lands directly on the member the last iteration draws.  The
results must be those of the full run: archives, final states and
energies, the four event counters and the (E1, E2, event) trace of every
iteration, bit for bit against the oracle, which runs every iteration --
and the shortcut must actually have been taken (stats[6] > 0)."""
import numpy as np
import pytest

from paper_2205_13399_gb300 import inputs
from parity import compare, gpu_run, oracle_run

pytestmark = pytest.mark.gpu

FAST = dict(delta0=2e6, deltaf=3e3, xi=0.02)


def _same(a, b, traces=None):
    assert np.array_equal(a.count, b.count)
    for r in range(len(a.count)):
        c = int(a.count[r])
        assert np.array_equal(a.E[r, :c], b.E[r, :c]), r
        assert np.array_equal(a.bits[r, :c], b.bits[r, :c]), r
    assert np.array_equal(a.x, b.x)
    assert np.array_equal(a.E_final, b.E_final)
    assert np.array_equal(a.stats[:, :4], b.stats[:, :4])
    if traces is not None:
        assert np.array_equal(traces[0], traces[1])


@pytest.mark.parametrize("cache", ["on", "off"])
@pytest.mark.parametrize("acc,arc", [(a, b) for a in ("strict", "lenient")
                                     for b in ("explore", "exploit")])
def test_traced_small_against_oracle(acc, arc, cache):
    """Ragged sizes and both archive rules: replicas whose archive settles
    stop early, replicas that keep a member able to accept run to the end;
    both give the oracle's full run, trace included."""
    fired = 0
    for n, bt in ((5, 0), (7, 0), (12, 32), (12, 0)):
        inst = inputs.uniform_instance(n, index=n, workload="P8")
        kw = dict(replicas=3, I_max=6000, seed=11 + n, accept=acc, archive=arc, **FAST)
        _, _, res, tr = gpu_run(inst, block_threads=bt, trace=True, field_cache=cache,
                                fast_forward=True, **kw)
        _, orc = oracle_run(inst, trace=True, **kw)
        compare(res, range(3), orc, n * n, gpu_trace=tr)
        assert np.all(res.stats[:, 6] < kw["I_max"])
        assert np.all(res.stats[:, 6] <= res.stats[:, 1])
        fired += int((res.stats[:, 6] > 0).sum())
    assert fired >= 6


@pytest.mark.parametrize("acc", ["strict", "lenient"])
def test_wide_variant_against_oracle(acc):
    """Penalty weights so large that Delta E needs int64 (the wide kernel)."""
    inst = inputs.uniform_instance(7, index=2, workload="P8")
    kw = dict(replicas=4, I_max=5000, seed=5, accept=acc, w=(2 * 10 ** 8, 3 * 10 ** 8), **FAST)
    _, _, res, tr = gpu_run(inst, trace=True, fast_forward=True, **kw)
    _, orc = oracle_run(inst, trace=True, **kw)
    compare(res, range(4), orc, 49, gpu_trace=tr)
    assert int((res.stats[:, 6] > 0).sum()) >= 1


@pytest.mark.parametrize("kw", [dict(prefetch=1), dict(prefetch=2), dict(prefetch=4),
                                dict(field_cache="off"), dict(block_threads=160)])
def test_equals_plain_run_p25_schedule(kw):
    """A 25-facility instance on the paper's schedule (delta0 = 1e9, deltaf =
    1e4, xi = 1e-3) for 3 x 10^4 iterations, in several layouts: the
    fast-forwarded run equals the full run, trace included."""
    inst = inputs.workload_instance("P25")
    run = dict(replicas=16, I_max=30000, seed=4)
    _, _, full, ftr = gpu_run(inst, trace=True, **run, **kw)
    _, _, fast, gtr = gpu_run(inst, trace=True, fast_forward=True, **run, **kw)
    _same(fast, full, (gtr, ftr))
    assert np.array_equal(full.stats[:, 6], np.zeros(16))
    assert np.all(fast.stats[:, 6] > 0)


def test_p25_full_config_sampled_replicas():
    """The n = 25 workload at full size (128 replicas, I_max = 10^5) with
    the shortcut: sampled replicas equal the oracle's full runs, and most
    iterations of every replica are settled without being executed."""
    inst = inputs.workload_instance("P25")
    run = inputs.WORKLOAD_RUN["P25"]
    _, _, res, _ = gpu_run(inst, replicas=run["replicas"], I_max=run["I_max"],
                           seed=run["seed"], fast_forward=True)
    rows = [0, 64, 127]
    _, orc = oracle_run(inst, replicas=rows, I_max=run["I_max"], seed=run["seed"])
    compare(res, rows, orc, 625)
    assert np.all(res.stats[:, :4].sum(1) == run["I_max"])
    assert np.all(res.stats[:, 6] > run["I_max"] // 2)


def test_batch_and_noalloc_paths():
    """The CUDA-graph batch launch and the allocation-free entry point take
    the fast-forward variant too and give the plain call's results."""
    import torch
    from paper_2205_13399_gb300 import moda
    qis = [inputs.uniform_instance(n, index=n, workload="P8") for n in (6, 9, 12)]
    insts = [moda.Instance(q.F1, q.F2, q.D) for q in qis]
    kws = [dict(replicas=3, I_max=4000, seed=k, fast_forward=True, **FAST) for k in range(3)]
    runs = moda.anneal_batch(insts, [moda.make_params(**kw) for kw in kws])
    for inst, kw, r in zip(insts, kws, runs):
        r.wait()
        plain = dict(kw, fast_forward=False)
        _same(r.read(), moda.anneal(inst, **plain).wait().read())
        assert np.array_equal(r.read().stats[:, 6], moda.anneal(inst, **kw).wait().read().stats[:, 6])
    q = qis[2]
    n, R = q.n, 3
    m, W = n * n, (n * n + 31) // 32
    dev = torch.device("cuda", torch.cuda.current_device())
    bufs = {"arch_E": torch.zeros(R * m * 2, dtype=torch.int64, device=dev),
            "arch_bits": torch.zeros(R * m * W + 8, dtype=torch.int32, device=dev),
            "arch_count": torch.zeros(R, dtype=torch.int32, device=dev),
            "x_final": torch.zeros(R * W, dtype=torch.int32, device=dev),
            "E_final": torch.zeros(R * 2, dtype=torch.int64, device=dev),
            "stats": torch.zeros(R * 8, dtype=torch.int64, device=dev),
            "error": torch.full((1,), -1, dtype=torch.int32, device=dev)}
    stream = torch.cuda.current_stream()
    moda.anneal_noalloc(q.F1, q.F2, q.D, bufs, stream=stream, **kws[2])
    stream.synchronize()
    assert int(bufs["error"].item()) == 0
    ref = moda.anneal(insts[2], stream=stream, **kws[2]).wait().read()
    assert np.array_equal(bufs["arch_count"].cpu().numpy(), ref.count)
    assert np.array_equal(bufs["x_final"].cpu().numpy().view(np.uint32).reshape(R, W), ref.x)
    assert np.array_equal(bufs["E_final"].cpu().numpy().reshape(R, 2), ref.E_final)
    st = bufs["stats"].cpu().numpy().reshape(R, 8)
    assert np.array_equal(st[:, :4], ref.stats[:, :4])
    assert np.array_equal(st[:, 6], ref.stats[:, 6])


def test_rejected_combinations():
    from paper_2205_13399_gb300 import moda
    q = inputs.uniform_instance(6, index=1, workload="P8")
    inst = moda.Instance(q.F1, q.F2, q.D)
    for bad in (dict(escape="offset"), dict(normalize=True), dict(snapshot_every=10)):
        with pytest.raises(moda.MODAError, match="MODA_EINVAL"):
            moda.anneal(inst, replicas=1, I_max=100, fast_forward=True, **bad)
    Q = inputs.random_qubo(1, 16)
    with pytest.raises(moda.MODAError, match="MODA_EUNSUPPORTED"):
        moda.Qubo(Q).anneal(replicas=1, I_max=100, fast_forward=True)
