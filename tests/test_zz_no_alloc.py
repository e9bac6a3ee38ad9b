"""moda_anneal_noalloc: the entry point for callers that must not allocate
device memory (their device memory belongs to their own pool or to a host
framework's allocator).  Its scratch and tables live in the library's
fixed-size device arrays; the test owns the output buffers (allocated here
with torch, outside the entry point) and checks, on two calls in a row with
different instances, that the results equal those of moda_anneal bit for
bit.  This file is collected last so that a run stopping at the first
failure has already run every other test."""
import numpy as np
import pytest

from paper_2205_13399_gb300 import inputs

pytestmark = pytest.mark.gpu

FAST = dict(delta0=2e6, deltaf=3e3, xi=0.02)


def _buffers(torch, R, s, W):
    dev = torch.device("cuda", torch.cuda.current_device())
    return {
        "arch_E": torch.zeros(R * s * 2, dtype=torch.int64, device=dev),
        "arch_bits": torch.zeros(R * s * W + 8, dtype=torch.int32, device=dev),  # + 32 bytes
        "arch_count": torch.zeros(R, dtype=torch.int32, device=dev),
        "x_final": torch.zeros(R * W, dtype=torch.int32, device=dev),
        "E_final": torch.zeros(R * 2, dtype=torch.int64, device=dev),
        "stats": torch.zeros(R * 8, dtype=torch.int64, device=dev),
        "error": torch.full((1,), -1, dtype=torch.int32, device=dev),
    }


def _run_both(torch, moda, inst, kw):
    n = inst.n
    m, W = n * n, (n * n + 31) // 32
    R = kw["replicas"]
    s = m
    bufs = _buffers(torch, R, s, W)
    stream = torch.cuda.current_stream()
    moda.anneal_noalloc(inst.F1, inst.F2, inst.D, bufs, stream=stream, **kw)
    stream.synchronize()
    assert int(bufs["error"].item()) == 0
    ref = moda.anneal(moda.Instance(inst.F1, inst.F2, inst.D), stream=stream, **kw).wait().read()
    count = bufs["arch_count"].cpu().numpy()
    E = bufs["arch_E"].cpu().numpy().reshape(R, s, 2)
    bits = bufs["arch_bits"].cpu().numpy()[:R * s * W].view(np.uint32).reshape(R, s, W)
    x = bufs["x_final"].cpu().numpy().view(np.uint32).reshape(R, W)
    E_final = bufs["E_final"].cpu().numpy().reshape(R, 2)
    stats = bufs["stats"].cpu().numpy().reshape(R, 8)
    assert np.array_equal(count, ref.count)
    assert np.array_equal(x, ref.x)
    assert np.array_equal(E_final, ref.E_final)
    assert np.array_equal(stats[:, :4], ref.stats[:, :4])
    for r in range(R):
        c = int(count[r])
        assert np.array_equal(E[r, :c], ref.E[r, :c])
        assert np.array_equal(bits[r, :c], ref.bits[r, :c])
    return stats


def test_noalloc_matches_anneal_twice():
    torch = pytest.importorskip("torch")
    from paper_2205_13399_gb300 import moda
    # first call: n = 12, a schedule that freezes quickly (many jumps)
    a = inputs.uniform_instance(12, index=12, workload="P8")
    st = _run_both(torch, moda, a, dict(replicas=6, I_max=3000, seed=21, **FAST))
    assert st[:, 1].sum() > 0  # jumps to the archive happened (the scratch was used)
    # second call, same arrays: the n = 8 workload at full size
    b = inputs.workload_instance("P8")
    run = inputs.WORKLOAD_RUN["P8"]
    _run_both(torch, moda, b, dict(replicas=run["replicas"], I_max=run["I_max"],
                                   seed=run["seed"]))


def test_noalloc_rejects_oversized_scratch():
    from paper_2205_13399_gb300 import moda
    inst = inputs.workload_instance("P25")
    fake = {k: 16 for k in ("arch_E", "arch_bits", "arch_count", "x_final", "E_final",
                            "stats", "error")}
    with pytest.raises(moda.MODAError) as ei:
        # 128 replicas x 625 slots x 7.5 KB records > 64 MiB
        moda.anneal_noalloc(inst.F1, inst.F2, inst.D, fake, replicas=128, I_max=10)
    assert ei.value.status == moda.EUNSUPPORTED
    assert "64 MiB" in str(ei.value)
