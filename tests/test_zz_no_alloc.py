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
    """Runs whose field cache would not fit the 64 MiB scratch array are
    refused; the same run with the offset escape, which uses no scratch,
    is not.  Real output buffers are passed, so nothing could be written
    out of bounds even if a check were missing."""
    torch = pytest.importorskip("torch")
    from paper_2205_13399_gb300 import moda
    inst = inputs.workload_instance("P25")
    m, W, R = 625, 20, 128
    bufs = _buffers(torch, R, m, W)
    with pytest.raises(moda.MODAError) as ei:
        # 128 replicas x 625 slots x 8 bytes x 632 bits (about 5 KB per
        # record, the int32 Delta E variant) = 405 MB > 64 MiB
        moda.anneal_noalloc(inst.F1, inst.F2, inst.D, bufs, replicas=R, I_max=10)
    assert ei.value.status == moda.EUNSUPPORTED
    assert "64 MiB" in str(ei.value)
    stream = torch.cuda.current_stream()
    moda.anneal_noalloc(inst.F1, inst.F2, inst.D, bufs, stream=stream, replicas=R, I_max=10,
                        escape="offset")
    stream.synchronize()
    assert int(bufs["error"].item()) == 0
    assert int(bufs["stats"].view(R, 8)[:, :4].sum().item()) == R * 10


def test_noalloc_refuses_stream_capture():
    """A call made while its stream is captured into a CUDA graph is
    refused: the call stages its instance in host arrays that the next call
    overwrites, so a replayed graph would anneal another call's instance."""
    torch = pytest.importorskip("torch")
    from paper_2205_13399_gb300 import moda
    inst = inputs.uniform_instance(6, index=6, workload="P8")
    bufs = _buffers(torch, 2, 36, 2)
    side = torch.cuda.Stream()
    x = torch.zeros(1, device=bufs["error"].device)
    g = torch.cuda.CUDAGraph()
    err = None
    with torch.cuda.graph(g, stream=side):
        x.add_(1)
        try:
            moda.anneal_noalloc(inst.F1, inst.F2, inst.D, bufs, stream=side, replicas=2,
                                I_max=100, **FAST)
        except moda.MODAError as e:
            err = e
    assert err is not None and err.status == moda.EUNSUPPORTED
    assert "captured" in str(err)
