"""Helpers shared by the GPU parity tests: run the CUDA path through the C ABI
and the CPU oracle on the same seeded instance and compare them element by
element.  The comparison is bit-exact: every quantity on the path is an
integer or an IEEE double decided identically on both sides."""
from __future__ import annotations

import numpy as np

import oracle


def gpu_run(inst_np, *, replicas, I_max, seed=0, accept="strict", archive="explore",
            escape="archive", delta0=1e9, deltaf=1e4, xi=1e-3, beta=None, archive_size=0,
            replica_base=0, block_threads=0, trace=False, w=None, stream=None,
            field_cache="auto", prefetch=0, normalize=False, fast_forward=False,
            engine="auto"):
    from paper_2205_13399_gb300 import moda
    inst = moda.Instance(inst_np.F1, inst_np.F2, inst_np.D, w=w)
    run = moda.anneal(inst, replicas=replicas, I_max=I_max, seed=seed, accept=accept,
                      archive=archive, escape=escape, delta0=delta0, deltaf=deltaf, xi=xi,
                      beta=beta, archive_size=archive_size, replica_base=replica_base,
                      block_threads=block_threads, trace=trace, stream=stream,
                      field_cache=field_cache, prefetch=prefetch, normalize=normalize,
                      fast_forward=fast_forward, engine=engine)
    run.wait()
    res = run.read()
    traces = None
    if trace:
        traces = np.stack([run.read_trace(r) for r in range(replicas)])
    return inst, run, res, traces


def oracle_run(inst_np, *, replicas, I_max, seed=0, accept="strict", archive="explore",
               escape="archive", delta0=1e9, deltaf=1e4, xi=1e-3, beta=None, archive_size=0,
               trace=False, w=None, threads=None, normalize=False, snapshot_every=0):
    oi = oracle.Instance(inst_np.F1, inst_np.F2, inst_np.D, w=w)
    out = oracle.run(oi, I_max=I_max, replicas=replicas, seed=seed, accept=accept,
                     archive=archive, escape=escape, delta0=delta0, deltaf=deltaf, xi=xi,
                     beta=beta, archive_size=archive_size, trace=trace, threads=threads,
                     normalize=normalize, snapshot_every=snapshot_every)
    return oi, out


def compare(gpu_res, gpu_rows, orc, m, gpu_trace=None):
    """Assert that replicas ``gpu_rows`` of the GPU result equal the oracle's
    replicas (same order), bit for bit."""
    from paper_2205_13399_gb300.moda import unpack_bits
    for k, g in enumerate(gpu_rows):
        if gpu_trace is not None:
            assert "trace" in orc
            ot = orc["trace"][k]
            gt = gpu_trace[g]
            if not np.array_equal(gt, ot):
                bad = int(np.argmax(np.any(gt != ot, axis=1)))
                lo = max(0, bad - 3)
                raise AssertionError(
                    f"row {g}: trace differs first at iteration {bad + 1}:\n"
                    f"gpu    {gt[lo:bad + 2].tolist()}\noracle {ot[lo:bad + 2].tolist()}")
        cnt = int(gpu_res.count[g])
        assert cnt == int(orc["count"][k]), f"archive size, replica row {g}"
        assert np.array_equal(gpu_res.E[g, :cnt], orc["E"][k, :cnt]), f"archive energies, row {g}"
        gb = unpack_bits(gpu_res.bits[g, :cnt], m)
        assert np.array_equal(gb, orc["bits"][k, :cnt]), f"archive states, row {g}"
        assert np.array_equal(unpack_bits(gpu_res.x[g], m), orc["x"][k]), f"final state, row {g}"
        assert np.array_equal(gpu_res.E_final[g], orc["E_final"][k]), f"final energies, row {g}"
        assert np.array_equal(gpu_res.stats[g, :4], orc["stats"][k]), f"counters, row {g}"


def oracle_merged_front(oi, orc):
    """The result of Alg. 3 over all replicas (its last line, and Sec. 4.2's
    merge of runs): the non-dominated members of the union of the oracle's
    replica archives, taken in (replica, slot) order so that among equal
    energy vectors the lowest (replica, slot) is kept (reading R16).  Each
    point carries its penalised energies, QAP costs, constraint value,
    feasibility, origin and decoded permutation, sorted by (E1, E2) as
    moda_read_archive returns them."""
    pts, where = [], []
    for k in range(len(orc["count"])):
        for slot in range(int(orc["count"][k])):
            pts.append((int(orc["E"][k, slot, 0]), int(orc["E"][k, slot, 1])))
            where.append((k, slot))
    out = []
    for i in oracle.nondominated(pts):
        k, slot = where[i]
        x = orc["bits"][k, slot]
        g = oi.constraint(x)
        out.append(dict(E1=pts[i][0], E2=pts[i][1], c1=oi.cost(0, x), c2=oi.cost(1, x), g=g,
                        feasible=g == 0, replica=k, slot=slot,
                        perm=oracle.decode_permutation(x) if g == 0 else None))
    return sorted(out, key=lambda d: (d["E1"], d["E2"]))
