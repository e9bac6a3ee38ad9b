"""Many anneals at once: moda_anneal_batch (one CUDA graph launch) and the
serving queue (moda_server_*).  Each request must give exactly what the
plain moda_anneal call gives on the same instance and params -- archives,
states, energies and counters, bit for bit -- whatever else runs beside it;
one request of each path is also checked against the oracle directly."""
import time

import numpy as np
import pytest

from paper_2205_13399_gb300 import inputs
from parity import compare, oracle_run

pytestmark = pytest.mark.gpu

FAST = dict(delta0=2e6, deltaf=3e3, xi=0.02)


def _requests():
    """Ragged sizes and every mode, small enough for the oracle."""
    from paper_2205_13399_gb300 import moda
    shapes = [(6, "strict", "explore", "archive"), (9, "lenient", "exploit", "archive"),
              (13, "strict", "exploit", "offset"), (20, "lenient", "explore", "offset"),
              (25, "strict", "explore", "archive"), (7, "strict", "explore", "archive")]
    out = []
    for k, (n, acc, arc, esc) in enumerate(shapes):
        qi = inputs.batch_instances(1, n_lo=n, n_hi=n)[0] if k % 2 else \
            inputs.uniform_instance(n, index=40 + k, workload="P8")
        kw = dict(replicas=3 + k % 3, I_max=1200 + 300 * k, seed=500 + k, accept=acc,
                  archive=arc, escape=esc, beta=900, **FAST)
        out.append((qi, moda.Instance(qi.F1, qi.F2, qi.D), kw))
    return out


def _same(a, b):
    """Two finished runs of the same request agree bit for bit."""
    ra, rb = a.read(), b.read()
    assert np.array_equal(ra.count, rb.count)
    for r in range(len(ra.count)):
        c = int(ra.count[r])
        assert np.array_equal(ra.E[r, :c], rb.E[r, :c])
        assert np.array_equal(ra.bits[r, :c], rb.bits[r, :c])
    assert np.array_equal(ra.x, rb.x)
    assert np.array_equal(ra.E_final, rb.E_final)
    assert np.array_equal(ra.stats[:, :4], rb.stats[:, :4])
    assert a.read_archive(-1) == b.read_archive(-1)


def _plain(inst, kw):
    from paper_2205_13399_gb300 import moda
    return moda.anneal(inst, **kw).wait()


def test_batch_equals_plain_runs():
    from paper_2205_13399_gb300 import moda
    reqs = _requests()
    params = [moda.make_params(**kw) for _, _, kw in reqs]
    runs = moda.anneal_batch([inst for _, inst, _ in reqs], params)
    for (qi, inst, kw), run in zip(reqs, runs):
        run.wait()
        _same(run, _plain(inst, kw))
    qi, inst, kw = reqs[1]
    _, orc = oracle_run(qi, **kw)
    compare(runs[1].read(), range(kw["replicas"]), orc, qi.n * qi.n)


def test_batch_many_instances_of_uneven_size():
    """A larger graph: 40 instances, n from 10 to 40, on a torch stream."""
    import torch
    from paper_2205_13399_gb300 import moda
    qis = inputs.batch_instances(40, n_lo=10, n_hi=40)
    insts = [moda.Instance(q.F1, q.F2, q.D) for q in qis]
    kws = [dict(replicas=4, I_max=2000, seed=k, **FAST) for k in range(len(qis))]
    stream = torch.cuda.Stream()
    runs = moda.anneal_batch(insts, [moda.make_params(**kw) for kw in kws], stream=stream)
    stream.synchronize()
    for k in (0, 7, 19, 33, 39):
        _same(runs[k].wait(), _plain(insts[k], kws[k]))


def test_batch_rejects_a_bad_request_without_enqueueing():
    from paper_2205_13399_gb300 import moda
    reqs = _requests()[:3]
    params = [moda.make_params(**kw) for _, _, kw in reqs]
    params[2].replicas = 0
    with pytest.raises(moda.MODAError, match="request 2"):
        moda.anneal_batch([inst for _, inst, _ in reqs], params)


def _drain(srv, tickets, timeout_s=120.0, watch=None, on_done=None):
    """Poll until every ticket finished; ``on_done(ticket, run)`` sees each
    finished run at once (it may close it, returning its memory)."""
    done = {}
    t0 = time.time()
    while len(done) < len(tickets):
        for t in tickets:
            if t not in done:
                r = srv.poll(t)
                if r is not None:
                    done[t] = r
                    if on_done is not None:
                        on_done(t, r)
        if watch is not None:
            watch(srv.info())
        assert time.time() - t0 < timeout_s, "server did not finish"
        time.sleep(0.002)
    return done


def test_server_results_equal_plain_runs():
    from paper_2205_13399_gb300 import moda
    reqs = _requests()
    srv = moda.Server()
    tickets = [srv.submit(inst, **kw) for _, inst, kw in reqs]
    done = _drain(srv, tickets)
    for t, (qi, inst, kw) in zip(tickets, reqs):
        _same(done[t], _plain(inst, kw))
    qi, inst, kw = reqs[4]
    _, orc = oracle_run(qi, **kw)
    compare(done[tickets[4]].read(), range(kw["replicas"]), orc, qi.n * qi.n)
    srv.close()


def test_server_admits_within_the_budget():
    """A budget that holds about one request at a time: requests queue,
    at most one runs, and all finish with the plain results."""
    from paper_2205_13399_gb300 import moda
    qi = inputs.uniform_instance(25, index=3, workload="P8")
    inst = moda.Instance(qi.F1, qi.F2, qi.D)
    kws = [dict(replicas=8, I_max=3000, seed=k, **FAST) for k in range(4)]
    # 2 MiB: one run's buffers without the field cache (about 0.5 MB) fit,
    # with it (about 25 MB) they do not, so each request runs alone
    srv = moda.Server(hbm_budget=1 << 21)
    seen = []
    tickets = [srv.submit(inst, **kw) for kw in kws]
    kw_of = dict(zip(tickets, kws))

    def check(t, run):  # compare, then free: the budget counts a run until then
        _same(run, _plain(inst, kw_of[t]))
        run.close()

    _drain(srv, tickets, watch=lambda i: seen.append(i["running"]), on_done=check)
    assert max(seen) <= 1
    assert srv.info()["bytes_in_use"] == 0
    srv.close()


def test_server_rejects_a_request_larger_than_the_budget():
    from paper_2205_13399_gb300 import moda
    qi = inputs.uniform_instance(8, index=1, workload="P8")
    inst = moda.Instance(qi.F1, qi.F2, qi.D)
    srv = moda.Server(hbm_budget=1)
    # field cache off everywhere, so even the leanest run needs > 1 byte
    t = srv.submit(inst, replicas=2, I_max=100, escape="offset", **FAST)
    with pytest.raises(moda.MODAError, match="MODA_ENOMEM"):
        for _ in range(2000):
            if srv.poll(t) is not None:
                break
            time.sleep(0.005)
    srv.close()


def test_server_overlaps_staggered_arrivals():
    """Continuous batching: requests submitted one by one while earlier ones
    are on the GPU are admitted at once and run beside them (the server
    reports two or more running at some moment), and every result equals
    the request's plain run, bit for bit."""
    from paper_2205_13399_gb300 import moda
    qis = [inputs.uniform_instance(n, index=500 + n, workload="P8") for n in (20, 26, 14, 31, 9, 23)]
    insts = [moda.Instance(q.F1, q.F2, q.D) for q in qis]
    kws = [dict(replicas=16 + 4 * k, I_max=60000, seed=70 + k, accept=("strict", "lenient")[k % 2],
                archive=("explore", "exploit")[k // 3], **FAST) for k in range(len(qis))]
    srv = moda.Server()
    seen = []
    tickets = []
    for k, (inst, kw) in enumerate(zip(insts, kws)):
        tickets.append(srv.submit(inst, **kw))
        # the next request arrives while this one (and its predecessors) run
        t0 = time.time()
        while time.time() - t0 < 0.01:
            seen.append(srv.info()["running"])
            time.sleep(0.001)
    done = _drain(srv, tickets, watch=lambda i: seen.append(i["running"]))
    assert max(seen) >= 2, seen
    for t, inst, kw in zip(tickets, insts, kws):
        _same(done[t], _plain(inst, kw))
    srv.close()
