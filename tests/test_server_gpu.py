"""Served graph building (continuous batching): every event's rows are the
same when it is built alone and when it is built in a mix with others, and
the trace replay reports a latency for every request."""
import threading
import time

import numpy as np
import pytest

from paper_2202_06929_b300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2202_06929_b300 as frnn  # noqa: E402

R, K, D = 0.1, 32, 8


def _events(sizes, seed):
    return [synth.clustered_grid(n, D, seed + i, max(n // 12, 1), 0.03, 0.15) for i, n in enumerate(sizes)]


def _alone(x):
    n = x.shape[0]
    with frnn.Plan(n_max=max(n, 1), d_max=D, k_max_cap=K) as plan:
        host = plan.build(torch.from_numpy(x).cuda(), R, K).to_host()
        assert plan.last_status() == 0
    return host


def test_served_rows_equal_rows_built_alone():
    rng = np.random.default_rng(11)
    sizes = [int(v) for v in rng.integers(0, 20000, size=22)] + [0, 1, 2, 19999]
    evs = _events(sizes, 500)
    with frnn.Server(d=D, r=R, k=K, batch_points=50000, batch_events=6, slots=3) as srv:
        # all at once: they are packed into batches that run on three streams
        outs = [srv.wait(t) for t in [srv.submit(x) for x in evs]]
        # staggered from another thread while this one waits
        tickets = []

        def feeder():
            for x in evs[::-1]:
                tickets.append(srv.submit(x))
                time.sleep(0.0005)

        th = threading.Thread(target=feeder)
        th.start()
        th.join()
        outs2 = [srv.wait(t) for t in tickets][::-1]
    for x, o, o2 in zip(evs, outs, outs2):
        ref = _alone(x)
        for got in (o, o2):
            np.testing.assert_array_equal(got["row_ptr"], ref["row_ptr"])
            np.testing.assert_array_equal(got["col"], ref["col"])
            assert got["latency_s"] > 0


def test_run_trace_poisson_arrivals():
    rng = np.random.default_rng(3)
    sizes = [int(v) for v in rng.integers(1000, 30000, size=12)]
    evs = _events(sizes, 900)
    x_all = np.concatenate(evs)
    start = np.concatenate([[0], np.cumsum(sizes)[:-1]]).astype(np.int64)
    req = rng.integers(0, len(evs), size=60)           # requests reuse the events
    arrivals = np.cumsum(rng.exponential(1 / 2000.0, size=req.size))
    with frnn.Server(d=D, r=R, k=K, batch_points=80000, batch_events=16, slots=2) as srv:
        res = srv.run_trace(x_all, start[req], np.array(sizes)[req], arrivals)
    assert np.all(res["latency_s"] > 0) and res["wall_s"] >= arrivals[-1]
    edges = [int(_alone(x)["row_ptr"][-1]) for x in evs]
    np.testing.assert_array_equal(res["n_edges"], np.array(edges)[req])


def test_server_memory_budget_and_capacity():
    with pytest.raises(frnn.FrnnError) as ei:
        frnn.Server(d=D, r=R, k=K, batch_points=100000, slots=2, mem_budget_bytes=1 << 20)
    assert ei.value.status == frnn.FRNN_ERR_OOM
    with frnn.Server(d=D, r=R, k=K, batch_points=1000, slots=1) as srv:
        assert 0 < srv.reserved_bytes() < 64 << 20
        with pytest.raises(frnn.FrnnError) as ei:
            srv.submit(np.zeros((1001, D), np.float32))
        assert ei.value.status == frnn.FRNN_ERR_CAPACITY
