"""Served graph building (continuous batching): every served event's rows
equal the CPU oracle's rows of that event alone, whatever mix of other events
it was batched and overlapped with, and the trace replay reports a latency
for every request."""
import threading
import time

import numpy as np
import pytest

import oracle
from paper_2202_06929_b300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2202_06929_b300 as frnn  # noqa: E402

R, K, D = 0.1, 32, 8


def _events(sizes, seed):
    return [synth.clustered_grid(n, D, seed + i, max(n // 12, 1), 0.03, 0.15) for i, n in enumerate(sizes)]


def _oracle_rows(x, r=R, k=K):
    """The oracle's graph of the event alone."""
    rp, col = oracle.radius_graph(x, r, k)
    return {"row_ptr": rp, "col": col}


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
        ref = _oracle_rows(x)
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
    edges = [int(_oracle_rows(x)["row_ptr"][-1]) for x in evs]
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


def _dense_event(n, seed):
    """A cap-binding event: dims 0-3 uniform in [-0.3, 0.3], the others within
    0.02 of 0, on the 1/256 grid (about 190 points within r = 0.1 of each)."""
    rng = np.random.default_rng(seed)
    x = np.empty((n, D))
    x[:, :4] = rng.uniform(-0.3, 0.3, size=(n, 4))
    x[:, 4:] = rng.uniform(-0.02, 0.02, size=(n, D - 4))
    return synth.quantise(x)


def test_dense_event_in_a_stream_is_readmitted_and_exact():
    """C2-like events mixed with a cap-binding one whose edges exceed a regular
    slot (4 edges per point here): the batch completes the requests that fit,
    re-queues the rest with their exact edge counts, and the dense event runs
    on the spill slot.  Every request returns OK and equals the oracle."""
    normal = [synth.make_event("c2", e, n=20_000) for e in range(6)]
    dense = _dense_event(30_000, 5)
    evs = normal[:3] + [dense] + normal[3:]
    with frnn.Server(d=D, r=R, k=K, batch_points=60_000, batch_events=8, slots=2, edges_per_point=4) as srv:
        tickets = [srv.submit(x) for x in evs]
        outs = [srv.wait(t) for t in tickets]
        st = srv.stats()
    assert st["spill_batches"] >= 1 and st["readmitted"] >= 1, st
    assert st["spill_edge_capacity"] >= 30_000 * K
    for x, o in zip(evs, outs):
        ref = _oracle_rows(x)
        np.testing.assert_array_equal(o["row_ptr"], ref["row_ptr"])
        np.testing.assert_array_equal(o["col"], ref["col"])
    assert int(outs[3]["row_ptr"][-1]) > 4 * 60_000  # more than a regular slot holds


def test_budget_limits_the_spill_slot():
    """A budget that leaves the spill slot fewer edges than the dense event
    needs: that request alone fails with OVERFLOW, the others are exact."""
    normal = [synth.make_event("c2", e, n=20_000) for e in range(3)]
    dense = _dense_event(30_000, 6)
    probe = frnn.Server(d=D, r=R, k=K, batch_points=60_000, batch_events=8, slots=1, edges_per_point=4,
                        mem_budget_bytes=0)
    try:
        full = probe.reserved_bytes()
        spill_full = probe.stats()["spill_edge_capacity"]
    finally:
        probe.close()
    # room for the spill slot's edges cut to a third
    budget = full - (2 * spill_full // 3) * 8
    with frnn.Server(d=D, r=R, k=K, batch_points=60_000, batch_events=8, slots=1, edges_per_point=4,
                     mem_budget_bytes=budget) as srv:
        assert srv.reserved_bytes() <= budget
        st = srv.stats()
        assert st["spill_edge_capacity"] < spill_full
        tickets = [srv.submit(x) for x in normal[:2] + [dense] + normal[2:]]
        results = []
        for t in tickets:
            try:
                results.append(srv.wait(t))
            except frnn.FrnnError as e:
                results.append(e.status)
    ref_dense = _oracle_rows(dense)
    assert int(ref_dense["row_ptr"][-1]) > st["spill_edge_capacity"]
    assert results[2] == frnn.FRNN_ERR_OVERFLOW
    for x, o in zip(normal, results[:2] + results[3:]):
        ref = _oracle_rows(x)
        np.testing.assert_array_equal(o["col"], ref["col"])


def test_nonfinite_event_fails_alone():
    """One event holding NaN in a batch: it alone reports NONFINITE_INPUT; the
    others of its batch are rerun one by one and equal the oracle."""
    evs = [synth.make_event("c2", e, n=15_000) for e in range(5)]
    bad = evs[2].copy()
    bad[100, 3] = np.nan
    evs[2] = bad
    with frnn.Server(d=D, r=R, k=K, batch_points=100_000, batch_events=8, slots=1) as srv:
        tickets = [srv.submit(x) for x in evs]
        res = []
        for t in tickets:
            try:
                res.append(srv.wait(t))
            except frnn.FrnnError as e:
                res.append(e.status)
    assert res[2] == frnn.FRNN_ERR_NONFINITE_INPUT
    for i in (0, 1, 3, 4):
        np.testing.assert_array_equal(res[i]["col"], _oracle_rows(evs[i])["col"])


def test_poll_is_non_blocking():
    x = synth.make_event("c2", 0, n=50_000)
    with frnn.Server(d=D, r=R, k=K, batch_points=60_000, batch_events=2, slots=1) as srv:
        t = srv.submit(x)
        seen_pending = not srv.poll(t)  # usually still running; never blocks
        deadline = time.time() + 30
        while not srv.poll(t):
            assert time.time() < deadline
            time.sleep(0.0002)
        assert srv.poll(t)
        o = srv.wait(t)
        with pytest.raises(frnn.FrnnError):
            srv.poll(t)          # a waited ticket is gone
    np.testing.assert_array_equal(o["col"], _oracle_rows(x)["col"])
    assert isinstance(seen_pending, bool)


def test_device_list_dispatch():
    """Replicas of the slots per listed device (here the one GPU listed twice:
    two independent sets of slots) with least-loaded dispatch; every request
    equals the oracle."""
    evs = [synth.make_event("c2", e, n=int(n)) for e, n in
           enumerate(np.random.default_rng(8).integers(5_000, 40_000, size=16))]
    with frnn.Server(d=D, r=R, k=K, batch_points=80_000, batch_events=4, slots=1, devices=[0, 0]) as srv:
        outs = [srv.wait(t) for t in [srv.submit(x) for x in evs]]
        st = srv.stats()
    assert st["batches"] >= 2
    for x, o in zip(evs, outs):
        ref = _oracle_rows(x)
        np.testing.assert_array_equal(o["row_ptr"], ref["row_ptr"])
        np.testing.assert_array_equal(o["col"], ref["col"])
