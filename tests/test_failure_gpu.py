"""Failure detection on the GPU without a GPU fault.

The scans' waits for a preceding tile are bounded (polls and time).  A test
hook makes the next build's cell scan wait for a predecessor that never
publishes, so the waits run out, the kernels return and FRNN_ERR_TIMEOUT is
latched.  The tests check that the build's outputs stay inside the plan's
buffers (an empty graph, singleton labels), that the status is reported, and
that the next build on the same plan is exact again.
"""
import time

import numpy as np
import pytest

import oracle
from paper_2202_06929_b300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2202_06929_b300 as frnn  # noqa: E402

R, K = 0.1, 64


def _events():
    xs = [synth.make_event("c1"), synth.clustered_grid(3000, 8, 5, 250, 0.03, 0.2)]
    off = np.cumsum([0] + [x.shape[0] for x in xs]).astype(np.int64)
    return xs, off, np.concatenate(xs)


def _assert_exact(plan, xs, off, xall):
    csr = plan.build_batched(torch.from_numpy(xall).cuda(), off, R, K)
    host = csr.to_host()
    assert plan.last_status() == frnn.FRNN_OK
    for b, x in enumerate(xs):
        rp, col = oracle.radius_graph(x, R, K)
        got_rp, got_col = csr.event_rows(host, b)
        np.testing.assert_array_equal(got_rp, rp)
        np.testing.assert_array_equal(got_col, col)


@pytest.mark.parametrize("use_graph", [False, True])
def test_stalled_scan_times_out_then_recovers(use_graph):
    xs, off, xall = _events()
    n = xall.shape[0]
    with frnn.Plan(n_max=n, d_max=8, k_max_cap=K, events_max=4, use_graph=use_graph) as plan:
        _assert_exact(plan, xs, off, xall)
        plan.test_stall_next_build()
        t0 = time.perf_counter()
        csr = plan.build_batched(torch.from_numpy(xall).cuda(), off, R, K)
        labels = plan.label_components()
        torch.cuda.synchronize()
        waited = time.perf_counter() - t0
        # every wait gave up after about a second, not after an unbounded spin
        assert waited < 20.0, waited
        rp = csr.row_ptr.cpu().numpy()
        np.testing.assert_array_equal(rp, np.zeros(n + 1, dtype=rp.dtype))
        # labeling of a timed-out build keeps every point alone
        lab = labels.cpu().numpy()
        local = np.concatenate([np.arange(x.shape[0]) for x in xs])
        np.testing.assert_array_equal(lab, local)
        assert plan.last_status() == frnn.FRNN_ERR_TIMEOUT
        # the reported build is forgotten
        with pytest.raises(frnn.FrnnError):
            plan.label_components()
        # the status was cleared and the plan restored: exact again
        assert plan.last_status() == frnn.FRNN_OK
        _assert_exact(plan, xs, off, xall)
        _assert_exact(plan, xs, off, xall)


def test_timeout_stays_latched_until_read():
    xs, off, xall = _events()
    with frnn.Plan(n_max=xall.shape[0], d_max=8, k_max_cap=K, events_max=4) as plan:
        plan.test_stall_next_build()
        xt = torch.from_numpy(xall).cuda()
        plan.build_batched(xt, off, R, K)
        # a second build before the status is read also skips its work
        csr = plan.build_batched(xt, off, R, K)
        torch.cuda.synchronize()
        assert int(csr.row_ptr[-1].item()) == 0
        assert plan.last_status() == frnn.FRNN_ERR_TIMEOUT
        _assert_exact(plan, xs, off, xall)


def test_stalled_knn_build_times_out_then_recovers():
    xs, off, xall = _events()
    k = 8
    with frnn.Plan(n_max=xall.shape[0], d_max=8, k_max_cap=K, events_max=4) as plan:
        xt = torch.from_numpy(xall).cuda()
        plan.test_stall_next_build()
        plan.knn_batched(xt, off, k)
        assert plan.last_status() == frnn.FRNN_ERR_TIMEOUT
        with pytest.raises(frnn.FrnnError):
            plan.edge_features(xt, 0, 1)
        csr = plan.knn_batched(xt, off, k)
        host = csr.to_host()
        assert plan.last_status() == frnn.FRNN_OK
        for b, x in enumerate(xs):
            rp, col = oracle.knn_graph(x, k)
            got_rp, got_col = csr.event_rows(host, b)
            np.testing.assert_array_equal(got_rp, rp)
            np.testing.assert_array_equal(got_col, col)
