"""The remaining workloads at full size: the batched stand-in (64 events of
N ~ U[40k, 140k], K=64), the pile-up-scale event (N=1,000,000, D=12, r=0.15,
K=128) and its cap-binding variant, checked exactly against the oracle (whole
events, or a seeded 50,000-query subset of the million-point events against
the oracle's rows over all points); and the autotuner, which may change speed
but never the result.  Both forms of the neighbour walk are checked."""
import functools

import numpy as np
import pytest

import oracle
from paper_2202_06929_b300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2202_06929_b300 as frnn  # noqa: E402

WALKS = [frnn._native.FRNN_WALK_CANDIDATES, frnn._native.FRNN_WALK_QUERIES]


def _subset(n, n_q, seed):
    return np.unique(np.concatenate([np.random.default_rng(seed).choice(n, size=min(n_q, n), replace=False),
                                     [0, n - 1]]))


def _rows_equal(rp, col, q, orp, ocol, what=""):
    """Rows q of a GPU graph (rp over all points) equal the oracle's rows for q."""
    lens = rp[q + 1] - rp[q]
    np.testing.assert_array_equal(lens, np.diff(orp), err_msg=f"{what} row lengths")
    starts = rp[q]
    idx = np.repeat(starts - orp[:-1], np.diff(orp)) + np.arange(orp[-1])
    np.testing.assert_array_equal(col[idx], ocol, err_msg=f"{what} columns")


@functools.lru_cache(maxsize=4)
def _c3_oracle(event):
    w = synth.WORKLOADS["c3"]
    return oracle.radius_graph(synth.make_event("c3", event), w.r, w.k)


@pytest.mark.parametrize("walk", WALKS, ids=["cand", "query"])
def test_c3_batched_events(walk):
    """64 events in one batched build: every row of events 0 and 63, a
    1,000-row sample of every eighth event."""
    w = synth.WORKLOADS["c3"]
    evs = [synth.make_event("c3", e) for e in range(64)]
    off = np.concatenate([[0], np.cumsum([e.shape[0] for e in evs])]).astype(np.int64)
    assert all(40_000 <= e.shape[0] <= 140_000 for e in evs)
    with frnn.Plan(n_max=int(off[-1]), d_max=w.d, k_max_cap=w.k, events_max=64, use_graph=True) as plan:
        plan.set_tuning(4, 1.0, walk)
        csr = plan.build_batched(torch.from_numpy(np.concatenate(evs)).cuda(), off, w.r, w.k)
        host = csr.to_host()
        assert plan.last_status() == 0
    for b in (0, 63):
        rp, col = csr.event_rows(host, b)
        orp, ocol = _c3_oracle(b)
        np.testing.assert_array_equal(rp, orp, err_msg=f"event {b}")
        np.testing.assert_array_equal(col, ocol, err_msg=f"event {b}")
    for b in range(0, 64, 8):
        rp, col = csr.event_rows(host, b)
        q = _subset(evs[b].shape[0], 1000, b)
        orp, ocol = oracle.radius_graph(evs[b], w.r, w.k, queries=q)
        _rows_equal(rp.astype(np.int64), col, q, orp, ocol, f"event {b}")


@functools.lru_cache(maxsize=2)
def _pileup_oracle(name):
    """The oracle's rows of a seeded 50,000-query subset of the event (each row
    against all 1,000,000 points)."""
    w = synth.WORKLOADS[name]
    x = synth.make_event(name)
    q = _subset(x.shape[0], 50_000, 77)
    orp, ocol = oracle.radius_graph(x, w.r, w.k, queries=q)
    return q, orp, ocol


@pytest.mark.parametrize("name", ["c5", "c5b"])
def test_pileup_scale_event(name):
    """One million points, D=12: a 50,000-query subset equals the oracle, for
    four and six gridded dims and both walks, with long rows walked again or
    sorted from their kept hits (c5b: the cap binds for most rows)."""
    w = synth.WORKLOADS[name]
    x = synth.make_event(name)
    assert x.shape == (1_000_000, 12)
    q, orp, ocol = _pileup_oracle(name)
    xt = torch.from_numpy(x).cuda()
    # a plan that keeps the hits of long rows (1.5 GB) and one that walks them again
    for hits in (0, 32 * 384 * (x.shape[0] // 32 + 1)):
        with frnn.Plan(n_max=x.shape[0], d_max=w.d, k_max_cap=w.k, edge_capacity=x.shape[0] * w.k,
                       cells_per_point=32, hit_capacity=hits) as plan:
            for tuning in [(4, 1.0, WALKS[0]), (4, 1.0, WALKS[1]), (6, 1.0, WALKS[0]), (6, 1.0, WALKS[1])]:
                if hits and tuning[1:] != (1.0, WALKS[0]):
                    continue  # only the candidate-major walk keeps hits
                plan.set_tuning(*tuning)
                host = plan.build(xt, w.r, w.k).to_host()
                assert plan.last_status() == 0
                _rows_equal(host["row_ptr"].astype(np.int64), host["col"], q, orp, ocol,
                            f"{name} {tuning} hits={hits}")
    capped = np.mean(np.diff(orp) == w.k)
    if name == "c5b":
        assert capped > 0.5, capped     # the cap binds for most rows
    else:
        assert capped < 0.01, capped


def test_autotune_keeps_result():
    """The autotuner (probe every grid, time the cheapest with both walk
    forms) may change speed, never the result; its choice is cached for the
    call's shape and an explicit tuning drops the cache."""
    evs = [synth.make_event("c2", e, n=30_000) for e in range(4)]
    off = np.concatenate([[0], np.cumsum([e.shape[0] for e in evs])]).astype(np.int64)
    xt = torch.from_numpy(np.concatenate(evs)).cuda()
    with frnn.Plan(n_max=int(off[-1]), d_max=8, k_max_cap=256, events_max=4, cells_per_point=32) as plan:
        ref = plan.build_batched(xt, off, 0.1, 256).to_host()
        assert plan.tuning_for(off, 8, 0.1, 256)[3] is False
        g, scale, ms = plan.autotune(xt, off, 0.1, 256)
        assert g in (2, 3, 4, 5, 6) and scale in (1.0, 1.25, 1.5, 2.0) and ms > 0
        g2, s2, walk, cached = plan.tuning_for(off, 8, 0.1, 256)
        assert (g2, s2) == (g, scale) and walk in (1, 2) and cached
        assert plan.get_tuning() == (g2, s2, walk)
        # another shape (one event) is not covered by the entry
        assert plan.tuning_for(off[:2], 8, 0.1, 256)[3] is False
        got = plan.build_batched(xt, off, 0.1, 256).to_host()
        assert plan.last_status() == 0
        plan.set_tuning(3, 1.5, 1)
        assert plan.tuning_for(off, 8, 0.1, 256) == (3, 1.5, 1, False)
    np.testing.assert_array_equal(got["row_ptr"], ref["row_ptr"])
    np.testing.assert_array_equal(got["col"], ref["col"])


def test_autotune_flag_tunes_each_new_shape():
    """FRNN_AUTOTUNE: the first build of a call shape autotunes it; the rows
    equal the oracle's for each shape."""
    evs = [synth.make_event("c3", e, n=20_000) for e in range(3)]
    w = synth.WORKLOADS["c3"]
    with frnn.Plan(n_max=60_000, d_max=8, k_max_cap=64, events_max=3, cells_per_point=32, autotune=True,
                   use_graph=True) as plan:
        for sel in ([0], [0, 1, 2]):
            x = np.concatenate([evs[i] for i in sel])
            off = np.concatenate([[0], np.cumsum([evs[i].shape[0] for i in sel])]).astype(np.int64)
            assert plan.tuning_for(off, 8, w.r, w.k)[3] is False
            csr = plan.build_batched(torch.from_numpy(x).cuda(), off, w.r, w.k)
            host = csr.to_host()
            assert plan.last_status() == 0
            assert plan.tuning_for(off, 8, w.r, w.k)[3] is True
            for b, i in enumerate(sel):
                rp, col = csr.event_rows(host, b)
                orp, ocol = oracle.radius_graph(evs[i], w.r, w.k)
                np.testing.assert_array_equal(rp, orp)
                np.testing.assert_array_equal(col, ocol)
