"""The debug checks of a build's output (FRNN_DEBUG, frnn_check_last_build),
through the C ABI.

Two directions:
  - a plan with FRNN_DEBUG builds the same graphs as the oracle and its
    checks find nothing: radius builds with and without a cap, kNN builds,
    an event holding NaN, edges that overflow the plan, both walk forms,
    query rows held in registers (d <= 16) or not, a full-size N=120k event
    checked by the brute-force pass on every row and a 200k-point event on
    sampled rows;
  - a mistake planted on the host into a correct build's output (one device
    word rewritten, in bounds) is reported by the check of the stage that
    owns that word, at that word's index, and the next build checks clean.
"""
import functools

import numpy as np
import pytest

import oracle
from paper_2202_06929_b300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2202_06929_b300 as frnn  # noqa: E402
from paper_2202_06929_b300 import _native  # noqa: E402


def _events(sizes, d, seed, sigma=0.03):
    out = []
    for b, n in enumerate(sizes):
        if n == 0:
            out.append(np.zeros((0, d), np.float32))
        else:
            out.append(synth.clustered_grid(n, d, seed + b, max(n // 10, 1), sigma, noise_frac=0.1))
    return out


def _build(plan, xs, r, k, knn=False):
    x = np.ascontiguousarray(np.concatenate(xs), dtype=np.float32)
    off = np.concatenate([[0], np.cumsum([len(a) for a in xs])]).astype(np.int64)
    xt = torch.from_numpy(x).cuda()
    csr = plan.knn_batched(xt, off, k) if knn else plan.build_batched(xt, off, r, k)
    return csr, xt


def _assert_oracle(csr, xs, r, k, knn=False):
    host = csr.to_host()
    for b, xb in enumerate(xs):
        rp, col = csr.event_rows(host, b)
        if knn:
            orp, ocol = oracle.knn_graph(xb, k)
        else:
            orp, ocol = oracle.radius_graph(xb, r, k)
        np.testing.assert_array_equal(rp, orp)
        if k != frnn._native.FRNN_NO_CAP:
            np.testing.assert_array_equal(col, ocol)
            continue
        for i in range(len(xb)):  # rows over 32 of a build without a cap come in no order
            a, o = col[rp[i]:rp[i + 1]], ocol[orp[i]:orp[i + 1]]
            if len(a) <= 32:
                np.testing.assert_array_equal(a, o)
            else:
                np.testing.assert_array_equal(np.sort(a), np.sort(o))


def _clean(plan):
    assert plan.last_status() == frnn.FRNN_OK
    assert plan.last_check() == ("none", -1)


CASES = {
    # name: (event sizes, d, r, k, knn)
    "capped_batch": ([3000, 0, 1, 2500, 40], 8, 0.1, 16, False),
    "no_cap_dense": ([4000], 3, 0.25, frnn._native.FRNN_NO_CAP, False),
    "k1": ([2000, 1500], 8, 0.1, 1, False),
    "d16": ([3000], 16, 0.3, 32, False),
    "d24_unrolled_off": ([2000, 700], 24, 0.4, 24, False),
    "knn": ([2500, 1, 2, 1800], 8, 0.0, 12, True),
    "knn_d24": ([1200], 24, 0.0, 7, True),
}


@pytest.mark.parametrize("walk", [_native.FRNN_WALK_CANDIDATES, _native.FRNN_WALK_QUERIES], ids=["cand", "query"])
@pytest.mark.parametrize("name", list(CASES))
def test_debug_plan_checks_clean_and_matches_oracle(name, walk):
    sizes, d, r, k, knn = CASES[name]
    xs = _events(sizes, d, 7100 + len(name))
    n = sum(sizes)
    with frnn.Plan(n_max=n, d_max=d, k_max_cap=max(k, 1), events_max=len(sizes), emit_d2=True, debug=True,
                   edge_capacity=n * 256 if k == frnn._native.FRNN_NO_CAP else 0) as plan:
        plan.set_tuning(walk=walk)
        csr, _ = _build(plan, xs, r, k, knn)
        _clean(plan)
        _assert_oracle(csr, xs, r, k, knn)


def test_debug_plan_with_graph_replay_checks_every_build():
    xs = _events([2500, 1700], 8, 7300)
    with frnn.Plan(n_max=4200, d_max=8, k_max_cap=32, events_max=2, use_graph=True, debug=True) as plan:
        for _ in range(3):
            csr, _ = _build(plan, xs, 0.1, 32)
            _clean(plan)
        _assert_oracle(csr, xs, 0.1, 32)


def test_checks_after_labeling_and_edge_features():
    """Labeling and edge features write nothing the checks read: checks run
    after them find a correct build clean."""
    xs = _events([2500, 1700], 8, 7350)
    with frnn.Plan(n_max=4200, d_max=8, k_max_cap=32, events_max=2, emit_d2=True) as plan:
        csr, xt = _build(plan, xs, 0.1, 32)
        plan.label_components()
        plan.edge_features(xt, 0, min(1000, csr.n_edges()))
        assert plan.last_status() == frnn.FRNN_OK
        plan.check_last_build()
        _clean(plan)


def test_nonfinite_event_and_overflow_are_statuses_not_check_failures():
    xs = _events([1500, 1200, 900], 8, 7400)
    xs[1] = xs[1].copy()
    xs[1][17, 3] = np.nan
    with frnn.Plan(n_max=3600, d_max=8, k_max_cap=16, events_max=3, emit_d2=True, debug=True) as plan:
        csr, _ = _build(plan, xs, 0.1, 16)
        assert plan.last_status() == frnn.FRNN_ERR_NONFINITE_INPUT
        assert plan.last_check() == ("none", -1)
        host = csr.to_host()
        for b in (0, 2):
            rp, col = csr.event_rows(host, b)
            orp, ocol = oracle.radius_graph(xs[b], 0.1, 16)
            np.testing.assert_array_equal(rp, orp)
            np.testing.assert_array_equal(col, ocol)
        csr, _ = _build(plan, xs, 0.0, 5, knn=True)
        assert plan.last_status() == frnn.FRNN_ERR_NONFINITE_INPUT
        assert plan.last_check() == ("none", -1)
    xs = _events([3000], 8, 7500, sigma=0.01)
    with frnn.Plan(n_max=3000, d_max=8, k_max_cap=64, edge_capacity=3000, debug=True) as plan:
        csr, _ = _build(plan, xs, 0.2, 64)
        assert int(csr.edge_off[-1].item()) > 3000
        assert plan.last_status() == frnn.FRNN_ERR_OVERFLOW
        assert plan.last_check() == ("none", -1)


def test_full_size_event_every_row_by_brute_force():
    """One N=120k event of the headline workload (D=8, r=0.1, K=256): the
    brute-force pass checks every row against all 120k points."""
    x = synth.make_event("c2", 0)
    with frnn.Plan(n_max=len(x), d_max=8, k_max_cap=256, debug=True) as plan:
        _build(plan, [x], 0.1, 256)
        _clean(plan)


def test_large_event_sampled_rows():
    """A 200k-point event: rows are checked every ceil(n^2 / 2^34) = 3rd."""
    x = synth.make_event("c4", 0, n=200_000)
    with frnn.Plan(n_max=len(x), d_max=8, k_max_cap=256, debug=True) as plan:
        _build(plan, [x], 0.1, 256)
        _clean(plan)


@functools.lru_cache(maxsize=1)
def _workload_batch(name, n_ev):
    evs = [synth.make_event(name, e) for e in range(n_ev)]
    off = np.concatenate([[0], np.cumsum([e.shape[0] for e in evs])]).astype(np.int64)
    return np.concatenate(evs), off


FULL = {
    # name: (workload, events, plan keyword arguments)
    "c2_bench_batch": ("c2", 64, dict(edge_capacity=64 * 120_000 * 64, cells_per_point=32, use_graph=True)),
    "c3_batch": ("c3", 64, dict(use_graph=True)),
    "c5": ("c5", 1, dict(cells_per_point=32, hit_capacity=32 * 384 * 31_251)),
    "c5b": ("c5b", 1, dict(cells_per_point=32, hit_capacity=32 * 384 * 31_251)),
}


@pytest.mark.parametrize("walk", [_native.FRNN_WALK_CANDIDATES, _native.FRNN_WALK_QUERIES], ids=["cand", "query"])
@pytest.mark.parametrize("name", list(FULL))
def test_full_size_workloads_pass_every_check(name, walk):
    """The workloads at full size, in the bench's plan configurations: every
    row of the 64-event N=120k batch and of the 64-event C3 batch checked by
    brute force against its whole event, and the million-point C5 and C5b
    events on every 59th row (each against all 10^6 points)."""
    wl, n_ev, kw = FULL[name]
    w = synth.WORKLOADS[wl]
    x, off = _workload_batch(wl, n_ev)
    with frnn.Plan(n_max=int(off[-1]), d_max=w.d, k_max_cap=w.k, events_max=n_ev, **kw) as plan:
        plan.set_tuning(4, 1.0, walk)
        plan.build_batched(torch.from_numpy(x).cuda(), off, w.r, w.k)
        assert plan.last_status() == frnn.FRNN_OK
        plan.check_last_build()
        _clean(plan)


# ------------------------------------------------------------ planted mistakes

def _planted(k=8, emit_d2=True):
    xs = _events([3000, 2500], 8, 7600, sigma=0.02)
    plan = frnn.Plan(n_max=5500, d_max=8, k_max_cap=k, events_max=2, emit_d2=emit_d2)
    csr, xt = _build(plan, xs, 0.1, k)
    assert plan.last_status() == frnn.FRNN_OK
    plan.check_last_build()
    _clean(plan)
    host = csr.to_host()
    return plan, csr, xs, host


def _row_with(host, pred, start=1):
    rp = host["row_ptr"]
    for p in range(start, len(rp) - 2):
        if pred(p, int(rp[p]), int(rp[p + 1])):
            return p, int(rp[p]), int(rp[p + 1])
    raise AssertionError("no such row")


def _expect(plan, name, index):
    plan.check_last_build()
    assert plan.last_status() == frnn.FRNN_ERR_CHECK
    assert plan.last_check() == (name, index)
    assert plan.last_check() == ("none", -1)


def test_planted_edge_offset():
    plan, csr, xs, host = _planted()
    with plan:
        csr.edge_off[1] += 1
        _expect(plan, "event_offsets", 1)


def test_planted_row_offset():
    plan, csr, xs, host = _planted()
    with plan:
        # a row offset past the next one: row p ends before it starts
        p, s0, s1 = _row_with(host, lambda p, a, b: 1 < p < 2900 and b > a)
        csr.row_ptr[p] = s1 + 1
        plan.check_last_build()
        assert plan.last_status() == frnn.FRNN_ERR_CHECK
        name, idx = plan.last_check()
        assert name == "row_ptr" and idx in (p - 1, p)


def test_planted_column_own_index():
    plan, csr, xs, host = _planted()
    with plan:
        p, s0, s1 = _row_with(host, lambda p, a, b: p < 3000 and b - a >= 2)
        csr.col(s1)[s0 + 1] = p  # event 0: local index = p
        _expect(plan, "column", s0 + 1)


def test_planted_column_beyond_radius():
    plan, csr, xs, host = _planted()
    with plan:
        x0 = xs[0].astype(np.float64)
        p, s0, s1 = _row_with(host, lambda p, a, b: p < 3000 and b - a >= 1)
        far = int(np.argmax(((x0 - x0[p]) ** 2).sum(1)))
        csr.col(s1)[s0] = far
        _expect(plan, "radius", s0)


def test_planted_d2_one_ulp():
    plan, csr, xs, host = _planted()
    with plan:
        p, s0, s1 = _row_with(host, lambda p, a, b: b - a >= 1)
        d2 = csr.d2(s1)
        d2.view(torch.int32)[s0] += 1
        _expect(plan, "d2", s0)


def test_planted_order_swap():
    plan, csr, xs, host = _planted()
    with plan:
        d2h = host["d2"]
        p, s0, s1 = _row_with(host, lambda p, a, b: b - a >= 2 and d2h[a] < d2h[a + 1])
        col = csr.col(s1)
        a, b = int(host["col"][s0]), int(host["col"][s0 + 1])
        col[s0], col[s0 + 1] = b, a
        d2 = csr.d2(s1)
        d2[s0], d2[s0 + 1] = float(d2h[s0 + 1]), float(d2h[s0])
        _expect(plan, "order", s0 + 1)


def test_planted_missing_neighbour():
    """A capped row whose last entry is replaced by the next point in (d2, j)
    order: every entry is within r, in order, with its d2; only the
    brute-force pass sees that the row skipped a point."""
    k = 8
    plan, csr, xs, host = _planted(k=k)
    with plan:
        x0 = xs[0]
        deg = oracle.degree(x0, 0.1)
        p = int(np.flatnonzero(deg > k)[0])
        orp, ocol, od2 = oracle.radius_graph(x0, 0.1, 0, queries=[p], with_d2=True)
        s0, s1 = int(host["row_ptr"][p]), int(host["row_ptr"][p + 1])
        assert s1 - s0 == k and list(host["col"][s0:s1]) == list(ocol[:k])
        csr.col(s1)[s1 - 1] = int(ocol[k])
        csr.d2(s1)[s1 - 1] = float(od2[k])
        _expect(plan, "complete", p)
        # the next build on the plan checks clean again
        _build(plan, xs, 0.1, k)
        plan.check_last_build()
        _clean(plan)
