"""Exact k-nearest-neighbour graphs on the GPU (no radius; Sec. 3.1's exact
kNN without its radius cut): every row equals the oracle's, column for column
and d2 for d2, on single and batched events, any tuning, ties and duplicates,
and the degenerate sizes (events of 0, 1 and 2 points; k above n - 1)."""
import numpy as np
import pytest

import oracle
from paper_2202_06929_b300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2202_06929_b300 as frnn  # noqa: E402


def knn_gpu(x, k, plan=None, tuning=None, ev_off=None):
    n, d = x.shape
    off = np.array([0, n], np.int64) if ev_off is None else np.asarray(ev_off, np.int64)
    own = plan is None
    if own:
        plan = frnn.Plan(n_max=max(n, 1), d_max=d, k_max_cap=k, events_max=len(off) - 1, emit_d2=True,
                         edge_capacity=max(n * k, 1))
    try:
        if tuning:
            plan.set_tuning(*tuning)
        csr = plan.knn_batched(torch.from_numpy(np.ascontiguousarray(x)).cuda(), off, k)
        host = csr.to_host()
        st = plan.last_status()
    finally:
        if own:
            plan.close()
    return host, st


def assert_rows_equal(host, x, k, lo=0):
    rp, col, d2 = oracle.knn_graph(x, k, with_d2=True)
    base = host["row_ptr"][lo]
    n = x.shape[0]
    np.testing.assert_array_equal(host["row_ptr"][lo:lo + n + 1] - base, rp)
    np.testing.assert_array_equal(host["col"][base:base + rp[-1]], col)
    np.testing.assert_array_equal(host["d2"][base:base + rp[-1]], d2)


CASES = [
    ("uniform", lambda: synth.uniform_grid(3000, 3, 1), 8),
    ("uniform_d8_k1", lambda: synth.uniform_grid(2500, 8, 2), 1),
    ("clustered_d8", lambda: synth.clustered_grid(4000, 8, 3, 200, 0.02), 16),
    ("clustered_d12_k40", lambda: synth.clustered_grid(3000, 12, 4, 100, 0.03), 40),
    ("offgrid_d5", lambda: synth.uniform_float(2000, 5, 5), 12),
    ("duplicates", lambda: synth.duplicates(1500, 4, 6, 60), 24),
    ("line_d1", lambda: synth.uniform_grid(1000, 1, 7), 5),
    ("d16_k64", lambda: synth.clustered_grid(2000, 16, 8, 80, 0.05), 64),
]


@pytest.mark.parametrize("name,make,k", CASES, ids=[c[0] for c in CASES])
def test_knn_equals_oracle(name, make, k):
    x = make()
    host, st = knn_gpu(x, k)
    assert st == 0
    assert_rows_equal(host, x, k)


@pytest.mark.parametrize("g_max,scale", [(1, 1.0), (2, 1.0), (3, 1.5), (4, 2.0), (6, 1.0)])
def test_knn_tuning_never_changes_result(g_max, scale):
    x = synth.clustered_grid(3000, 8, 9, 150, 0.03)
    host, st = knn_gpu(x, 10, tuning=(g_max, scale))
    assert st == 0
    assert_rows_equal(host, x, 10)


def test_knn_batched_with_degenerate_events():
    sizes = [0, 1, 2, 5, 2500, 0, 3000]
    k = 6
    evs = [synth.clustered_grid(n, 8, 20 + i, max(n // 20, 1), 0.03) if n else np.zeros((0, 8), np.float32)
           for i, n in enumerate(sizes)]
    off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    x = np.concatenate(evs)
    plan = frnn.Plan(n_max=int(off[-1]), d_max=8, k_max_cap=k, events_max=len(sizes), emit_d2=True,
                     edge_capacity=int(off[-1]) * k)
    try:
        for _ in range(2):  # twice: counters and states return to zero
            host, st = knn_gpu(x, k, plan=plan, ev_off=off)
            assert st == 0
            for b, e in enumerate(evs):
                if sizes[b]:
                    assert_rows_equal(host, e, k, lo=int(off[b]))
            want = np.concatenate([[0], np.cumsum([n * min(k, max(n - 1, 0)) for n in sizes])])
            np.testing.assert_array_equal(host["edge_off"], want)
    finally:
        plan.close()


def test_knn_identical_points_and_large_k():
    x = np.zeros((1200, 3), np.float32)
    host, st = knn_gpu(x, 1024)
    assert st == 0
    assert_rows_equal(host, x, 1024)


def test_knn_sampled_rows_of_a_full_size_event():
    x = synth.make_event("c2", 0)
    k = 16
    plan = frnn.Plan(n_max=x.shape[0], d_max=8, k_max_cap=k, emit_d2=True, edge_capacity=x.shape[0] * k)
    try:
        host, st = knn_gpu(x, k, plan=plan)
    finally:
        plan.close()
    assert st == 0
    q = np.random.default_rng(0).choice(x.shape[0], 3000, replace=False)
    rp, col, d2 = oracle.knn_graph(x, k, queries=q, with_d2=True)
    for i, qi in enumerate(q):
        np.testing.assert_array_equal(host["col"][qi * k:(qi + 1) * k], col[rp[i]:rp[i + 1]])
        np.testing.assert_array_equal(host["d2"][qi * k:(qi + 1) * k], d2[rp[i]:rp[i + 1]])


def test_knn_labels_equal_oracle():
    x = synth.clustered_grid(4000, 8, 11, 300, 0.02, 0.2)
    k = 4
    plan = frnn.Plan(n_max=x.shape[0], d_max=8, k_max_cap=k, edge_capacity=x.shape[0] * k)
    try:
        plan.knn_batched(torch.from_numpy(x).cuda(), np.array([0, x.shape[0]]), k)
        labels = plan.label_components(float("inf")).cpu().numpy()
        assert plan.last_status() == 0
    finally:
        plan.close()
    rp, col = oracle.knn_graph(x, k)
    np.testing.assert_array_equal(labels, oracle.components(rp, col))


def test_knn_nonfinite_event_and_capacity():
    x = synth.uniform_grid(600, 4, 12)
    bad = x.copy()
    bad[3, 1] = np.inf
    k = 5
    plan = frnn.Plan(n_max=1200, d_max=4, k_max_cap=k, events_max=2, emit_d2=True, edge_capacity=1200 * k)
    try:
        host, st = knn_gpu(np.concatenate([bad, x]), k, plan=plan, ev_off=[0, 600, 1200])
        assert st == frnn.FRNN_ERR_NONFINITE_INPUT
        assert np.all(host["col"][:600 * k] == -1)
        assert_rows_equal(host, x, k, lo=600)
        host, st = knn_gpu(x, k, plan=plan)
        assert st == 0
        assert_rows_equal(host, x, k)
    finally:
        plan.close()
    small = frnn.Plan(n_max=600, d_max=4, k_max_cap=k, edge_capacity=600 * k - 1)
    try:
        with pytest.raises(frnn.FrnnError):
            small.knn_batched(torch.from_numpy(x).cuda(), np.array([0, 600]), k)
    finally:
        small.close()


def test_knn_far_outlier_takes_the_whole_event_scan():
    # one point far from a tight cloud stretches the grid; its rings would
    # grow past the ring limits, so its row comes from the whole-event scan
    x = synth.clustered_grid(2000, 4, 13, 40, 0.02)
    x = np.concatenate([x, np.array([[60.0, 60.0, -60.0, 60.0]], np.float32)])
    host, st = knn_gpu(x, 8)
    assert st == 0
    assert_rows_equal(host, x, 8)


def test_knn_and_radius_builds_alternate_on_one_plan():
    # the two launch sequences share the plan's counters and tile states:
    # each must leave them as the other expects (radius builds replayed from
    # a captured graph)
    x = synth.clustered_grid(3000, 8, 14, 150, 0.03)
    xt = torch.from_numpy(x).cuda()
    off = np.array([0, x.shape[0]], np.int64)
    rp_r, col_r = oracle.radius_graph(x, 0.1, 16)
    rp_k, col_k = oracle.knn_graph(x, 12)
    plan = frnn.Plan(n_max=x.shape[0], d_max=8, k_max_cap=16, edge_capacity=x.shape[0] * 16, use_graph=True)
    try:
        for _ in range(2):
            h = plan.build_batched(xt, off, 0.1, 16).to_host()
            assert plan.last_status() == 0
            np.testing.assert_array_equal(h["row_ptr"], rp_r)
            np.testing.assert_array_equal(h["col"], col_r)
            h = plan.knn_batched(xt, off, 12).to_host()
            assert plan.last_status() == 0
            np.testing.assert_array_equal(h["row_ptr"], rp_k)
            np.testing.assert_array_equal(h["col"], col_k)
    finally:
        plan.close()


def test_knn_edge_features_equal_oracle():
    x = synth.uniform_grid(1500, 6, 15)
    k = 5
    plan = frnn.Plan(n_max=x.shape[0], d_max=6, k_max_cap=k, edge_capacity=x.shape[0] * k)
    try:
        xt = torch.from_numpy(x).cuda()
        plan.knn_batched(xt, np.array([0, x.shape[0]]), k)
        feats = plan.edge_features(xt, 0, x.shape[0] * k).cpu().numpy()
        assert plan.last_status() == 0
    finally:
        plan.close()
    rp, col, d2 = oracle.knn_graph(x, k, with_d2=True)
    src = np.repeat(np.arange(x.shape[0]), np.diff(rp))
    np.testing.assert_array_equal(feats[:, :6], x[src])
    np.testing.assert_array_equal(feats[:, 6:12], x[col])
    np.testing.assert_array_equal(feats[:, 12], d2)


@pytest.mark.parametrize("k", [6, 18, 26, 32, 80])
def test_knn_lattice_ties_at_shell_boundaries(k):
    """A regular lattice in 3 of 8 dims: neighbour shells of equal d2 (6 at
    one spacing, 12 at sqrt 2, 8 at sqrt 3, ...), so the k-th key often ties
    with keys of several other cells and ring slots; the rings' gap pruning
    must keep every tied candidate whose index sorts first."""
    m = 12
    g = np.stack(np.meshgrid(np.arange(m), np.arange(m), np.arange(m), indexing="ij"), -1).reshape(-1, 3)
    x = np.zeros((g.shape[0], 8), np.float32)
    x[:, :3] = (g * 8 - 44).astype(np.float32) / 256.0  # on the 1/256 grid
    rng = np.random.default_rng(2202069290)
    x = x[rng.permutation(x.shape[0])]
    host, st = knn_gpu(x, k)
    assert st == frnn.FRNN_OK
    assert_rows_equal(host, x, k)
