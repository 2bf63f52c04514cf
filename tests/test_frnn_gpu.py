"""Parity of the CUDA graph build with the CPU oracle, through the C ABI.

Every comparison is exact: row_ptr and col equal element by element (and d2
bit for bit when emitted).  The CUDA path computes each squared distance with
the same float32 operations in the same order as the oracle (or, when every
coordinate is on the 1/256 grid and every partial sum is exact, with fused
multiply-adds that give the same bits), so the edge sets agree on any input,
on the 1/256 grid or off it.  Both forms of the
neighbour walk (candidates across the lanes, or a lane per query) are
checked on the seeded sweep, the tunings and the full-size events.
"""
import functools

import numpy as np
import pytest

import oracle
from paper_2202_06929_b300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2202_06929_b300 as frnn  # noqa: E402

WALKS = [frnn._native.FRNN_WALK_CANDIDATES, frnn._native.FRNN_WALK_QUERIES]
WALK_IDS = ["cand", "query"]


def gpu_csr(x, r, k, emit_d2=False, use_graph=False, tuning=None, plan=None, cells_per_point=0):
    x = np.ascontiguousarray(x, dtype=np.float32)
    n, d = x.shape
    own = plan is None
    if own:
        plan = frnn.Plan(n_max=max(n, 1), d_max=d, k_max_cap=max(k, 1), emit_d2=emit_d2,
                         use_graph=use_graph, cells_per_point=cells_per_point)
    try:
        if tuning:
            plan.set_tuning(*tuning)
        xt = torch.from_numpy(x).cuda()
        csr = plan.build(xt, r, k)
        host = csr.to_host()
        st = plan.last_status()
        return host, st
    finally:
        if own:
            plan.close()


def assert_same_as_oracle(x, r, k, **kw):
    host, st = gpu_csr(x, r, k, emit_d2=True, **kw)
    assert st == frnn.FRNN_OK, frnn.status_string(st)
    rp, col, d2 = oracle.radius_graph(x, r, k, with_d2=True)
    np.testing.assert_array_equal(host["row_ptr"].astype(np.int64), rp)
    np.testing.assert_array_equal(host["col"], col)
    np.testing.assert_array_equal(host["d2"].view(np.uint32), d2.view(np.uint32))
    return host


# ------------------------------------------------------------------ workloads

def test_c1_plain_event():
    x = synth.make_event("c1")
    assert_same_as_oracle(x, 0.1, 64)


@pytest.mark.parametrize("use_graph", [False, True])
def test_c1_graph_replay(use_graph):
    x = synth.make_event("c1")
    plan = frnn.Plan(n_max=4000, d_max=8, k_max_cap=64, use_graph=use_graph, emit_d2=True)
    try:
        rp, col = oracle.radius_graph(x, 0.1, 64)
        for rep in range(3):  # replays of the same captured graph
            host, st = gpu_csr(x, 0.1, 64, plan=plan)
            assert st == 0
            np.testing.assert_array_equal(host["row_ptr"], rp)
            np.testing.assert_array_equal(host["col"], col)
        # a different event through the same plan (and graph)
        x2 = synth.clustered_grid(3500, 8, 77, 300, 0.03, 0.2)
        rp2, col2 = oracle.radius_graph(x2, 0.1, 64)
        host, st = gpu_csr(x2, 0.1, 64, plan=plan)
        np.testing.assert_array_equal(host["row_ptr"], rp2)
        np.testing.assert_array_equal(host["col"], col2)
    finally:
        plan.close()


# ------------------------------------------------------------------ seeded property sweep

SWEEP = []
_rng = np.random.default_rng(2202)
for _case in range(28):
    _d = [1, 2, 3, 5, 8, 12, 16][_case % 7]
    _k = [1, 2, 31, 32, 33, 64, 256][(_case // 7 + _case) % 7]
    _n = int(_rng.integers(0, 5001)) if _case % 9 else int(_rng.integers(0, 40))
    _kind = ["grid", "cluster", "float", "dups"][_case % 4]
    _r = [0.1, 0.0625, 0.137, 0.25][(_case // 4) % 4]
    SWEEP.append((_case, _n, _d, _k, _kind, _r))


def _make(kind, n, d, seed):
    if kind == "grid":
        return synth.uniform_grid(n, d, seed, -64, 64)
    if kind == "cluster":
        return synth.clustered_grid(n, d, seed, max(n // 12, 1), 0.04, 0.1)
    if kind == "float":
        return synth.uniform_float(n, d, seed, 0.4)
    return synth.duplicates(n, d, seed, max(n // 20, 1))


@pytest.mark.parametrize("walk", WALKS, ids=WALK_IDS)
@pytest.mark.parametrize("case,n,d,k,kind,r", SWEEP, ids=[f"c{c[0]}-n{c[1]}-d{c[2]}-k{c[3]}-{c[4]}" for c in SWEEP])
def test_property_sweep(case, n, d, k, kind, r, walk):
    x = _make(kind, n, d, 1000 + case)
    assert_same_as_oracle(x, r, k, tuning=(0, 0.0, walk))


@pytest.mark.parametrize("walk", WALKS, ids=WALK_IDS)
@pytest.mark.parametrize("g_max,scale", [(1, 1.0), (2, 1.0), (3, 1.0), (4, 1.0), (4, 1.5), (3, 2.0), (2, 3.7),
                                         (5, 1.0), (6, 1.0), (6, 1.5), (5, 2.0)])
def test_tuning_never_changes_result(g_max, scale, walk):
    # a cell budget large enough for five and six gridded dims (81 and 243 runs per cell)
    x = synth.clustered_grid(4000, 8, 5, 300, 0.03, 0.15)
    assert_same_as_oracle(x, 0.1, 16, tuning=(g_max, scale, walk), cells_per_point=512)


@pytest.mark.parametrize("walk", WALKS, ids=WALK_IDS)
def test_six_gridded_dims_high_dimensional_event(walk):
    x = synth.clustered_grid(20000, 12, 8, 1500, 0.03, 0.25)
    assert_same_as_oracle(x, 0.15, 40, tuning=(6, 1.0, walk), cells_per_point=256)


def test_query_major_run_list_overflow():
    """Dense single-point cells: a 32-query chunk holds up to 32 segments of
    27 non-empty runs each, more than one run list holds, so the lane-per-query
    walk takes the chunk's segments in several batches."""
    x = synth.uniform_grid(6000, 4, 31, -256, 256)
    assert_same_as_oracle(x, 0.18, 64, tuning=(4, 1.0, frnn._native.FRNN_WALK_QUERIES))


# ------------------------------------------------------------------ edge cases

def test_empty_and_single_point():
    for n in (0, 1):
        x = np.zeros((n, 5), np.float32)
        host, st = gpu_csr(x, 0.1, 4, plan=None)
        assert st == 0
        assert host["row_ptr"].tolist() == [0] * (n + 1)
        assert host["col"].size == 0


def test_all_identical_points():
    n, k = 3000, 37
    x = np.tile(np.array([[0.1, -0.2, 0.3, 0.4, 0.5]], np.float32), (n, 1))
    host = assert_same_as_oracle(x, 0.01, k)
    rp, col = host["row_ptr"], host["col"]
    for i in (0, 1, 36, 37, 2999):
        assert col[rp[i]:rp[i + 1]].tolist() == [j for j in range(n) if j != i][:k]


def test_single_dense_cell_cap_binds():
    # every point within r of most others: |S_i| >> k, deep top-k selection
    x = synth.uniform_grid(2500, 3, 9, -6, 6)
    assert_same_as_oracle(x, 0.05, 100)


@pytest.mark.parametrize("case", ["dense-k100", "grid-k1024", "dense-nocap", "small-area"])
def test_long_rows_from_kept_hits(case):
    """Rows longer than 24 whose every neighbour the walk kept in the plan's
    spill area (hit_capacity): their k nearest are sorted from those.  With a
    small area only some chunks get room and the others' rows are walked
    again; the rows are the oracle's either way."""
    walk = frnn._native.FRNN_WALK_CANDIDATES
    if case == "dense-k100":
        x, r, k, cap = synth.uniform_grid(2500, 3, 9, -6, 6), 0.05, 100, 1 << 22
    elif case == "grid-k1024":
        x, r, k, cap = synth.uniform_grid(3000, 2, 17, -40, 40), 0.06, 1024, 1 << 22
    elif case == "dense-nocap":
        x, r, k, cap = synth.uniform_grid(4000, 3, 92, -20, 20), 0.05, 0, 1 << 22
    else:
        x, r, k, cap = synth.uniform_grid(4000, 3, 93, -12, 12), 0.05, 64, 3 * 32 * 384
    n, d = x.shape
    rp, col, d2 = oracle.radius_graph(x, r, k, with_d2=True)
    assert np.sum(np.diff(rp) > 24) > 100
    with frnn.Plan(n_max=n, d_max=d, k_max_cap=max(k, 1), emit_d2=True, hit_capacity=cap,
                   edge_capacity=int(rp[-1]) if k == 0 else 0) as plan:
        plan.set_tuning(0, 0.0, walk)
        for rep in range(2):
            host = plan.build(torch.from_numpy(x).cuda(), r, k).to_host()
            assert plan.last_status() == 0
            np.testing.assert_array_equal(host["row_ptr"].astype(np.int64), rp)
            if k > 0:
                np.testing.assert_array_equal(host["col"], col)
                np.testing.assert_array_equal(host["d2"].view(np.uint32), d2.view(np.uint32))
            else:  # no cap: long rows as sets
                for i in range(n):
                    a, b = rp[i], rp[i + 1]
                    assert sorted(col[a:b].tolist()) == sorted(host["col"][a:b].tolist())


def test_points_outside_unit_box_and_large_values():
    rng = np.random.default_rng(4)
    x = (rng.normal(0, 30.0, size=(3000, 4)) + 1000.0).astype(np.float32)
    assert_same_as_oracle(x, 3.0, 8)


@pytest.mark.parametrize("d", [7, 13, 33, 64])
def test_dims_not_multiple_of_four_and_wide(d):
    x = synth.clustered_grid(1500, d, 40 + d, 100, 0.02, 0.1)
    assert_same_as_oracle(x, 0.05 * np.sqrt(d / 8), 12)


@pytest.mark.parametrize("k", [1, 1024])
def test_extreme_caps(k):
    x = synth.uniform_grid(3000, 2, 17, -40, 40)
    assert_same_as_oracle(x, 0.06, k)


@pytest.mark.parametrize("outlier", [False, True])
@pytest.mark.parametrize("walk", WALKS, ids=WALK_IDS)
def test_pairs_at_the_radius_along_filter_dims(outlier, walk):
    """Partners placed at distances within a few ulps of r, displaced only
    along the dims the grid leaves out (those the one-byte key filter reads),
    off the 1/256 grid.  With outliers (five points at 100 along dims 0-4)
    only one dim is gridded and the filter's key step is about 4 r, so most
    candidates pass the filter and rows overflow their slots (the candidates
    past them are tested at once).  The key filter may only skip pairs
    farther than r, so every row still equals the oracle's."""
    rng = np.random.default_rng(2202)
    n0, d, r = 1200, 8, 0.1
    base = rng.uniform(-1, 1, size=(n0, d)).astype(np.float32)
    parts = [base]
    for scale in (1 - 2**-22, 1.0, 1 + 2**-22, 1 - 2**-12, 1 + 2**-12):
        u = rng.normal(size=(n0, d))
        u[:, :4] = 0.0  # the four widest dims are gridded; move along the others
        u /= np.linalg.norm(u, axis=1, keepdims=True)
        parts.append((base + (r * scale) * u).astype(np.float32))
    x = np.concatenate(parts)
    x[:, :4] *= np.float32(1.5)  # keep dims 0-3 the widest
    if outlier:
        for t in range(5):
            x[t, t] = np.float32(100.0)
    x = x[rng.permutation(x.shape[0])]
    host = assert_same_as_oracle(x, r, 16, tuning=(4, 1.0, walk))
    assert host["row_ptr"][-1] > 0


@pytest.mark.parametrize("case", ["flat-filter-dims", "tiny-radius", "huge-extent", "three-dims"])
@pytest.mark.parametrize("walk", WALKS, ids=WALK_IDS)
def test_key_filter_degenerate_events(case, walk):
    """Events where the key filter has nothing to go on, or is switched off:
    the dims it reads are constant (every key equal), the radius is so small
    that r^2 is below 2^-100, the extent is beyond 2^100, or every dim is
    gridded (the filter then reads gridded dims).  The rows still equal the
    oracle's."""
    rng = np.random.default_rng(77)
    if case == "flat-filter-dims":
        x = rng.uniform(-1, 1, size=(3000, 8)).astype(np.float32)
        x[:, 4:] = np.float32(0.25)
        x[:, :4] *= np.float32(0.3)
        r, k = 0.1, 32
    elif case == "tiny-radius":
        base = rng.uniform(-1, 1, size=(1500, 8)).astype(np.float32)
        x = np.concatenate([base, base[:700]])  # exact duplicates: d2 = 0 <= r2
        r, k = 1e-16, 8
    elif case == "huge-extent":
        base = (rng.normal(0, 1, size=(2000, 8)) * 1e30).astype(np.float32)
        x = np.concatenate([base, base[:600]])  # at this scale only duplicates are within r
        r, k = 1e18, 16
    else:
        x = synth.uniform_grid(4000, 3, 12, -40, 40)
        r, k = 0.05, 24
    x = x[rng.permutation(x.shape[0])]
    assert_same_as_oracle(x, r, k, tuning=(0, 0.0, walk))


def test_radius_boundary_inclusive():
    x = np.array([[0.0, 0.0], [0.125, 0.0], [0.0, 0.12890625]], dtype=np.float32)
    host = assert_same_as_oracle(x, 0.125, 4)
    assert host["row_ptr"].tolist() == [0, 1, 2, 2]


def test_nonfinite_input_is_reported_and_plan_recovers():
    x = synth.uniform_grid(500, 4, 3, -20, 20)
    bad = x.copy()
    bad[17, 2] = np.nan
    plan = frnn.Plan(n_max=1000, d_max=4, k_max_cap=8)
    try:
        host, st = gpu_csr(bad, 0.1, 8, plan=plan)
        assert st == frnn.FRNN_ERR_NONFINITE_INPUT
        assert host["row_ptr"][-1] == 0
        host, st = gpu_csr(x, 0.1, 8, plan=plan)
        assert st == 0
        rp, col = oracle.radius_graph(x, 0.1, 8)
        np.testing.assert_array_equal(host["col"], col)
    finally:
        plan.close()


def test_edge_overflow_is_reported_and_plan_recovers():
    x = synth.clustered_grid(2000, 4, 8, 50, 0.03)
    rp, col = oracle.radius_graph(x, 0.1, 16)
    plan = frnn.Plan(n_max=2000, d_max=4, k_max_cap=16, edge_capacity=int(rp[-1]) - 1)
    try:
        _, st = gpu_csr(x, 0.1, 16, plan=plan)
        assert st == frnn.FRNN_ERR_OVERFLOW
        small = x[:200]
        rps, cols = oracle.radius_graph(small, 0.1, 16)
        host, st = gpu_csr(small, 0.1, 16, plan=plan)
        assert st == 0
        np.testing.assert_array_equal(host["col"], cols)
    finally:
        plan.close()


def test_invalid_arguments():
    plan = frnn.Plan(n_max=100, d_max=4, k_max_cap=8)
    x = torch.zeros((50, 4), device="cuda")
    try:
        for r, k, err in [(0.0, 4, 1), (float("nan"), 4, 1), (-1.0, 4, 1), (0.1, -1, 1), (0.1, 9, 7)]:
            with pytest.raises(frnn.FrnnError) as ei:
                plan.build(x, r, k)
            assert ei.value.status == err
        with pytest.raises(frnn.FrnnError) as ei:
            plan.build(torch.zeros((200, 4), device="cuda"), 0.1, 4)
        assert ei.value.status == frnn.FRNN_ERR_CAPACITY
        with pytest.raises(frnn.FrnnError) as ei:
            plan.build(torch.zeros((10, 5), device="cuda"), 0.1, 4)
        assert ei.value.status == frnn.FRNN_ERR_CAPACITY
        with pytest.raises(frnn.FrnnError):
            plan.build_batched(x, [0, 30, 20, 50], 0.1, 4)
    finally:
        plan.close()


def test_plan_memory_budget():
    """mem_budget_bytes: a plan whose device bytes exceed the budget is
    refused with OOM; one at exactly its own size is created, and the device
    memory it takes is its stated size plus allocation granularity."""
    kw = dict(n_max=200_000, d_max=8, k_max_cap=64, events_max=4, emit_d2=True)
    need = frnn.plan_bytes(**kw)
    with pytest.raises(frnn.FrnnError) as ei:
        frnn.Plan(mem_budget_bytes=need - 1, **kw)
    assert ei.value.status == frnn.FRNN_ERR_OOM
    frnn.Plan(n_max=10, d_max=8, k_max_cap=8).close()  # module and context set-up outside the window
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    with frnn.Plan(mem_budget_bytes=need, **kw) as plan:
        torch.cuda.synchronize()
        used = free0 - torch.cuda.mem_get_info()[0]
        assert need <= used <= need + 48 * (2 << 20), (need, used)
        x = synth.uniform_grid(3000, 8, 5)
        host = plan.build(torch.from_numpy(x).cuda(), 0.3, 64).to_host()
        assert plan.last_status() == frnn.FRNN_OK
    rp, col = oracle.radius_graph(x, 0.3, 64)
    np.testing.assert_array_equal(host["row_ptr"], rp)
    np.testing.assert_array_equal(host["col"], col)


# ------------------------------------------------------------------ batched form

def _events(kind, sizes, d, seed):
    return [_make(kind, n, d, seed + i) for i, n in enumerate(sizes)]


@pytest.mark.parametrize("use_graph", [False, True])
def test_batched_equals_each_event_alone(use_graph):
    sizes = [1200, 0, 1, 3500, 777, 2048, 2049, 5]
    evs = _events("cluster", sizes, 8, 300)
    off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    allx = np.concatenate(evs).astype(np.float32)
    plan = frnn.Plan(n_max=int(off[-1]), d_max=8, k_max_cap=32, events_max=16, use_graph=use_graph)
    try:
        csr = plan.build_batched(torch.from_numpy(allx).cuda(), off, 0.1, 32)
        host = csr.to_host()
        assert plan.last_status() == 0
        for b, x in enumerate(evs):
            rp, col = csr.event_rows(host, b)
            orp, ocol = oracle.radius_graph(x, 0.1, 32)
            np.testing.assert_array_equal(rp, orp)
            np.testing.assert_array_equal(col, ocol)
    finally:
        plan.close()


@pytest.mark.parametrize("off_grid_event", [None, 0, 2])
def test_candidate_major_fused_and_exact_sums_on_one_plan(off_grid_event):
    """The candidate-major walk adds squares with fused multiply-adds only
    when every coordinate of the call is on the 1/256 grid (small enough that
    every partial sum is exact); one event off the grid makes the whole call
    take the sequential sum.  Builds of both kinds alternate on one plan (and
    its captured graph), and every row equals the oracle's, d2 included."""
    sizes = [3000, 1500, 2500]
    evs = _events("cluster", sizes, 12, 400)
    if off_grid_event is not None:
        rng = np.random.default_rng(5)
        x = evs[off_grid_event].astype(np.float64)
        evs[off_grid_event] = (x + rng.uniform(-1e-3, 1e-3, size=x.shape)).astype(np.float32)
    off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    allx = np.concatenate(evs).astype(np.float32)
    grid = _events("grid", sizes, 12, 401)
    gx = np.concatenate(grid).astype(np.float32)
    with frnn.Plan(n_max=int(off[-1]), d_max=12, k_max_cap=24, events_max=4, emit_d2=True, use_graph=True) as plan:
        plan.set_tuning(0, 0.0, frnn._native.FRNN_WALK_CANDIDATES)
        for batch, xs_ in ((allx, evs), (gx, grid), (allx, evs)):
            csr = plan.build_batched(torch.from_numpy(batch).cuda(), off, 0.15, 24)
            host = csr.to_host()
            assert plan.last_status() == 0
            for b, x in enumerate(xs_):
                rp, col = csr.event_rows(host, b)
                orp, ocol, od2 = oracle.radius_graph(x, 0.15, 24, with_d2=True)
                np.testing.assert_array_equal(rp, orp)
                np.testing.assert_array_equal(col, ocol)
                e0 = int(host["edge_off"][b])
                d2 = host["d2"][e0:e0 + int(orp[-1])]
                np.testing.assert_array_equal(d2.view(np.uint32), od2.view(np.uint32))


def test_host_to_host_call_matches_device_call():
    sizes = [900, 1500, 3]
    evs = _events("grid", sizes, 5, 900)
    off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    allx = np.concatenate(evs).astype(np.float32)
    plan = frnn.Plan(n_max=int(off[-1]), d_max=5, k_max_cap=16, events_max=4)
    try:
        out = plan.build_host(allx, off, 0.09, 16)
        for b, x in enumerate(evs):
            lo, hi = off[b], off[b + 1]
            e0 = out["edge_off"][b]
            rp = out["row_ptr"][lo:hi + 1].astype(np.int64) - e0
            col = out["col"][e0:e0 + rp[-1]]
            orp, ocol = oracle.radius_graph(x, 0.09, 16)
            np.testing.assert_array_equal(rp, orp)
            np.testing.assert_array_equal(col, ocol)
        with pytest.raises(frnn.FrnnError) as ei:
            plan.build_host(allx, off, 0.09, 16, col_capacity=3)
        assert ei.value.status == frnn.FRNN_ERR_OVERFLOW
    finally:
        plan.close()


# ------------------------------------------------------------------ full-size workloads

def _sample_queries(n, m, seed):
    rng = np.random.default_rng(seed)
    q = rng.choice(n, size=min(m, n), replace=False)
    return np.unique(np.concatenate([q, [0, n - 1]]))


def _check_sampled(x, r, k, host_rp, host_col, queries):
    orp, ocol = oracle.radius_graph(x, r, k, queries=queries)
    for qi, i in enumerate(queries):
        got = host_col[host_rp[i]:host_rp[i + 1]]
        want = ocol[orp[qi]:orp[qi + 1]]
        np.testing.assert_array_equal(got, want, err_msg=f"row {i}")


@functools.lru_cache(maxsize=8)
def _c2_oracle(event):
    """The whole oracle graph of event `event` of the N=120,000 workload
    (every row; about 8 s on 16 host cores)."""
    return oracle.radius_graph(synth.make_event("c2", event), 0.1, 256)


@pytest.mark.parametrize("walk", WALKS, ids=WALK_IDS)
def test_c2_full_event_every_row(walk):
    """N=120,000, D=8, r=0.1, K=256: the whole graph (row_ptr and every col
    entry) equals the oracle's; the cap never binds at this density, so the
    graph is also symmetric and every edge lies within r."""
    x = synth.make_event("c2")
    host, st = gpu_csr(x, 0.1, 256, use_graph=True, tuning=(0, 0.0, walk))
    assert st == 0
    orp, ocol = _c2_oracle(0)
    rp, col = host["row_ptr"].astype(np.int64), host["col"]
    np.testing.assert_array_equal(rp, orp)
    np.testing.assert_array_equal(col, ocol)
    n = x.shape[0]
    src = np.repeat(np.arange(n), np.diff(rp))
    a = src.astype(np.int64) * n + col
    b = col.astype(np.int64) * n + src
    np.testing.assert_array_equal(np.sort(a), np.sort(b))
    assert np.all(col != src)
    # every edge within r: exact grid arithmetic in float64
    xd = x.astype(np.float64)
    d2 = ((xd[src] - xd[col]) ** 2).sum(1)
    assert np.all(d2 * 65536 <= oracle.grid_threshold(0.1))


@pytest.mark.parametrize("walk", WALKS, ids=WALK_IDS)
def test_c2_batched_bench_configuration(walk):
    """The benchmark's configuration: 64 events of N=120,000 (seeded per event),
    one batched build replayed from a CUDA graph: every row of four events
    (first, last and two between) equals the oracle's, and sampled rows of
    every third event."""
    n_ev = 64
    evs = [synth.make_event("c2", e) for e in range(n_ev)]
    off = np.concatenate([[0], np.cumsum([e.shape[0] for e in evs])]).astype(np.int64)
    allx = torch.from_numpy(np.concatenate(evs)).cuda()
    plan = frnn.Plan(n_max=int(off[-1]), d_max=8, k_max_cap=256, events_max=n_ev,
                     edge_capacity=int(off[-1]) * 64, cells_per_point=32, use_graph=True)
    try:
        plan.set_tuning(4, 1.0, walk)
        for rep in range(2):
            csr = plan.build_batched(allx, off, 0.1, 256)
            host = csr.to_host()
            assert plan.last_status() == 0
        for b in (0, 21, 42, 63):
            rp, col = csr.event_rows(host, b)
            orp, ocol = _c2_oracle(b)
            np.testing.assert_array_equal(rp, orp, err_msg=f"event {b}")
            np.testing.assert_array_equal(col, ocol, err_msg=f"event {b}")
        for b in range(0, n_ev, 3):
            rp, col = csr.event_rows(host, b)
            _check_sampled(evs[b], 0.1, 256, rp, col, _sample_queries(evs[b].shape[0], 150, b))
    finally:
        plan.close()


def test_plans_with_different_caps_coexist():
    """A plan with a small cap must not shrink the shared-memory limit that a
    plan with k = 1024 (the largest per-warp key buffer) launches with."""
    x = synth.uniform_grid(3000, 2, 23, -30, 30)
    big = frnn.Plan(n_max=3000, d_max=2, k_max_cap=1024)
    small = frnn.Plan(n_max=3000, d_max=2, k_max_cap=32)
    try:
        rp, col = oracle.radius_graph(x, 0.06, 1024)
        rps, cols = oracle.radius_graph(x, 0.06, 32)
        for plan, k, want in [(big, 1024, col), (small, 32, cols), (big, 1024, col)]:
            host, st = gpu_csr(x, 0.06, k, plan=plan)
            assert st == 0
            np.testing.assert_array_equal(host["col"], want)
    finally:
        big.close()
        small.close()


@pytest.mark.parametrize("kind", ["cluster", "dense"])
def test_no_cap_rows_equal_uncapped_oracle(kind):
    """k = FRNN_NO_CAP: the paper's own FRNN list, every neighbour within r.
    Rows of at most 32 neighbours are sorted; longer ones are compared as sets."""
    x = (synth.clustered_grid(5000, 8, 91, 300, 0.03, 0.1) if kind == "cluster"
         else synth.uniform_grid(4000, 3, 92, -20, 20))
    r = 0.1 if kind == "cluster" else 0.05
    rp, col, d2 = oracle.radius_graph(x, r, 0, with_d2=True)
    with frnn.Plan(n_max=x.shape[0], d_max=x.shape[1], k_max_cap=1, edge_capacity=int(rp[-1]),
                   emit_d2=True) as plan:
        host = plan.build(torch.from_numpy(x).cuda(), r, frnn._native.FRNN_NO_CAP).to_host()
        assert plan.last_status() == 0
    np.testing.assert_array_equal(host["row_ptr"], rp)
    long_rows = 0
    for i in range(x.shape[0]):
        a, b = rp[i], rp[i + 1]
        if b - a <= 32:
            np.testing.assert_array_equal(host["col"][a:b], col[a:b])
            np.testing.assert_array_equal(host["d2"][a:b], d2[a:b])
        else:
            long_rows += 1
            o = np.argsort(host["col"][a:b])
            assert sorted(zip(col[a:b].tolist(), d2[a:b].tolist())) == \
                list(zip(host["col"][a:b][o].tolist(), host["d2"][a:b][o].tolist()))
    if kind == "dense":
        assert long_rows > 1000
