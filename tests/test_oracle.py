"""Pins for the CPU oracle, checked against things other than the oracle itself.

* hand-enumerated fixtures (tests/golden/), read from the definition of the
  graph (Sec. 2, Sec. 3.4) and of the neighbour cap (Sec. 3.1);
* closed forms: points on a line, lattice ball counts;
* a host library: scipy's cKDTree (ball query for the uncapped graph, k-nearest
  query for the capped rows);
* exact rational arithmetic (float64 / integer) for every distance decision on
  grid inputs, and the float32 rounding bound off the grid;
* invariants of the radius graph (symmetry, no self loops, ordering, the cap);
* mutation checks: a copy of the oracle with one plausible mistake planted
  must fail at least one pin.
"""
import os
import re
import shutil
import subprocess
import tempfile

import numpy as np
import pytest
from scipy.spatial import cKDTree

import oracle
from paper_2202_06929_b300 import synth
from tests import golden_io


# --------------------------------------------------------------------------- helpers

def exact_q(m, i, j):
    """Squared distance in grid units (integer), from integer coordinates."""
    diff = m[i].astype(np.int64) - m[j].astype(np.int64)
    return int(np.dot(diff, diff))


def rows_of(row_ptr, col):
    return [col[row_ptr[i]:row_ptr[i + 1]].tolist() for i in range(len(row_ptr) - 1)]


def ckdtree_ball(x, r):
    """Uncapped neighbour sets from cKDTree for grid inputs.

    Grid squared distances are integers q / 65536, and the edge test is
    q <= thr; a ball of radius sqrt((thr + 0.5) / 65536) separates q = thr from
    q = thr + 1 with room to spare for double rounding."""
    thr = oracle.grid_threshold(r)
    rb = np.sqrt((thr + 0.5) / 65536.0)
    tree = cKDTree(x.astype(np.float64))
    sets = tree.query_ball_point(x.astype(np.float64), rb, p=2.0)
    return [sorted(j for j in s if j != i) for i, s in enumerate(sets)]


# --------------------------------------------------------------------------- fixtures

@pytest.mark.parametrize("name", golden_io.names())
def test_golden_float(name):
    g = golden_io.load(name)
    rp, col = oracle.radius_graph(g["x"], g["r"], g["k"])
    assert rp.tolist() == g["row_ptr"].tolist()
    assert col.tolist() == g["col"].tolist()


@pytest.mark.parametrize("name", golden_io.names())
def test_golden_grid(name):
    g = golden_io.load(name)
    rp, col = oracle.radius_graph_grid(g["m"], oracle.grid_threshold(g["r"]), g["k"])
    assert rp.tolist() == g["row_ptr"].tolist()
    assert col.tolist() == g["col"].tolist()


def test_grid_threshold_values():
    # r = 0.1: r2 = fl32(0.1f * 0.1f) = 0.010000000707805156..., * 65536 = 655.36...
    assert oracle.grid_threshold(0.1) == 655
    # r = 0.15: 1474.56 -> 1474;  r = 0.125: exactly 1024 (boundary kept)
    assert oracle.grid_threshold(0.15) == 1474
    assert oracle.grid_threshold(0.125) == 1024
    assert oracle.grid_threshold(5 / 256) == 25


# --------------------------------------------------------------------------- closed forms

@pytest.mark.parametrize("L", [1, 2, 3, 4, 5, 17, 64])
def test_line_closed_form(L):
    """Points m/256, m = 0..L-1, radius 2.5 steps: rows are m +- 1, m +- 2."""
    x = np.zeros((L, 3), dtype=np.float32)
    x[:, 0] = np.arange(L) / 256.0
    rp, col = oracle.radius_graph(x, 2.5 / 256, 0)
    expect_e = {1: 0, 2: 2, 3: 6}.get(L, 4 * L - 6)
    assert rp[-1] == expect_e
    rows = rows_of(rp, col)
    for m in range(L):
        want = [j for j in (m - 1, m + 1, m - 2, m + 2) if 0 <= j < L]
        assert rows[m] == want
    rp3, col3 = oracle.radius_graph(x, 2.5 / 256, 3)
    for m, row in enumerate(rows_of(rp3, col3)):
        want = [j for j in (m - 1, m + 1, m - 2, m + 2) if 0 <= j < L][:3]
        assert row == want


def lattice_pair_count(side, q_max, d):
    """Ordered pairs of a side^d integer lattice at squared distance 1..q_max,
    counted over offset vectors v: each v fits prod(side - |v_t|) times."""
    import itertools
    tot = 0
    rng = range(-(side - 1), side)
    for v in itertools.product(rng, repeat=d):
        q = sum(c * c for c in v)
        if 0 < q <= q_max:
            tot += int(np.prod([side - abs(c) for c in v]))
    return tot


@pytest.mark.parametrize("r_steps,q_max,centre_deg", [(1.5, 2, 18), (1.8, 3, 26), (2.1, 4, 32)])
def test_lattice_ball(r_steps, q_max, centre_deg):
    side = 7
    g = np.stack(np.meshgrid(*[np.arange(side) - 3] * 3, indexing="ij"), -1).reshape(-1, 3)
    x = (g / 256.0).astype(np.float32)
    r = r_steps / 256
    deg = oracle.degree(x, r)
    centre = int(np.flatnonzero((g == 0).all(1))[0])
    assert deg[centre] == centre_deg
    assert deg.sum() == lattice_pair_count(side, q_max, 3)


def test_identical_points_keep_lowest_indices():
    n, k = 50, 7
    x = np.tile(np.array([[0.25, -0.5, 0.75, 0.0]], dtype=np.float32), (n, 1))
    rp, col = oracle.radius_graph(x, 1 / 256, k)
    for i, row in enumerate(rows_of(rp, col)):
        assert row == [j for j in range(n) if j != i][:k]


def test_radius_boundary_is_inclusive():
    # r = 0.125 -> r2 = 1/64 exactly; a pair exactly 32 grid steps apart is kept
    x = np.array([[0.0, 0.0], [0.125, 0.0], [0.0, 0.12890625]], dtype=np.float32)
    rp, col = oracle.radius_graph(x, 0.125, 0)
    assert rows_of(rp, col) == [[1], [0], []]


def test_empty_and_single():
    rp, col = oracle.radius_graph(np.zeros((0, 4), np.float32), 0.1, 8)
    assert rp.tolist() == [0] and col.size == 0
    rp, col = oracle.radius_graph(np.zeros((1, 4), np.float32), 0.1, 8)
    assert rp.tolist() == [0, 0] and col.size == 0


# --------------------------------------------------------------------------- library: cKDTree

CASES = [
    ("uniform", lambda: synth.uniform_grid(1500, 3, 11, -40, 40), 0.05),
    ("clustered8", lambda: synth.clustered_grid(2500, 8, 12, 150, 0.03, 0.2), 0.1),
    ("clustered5", lambda: synth.clustered_grid(1200, 5, 13, 60, 0.02, 0.1), 0.07),
    ("c1", lambda: synth.make_event("c1"), 0.1),
    ("dups", lambda: synth.duplicates(800, 4, 14, 90), 0.03),
]


@pytest.mark.parametrize("name,make,r", CASES, ids=[c[0] for c in CASES])
def test_uncapped_equals_ckdtree_ball(name, make, r):
    x = make()
    rp, col = oracle.radius_graph(x, r, 0)
    want = ckdtree_ball(x, r)
    got = [sorted(row) for row in rows_of(rp, col)]
    assert got == want


@pytest.mark.parametrize("name,make,r", CASES, ids=[c[0] for c in CASES])
@pytest.mark.parametrize("k", [1, 3, 16])
def test_capped_distances_equal_ckdtree_knn(name, make, r, k):
    """The capped row's distances are the k smallest within r (tie-insensitive)."""
    x = make()
    m = oracle.to_grid_ints(x)
    rp, col = oracle.radius_graph(x, r, k)
    thr = oracle.grid_threshold(r)
    rb = np.sqrt((thr + 0.5) / 65536.0)
    tree = cKDTree(m.astype(np.float64))
    dist, _ = tree.query(m.astype(np.float64), k=k + 1, distance_upper_bound=np.sqrt(thr + 0.5))
    for i in range(x.shape[0]):
        dd = dist[i][np.isfinite(dist[i])]
        q_tree = sorted(int(round(v * v)) for v in dd)
        q_tree.remove(0)  # the query itself (or an equal duplicate: same value)
        q_row = [exact_q(m, i, j) for j in col[rp[i]:rp[i + 1]]]
        assert q_row == q_tree[:k], i
    assert rb > 0


# --------------------------------------------------------------------------- invariants

@pytest.mark.parametrize("name,make,r", CASES, ids=[c[0] for c in CASES])
def test_invariants(name, make, r):
    x = make()
    n = x.shape[0]
    m = oracle.to_grid_ints(x)
    thr = oracle.grid_threshold(r)
    k = 4
    rp0, col0 = oracle.radius_graph(x, r, 0)
    rows0 = rows_of(rp0, col0)
    rp, col, d2 = oracle.radius_graph(x, r, k, with_d2=True)
    rows = rows_of(rp, col)
    edges0 = set()
    for i, row in enumerate(rows0):
        assert i not in row
        for j in row:
            assert exact_q(m, i, j) <= thr
            edges0.add((i, j))
    assert all((j, i) in edges0 for (i, j) in edges0)          # symmetric before the cap
    # an independent pair count: each unordered pair once, times two
    d2all = ((m[:, None, :].astype(np.int64) - m[None, :, :]) ** 2).sum(-1)
    iu = np.triu_indices(n, 1)
    assert 2 * int((d2all[iu] <= thr).sum()) == rp0[-1]
    assert rp[-1] == sum(min(len(r0), k) for r0 in rows0)
    for i, row in enumerate(rows):
        keys = [(exact_q(m, i, j), j) for j in row]
        assert keys == sorted(keys) and len(set(keys)) == len(keys)  # strictly increasing
        assert set(row) <= set(rows0[i])
        if len(rows0[i]) > k:
            last = keys[-1]
            for j in set(rows0[i]) - set(row):
                assert (exact_q(m, i, j), j) > last
        # reported d2 is the exact grid value
        np.testing.assert_array_equal(d2[rp[i]:rp[i + 1]] * 65536.0,
                                      np.array([q for q, _ in keys], dtype=np.float64))


@pytest.mark.parametrize("r,k", [(0.1, 64), (0.1, 5), (0.15, 0), (0.05, 2)])
def test_grid_oracle_equals_float_oracle(r, k):
    x = synth.make_event("c1")
    rp, col = oracle.radius_graph(x, r, k)
    rpg, colg = oracle.radius_graph_grid(oracle.to_grid_ints(x), oracle.grid_threshold(r), k)
    np.testing.assert_array_equal(rp, rpg)
    np.testing.assert_array_equal(col, colg)


def test_query_subset_rows_match_full_rows():
    x = synth.clustered_grid(3000, 8, 21, 200, 0.03, 0.15)
    rp, col = oracle.radius_graph(x, 0.1, 8)
    q = np.random.default_rng(0).choice(3000, 300, replace=False)
    rpq, colq = oracle.radius_graph(x, 0.1, 8, queries=q)
    full = rows_of(rp, col)
    assert rows_of(rpq, colq) == [full[i] for i in q]


@pytest.mark.parametrize("d", [1, 3, 8, 13])
def test_offgrid_float32_within_rounding_bound(d):
    """Off the grid the float32 squared distance is rounded; it must lie within
    (d + 2) * 2^-24 (relative) of the exact value, and the edge decision must
    agree with the exact test outside that band."""
    x = synth.uniform_float(700, d, 30 + d, 0.3)
    r = 0.11
    r2 = float(np.float32(np.float32(r) * np.float32(r)))
    rp, col, d2 = oracle.radius_graph(x, r, 0, with_d2=True)
    xd = x.astype(np.float64)
    exact = ((xd[:, None, :] - xd[None, :, :]) ** 2).sum(-1)
    tol = (d + 2) * 2.0 ** -24
    rows = rows_of(rp, col)
    for i in range(x.shape[0]):
        ex = exact[i, col[rp[i]:rp[i + 1]]]
        assert np.all(np.abs(d2[rp[i]:rp[i + 1]] - ex) <= tol * ex + 1e-30)
        sure_in = set(np.flatnonzero(exact[i] <= r2 * (1 - tol)).tolist()) - {i}
        sure_out = set(np.flatnonzero(exact[i] > r2 * (1 + tol)).tolist())
        assert sure_in <= set(rows[i])
        assert not (sure_out & set(rows[i]))


# --------------------------------------------------------------------------- mutations

def _pins_pass():
    """A compact set of the pins above; False if any fails or raises."""
    try:
        for name in golden_io.names():
            g = golden_io.load(name)
            rp, col = oracle.radius_graph(g["x"], g["r"], g["k"])
            if rp.tolist() != g["row_ptr"].tolist() or col.tolist() != g["col"].tolist():
                return False
        x = synth.clustered_grid(600, 8, 5, 40, 0.03, 0.2)
        rp, col = oracle.radius_graph(x, 0.1, 0)
        if [sorted(r) for r in rows_of(rp, col)] != ckdtree_ball(x, 0.1):
            return False
        n = 12
        xi = np.tile(np.array([[0.5, 0.5]], np.float32), (n, 1))
        rp, col = oracle.radius_graph(xi, 1 / 256, 3)
        if rows_of(rp, col) != [[j for j in range(n) if j != i][:3] for i in range(n)]:
            return False
        return True
    except Exception:
        return False


MUTANTS = {
    "strict_radius": [("if (v <= r2)", "if (v < r2)"), ("<= r2) ++c", "< r2) ++c")],
    "dropped_last_term": [("for (int t = 0; t < d; ++t) {\n        float diff",
                           "for (int t = 0; t < d - 1; ++t) {\n        float diff")],
    "wrong_sign": [("float diff = a[t] - b[t];", "float diff = a[t] + b[t];")],
    "tie_break_reversed": [("    return (u->j > v->j) - (u->j < v->j);\n}\n\nstatic int fo_cmp_hit_grid",
                            "    return (u->j < v->j) - (u->j > v->j);\n}\n\nstatic int fo_cmp_hit_grid")],
    "self_loops": [("if (j == i) continue;\n            if (fo_dist2", "if (fo_dist2"),
                   ("if (j == i) continue;\n                float v", "float v")],
    "transposed_index": [("fo_dist2(x + i * d, x + j * d, d)", "fo_dist2(x + i * d, x + j, d)")],
    "cap_off_by_one": [("int64_t keep = (k > 0 && m > k) ? k : m;",
                        "int64_t keep = (k > 0 && m >= k) ? k - 1 : m;")],
}


@pytest.mark.parametrize("mutant", sorted(MUTANTS))
def test_pins_reject_planted_mistake(mutant):
    src = open(oracle._SRC).read()
    for old, new in MUTANTS[mutant]:
        assert old in src, (mutant, old)
        src = src.replace(old, new)
    tmp = tempfile.mkdtemp(prefix="oracle_mut_")
    try:
        c = os.path.join(tmp, "m.c")
        so = os.path.join(tmp, "m.so")
        open(c, "w").write(src)
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-std=c11",
                               "-shared", "-fPIC", "-o", so, c])
        prev = oracle.use_library(so)
        try:
            assert not _pins_pass(), f"pins did not notice mutant {mutant}"
        finally:
            oracle.use_library(prev)
    finally:
        shutil.rmtree(tmp, ignore_errors=True)


def test_pins_pass_on_the_real_oracle():
    assert _pins_pass()


# --------------------------------------------------------------------------- track labeling

def test_components_closed_forms():
    # a chain 0-1-2-3 given by one directed edge per link, and two isolated points
    rp = np.array([0, 1, 2, 3, 3, 3, 3])
    col = np.array([1, 2, 3], np.int32)
    assert oracle.components(rp, col).tolist() == [0, 0, 0, 0, 4, 5]
    # the same links pointing the other way: weak connectivity ignores direction
    rp = np.array([0, 0, 1, 2, 3, 3, 3])
    col = np.array([0, 1, 2], np.int32)
    assert oracle.components(rp, col).tolist() == [0, 0, 0, 0, 4, 5]
    # a weight cut splits the chain
    w = np.array([0.1, 0.9, 0.1], np.float32)
    assert oracle.components(rp, col, w, 0.5).tolist() == [0, 0, 2, 2, 4, 5]


@pytest.mark.parametrize("cut", [1.0, 0.5, 0.2])
def test_components_equal_networkx(cut):
    import networkx as nx
    x = synth.clustered_grid(2500, 8, 41, 120, 0.03, 0.2)
    r, k = 0.1, 8
    rp, col, d2 = oracle.radius_graph(x, r, k, with_d2=True)
    d2_max = float(np.float32(cut * cut * r * r))
    labels = oracle.components(rp, col, d2, d2_max)
    g = nx.Graph()
    g.add_nodes_from(range(x.shape[0]))
    for i in range(x.shape[0]):
        for e in range(rp[i], rp[i + 1]):
            if d2[e] <= np.float32(d2_max):
                g.add_edge(i, int(col[e]))
    want = np.empty(x.shape[0], np.int32)
    for comp in nx.connected_components(g):
        want[list(comp)] = min(comp)
    np.testing.assert_array_equal(labels, want)


# --------------------------------------------------------------------------
# exact kNN (no radius cut), Sec. 3.1 without the cut

def test_knn_line_closed_form():
    # points m/256 on axis 0, m = 0..L-1: row m takes its k nearest by (d2, j);
    # with k = 3 an interior row is [m-1, m+1, m-2] (d2 1, 1, 4 grid steps^2,
    # the tie broken by index), the ends reach three steps along the line
    L = 12
    x = np.zeros((L, 2), np.float32)
    x[:, 0] = np.arange(L) / 256.0
    rp, col, d2 = oracle.knn_graph(x, 3, with_d2=True)
    rows = rows_of(rp, col)
    step2 = np.float32(1 / 256.0) ** 2
    assert rows[0] == [1, 2, 3] and rows[L - 1] == [L - 2, L - 3, L - 4]
    assert rows[1] == [0, 2, 3]
    for m in range(2, L - 2):
        assert rows[m] == [m - 1, m + 1, m - 2]
    assert np.allclose(d2[rp[5]:rp[6]], np.array([1, 1, 4], np.float32) * step2)


def test_knn_small_event_takes_every_point():
    # n <= k + 1: every other point, sorted by (d2, j)
    x = np.array([[0, 0], [3, 0], [1, 0], [1, 0]], np.float32) / 256.0
    rp, col = oracle.knn_graph(x, 8)
    assert rows_of(rp, col) == [[2, 3, 1], [2, 3, 0], [3, 0, 1], [2, 0, 1]]


def test_knn_identical_points_keep_lowest_indices():
    x = np.zeros((9, 3), np.float32)
    rp, col = oracle.knn_graph(x, 4)
    rows = rows_of(rp, col)
    for i in range(9):
        assert rows[i] == [j for j in range(9) if j != i][:4]


@pytest.mark.parametrize("seed,n,d,k", [(0, 400, 3, 1), (1, 700, 8, 16), (2, 300, 12, 40)])
def test_knn_distances_equal_ckdtree(seed, n, d, k):
    # on the 1/256 grid d2 is exact in float32, so the row's d2 sequence
    # equals cKDTree's k nearest distances squared (ties are index-free here)
    from scipy.spatial import cKDTree
    rng = np.random.default_rng(seed)
    x = (np.rint(rng.uniform(-1, 1, (n, d)) * 256) / 256).astype(np.float32)
    rp, col, d2 = oracle.knn_graph(x, k, with_d2=True)
    dist, idx = cKDTree(x.astype(np.float64)).query(x.astype(np.float64), k + 1)
    for i in range(n):
        ref = np.sort(dist[i] ** 2)[1:]  # the query itself is one of the zero distances
        got = d2[rp[i]:rp[i + 1]].astype(np.float64)
        assert got.size == k
        assert np.allclose(got, ref, rtol=1e-9, atol=0)
        assert np.all(np.diff(got) >= 0)
        assert i not in set(col[rp[i]:rp[i + 1]].tolist())
