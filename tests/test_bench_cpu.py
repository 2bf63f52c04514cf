"""Host-side helpers of bench.py: the candidate recount that feeds the
reported arithmetic view, checked against a direct count of the points in
each query's neighbouring cells."""
import importlib.util
import itertools
import os

import numpy as np

from paper_2202_06929_b300 import synth

_spec = importlib.util.spec_from_file_location(
    "bench_module", os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "bench.py"))
bench = importlib.util.module_from_spec(_spec)
_spec.loader.exec_module(bench)


def direct_candidates(x, r, g, cells_per_point=32):
    # same grid rule (widest dims first, >= 4 cells each, table within the
    # event's budget of cells_per_point * n + 4096 cells), counted query by
    # query with a dictionary of cells
    x = x.astype(np.float32)
    lo = x.min(0)
    w = (x.max(0) - lo).astype(np.float32)
    order = np.argsort(-w, kind="stable")
    s = np.float32(r) * np.float32(1.0) * np.float32(1 + 1 / 64)
    dims, ncs, cells = [], [], 1
    budget = cells_per_point * x.shape[0] + 4096
    for i in range(g):
        t = int(order[i])
        nc = int(w[t] / s) + 1
        if dims and (nc < 4 or cells * nc > budget):
            break
        dims.append(t)
        ncs.append(nc)
        cells *= nc
    k = np.minimum(((x[:, dims] - lo[dims]) * (np.float32(1) / s)).astype(np.int64), np.array(ncs) - 1)
    cells = {}
    for c in map(tuple, k):
        cells[c] = cells.get(c, 0) + 1
    tot = []
    for c in map(tuple, k):
        n = 0
        for off in itertools.product((-1, 0, 1), repeat=len(dims)):
            n += cells.get(tuple(a + b for a, b in zip(c, off)), 0)
        tot.append(n)
    return float(np.mean(tot)), len(dims)


def test_host_candidates_equal_direct_count():
    x = synth.clustered_grid(3000, 8, 3, 150, 0.03)
    for g, cpp in ((2, 32), (3, 32), (4, 32), (4, 64)):
        want, g_want = direct_candidates(x, 0.1, g, cpp)
        got, g_got = bench.host_candidates(x, 0.1, g, 1.0, cpp, sample=10 ** 9)
        assert g_got == g_want
        assert abs(got - want) < 1e-9


def test_host_cell_slots_sum_each_events_grid():
    # the grid rule restated here (widest dims first while each has >= 4 cells
    # and the table stays within the budget), one slot for an empty event
    def direct(x, r, g, cpp):
        lo = x.min(0)
        w = (x.max(0) - lo).astype(np.float32)
        order = np.argsort(-w, kind="stable")
        s = np.float32(r) * np.float32(1 + 1 / 64)
        cells, used = 1, 0
        for i in range(g):
            nc = int(w[int(order[i])] / s) + 1
            if used and (nc < 4 or cells * nc > cpp * x.shape[0] + 4096):
                break
            cells *= nc
            used += 1
        return cells
    evs = [synth.clustered_grid(n, 8, 11 + n, max(n // 10, 1), 0.03) for n in (3000, 500, 40)]
    evs.insert(1, np.zeros((0, 8), np.float32))
    off = np.concatenate([[0], np.cumsum([len(e) for e in evs])])
    x = np.concatenate(evs)
    for g, cpp in ((2, 32), (4, 32), (6, 4)):
        want = sum(direct(e, 0.1, g, cpp) if len(e) else 1 for e in evs)
        assert bench.host_cell_slots(x, off, 0.1, g, 1.0, cpp) == want


def test_stage_bytes_total_matches_whole_build_terms():
    b = bench.stage_bytes(1000, 5000, 8, cells=777)
    assert b["scan_cells"] == 12 * 777
    assert b["walk_collect"] == 4 * 1000 * 8 + 12 * 1000 + 4 * 5000
    assert b["scan_rows"] == 12 * 1000 + 8 * 5000
    # scatter stage: the scatter's moves and the filter keys read back from the sorted rows
    assert b["scatter"] == (4 * 1000 * 8 + 16 * 1000 + 4 * 1000 * 8) + (4 * 1000 * 8 + 4 * 1000)


def test_edge_feature_bytes_counts_outputs_columns_and_rows():
    # per edge: (2d + 1) float32 outputs, its column, the neighbour's row;
    # per row: the query's row and its offset
    d = 8
    assert bench.edge_feature_bytes(1, 0, d) == 4 * 17 + 4 + 32
    assert bench.edge_feature_bytes(800_000, 70_000, d) == 800_000 * 104 + 70_000 * 36
    assert bench.edge_feature_bytes(0, 5, 12) == 5 * 52
