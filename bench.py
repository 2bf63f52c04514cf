"""Benchmark of the fixed-radius nearest-neighbour graph build on B300.

Workload (the graph-building step of the paper's pipeline, Sec. 3.4 / Table 1,
on synthetic TrackML-shaped embeddings): events of N=120,000 points, D=8
float32 coordinates on the 1/256 grid, r=0.1, K=256.  A step builds the graphs
of a batch of 64 such events (each with its own seed) in one batched build
replayed from a captured CUDA graph.  Beside it:

* plain: the same events built one per call (one graph replay per event),
  with per-event device latency p50/p99;
* e2e: the batched build through the host-to-host C call
  (frnn_build_graph_host): points copied from pinned host memory, the whole
  CSR copied back, all inside the timed region;
* roofline: per-stage device times from CUDA events between the stages
  (frnn_build_graph_profiled) for the dominant kernel, against the measured
  HBM bandwidth;
* cpu_baseline: the CPU oracle (brute force, OpenMP) on a bounded sample of
  queries of one event, scaled to events/s.

`--impl reference` times the CPU oracle alone as the reference arm.
Multi-GPU (torchrun): every rank builds its own events (replicas, no
collective on the data path); the step time is the max over ranks.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_2202_06929_b300 import synth  # noqa: E402

METRIC = "FRNN graph-build events/s at N=120k,D=8 batched vs plain; p50/p99 latency"
UNIT = "events/s"
N_PER_EVENT, D, R, K = 120_000, 8, 0.1, 256
KERNELS_PER_BUILD = 9  # with the query-major walk; the candidate-major walk is launched twice (one returns at once)
STAGES = ("bbox_plan", "key_hist", "scan_cells", "scatter", "walk_collect", "scan_rows", "walk_emit")
L2_BYTES = 126 * 1024 * 1024
KFAST_ROWS = 24  # rows longer than this are walked a second time by the emit walk
KNN_K = 16       # k of the exact-kNN measurement
AUTOTUNE_SPACE = ("20 grids (g_max in {6,5,4,3,2} x cell_scale in {1,1.25,1.5,2}) probed for their exact "
                  "candidate tests, non-empty cells and cell slots; the 3 cheapest timed with both walk forms "
                  "(best of 3 builds)")
# DRAM read + write bytes per point and warp instructions per query of the
# collect walk, from one ncu capture of the N=120k workload (40 events, 4.8 M
# points); valid only for the kernel code it was taken on (the sha1 of the
# kernel file without comments) and the walk form it ran.
MEASURED_COLLECT = {"workload": "c2", "stage": "walk_collect", "walk": 2, "source_sha1_prefix": "92bbb52820ee",
                    "bytes_per_point": (240_564_224 + 212_406_784) / 4_800_000,
                    "instr_per_query": 1_008_893_392 / 4_800_000}


def parse_args(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--workload", choices=["c2", "c3", "c5", "c5b"], default="c2",
                    help="c2: N=120k events (the headline); c3: N~U[40k,140k], K=64; "
                         "c5/c5b: N=1M, D=12, r=0.15, K=128 (c5b: the cap binds)")
    ap.add_argument("--events", type=int, default=None, help="events per batched step (64; 8 for c5/c5b)")
    ap.add_argument("--no-autotune", action="store_true")
    ap.add_argument("--walk", choices=["tuned", "auto", "candidates", "queries"], default="tuned",
                    help="form of the neighbour walk: the autotuner's choice (tuned), or forced")
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--cpu-queries", type=int, default=40_000,
                    help="queries of the CPU oracle sample (bounded CPU work)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--e2e-slots", type=int, default=3, help="server slots of the end-to-end measurement")
    ap.add_argument("--e2e-batch", type=int, default=0, help="events per server batch (default: an eighth of a step)")
    ap.add_argument("--no-served", action="store_true")
    ap.add_argument("--served-requests", type=int, default=2000,
                    help="measured requests per offered load (plus 200 warm-up)")
    return ap.parse_args(argv)


# --------------------------------------------------------------------------- distributed

def dist_setup(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    pg = None
    if world > 1:
        import torch
        import torch.distributed as dist
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        dist.init_process_group(backend=backend)
        pg = dist
    return rank, world, local, pg


def barrier(pg):
    if pg is not None:
        pg.barrier()


def max_over_ranks(pg, value: float, device=None) -> float:
    if pg is None:
        return value
    import torch
    t = torch.tensor([value], dtype=torch.float64, device=device)
    pg.all_reduce(t, op=pg.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(pg, value: float, device=None) -> float:
    if pg is None:
        return value
    import torch
    t = torch.tensor([value], dtype=torch.float64, device=device)
    pg.all_reduce(t, op=pg.ReduceOp.SUM)
    return float(t.item())


# --------------------------------------------------------------------------- workload

def make_batch(rank: int, n_events: int, workload: str = "c2"):
    """Events rank*n_events .. of a workload, concatenated (ranks never share events)."""
    evs = [synth.make_event(workload, rank * n_events + e) for e in range(n_events)]
    off = np.zeros(n_events + 1, dtype=np.int64)
    off[1:] = np.cumsum([e.shape[0] for e in evs])
    return np.ascontiguousarray(np.concatenate(evs)), off


def percentile(v, q):
    return float(np.percentile(np.asarray(v, dtype=np.float64), q)) if len(v) else None


# --------------------------------------------------------------------------- clocks

class ClockSampler:
    """nvidia-smi sampled every 100 ms; each sample is stamped with the host
    time it arrived.  Start it before the warm-up (`wait_first` waits for the
    first sample), bracket the timed region with `mark_start` / `mark_end`
    (which waits for one sample after the region); the summary uses the
    samples within 0.25 s of the region, so a region shorter than the
    sampling period still gets the samples on either side of it, taken while
    the warm-up or the region kept the GPU busy."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    PERIOD_MS = 100

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []
        self._t = None
        self.t0 = None
        self.t1 = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.QUERY}", "--format=csv,noheader,nounits",
                 "-lms", str(self.PERIOD_MS)], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self._t = threading.Thread(target=self._read, daemon=True)
            self._t.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append((time.perf_counter(), line.strip()))

    def _wait_until(self, cond, timeout: float):
        t_end = time.perf_counter() + timeout
        while self.proc is not None and not cond() and time.perf_counter() < t_end:
            time.sleep(0.01)

    def wait_first(self, timeout: float = 5.0):
        self._wait_until(lambda: len(self.lines) > 0, timeout)

    def mark_start(self):
        self.t0 = time.perf_counter()

    def mark_end(self):
        self.t1 = time.perf_counter()
        self._wait_until(lambda: any(t > self.t1 for t, _ in self.lines), 3 * self.PERIOD_MS / 1e3 + 1.0)

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            if self._t:
                self._t.join(timeout=2)

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        lo = (self.t0 if self.t0 is not None else -1e30) - 0.25
        hi = (self.t1 if self.t1 is not None else 1e30) + 0.25
        for t, ln in self.lines:
            if not (lo <= t <= hi):
                continue
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


# --------------------------------------------------------------------------- peaks

EDGE_BATCH = 800_000   # edges per filter batch (Sec. 3)


def edge_feature_bytes(batch_edges: int, rows: int, d: int) -> int:
    """Algorithmic bytes of one edge-feature batch: per edge the (2d + 1)
    float32 output, its column and the neighbour's row; per row touched the
    query's row and its row offset."""
    return batch_edges * (4 * (2 * d + 1) + 4 + 4 * d) + rows * (4 * d + 4)


def edge_feature_bench(plan, x_dev, csr, n_total, d, stream, dev, max_batches=20):
    import torch
    n_edges = csr.n_edges()
    nb = min(n_edges // EDGE_BATCH, max_batches)
    if nb < 1:
        return None
    outs = [torch.empty((EDGE_BATCH, 2 * d + 1), dtype=torch.float32, device=dev) for _ in range(4)]
    with torch.cuda.stream(stream):
        plan.edge_features(x_dev, 0, EDGE_BATCH, stream=stream, out=outs[0])
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for bi in range(nb):
            plan.edge_features(x_dev, bi * EDGE_BATCH, (bi + 1) * EDGE_BATCH, stream=stream, out=outs[bi % 4])
        e1.record(stream)
        e1.synchronize()
    if plan.last_status(stream) != 0:
        return None
    ms = e0.elapsed_time(e1) / nb
    row_ptr = csr.row_ptr[: n_total + 1].cpu().numpy().astype(np.int64)
    last = nb * EDGE_BATCH
    rows = int(np.searchsorted(row_ptr, last, side="left"))  # rows whose edges start before the last edge timed
    byts = edge_feature_bytes(EDGE_BATCH, max(1, rows // nb), d)
    hbm, kind = measured_peaks()
    gbs = byts / (ms / 1e3) / 1e9
    return {"batch_edges": EDGE_BATCH, "batches": nb, "ms_per_batch": ms, "edges_per_s": EDGE_BATCH / (ms / 1e3),
            "algorithmic_bytes_per_batch": byts, "achieved_gbs": gbs, "frac_of_hbm": gbs / hbm, "peak_kind": kind,
            "note": "frnn_edge_features over the step's first edges, device time per batch; bytes per edge: "
                    "(2d+1) float32 out + column + neighbour row; per row: its row and offset"}


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            m = json.load(f)
        return float(m["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6400.0, "fallback"


def walk_form(walk: int, d: int) -> int:
    """The collect walk a build runs (the rule of frnn_tuning.walk): the
    query-major form (2) for d <= 12 unless the candidate-major form (1) is
    asked for; candidate-major above."""
    return 1 if ((d + 3) // 4 > 3 or walk == 1) else 2


def kernel_source_sha1() -> str:
    """sha1 of the kernel source with // comments removed and whitespace runs
    collapsed: a capture stays valid across comment edits, not code edits."""
    import hashlib
    import re
    src = open(os.path.join(ROOT, "paper_2202_06929_b300", "csrc", "frnn_kernels.cu")).read()
    src = re.sub(r"\s+", " ", re.sub(r"//[^\n]*", "", src)).strip()
    return hashlib.sha1(src.encode()).hexdigest()


def measured_collect(stage: str, workload: str, walk: int):
    """The captured figures of the collect walk (MEASURED_COLLECT) when they
    describe this launch: same stage, workload, walk form and kernel code;
    else None."""
    m = MEASURED_COLLECT
    if workload != m["workload"] or stage != m["stage"] or walk != m["walk"]:
        return None
    try:
        sha = kernel_source_sha1()
    except OSError:
        return None
    return m if sha.startswith(m["source_sha1_prefix"]) else None


def stage_bytes(n_total: int, n_edges: int, d: int, long_edges: int = 0, long_rows: int = 0, cells: int = 0):
    """Algorithmic bytes of each stage for a batch (each stage's unavoidable
    reads of its inputs and writes of its outputs, counted once).  long_edges
    / long_rows: the edges and rows of the rows longer than the collect walk
    parks (the emit walk writes those); cells: the cell-table slots of the
    batch's grids."""
    dp = (d + 3) // 4 * 4
    parked = n_edges - long_edges
    return {
        "bbox_plan": 4 * n_total * d,
        "key_hist": 4 * n_total * d + 8 * n_total,
        # per cell slot its count read, its start written, its count cleared
        # for the next build
        "scan_cells": 12 * cells,
        # scatter (points moved, key and rank read, perm and cell id written)
        # and filter keys (sorted rows read, one 4-byte key written)
        "scatter": 4 * n_total * d + 8 * n_total + 4 * n_total * dp + 8 * n_total + 4 * n_total * dp + 4 * n_total,
        # sorted points read once; per point its cell id, count and pool slot; rows parked
        "walk_collect": 4 * n_total * dp + 4 * n_total + 8 * n_total + 4 * parked,
        # per point its count and pool slot read, row_ptr written; parked rows
        # read from the pool and written to col
        "scan_rows": 12 * n_total + 8 * parked,
        # the long rows: per row its list entry, count and offset read, its
        # columns written
        "walk_emit": 12 * long_rows + 4 * long_edges,
    }


def measure_link(torch, dev, h2d_bytes: int, d2h_bytes: int, reps: int = 5):
    """Pinned host <-> device copy bandwidth for a step's bytes: each
    direction alone and both at once on two streams (the bound of the end to
    end path, whose copies in and out overlap across server slots)."""
    hi = torch.empty(h2d_bytes // 4, dtype=torch.int32).pin_memory()
    ho = torch.empty(d2h_bytes // 4, dtype=torch.int32).pin_memory()
    di = torch.empty(h2d_bytes // 4, dtype=torch.int32, device=dev)
    do = torch.empty(d2h_bytes // 4, dtype=torch.int32, device=dev)
    s1, s2 = torch.cuda.Stream(dev), torch.cuda.Stream(dev)

    def timed(fn):
        fn()
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        for _ in range(reps):
            fn()
        torch.cuda.synchronize(dev)
        return (time.perf_counter() - t0) / reps

    def both():
        with torch.cuda.stream(s1):
            di.copy_(hi, non_blocking=True)
        with torch.cuda.stream(s2):
            ho.copy_(do, non_blocking=True)

    t_in = timed(lambda: di.copy_(hi, non_blocking=True))
    t_out = timed(lambda: ho.copy_(do, non_blocking=True))
    t_both = timed(both)
    return {"h2d_gbs": h2d_bytes / t_in / 1e9, "d2h_gbs": d2h_bytes / t_out / 1e9,
            "both_gbs": (h2d_bytes + d2h_bytes) / t_both / 1e9,
            "note": "pinned copies of one step's input and result sizes, each direction alone and both at once"}


def host_grid(x, r: float, g_max: int, cell_scale: float, cells_per_point: int):
    """The cell grid of one event, restated on the host from the planning
    rule (widest dims first, cell edge r * cell_scale * (1 + 2^-6), stop below
    4 cells or over the event's cell budget): (lo, cell edge, gridded dims,
    cells along each)."""
    x = np.ascontiguousarray(x, dtype=np.float32)
    n, dd = x.shape
    lo = x.min(0)
    w = (x.max(0) - lo).astype(np.float32)
    order = np.argsort(-w, kind="stable")
    npick = min(g_max or 4, 6, dd)
    s = np.float32(r) * np.float32(cell_scale or 1.0) * np.float32(1 + 1 / 64)
    budget = cells_per_point * n + 4096
    maxc0 = min(budget, 32768)
    if w[order[0]] / s > maxc0 - 3:
        s = np.float32(w[order[0]] / np.float32(maxc0 - 3) * np.float32(1 + 1 / 64))
    dims, ncs, cells = [], [], 1
    for i in range(npick):
        t = int(order[i])
        a = w[t] / s
        nc = 32768 if a >= 32767 else int(a) + 1
        if dims and (nc < 4 or cells * nc > budget):
            break
        dims.append(t)
        ncs.append(nc)
        cells *= nc
    return lo, s, dims, np.array(ncs)


def host_cell_slots(x, off, r: float, g_max: int, cell_scale: float, cells_per_point: int) -> int:
    """Cell-table slots of a batch (the cell scan's items): the product of the
    cells along the gridded dims of every event (one for an empty event)."""
    tot = 0
    for b in range(len(off) - 1):
        xb = x[off[b]:off[b + 1]]
        tot += int(np.prod(host_grid(xb, r, g_max, cell_scale, cells_per_point)[3])) if len(xb) else 1
    return tot


def host_candidates(x, r: float, g_max: int, cell_scale: float, cells_per_point: int, sample: int = 100_000,
                    seed: int = 3):
    """Mean number of candidates a query of this event is tested against by
    the walk (the points of the 3^g cells around its cell), recounted on the
    host over the grid of host_grid, over a random sample of queries."""
    x = np.ascontiguousarray(x, dtype=np.float32)
    n = x.shape[0]
    lo, s, dims, ncs = host_grid(x, r, g_max, cell_scale, cells_per_point)
    inv_s = np.float32(1) / s
    k = np.minimum(((x[:, dims] - lo[dims]) * inv_s).astype(np.int64), ncs - 1)
    cid = np.ravel_multi_index(k.T, ncs)
    start = np.concatenate([[0], np.cumsum(np.bincount(cid, minlength=int(np.prod(ncs))))])
    q = np.random.default_rng(seed).choice(n, size=min(sample, n), replace=False)
    kq = k[q]
    g = len(dims)
    tot = np.zeros(len(q), np.int64)
    import itertools
    for offs in itertools.product((-1, 0, 1), repeat=g - 1):
        kk = kq[:, :g - 1] + np.array(offs, dtype=np.int64)
        ok = np.all((kk >= 0) & (kk < ncs[:g - 1]), axis=1)
        kk = np.clip(kk, 0, ncs[:g - 1] - 1)
        c0 = np.ravel_multi_index(np.concatenate([kk, np.maximum(kq[:, g - 1:] - 1, 0)], 1).T, ncs)
        c1 = np.ravel_multi_index(np.concatenate([kk, np.minimum(kq[:, g - 1:] + 1, ncs[g - 1] - 1)], 1).T, ncs)
        tot += np.where(ok, start[c1 + 1] - start[c0], 0)
    return float(tot.mean()), g


# --------------------------------------------------------------------------- CPU oracle

def cpu_model() -> str:
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.startswith("model name"):
                    return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return "unknown"


def run_cpu_baseline(x, queries: int, seed: int = 0, r: float = R, k: int = K):
    import oracle
    n = x.shape[0]
    q = np.random.default_rng(seed).choice(n, size=min(queries, n), replace=False)
    t0 = time.perf_counter()
    oracle.radius_graph(x, r, k, queries=q)
    dt = time.perf_counter() - t0
    return {"value": (len(q) / n) / dt, "unit": UNIT, "cores": oracle.num_threads(), "cpu_model": cpu_model(),
            "kind": "oracle",
            "sample": f"{len(q)} random query rows of one N={n} event (brute force over all {n} points), "
                      f"{dt:.2f} s; events/s = (rows / N) / s"}


def run_cpu_single_core(x, queries: int, seed: int = 7, r: float = R, k: int = K):
    """The same oracle on one host core (OMP_NUM_THREADS=1, in a child process
    so that this process's OpenMP runtime keeps its thread count)."""
    import subprocess
    import tempfile
    with tempfile.TemporaryDirectory() as td:
        path = os.path.join(td, "event.npy")
        np.save(path, np.ascontiguousarray(x, dtype=np.float32))
        code = ("import json, sys, time; import numpy as np; sys.path.insert(0, {root!r}); import oracle; "
                "x = np.load({path!r}); n = x.shape[0]; "
                "q = np.random.default_rng({seed}).choice(n, size=min({queries}, n), replace=False); "
                "t0 = time.perf_counter(); oracle.radius_graph(x, {r!r}, {k}, queries=q); "
                "dt = time.perf_counter() - t0; "
                "print(json.dumps({{'rows': int(len(q)), 'n': int(n), 's': dt, 'threads': oracle.num_threads()}}))"
                ).format(root=ROOT, path=path, seed=seed, queries=int(queries), r=float(r), k=int(k))
        env = dict(os.environ, OMP_NUM_THREADS="1")
        res = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=600)
    if res.returncode != 0:
        return {"error": res.stderr.strip().splitlines()[-1] if res.stderr.strip() else f"exit {res.returncode}"}
    o = json.loads(res.stdout.strip().splitlines()[-1])
    return {"value": (o["rows"] / o["n"]) / o["s"], "unit": UNIT, "cores": o["threads"],
            "sample": f"{o['rows']} random query rows of the same event, {o['s']:.2f} s on one core"}


def reference_arm(args, rank, world):
    if rank != 0:
        return 0
    x = synth.make_event("c2", 0)
    steps, warm = [], []
    for i in range(args.warmup):
        warm.append(run_cpu_baseline(x, max(args.cpu_queries // 20, 100), seed=1000 + i))
    per_step_q = max(args.cpu_queries // max(args.steps, 1), 200)
    t0 = time.perf_counter()
    for i in range(args.steps):
        steps.append(run_cpu_baseline(x, per_step_q, seed=i))
    wall = time.perf_counter() - t0
    value = (args.steps * per_step_q / x.shape[0]) / wall
    cores = steps[0]["cores"]
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * wall / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": "c2: N=120000, D=8, r=0.1, K=256 (CPU oracle on a query sample per step)",
                   "n_per_event": N_PER_EVENT, "d": D, "r": R, "k": K},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": f"{per_step_q} random query rows of one N={N_PER_EVENT} event per step"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# --------------------------------------------------------------------------- served

def _trace_loads(srv, x_all, start, sizes, req, traces, warm, n_requests):
    out = []
    for f, rate, arr in traces:
        res = srv.run_trace(x_all, start[req], sizes[req], arr)
        lat = res["latency_s"][warm:] * 1e3
        span = arr[-1] - arr[warm] if req.size > warm + 1 else res["wall_s"]
        done_eps = n_requests / max(res["wall_s"] - arr[warm], 1e-9)
        out.append({"offered_x_capacity": f, "offered_events_per_s": rate,
                    "achieved_events_per_s": done_eps, "latency_ms_p50": percentile(lat, 50),
                    "latency_ms_p99": percentile(lat, 99), "arrival_span_s": span})
    return out


def run_served(frnn, torch, n_requests: int, pool_events: int = 48, seed: int = 7):
    """Served workload: events of N ~ U[20k, 200k] (the N=120k generator),
    D=8, r=0.1, K=256, Poisson arrivals at 0.25x..1.5x of the continuous
    batching server's measured capacity, host arrival to host rows.  The same
    arrival traces go through two servers within a 40 GB device budget:
    continuous batching (3 slots, up to 64 events per launch) and the plain
    form (1 slot, one event per launch).  Requests draw from a pool of
    distinct events (seeded)."""
    evs = [synth.make_event("c4", e) for e in range(pool_events)]
    sizes = np.array([e.shape[0] for e in evs], dtype=np.int64)
    start = np.concatenate([[0], np.cumsum(sizes)[:-1]]).astype(np.int64)
    x_all = torch.from_numpy(np.concatenate(evs)).pin_memory().numpy()
    rng = np.random.default_rng(seed)
    warm = 200
    req = rng.integers(0, pool_events, size=warm + n_requests)
    forms = {"batching": dict(batch_points=2_000_000, batch_events=64, slots=3),
             "plain": dict(batch_points=int(sizes.max()), batch_events=1, slots=1)}
    out = {"workload": "c4: N ~ U[20000, 200000] per event, D=8, r=0.1, K=256, Poisson arrivals",
           "requests_per_load": n_requests, "warmup_requests": warm, "event_pool": pool_events,
           "mem_budget_gb": 40, "latency_note": "arrival (host clock) to the event's CSR on the host"}
    traces = None
    for name in ("batching", "plain"):
        srv = frnn.Server(d=D, r=R, k=K, edges_per_point=32, mem_budget_bytes=40 << 30, **forms[name])
        try:
            # capacity: every request present at t = 0
            sat = srv.run_trace(x_all, start[req], sizes[req], np.zeros(req.size))
            capacity = req.size / sat["wall_s"]
            if traces is None:  # offered loads are fractions of the batching server's capacity
                traces = []
                for f in (0.25, 0.5, 1.0, 1.5):
                    rate = f * capacity
                    arr = np.cumsum(rng.exponential(1.0 / rate, size=req.size))
                    traces.append((f, rate, arr - arr[0]))
            loads = _trace_loads(srv, x_all, start, sizes, req, traces, warm, n_requests)
            out[name] = {**forms[name], "reserved_gb": srv.reserved_bytes() / 1e9,
                         "capacity_events_per_s": capacity, "loads": loads, "stats": srv.stats()}
        finally:
            srv.close()
    out["p99_winner_per_load"] = [
        {"offered_x_capacity": b["offered_x_capacity"],
         "winner": "batching" if b["latency_ms_p99"] <= p["latency_ms_p99"] else "plain",
         "p99_ms": {"batching": b["latency_ms_p99"], "plain": p["latency_ms_p99"]}}
        for b, p in zip(out["batching"]["loads"], out["plain"]["loads"])]
    return out


# --------------------------------------------------------------------------- GPU arm

def main(argv=None):
    args = parse_args(argv)
    rank, world, local, pg = dist_setup(args)
    if args.impl == "reference":
        rc = reference_arm(args, rank, world)
        if pg is not None:
            pg.destroy_process_group()
        return rc

    import torch
    import paper_2202_06929_b300 as frnn

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    wl = synth.WORKLOADS[args.workload]
    d, r, k = wl.d, wl.r, wl.k
    B = args.events or (8 if args.workload in ("c5", "c5b") else 64)
    x_host, off = make_batch(rank, B, args.workload)
    n_total = int(off[-1])
    n_max_event = int(np.max(np.diff(off)))
    x_dev = torch.from_numpy(x_host).to(dev)
    stream = torch.cuda.Stream(device=dev)
    epp = k if args.workload == "c5b" else 64  # edge slots per point (C5b rows hold up to K)

    cpp = 32  # cell slots per point: room for five or six gridded dims (the autotuner decides)
    # the million-point workloads have rows longer than the walk parks: room
    # to keep their neighbours (384 slots per row, 32 rows at a time)
    hits = (lambda n: 32 * 384 * (n // 32 + B)) if args.workload in ("c5", "c5b") else (lambda n: 0)
    plan = frnn.Plan(n_max=n_total, d_max=d, k_max_cap=k, events_max=B, edge_capacity=n_total * epp,
                     cells_per_point=cpp, use_graph=True, device=local, hit_capacity=hits(n_total))
    plan_one = frnn.Plan(n_max=n_max_event, d_max=d, k_max_cap=k, events_max=1,
                         edge_capacity=n_max_event * epp, cells_per_point=cpp, use_graph=True, device=local,
                         hit_capacity=hits(n_max_event))
    tuned = None
    if not args.no_autotune:
        t0 = time.perf_counter()
        with torch.cuda.stream(stream):
            g, scale, ms = plan.autotune(x_dev, off, r, k, stream=stream)
            g1, scale1, ms1 = plan_one.autotune(x_dev[int(off[0]):int(off[1])], off[:2], r, k, stream=stream)
        tuned = {"batched": {"g_max": g, "cell_scale": scale, "walk": plan.get_tuning()[2], "build_ms": ms},
                 "plain": {"g_max": g1, "cell_scale": scale1, "walk": plan_one.get_tuning()[2], "build_ms": ms1},
                 "seconds": time.perf_counter() - t0,
                 "searched": AUTOTUNE_SPACE, "cells_per_point": cpp}
    if args.walk != "tuned":
        w = {"auto": 0, "candidates": 1, "queries": 2}[args.walk]
        for pl in (plan, plan_one):
            g_, s_, _ = pl.get_tuning()
            pl.set_tuning(g_, s_, w)
    walk_used = walk_form(plan.get_tuning()[2], d)

    # ---- batched: the timed step
    with torch.cuda.stream(stream), ClockSampler(local) as clk:
        clk.wait_first()
        for _ in range(args.warmup):
            plan.build_batched(x_dev, off, r, k, stream=stream)
        st = plan.last_status(stream)
        if st != 0:
            raise RuntimeError(f"warm-up status: {frnn.status_string(st)}")
        n_edges = int(plan.build_batched(x_dev, off, r, k, stream=stream).n_edges())
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
        barrier(pg)
        torch.cuda.synchronize(dev)
        clk.mark_start()
        ev[0].record(stream)
        for i in range(args.steps):
            plan.build_batched(x_dev, off, r, k, stream=stream)
            ev[i + 1].record(stream)
        torch.cuda.synchronize(dev)
        clk.mark_end()
        barrier(pg)
    st = plan.last_status(stream)
    if st != 0:
        raise RuntimeError(f"timed-region status: {frnn.status_string(st)}")
    step_ms = [ev[i].elapsed_time(ev[i + 1]) for i in range(args.steps)]
    total_ms = ev[0].elapsed_time(ev[-1])
    total_ms_max = max_over_ranks(pg, total_ms, dev)
    events_all = sum_over_ranks(pg, float(B * args.steps), dev)
    value = events_all / (total_ms_max / 1e3)

    # ---- plain: one event per call plus a stream sync, timed per event with
    # CUDA events (device latency) and the host clock (call to sync), cycling
    # through the batch's events (the batch is 2x larger than L2, so each
    # event's input is cold when reused)
    plain_ms = []
    plain_host_ms = []
    with torch.cuda.stream(stream):
        for e in range(min(B, 4)):
            lo, hi = int(off[e]), int(off[e + 1])
            plan_one.build(x_dev[lo:hi], r, k, stream=stream)
        pe0, pe1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize(dev)
        for e in range(B):
            lo, hi = int(off[e]), int(off[e + 1])
            t0 = time.perf_counter()
            pe0.record(stream)
            plan_one.build(x_dev[lo:hi], r, k, stream=stream)
            pe1.record(stream)
            pe1.synchronize()
            plain_host_ms.append(1e3 * (time.perf_counter() - t0))
            plain_ms.append(pe0.elapsed_time(pe1))
    st = plan_one.last_status(stream)
    if st != 0:
        raise RuntimeError(f"plain status: {frnn.status_string(st)}")
    plain_value = B / (sum(plain_host_ms) / 1e3)

    # ---- track labeling (connected components of the built graph, every edge kept)
    labeling = None
    with torch.cuda.stream(stream):
        csr_last = plan.build_batched(x_dev, off, r, k, stream=stream)
        lab = torch.empty(n_total, dtype=torch.int32, device=dev)
        plan.label_components(float("inf"), stream=stream, out=lab)
        le0, le1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        lab_ms = []
        for _ in range(5):
            le0.record(stream)
            plan.label_components(float("inf"), stream=stream, out=lab)
            le1.record(stream)
            le1.synchronize()
            lab_ms.append(le0.elapsed_time(le1))
    if plan.last_status(stream) == 0:
        n_tracks = int((lab.cpu().numpy() == np.arange(n_total) - np.repeat(off[:-1], np.diff(off))).sum())
        lab_bytes = 4 * (n_total + 1) + 4 * n_edges + 4 * n_total  # row offsets and columns read, labels written
        lab_gbs = lab_bytes / (float(np.median(lab_ms)) / 1e3) / 1e9
        labeling = {"ms_per_step": float(np.median(lab_ms)), "components_per_step": n_tracks,
                    "algorithmic_bytes": lab_bytes, "achieved_gbs": lab_gbs,
                    "frac_of_hbm": lab_gbs / measured_peaks()[0],
                    "note": "frnn_label_components: weakly connected components of the step's graphs "
                            "(all edges kept), 4 kernels, after the build on the same stream; bytes: row "
                            "offsets and columns read once, labels written once"}

    # ---- edge features for the filter stage: [x_i, x_j, d2] per edge of the same
    # graph, in 800k-edge batches (the filter network's batch, Sec. 3); outputs
    # rotate over 4 buffers (218 MB, more than L2)
    edge_features = edge_feature_bench(plan, x_dev, csr_last, n_total, d, stream, dev)

    # ---- exact k nearest neighbours (no radius) of the same batch
    knn = None
    knn_k = KNN_K
    if n_total * knn_k <= plan.edge_capacity:
        with torch.cuda.stream(stream):
            plan.knn_batched(x_dev, off, knn_k, stream=stream)
            ke0, ke1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            knn_ms = []
            for _ in range(5):
                ke0.record(stream)
                plan.knn_batched(x_dev, off, knn_k, stream=stream)
                ke1.record(stream)
                ke1.synchronize()
                knn_ms.append(ke0.elapsed_time(ke1))
        if plan.last_status(stream) == 0:
            kms = float(np.median(knn_ms))
            knn_bytes = 4 * n_total * d + 4 * (n_total + 1) + 4 * n_total * knn_k
            knn_gbs = knn_bytes / (kms / 1e3) / 1e9
            knn = {"k": knn_k, "ms_per_step": kms, "events_per_s": B / (kms / 1e3),
                   "algorithmic_bytes": knn_bytes, "achieved_gbs": knn_gbs,
                   "frac_of_hbm": knn_gbs / measured_peaks()[0],
                   "note": "frnn_knn_graph_batched: the k nearest of every point (no radius) over the step's "
                           "events, device time per step, median of 5 after one warm-up; bytes: points read "
                           "once, CSR written once"}

    # ---- per-stage times of the batched build (CUDA events between stages)
    stage_ms = {s: [] for s in STAGES}
    with torch.cuda.stream(stream):
        for _ in range(5):
            _, ms = plan.build_profiled(x_dev, off, r, k, stream=stream)
            for s in STAGES:
                stage_ms[s].append(ms[s])
    stage_avg = {s: float(np.mean(v[1:])) for s, v in stage_ms.items()}
    dom = max(stage_avg, key=stage_avg.get)
    row_len = np.diff(plan.build_batched(x_dev, off, r, k, stream=stream).to_host()["row_ptr"].astype(np.int64))
    torch.cuda.synchronize(dev)
    long_mask = row_len > KFAST_ROWS
    g_tu, s_tu, _ = plan.get_tuning()
    cell_slots = host_cell_slots(x_host, off, r, g_tu, s_tu, cpp)
    sbytes = stage_bytes(n_total, n_edges, d, int(row_len[long_mask].sum()), int(long_mask.sum()), cell_slots)
    hbm_peak, peak_kind = measured_peaks()
    # the build's algorithmic bytes (read the points once, write the CSR once)
    whole_bytes = 4 * n_total * d + 4 * (n_total + 1) + 4 * n_edges
    achieved = whole_bytes / (stage_avg[dom] / 1e3) / 1e9
    stages = {}
    for sname in STAGES:
        ms_ = stage_avg[sname]
        gbs = sbytes[sname] / (ms_ / 1e3) / 1e9 if ms_ > 0 and sbytes[sname] > 0 else None
        stages[sname] = {"ms": ms_, "algorithmic_bytes": sbytes[sname], "achieved_gbs": gbs,
                         "frac": gbs / hbm_peak if gbs is not None else None}
        if sname == "walk_emit" and sbytes[sname] == 0:
            stages[sname]["note"] = ("no row of this batch is longer than the collect walk parks; the emit walk "
                                     "only took the rows whose filter passes outnumbered their row slots, which "
                                     "the host cannot count, so no fraction is given")

    # ---- e2e: host buffers in, host CSR out.  Main figure: the server's trace
    # call (frnn_server_run_trace) with every event of K steps present at t = 0:
    # copies in, builds and copies out overlap across slots.  Also reported: the
    # synchronous host-to-host call (frnn_build_graph_host), one step at a time.
    e2e = None
    if not args.no_e2e:
        pinned_x = torch.from_numpy(x_host).pin_memory()
        xin = pinned_x.numpy()
        e2e_steps = max(3, min(args.steps, 10))
        sizes = np.diff(off)
        per_batch = args.e2e_batch or max(1, B // 8)
        srv = frnn.Server(d=d, r=r, k=k, batch_points=int(per_batch * n_max_event), batch_events=per_batch,
                          slots=args.e2e_slots, edges_per_point=epp, device=local)
        try:
            req_start = np.tile(off[:-1], e2e_steps)
            req_len = np.tile(sizes, e2e_steps)
            srv.run_trace(xin, off[:-1], sizes, np.zeros(B))  # warm-up
            barrier(pg)
            res = srv.run_trace(xin, req_start, req_len, np.zeros(req_start.size))
            barrier(pg)
        finally:
            srv.close()
        e2e_s = max_over_ranks(pg, res["wall_s"], dev)
        d2h = int(4 * (n_total + B) + 4 * n_edges)
        link = measure_link(torch, dev, int(x_host.nbytes), d2h)
        e2e = {"value": sum_over_ranks(pg, float(B * e2e_steps), dev) / e2e_s, "unit": UNIT,
               "h2d_bytes_per_step": int(x_host.nbytes), "d2h_bytes_per_step": d2h,
               "steps": e2e_steps, "ms_per_step": 1e3 * e2e_s / e2e_steps,
               "link": link,
               "frac_of_link": ((x_host.nbytes + d2h) * e2e_steps / e2e_s / 1e9) / link["both_gbs"],
               "note": (f"frnn_server_run_trace: {B * e2e_steps} events present at t=0, {per_batch} events per "
                        f"batch on {args.e2e_slots} slots; each batch: H2D of its points from pinned host memory, build, D2H "
                        "of row_ptr, edge_off and col into pinned host memory; host wall clock")}
        out = dict(row_ptr=torch.zeros(n_total + 1, dtype=torch.int32).pin_memory().numpy(),
                   col=torch.zeros(n_total * epp, dtype=torch.int32).pin_memory().numpy(),
                   edge_off=np.zeros(B + 1, np.int32))
        plan.build_host(xin, off, r, k, out=out, stream=stream)
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        for _ in range(e2e_steps):
            plan.build_host(xin, off, r, k, out=out, stream=stream)
        t1 = time.perf_counter()
        e2e["sync_host_call"] = {"value": B * e2e_steps / (t1 - t0), "unit": UNIT,
                                 "note": "frnn_build_graph_host, one step per call (copy in, build, copy out)"}

    # ---- served (continuous batching), rank 0 at N=1 only
    served = None
    if rank == 0 and world == 1 and not args.no_served and args.workload == "c2":
        served = run_served(frnn, torch, args.served_requests)

    # ---- CPU oracle baseline (rank 0, N=1 only)
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = run_cpu_baseline(x_host[off[0]:off[1]], args.cpu_queries, r=r, k=k)
        cpu["single_core"] = run_cpu_single_core(x_host[off[0]:off[1]], max(args.cpu_queries // 16, 100), r=r, k=k)

    clocks = clk.summary()
    # ---- arithmetic view of the walks: candidate distance tests per step
    # (every query against its candidates in the collect walk, and the long
    # rows once more in the emit walk unless the plan keeps their hits, whose
    # recomputed distances are not counted), FP32 operations 3 D per test (one
    # subtraction, one product, one addition per dim), against the FP32 rate
    # derived from the SM count, 128 FP32 lanes per SM, two operations per
    # lane per packed f32x2 instruction, and the maximum SM clock
    alu = None
    issue = None
    if rank == 0:
        g_used, s_used, _ = plan.get_tuning()
        mean_cand, g_grid = host_candidates(x_host[off[0]:off[1]], r, g_used, s_used, cpp)
        long_frac = float(np.mean(long_mask))
        kept = hits(n_total) > 0 and walk_used == 1  # the candidate-major walk keeps long rows' hits
        evals = mean_cand * n_total * (1.0 + (0.0 if kept else long_frac))
        ops = evals * 3 * d
        n_sm = torch.cuda.get_device_properties(dev).multi_processor_count
        peak_tops = n_sm * 128 * 2 * clocks["sm_max_mhz"] * 1e6 / 1e12 if clocks["sm_max_mhz"] else None
        achieved_tops = ops / (total_ms_max / args.steps / 1e3) / 1e12
        cap = measured_collect(dom, args.workload, walk_used)
        if cap is not None and clocks["sm_max_mhz"]:
            instr = cap["instr_per_query"] * n_total
            peak_g = 4 * n_sm * clocks["sm_max_mhz"] * 1e6 / 1e9
            ach_g = instr / (stage_avg[dom] / 1e3) / 1e9
            issue = {"warp_instructions_per_launch": instr, "achieved_g_per_s": ach_g, "peak_g_per_s": peak_g,
                     "frac": ach_g / peak_g,
                     "note": "instructions per query from the ncu capture of the same kernel code, scaled to this "
                             "launch; peak = 4 warp instructions per cycle per SM x SMs x max SM clock"}
        alu = {"candidate_tests_per_step": evals, "mean_candidates_per_query": mean_cand,
               "gridded_dims": g_grid, "long_row_fraction": long_frac, "long_rows_walked_again": not kept,
               "candidate_tests_per_s": evals / (total_ms_max / args.steps / 1e3),
               "fp32_ops_per_test": 3 * d, "achieved_tops": achieved_tops, "peak_tops_derived": peak_tops,
               "frac": achieved_tops / peak_tops if peak_tops else None,
               "note": "candidates recounted on the host (event 0, 100k sampled queries, the plan's grid rule); "
                       "peak = SMs x 128 FP32 lanes x 2 (packed f32x2) x max SM clock, derived, not measured"}
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {
                "workload": (f"{args.workload} batched: {B} events x "
                             + (f"N={N_PER_EVENT}" if args.workload == "c2" else
                                f"N in [{int(np.min(np.diff(off)))}, {n_max_event}]")
                             + f" (seeded per event), D={d}, r={r}, K={k}, "
                               "one batched build per step replayed from a CUDA graph"),
                "events_per_step": B, "n_per_event": N_PER_EVENT if args.workload == "c2" else None,
                "d": d, "r": r, "k": k, "autotune": tuned, "hit_capacity": hits(n_total),
                "points_per_step": n_total, "edges_per_step": n_edges,
                "l2": f"inputs larger than L2 ({x_host.nbytes / 1e6:.0f} MB of points per step, "
                      f"plus {4 * n_edges / 1e6:.0f} MB of col written)",
                "parallelism": f"replicas x{world}",
            },
            "batched": {"events_per_s": value, "step_ms_p50": percentile(step_ms, 50),
                        "step_ms_p99": percentile(step_ms, 99),
                        "event_latency_note": "every event of a batch completes with its step"},
            "plain": {"events_per_s": plain_value, "latency_ms_p50": percentile(plain_ms, 50),
                      "latency_ms_p99": percentile(plain_ms, 99),
                      "host_ms_p50": percentile(plain_host_ms, 50), "host_ms_p99": percentile(plain_host_ms, 99),
                      "note": "one event per call (CUDA graph replay per event) plus a stream sync; latency = "
                              "device time per event (CUDA events), host_ms = call to sync; events/s from the host "
                              "times"},
            "batched_over_plain": value / plain_value / world,
            "walk": {1: "candidate-major", 2: "query-major"}[walk_used],
            "stages_ms": stage_avg,
            "stages": stages,
            "roofline": {"bound": "hbm", "kernel": "k_" + dom,
                         "achieved": achieved, "peak": hbm_peak, "unit": "GB/s", "frac": achieved / hbm_peak,
                         "traffic": (cap["bytes_per_point"] * n_total
                                     if (cap := measured_collect(dom, args.workload, walk_used)) else None),
                         "peak_kind": peak_kind,
                         "algorithmic_bytes_per_launch": whole_bytes,
                         "algorithmic_bytes_note": "4 N D + 4 (N + 1) + 4 E: the points read once and the CSR "
                                                   "written once, over the dominant kernel's CUDA-event time",
                         "launch_ms": stage_avg[dom],
                         "stage_bytes_view": {"bytes": sbytes[dom], "frac": stages[dom]["frac"],
                                              "note": "the kernel's own unavoidable reads and writes"},
                         "whole_build": {"algorithmic_bytes": whole_bytes,
                                         "achieved_gbs": whole_bytes / (total_ms_max / args.steps / 1e3) / 1e9,
                                         "frac": whole_bytes / (total_ms_max / args.steps / 1e3) / 1e9 / hbm_peak},
                         "alu_view": alu, "issue_view": issue},
            "e2e": e2e,
            "labeling": labeling,
            "edge_features": edge_features,
            "knn": knn,
            "served": served,
            "cpu_baseline": cpu,
            "gpu_launches": (KERNELS_PER_BUILD + (1 if walk_used == 1 else 0)) * args.steps,
            "clocks": {"sm_mhz": clocks["sm_mhz"], "sm_max_mhz": clocks["sm_max_mhz"],
                       "reasons": clocks["reasons"], "samples": clocks["samples"]},
        }
        print(json.dumps(line), flush=True)
    plan.close()
    plan_one.close()
    if pg is not None:
        pg.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
