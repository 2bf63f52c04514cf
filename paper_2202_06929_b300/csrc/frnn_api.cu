// Host side of libfrnn: plans, the C ABI declared in include/frnn.h, and the
// CUDA-graph replay of a build.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <limits>
#include <new>

#include "frnn.h"
#include "frnn_internal.h"

using namespace frnn;

namespace {

constexpr int kRing = 4;  // pinned staging slots for the per-call header
constexpr int kMaxAllocs = 48;  // device allocations of a plan, at most
constexpr int kVersion = 10000;

struct DeviceGuard {
    int prev = -1;
    bool ok = false;
    explicit DeviceGuard(int dev)
    {
        if (cudaGetDevice(&prev) != cudaSuccess) return;
        ok = (prev == dev) || (cudaSetDevice(dev) == cudaSuccess);
    }
    ~DeviceGuard()
    {
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

int next_pow2(int v)
{
    int p = 1;
    while (p < v) p <<= 1;
    return p;
}

// The shape of a call that a tuning is cached for: mean points per event
// (two buckets per octave), events (one per octave), dimension, radius, cap.
struct TuneKey {
    int n_bucket = -1, ev_bucket = -1, d = 0, k = 0;
    float r = 0.f;
    bool operator==(const TuneKey& o) const
    {
        return n_bucket == o.n_bucket && ev_bucket == o.ev_bucket && d == o.d && k == o.k && r == o.r;
    }
};

struct TuneEntry {
    TuneKey key;
    frnn_tuning t{};
};

constexpr int kTuneCache = 16;

TuneKey tune_key(const int64_t* ev_off, int n_events, int d, float r, int k)
{
    TuneKey key;
    const double mean = (double)ev_off[n_events] / (double)n_events;
    key.n_bucket = mean >= 1.0 ? (int)std::floor(2.0 * std::log2(mean)) : -1;
    key.ev_bucket = (int)std::floor(std::log2((double)n_events));
    key.d = d;
    key.k = k;
    key.r = r;
    return key;
}

struct GraphEntry {
    int dp4 = 0;
    int cap = 0;
    int walk = 0;
    cudaGraphExec_t exec = nullptr;
};

}  // namespace

struct frnn_plan {
    frnn_plan_params prm{};
    frnn_tuning tuning{4, 1.0f, 0};
    int n_sm = 0;
    int dp_max = 0;
    long long cells_max = 0;
    long long edge_cap = 0;
    int tiles_cells = 0, tiles_rows = 0;
    LaunchCfg base_cfg{};
    DevState st{};
    // per-call header + event table (device) and its pinned staging ring
    char* d_call = nullptr;
    size_t call_bytes = 0;
    char* h_call[kRing] = {};
    cudaEvent_t ring_ev[kRing] = {};
    int ring_pos = 0;
    // allocations to free
    void* allocs[kMaxAllocs] = {};
    int n_allocs = 0;
    // graph cache (FRNN_USE_GRAPH)
    cudaStream_t cap_stream = nullptr;
    GraphEntry graphs[32];
    int n_graphs = 0;
    // walk launch shapes per (dp4, cap)
    LaunchCfg walk_cfg[17][12];
    bool walk_ok[17][12] = {};
    // device input of the host-to-host call
    float* d_input = nullptr;
    long long d_input_floats = 0;
    frnn_csr last{};
    float last_r2 = 0.f;
    int last_d = 0;
    bool has_last = false;
    bool stall_next = false;  // frnn_plan_test_stall_next_build
    // debug checks: first failure (check id << 48 | index, ~0 if none) and
    // one bit per point of scratch
    unsigned long long* chk_first = nullptr;
    unsigned* chk_bits = nullptr;
    // autotuner: probe output (device, 3 x u64) and the tunings it found,
    // keyed by the shape of the call
    unsigned long long* probe = nullptr;
    TuneEntry tune_cache[kTuneCache];
    int n_tune = 0, tune_next = 0;
    bool tuning_fixed = false;  // the autotuner is timing p->tuning itself: no lookup
};

namespace {

// The tuning a call uses: the autotuner's entry for the call's shape if there
// is one, else the plan's tuning.
frnn_tuning tuning_for(const frnn_plan* p, const int64_t* ev_off, int n_events, int d, float r, int k,
                       bool* cached = nullptr)
{
    if (cached) *cached = false;
    if (!p->tuning_fixed && p->n_tune > 0) {
        const TuneKey key = tune_key(ev_off, n_events, d, r, k);
        for (int i = 0; i < p->n_tune; ++i)
            if (p->tune_cache[i].key == key) {
                if (cached) *cached = true;
                return p->tune_cache[i].t;
            }
    }
    return p->tuning;
}

void cache_tuning(frnn_plan* p, const TuneKey& key, const frnn_tuning& t)
{
    for (int i = 0; i < p->n_tune; ++i)
        if (p->tune_cache[i].key == key) {
            p->tune_cache[i].t = t;
            return;
        }
    const int i = p->n_tune < kTuneCache ? p->n_tune++ : (p->tune_next++ % kTuneCache);
    p->tune_cache[i].key = key;
    p->tune_cache[i].t = t;
}

template <typename T>
int plan_alloc(frnn_plan* p, T** out, long long count)
{
    *out = nullptr;
    if (count <= 0) count = 1;
    if (p->n_allocs >= kMaxAllocs) return FRNN_ERR_OOM;
    void* ptr = nullptr;
    if (cudaMalloc(&ptr, (size_t)count * sizeof(T)) != cudaSuccess) {
        cudaGetLastError();
        return FRNN_ERR_OOM;
    }
    p->allocs[p->n_allocs++] = ptr;
    *out = static_cast<T*>(ptr);
    return FRNN_OK;
}

void plan_free_all(frnn_plan* p)
{
    for (int i = 0; i < p->n_graphs; ++i)
        if (p->graphs[i].exec) cudaGraphExecDestroy(p->graphs[i].exec);
    p->n_graphs = 0;
    if (p->cap_stream) cudaStreamDestroy(p->cap_stream);
    for (int i = 0; i < kRing; ++i) {
        if (p->ring_ev[i]) cudaEventDestroy(p->ring_ev[i]);
        if (p->h_call[i]) cudaFreeHost(p->h_call[i]);
    }
    for (int i = 0; i < p->n_allocs; ++i) cudaFree(p->allocs[i]);
    p->n_allocs = 0;
}

// Restore every buffer that must be zero (or +-inf encoded) between builds.
int reset_device_state(frnn_plan* p, cudaStream_t s)
{
    const DevState& st = p->st;
    const long long ev = p->prm.events_max;
    bool ok = true;
    ok &= cudaMemsetAsync(st.bb_min, 0xff, sizeof(unsigned) * ev * kMaxDims, s) == cudaSuccess;
    ok &= cudaMemsetAsync(st.bb_max, 0, sizeof(unsigned) * ev * kMaxDims, s) == cudaSuccess;
    ok &= cudaMemsetAsync(st.chunk_done, 0, sizeof(unsigned) * ev, s) == cudaSuccess;
    ok &= cudaMemsetAsync(st.nonfinite, 0, sizeof(unsigned) * ev, s) == cudaSuccess;
    ok &= cudaMemsetAsync(st.counters, 0, sizeof(unsigned) * kCtrCount, s) == cudaSuccess;
    ok &= cudaMemsetAsync(st.pool_ctr, 0, sizeof(unsigned long long), s) == cudaSuccess;
    if (st.spill_ctr) ok &= cudaMemsetAsync(st.spill_ctr, 0, sizeof(unsigned long long), s) == cudaSuccess;
    ok &= cudaMemsetAsync(st.cell_count, 0, sizeof(unsigned) * p->cells_max, s) == cudaSuccess;
    ok &= cudaMemsetAsync(st.scan_cells, 0, sizeof(unsigned long long) * p->tiles_cells, s) == cudaSuccess;
    ok &= cudaMemsetAsync(st.scan_rows, 0, sizeof(unsigned long long) * p->tiles_rows, s) == cudaSuccess;
    return ok ? FRNN_OK : FRNN_ERR_CUDA;
}

int get_walk_cfg(frnn_plan* p, int dp4, int cap, LaunchCfg* out)
{
    int ci = 0;
    while ((1 << ci) < cap) ++ci;
    if (dp4 < 1 || dp4 > 16 || ci >= 12) return FRNN_ERR_INVALID_ARG;
    if (!p->walk_ok[dp4][ci]) {
        LaunchCfg c = p->base_cfg;
        if (config_walk(dp4, cap, p->n_sm, &c) != 0) {
            cudaGetLastError();
            return FRNN_ERR_CUDA;
        }
        p->walk_cfg[dp4][ci] = c;
        p->walk_ok[dp4][ci] = true;
    }
    *out = p->walk_cfg[dp4][ci];
    return FRNN_OK;
}

int launch(frnn_plan* p, int dp4, int cap, int walk_tuning, cudaStream_t s, cudaEvent_t* stage_ev)
{
    LaunchCfg cfg;
    int rc = get_walk_cfg(p, dp4, cap, &cfg);
    if (rc != FRNN_OK) return rc;
    const int walk = resolve_walk(walk_tuning, dp4);
    if (stage_ev || !(p->prm.flags & FRNN_USE_GRAPH))
        return launch_build(p->st, dp4, cfg, walk, s, stage_ev) == 0 ? FRNN_OK : FRNN_ERR_CUDA;
    GraphEntry* ge = nullptr;
    for (int i = 0; i < p->n_graphs; ++i)
        if (p->graphs[i].dp4 == dp4 && p->graphs[i].cap == cap && p->graphs[i].walk == walk) ge = &p->graphs[i];
    if (!ge) {
        if (p->n_graphs >= 32) return FRNN_ERR_CAPACITY;
        cudaGraph_t g = nullptr;
        if (cudaStreamBeginCapture(p->cap_stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
            return FRNN_ERR_CUDA;
        const int lrc = launch_build(p->st, dp4, cfg, walk, p->cap_stream, nullptr);
        const cudaError_t ce = cudaStreamEndCapture(p->cap_stream, &g);
        if (lrc != 0 || ce != cudaSuccess) {
            if (g) cudaGraphDestroy(g);
            cudaGetLastError();
            return FRNN_ERR_CUDA;
        }
        cudaGraphExec_t ex = nullptr;
        const cudaError_t ie = cudaGraphInstantiate(&ex, g, 0);
        cudaGraphDestroy(g);
        if (ie != cudaSuccess) {
            cudaGetLastError();
            return FRNN_ERR_CUDA;
        }
        ge = &p->graphs[p->n_graphs++];
        ge->dp4 = dp4;
        ge->cap = cap;
        ge->walk = walk;
        ge->exec = ex;
    }
    return cudaGraphLaunch(ge->exec, s) == cudaSuccess ? FRNN_OK : FRNN_ERR_CUDA;
}

// Points per chunk of the per-point kernels: the smallest power of two from
// kChunkMin that leaves at most about two chunks per block of those kernels,
// up to kChunk (a single event spreads over every SM; big batches keep the
// per-chunk overhead low).
int chunk_points(const frnn_plan* p, long long n_total)
{
    const long long want = 2ll * p->base_cfg.grid_pt;
    int c = kChunkMin;
    while (c < kChunk && (n_total + c - 1) / c > want) c *= 2;
    return c;
}

// Chunks the bounding-box kernel takes at a time: its per-chunk reduction,
// barriers and atomics cost about as much as reading a chunk, so a batch much
// larger than the grid is read a few chunks (of one event) per step.
int bbox_group(const frnn_plan* p, int chunks)
{
    int g = 1;
    while (g < 8 && chunks > 2ll * g * p->base_cfg.grid_pt) g *= 2;
    return g;
}

int check_build_args(const frnn_plan* p, const float* emb, const int64_t* ev_off, int n_events,
                     int d, float r, int k, frnn_csr* out, long long* n_total)
{
    if (!p || !out || !ev_off) return FRNN_ERR_INVALID_ARG;
    if (n_events < 1 || d < 1 || d > kMaxDims || k < 0 || k > 1024) return FRNN_ERR_INVALID_ARG;
    if (!(r > 0.0f) || !std::isfinite(r)) return FRNN_ERR_INVALID_ARG;
    if (ev_off[0] != 0) return FRNN_ERR_INVALID_ARG;
    for (int b = 0; b < n_events; ++b)
        if (ev_off[b + 1] < ev_off[b]) return FRNN_ERR_INVALID_ARG;
    const long long n = ev_off[n_events];
    if (n > 0 && (!emb || (reinterpret_cast<uintptr_t>(emb) & 3u))) return FRNN_ERR_INVALID_ARG;
    if (n * (long long)k >= (1ll << 31)) return FRNN_ERR_INVALID_ARG;  // k = 0 (no cap): bounded by the edge capacity
    if (n_events > p->prm.events_max || n > p->prm.n_max || d > p->prm.d_max || k > p->prm.k_max_cap)
        return FRNN_ERR_CAPACITY;
    float r2 = r * r;
    if (!(r2 > 0.0f) || !std::isfinite(r2)) return FRNN_ERR_INVALID_ARG;
    *n_total = n;
    return FRNN_OK;
}

int autotune(frnn_plan* p, const float* emb, const int64_t* ev_off, int n_events, int d, float r, int k,
             cudaStream_t s, frnn_tuning* best, float* best_ms);

// The debug checks of the plan's last build (p->last), on stream s.
int run_checks(frnn_plan* p, cudaStream_t s)
{
    if (p->last.n_total == 0) return FRNN_OK;
    return launch_checks(p->st, p->chk_first, p->chk_bits, p->last.n_total, p->last.n_events, p->cells_max,
                         p->last_d, p->n_sm, s) == 0
               ? FRNN_OK : FRNN_ERR_CUDA;
}

// One radius build, or with probe_out set the autotuner's probe of the grid
// (stages 1-3 and the candidate count; the outputs are not written).
int build_batched(frnn_plan* p, const float* emb, const int64_t* ev_off, int n_events, int d,
                  float r, int k, cudaStream_t s, frnn_csr* out, cudaEvent_t* stage_ev = nullptr,
                  unsigned long long* probe_out = nullptr)
{
    long long n_total = 0;
    int rc = check_build_args(p, emb, ev_off, n_events, d, r, k, out, &n_total);
    if (rc != FRNN_OK) return rc;
    bool cached = false;
    frnn_tuning tu = tuning_for(p, ev_off, n_events, d, r, k, &cached);
    if (!cached && !p->tuning_fixed && (p->prm.flags & FRNN_AUTOTUNE) && n_total > 0 && !probe_out) {
        // first call of this shape: tune it (synchronous, off the steady-state path)
        rc = autotune(p, emb, ev_off, n_events, d, r, k, s, &tu, nullptr);
        if (rc != FRNN_OK) return rc;
    }
    const DevState& st = p->st;
    out->row_ptr = st.row_ptr;
    out->col = st.col;
    out->d2 = (p->prm.flags & FRNN_EMIT_D2) ? st.d2 : nullptr;
    out->edge_off = st.edge_off;
    out->n_edges = st.edge_off + n_events;
    out->n_events = n_events;
    out->n_total = n_total;
    if (n_total == 0) {
        if (cudaMemsetAsync(st.row_ptr, 0, sizeof(int), s) != cudaSuccess ||
            cudaMemsetAsync(st.edge_off, 0, sizeof(int) * (n_events + 1), s) != cudaSuccess)
            return FRNN_ERR_CUDA;
        p->last = *out;
        p->last_r2 = r * r;
        p->last_d = d;
        p->has_last = true;
        return FRNN_OK;
    }
    // stage the per-call header and event table
    const int slot = p->ring_pos;
    p->ring_pos = (p->ring_pos + 1) % kRing;
    if (cudaEventSynchronize(p->ring_ev[slot]) != cudaSuccess) return FRNN_ERR_CUDA;
    CallHdr* h = reinterpret_cast<CallHdr*>(p->h_call[slot]);
    EvDesc* ev = reinterpret_cast<EvDesc*>(p->h_call[slot] + sizeof(CallHdr));
    const int cpp = p->prm.cells_per_point;
    const int chunk = chunk_points(p, n_total);
    int chunks = 0;
    for (int b = 0; b < n_events; ++b) {
        const long long nb = ev_off[b + 1] - ev_off[b];
        const int nc = nb > 0 ? (int)((nb + chunk - 1) / chunk) : 1;
        ev[b].pt_off = ev_off[b];
        ev[b].n = (int)nb;
        ev[b].chunk_off = chunks;
        ev[b].nchunk = nc;
        ev[b].cell_budget = (int)(cpp * nb + 4096);
        ev[b].edge0 = ev[b].pad1 = 0;
        chunks += nc;
    }
    h->emb = emb;
    h->n_total = n_total;
    h->n_events = n_events;
    h->total_chunks = chunks;
    h->chunk = chunk;
    h->d = d;
    h->dp = (d + 3) & ~3;
    h->k = (k == FRNN_NO_CAP) ? 0x7fffffff : k;
    h->r = r;
    h->r2 = r * r;
    h->g_max = tu.g_max;
    h->cell_scale = tu.cell_scale;
    h->emit_d2 = (p->prm.flags & FRNN_EMIT_D2) ? 1 : 0;
    h->knn = 0;
    h->stall = p->stall_next ? 1 : 0;
    p->stall_next = false;
    h->edge_capacity = p->edge_cap;
    const int cap = next_pow2((k > 32 ? k : 32) + 32);
    // long rows keep every hit when the plan has room (rows of up to 16 floats)
    h->spill_capacity = p->prm.hit_capacity;
    h->spill_max = (p->prm.hit_capacity > 0 && h->dp / 4 <= 4) ? kSpillSlots : 0;
    h->bbox_group = bbox_group(p, chunks);
    const size_t bytes = sizeof(CallHdr) + sizeof(EvDesc) * (size_t)n_events;
    if (cudaMemcpyAsync(p->d_call, p->h_call[slot], bytes, cudaMemcpyHostToDevice, s) != cudaSuccess)
        return FRNN_ERR_CUDA;
    if (cudaEventRecord(p->ring_ev[slot], s) != cudaSuccess) return FRNN_ERR_CUDA;
    if (probe_out) {
        p->has_last = false;  // a probe leaves no graph behind
        return launch_probe(p->st, p->base_cfg, probe_out, s) == 0 ? FRNN_OK : FRNN_ERR_CUDA;
    }
    rc = launch(p, h->dp / 4, cap, tu.walk, s, stage_ev);
    if (rc != FRNN_OK) return rc;
    p->last = *out;
    p->last_r2 = r * r;
    p->last_d = d;
    p->has_last = true;
    // the autotuner's timed builds are not checked
    if ((p->prm.flags & FRNN_DEBUG) && !p->tuning_fixed) return run_checks(p, s);
    return FRNN_OK;
}

// Checks plan parameters and fills in their defaults.
int normalize_params(const frnn_plan_params* prm, frnn_plan_params* out, long long* cells_max)
{
    frnn_plan_params q = *prm;
    if (q.d_max < 1 || q.d_max > kMaxDims || q.n_max < 0 || q.events_max < 1 ||
        q.k_max_cap < 1 || q.k_max_cap > 1024 || q.edge_capacity < 0 || q.cells_per_point < 0 ||
        q.hit_capacity < 0)
        return FRNN_ERR_INVALID_ARG;
    if (q.cells_per_point == 0) q.cells_per_point = 4;
    if (q.edge_capacity == 0) {
        if (q.n_max * (long long)q.k_max_cap >= (1ll << 31)) return FRNN_ERR_INVALID_ARG;
        q.edge_capacity = q.n_max * (long long)q.k_max_cap;
    }
    if (q.edge_capacity >= (1ll << 31)) return FRNN_ERR_INVALID_ARG;
    const long long cm = q.cells_per_point * q.n_max + 4096ll * q.events_max;
    if (cm >= (1ll << 31) || q.n_max >= (1ll << 31) - 1) return FRNN_ERR_INVALID_ARG;
    *out = q;
    *cells_max = cm;
    return FRNN_OK;
}

// Device bytes frnn_plan_create allocates for these (normalised) parameters.
unsigned long long plan_device_bytes(const frnn_plan_params& q, long long cells_max)
{
    const unsigned long long n = (unsigned long long)q.n_max, ev = (unsigned long long)q.events_max;
    const unsigned long long dp = (unsigned long long)((q.d_max + 3) & ~3);
    const unsigned long long ec = (unsigned long long)q.edge_capacity;
    const unsigned long long tiles_c = (unsigned long long)(cells_max + kScanTile - 1) / kScanTile + 1;
    const unsigned long long tiles_r = (n + kRowScanTile - 1) / kRowScanTile + 1;
    const bool d2 = (q.flags & FRNN_EMIT_D2) != 0;
    unsigned long long b = sizeof(CallHdr) + sizeof(EvDesc) * ev + sizeof(EvPlan) * ev + sizeof(int2) * kMaxRuns * ev;
    b += 2 * sizeof(unsigned) * ev * kMaxDims + 2 * sizeof(unsigned) * ev + sizeof(unsigned) * kCtrCount + 4;
    b += 4 * sizeof(unsigned) * n + sizeof(float) * n * dp + 2 * sizeof(int) * n + sizeof(int) * (n + 1);
    b += sizeof(unsigned) * (((n + 7) & ~7ull) + 8) + sizeof(FiltPlan) * ev;  // filter keys and plans
    b += sizeof(unsigned) * (unsigned long long)cells_max + sizeof(int) * ((unsigned long long)cells_max + 1);
    b += sizeof(unsigned long long) * (tiles_c + tiles_r);
    b += sizeof(int) * ec * 2 + (d2 ? 2 * sizeof(float) * ec : 0);
    b += 8 + sizeof(int) * (ev + 1) + 4 + sizeof(unsigned);
    b += 3 * sizeof(unsigned long long);  // autotuner probe
    b += sizeof(unsigned long long) + sizeof(unsigned) * ((n + 31) / 32 + 1);  // debug checks
    b += sizeof(float) * n * (unsigned long long)q.d_max;  // input of the host-to-host call
    if (q.hit_capacity > 0)  // neighbours of long rows, and per long row its entry
        b += sizeof(int) * (unsigned long long)q.hit_capacity + 8 + (sizeof(long long) + sizeof(int)) * n;
    return b;
}

// The autotuner (the choice of gridded dimensions that the paper makes by
// hand, Sec. 3.4, plus the form of the walk).  Every grid of the search
// (g_max x cell_scale) is first probed: stages 1-3 and a count of the exact
// candidate tests, non-empty cells and cell slots the walk and the scans
// would handle.  A cost in candidate-test units, tests + 20 x non-empty cells
// (a segment's set-up) + 2 x cell slots (the scans), keeps the three cheapest
// grids; those are timed with each walk form (best of three builds after a
// warm-up) and the fastest is set on the plan and cached for the call's shape.
int autotune(frnn_plan* p, const float* emb, const int64_t* ev_off, int n_events, int d, float r, int k,
             cudaStream_t s, frnn_tuning* best, float* best_ms)
{
    static const int kG[] = {6, 5, 4, 3, 2};
    static const float kScale[] = {1.0f, 1.25f, 1.5f, 2.0f};
    constexpr int kGrids = 20, kFinalists = 3;
    frnn_csr out;
    long long n_total = 0;
    int rc = check_build_args(p, emb, ev_off, n_events, d, r, k, &out, &n_total);
    if (rc != FRNN_OK) return rc;
    const frnn_tuning saved = p->tuning;
    if (n_total == 0) {
        if (best) *best = saved;
        if (best_ms) *best_ms = 0.f;
        return FRNN_OK;
    }
    p->tuning_fixed = true;
    // probe every grid
    struct Cand {
        frnn_tuning t;
        double cost;
    };
    Cand cand[kGrids];
    unsigned long long h_probe[3];
    for (int i = 0; i < kGrids && rc == FRNN_OK; ++i) {
        p->tuning.g_max = kG[i / 4];
        p->tuning.cell_scale = kScale[i % 4];
        p->tuning.walk = kWalkAuto;
        rc = build_batched(p, emb, ev_off, n_events, d, r, k, s, &out, nullptr, p->probe);
        if (rc != FRNN_OK) break;
        if (cudaMemcpyAsync(h_probe, p->probe, sizeof(h_probe), cudaMemcpyDeviceToHost, s) != cudaSuccess) {
            rc = FRNN_ERR_CUDA;
            break;
        }
        unsigned bits = 0;
        rc = read_status_bits(p, s, &bits);  // synchronises the stream
        if (rc == FRNN_OK && (bits & kStTimeout)) rc = FRNN_ERR_TIMEOUT;
        cand[i].t = p->tuning;
        cand[i].cost = (double)h_probe[0] + 20.0 * (double)h_probe[1] + 2.0 * (double)h_probe[2];
    }
    // time the cheapest grids with each walk form
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (rc == FRNN_OK && (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)) {
        cudaGetLastError();
        rc = FRNN_ERR_CUDA;
    }
    frnn_tuning win = saved;
    float win_ms = -1.f;
    if (rc == FRNN_OK) {
        std::sort(cand, cand + kGrids, [](const Cand& a, const Cand& b) { return a.cost < b.cost; });
        const int dp4 = (d + 3) / 4;
        const int n_walks = dp4 <= kMaxDp4QueryMajor ? 2 : 1;
        for (int f = 0; f < kFinalists && rc == FRNN_OK; ++f) {
            for (int w = 0; w < n_walks && rc == FRNN_OK; ++w) {
                p->tuning = cand[f].t;
                p->tuning.walk = w == 0 ? kWalkCandMajor : kWalkQueryMajor;
                rc = build_batched(p, emb, ev_off, n_events, d, r, k, s, &out);  // warm-up (and graph capture)
                float best_rep = -1.f;
                for (int rep = 0; rep < 3 && rc == FRNN_OK; ++rep) {
                    cudaEventRecord(e0, s);
                    rc = build_batched(p, emb, ev_off, n_events, d, r, k, s, &out);
                    cudaEventRecord(e1, s);
                    if (rc != FRNN_OK) break;
                    float ms = 0.f;
                    if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
                        rc = FRNN_ERR_CUDA;
                        break;
                    }
                    if (best_rep < 0.f || ms < best_rep) best_rep = ms;
                }
                if (rc != FRNN_OK) break;
                unsigned bits = 0;
                rc = read_status_bits(p, s, &bits);
                if (rc == FRNN_OK && (bits & kStTimeout)) rc = FRNN_ERR_TIMEOUT;
                if (rc == FRNN_OK && (win_ms < 0.f || best_rep < win_ms)) {
                    win_ms = best_rep;
                    win = p->tuning;
                }
            }
        }
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    p->tuning_fixed = false;
    p->tuning = (rc == FRNN_OK && win_ms >= 0.f) ? win : saved;
    if (rc == FRNN_OK && win_ms < 0.f) rc = FRNN_ERR_CUDA;
    if (rc == FRNN_OK) cache_tuning(p, tune_key(ev_off, n_events, d, r, k), win);
    if (best) *best = p->tuning;
    if (best_ms) *best_ms = win_ms;
    return rc;
}

}  // namespace

extern "C" {

int frnn_version(void) { return kVersion; }

const char* frnn_status_string(int status)
{
    switch (status) {
        case FRNN_OK: return "ok";
        case FRNN_ERR_INVALID_ARG: return "invalid argument";
        case FRNN_ERR_CUDA: return "CUDA runtime error";
        case FRNN_ERR_OOM: return "device out of memory";
        case FRNN_ERR_NONFINITE_INPUT: return "input holds NaN or Inf; that event's rows are empty";
        case FRNN_ERR_TIMEOUT: return "a bounded device-side wait ran out";
        case FRNN_ERR_OVERFLOW: return "edges exceed the edge capacity";
        case FRNN_ERR_CAPACITY: return "call exceeds a plan capacity";
        case FRNN_ERR_CHECK: return "a debug check of the build's output failed";
        default: return "unknown status";
    }
}

int frnn_plan_bytes(const frnn_plan_params* prm, uint64_t* bytes)
{
    if (!prm || !bytes) return FRNN_ERR_INVALID_ARG;
    frnn_plan_params q;
    long long cm = 0;
    const int rc = normalize_params(prm, &q, &cm);
    if (rc != FRNN_OK) return rc;
    *bytes = plan_device_bytes(q, cm);
    return FRNN_OK;
}

int frnn_plan_create(frnn_plan** out, const frnn_plan_params* prm)
{
    frnn::NvtxRange nvtx("frnn_plan_create");
    if (!out || !prm) return FRNN_ERR_INVALID_ARG;
    *out = nullptr;
    frnn_plan_params q;
    long long cells_max = 0;
    const int nrc = normalize_params(prm, &q, &cells_max);
    if (nrc != FRNN_OK) return nrc;
    if (q.mem_budget_bytes > 0 && plan_device_bytes(q, cells_max) > q.mem_budget_bytes) return FRNN_ERR_OOM;
    int n_dev = 0;
    if (cudaGetDeviceCount(&n_dev) != cudaSuccess || q.device < 0 || q.device >= n_dev) {
        cudaGetLastError();
        return q.device < 0 ? FRNN_ERR_INVALID_ARG : FRNN_ERR_CUDA;
    }
    DeviceGuard dg(q.device);
    if (!dg.ok) return FRNN_ERR_CUDA;
    frnn_plan* p = new (std::nothrow) frnn_plan();
    if (!p) return FRNN_ERR_OOM;
    p->prm = q;
    p->dp_max = (q.d_max + 3) & ~3;
    p->cells_max = cells_max;
    p->edge_cap = q.edge_capacity;
    p->tiles_cells = (int)((cells_max + kScanTile - 1) / kScanTile) + 1;
    p->tiles_rows = (int)((q.n_max + kRowScanTile - 1) / kRowScanTile) + 1;
    cudaDeviceGetAttribute(&p->n_sm, cudaDevAttrMultiProcessorCount, q.device);
    int rc = FRNN_OK;
    DevState& st = p->st;
    const long long n = q.n_max, ev = q.events_max;
    p->call_bytes = sizeof(CallHdr) + sizeof(EvDesc) * (size_t)ev;
#define ALLOC(ptr, cnt) \
    if (rc == FRNN_OK) rc = plan_alloc(p, &(ptr), (cnt))
    ALLOC(p->d_call, (long long)p->call_bytes);
    st.hdr = reinterpret_cast<const CallHdr*>(p->d_call);
    st.ev = reinterpret_cast<const EvDesc*>(p->d_call + sizeof(CallHdr));
    ALLOC(st.plan, ev);
    ALLOC(st.run_tab, ev * kMaxRuns);
    ALLOC(st.bb_min, ev * kMaxDims);
    ALLOC(st.bb_max, ev * kMaxDims);
    ALLOC(st.chunk_done, ev);
    ALLOC(st.nonfinite, ev);
    ALLOC(st.counters, (long long)kCtrCount);
    ALLOC(st.cells_total, 1);
    ALLOC(st.key, n);
    ALLOC(st.rank, n);
    ALLOC(st.perm, n);
    ALLOC(st.cell_s, n);
    ALLOC(st.xs, n * p->dp_max);
    ALLOC(st.xq, ((n + 7) & ~7LL) + 8);
    ALLOC(st.fplan, ev);
    ALLOC(st.pool_off, n);
    ALLOC(st.cnt_o, n);
    ALLOC(st.row_ptr, n + 1);
    ALLOC(st.cell_count, cells_max);
    ALLOC(st.cell_start, cells_max + 1);
    ALLOC(st.scan_cells, (long long)p->tiles_cells);
    ALLOC(st.scan_rows, (long long)p->tiles_rows);
    ALLOC(st.col, q.edge_capacity);
    if (q.flags & FRNN_EMIT_D2) ALLOC(st.d2, q.edge_capacity);
    ALLOC(st.pool, q.edge_capacity);
    if (q.flags & FRNN_EMIT_D2) ALLOC(st.pool_d2, q.edge_capacity);
    ALLOC(st.pool_ctr, 1);
    ALLOC(st.edge_off, ev + 1);
    ALLOC(st.status, 1);
    ALLOC(st.offgrid, 1);
    ALLOC(p->probe, 3);
    ALLOC(p->chk_first, 1);
    ALLOC(p->chk_bits, (n + 31) / 32 + 1);
    ALLOC(p->d_input, n * q.d_max);  // the device copy of frnn_build_graph_host's input
    p->d_input_floats = n * q.d_max;
    if (q.hit_capacity > 0) {
        ALLOC(st.spill, q.hit_capacity);
        ALLOC(st.spill_ctr, 1);
        ALLOC(st.spill_at, n);
        ALLOC(st.spill_n, n);
    }
#undef ALLOC
    for (int i = 0; rc == FRNN_OK && i < kRing; ++i) {
        if (cudaHostAlloc(reinterpret_cast<void**>(&p->h_call[i]), p->call_bytes, cudaHostAllocDefault) != cudaSuccess ||
            cudaEventCreateWithFlags(&p->ring_ev[i], cudaEventDisableTiming) != cudaSuccess)
            rc = FRNN_ERR_OOM;
    }
    if (rc == FRNN_OK && cudaStreamCreateWithFlags(&p->cap_stream, cudaStreamNonBlocking) != cudaSuccess)
        rc = FRNN_ERR_CUDA;
    if (rc == FRNN_OK && config_pt(p->n_sm, &p->base_cfg) != 0) rc = FRNN_ERR_CUDA;
    if (rc == FRNN_OK) {
        rc = reset_device_state(p, nullptr);
        if (rc == FRNN_OK && cudaMemset(st.status, 0, sizeof(unsigned)) != cudaSuccess) rc = FRNN_ERR_CUDA;
        if (rc == FRNN_OK && cudaMemset(p->chk_first, 0xff, sizeof(unsigned long long)) != cudaSuccess)
            rc = FRNN_ERR_CUDA;
        if (rc == FRNN_OK && cudaDeviceSynchronize() != cudaSuccess) rc = FRNN_ERR_CUDA;
    }
    if (rc != FRNN_OK) {
        cudaGetLastError();
        plan_free_all(p);
        delete p;
        return rc;
    }
    *out = p;
    return FRNN_OK;
}

int frnn_plan_destroy(frnn_plan* p)
{
    if (!p) return FRNN_OK;
    DeviceGuard dg(p->prm.device);
    cudaDeviceSynchronize();
    plan_free_all(p);
    delete p;
    return FRNN_OK;
}

int frnn_plan_set_tuning(frnn_plan* p, const frnn_tuning* t)
{
    if (!p || !t) return FRNN_ERR_INVALID_ARG;
    const int g = t->g_max == 0 ? 4 : t->g_max;  // default 4; up to kMaxG when the cell budget allows
    const float cs = t->cell_scale == 0.f ? 1.0f : t->cell_scale;
    if (g < 1 || g > kMaxG || !(cs >= 1.0f) || !std::isfinite(cs) || cs > 1e6f) return FRNN_ERR_INVALID_ARG;
    if (t->walk < kWalkAuto || t->walk > kWalkQueryMajor) return FRNN_ERR_INVALID_ARG;
    p->tuning.g_max = g;
    p->tuning.cell_scale = cs;
    p->tuning.walk = t->walk;
    p->n_tune = 0;  // an explicit tuning replaces every autotuned one
    p->tune_next = 0;
    return FRNN_OK;
}

int frnn_plan_get_tuning(const frnn_plan* p, frnn_tuning* t)
{
    if (!p || !t) return FRNN_ERR_INVALID_ARG;
    *t = p->tuning;
    return FRNN_OK;
}

int frnn_build_graph(frnn_plan* p, const float* emb, int64_t n, int d, float r, int k_max,
                     void* stream, frnn_csr* out)
{
    frnn::NvtxRange nvtx("frnn_build_graph");
    if (!p) return FRNN_ERR_INVALID_ARG;
    if (n < 0) return FRNN_ERR_INVALID_ARG;
    const int64_t off[2] = {0, n};
    DeviceGuard dg(p->prm.device);
    if (!dg.ok) return FRNN_ERR_CUDA;
    return build_batched(p, emb, off, 1, d, r, k_max, static_cast<cudaStream_t>(stream), out);
}

int frnn_build_graph_batched(frnn_plan* p, const float* emb, const int64_t* ev_off, int n_events,
                             int d, float r, int k_max, void* stream, frnn_csr* out)
{
    frnn::NvtxRange nvtx("frnn_build_graph_batched");
    if (!p) return FRNN_ERR_INVALID_ARG;
    DeviceGuard dg(p->prm.device);
    if (!dg.ok) return FRNN_ERR_CUDA;
    return build_batched(p, emb, ev_off, n_events, d, r, k_max, static_cast<cudaStream_t>(stream), out);
}

int frnn_knn_graph_batched(frnn_plan* p, const float* emb, const int64_t* ev_off, int n_events, int d, int k,
                           void* stream, frnn_csr* out)
{
    frnn::NvtxRange nvtx("frnn_knn_graph_batched");
    if (!p) return FRNN_ERR_INVALID_ARG;
    if (k < 1) return FRNN_ERR_INVALID_ARG;
    long long n_total = 0;
    // the argument checks of the radius build, with a radius that passes them
    int rc = check_build_args(p, emb, ev_off, n_events, d, 1.0f, k, out, &n_total);
    if (rc != FRNN_OK) return rc;
    long long edges = 0;
    for (int b = 0; b < n_events; ++b) {
        const long long nb = ev_off[b + 1] - ev_off[b];
        edges += nb * (long long)(nb - 1 < k ? (nb > 0 ? nb - 1 : 0) : k);
    }
    if (edges > p->edge_cap) return FRNN_ERR_CAPACITY;
    DeviceGuard dg(p->prm.device);
    if (!dg.ok) return FRNN_ERR_CUDA;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const DevState& st = p->st;
    out->row_ptr = st.row_ptr;
    out->col = st.col;
    out->d2 = (p->prm.flags & FRNN_EMIT_D2) ? st.d2 : nullptr;
    out->edge_off = st.edge_off;
    out->n_edges = st.edge_off + n_events;
    out->n_events = n_events;
    out->n_total = n_total;
    const float inf = std::numeric_limits<float>::infinity();
    if (n_total == 0) {
        if (cudaMemsetAsync(st.row_ptr, 0, sizeof(int), s) != cudaSuccess ||
            cudaMemsetAsync(st.edge_off, 0, sizeof(int) * (n_events + 1), s) != cudaSuccess)
            return FRNN_ERR_CUDA;
        p->last = *out;
        p->last_r2 = inf;
        p->last_d = d;
        p->has_last = true;
        return FRNN_OK;
    }
    const int slot = p->ring_pos;
    p->ring_pos = (p->ring_pos + 1) % kRing;
    if (cudaEventSynchronize(p->ring_ev[slot]) != cudaSuccess) return FRNN_ERR_CUDA;
    CallHdr* h = reinterpret_cast<CallHdr*>(p->h_call[slot]);
    EvDesc* ev = reinterpret_cast<EvDesc*>(p->h_call[slot] + sizeof(CallHdr));
    const int cpp = p->prm.cells_per_point;
    const int chunk = chunk_points(p, n_total);
    int chunks = 0;
    long long e0 = 0;
    for (int b = 0; b < n_events; ++b) {
        const long long nb = ev_off[b + 1] - ev_off[b];
        const int nc = nb > 0 ? (int)((nb + chunk - 1) / chunk) : 1;
        ev[b].pt_off = ev_off[b];
        ev[b].n = (int)nb;
        ev[b].chunk_off = chunks;
        ev[b].nchunk = nc;
        ev[b].cell_budget = (int)(cpp * nb + 4096);
        ev[b].edge0 = (int)e0;
        ev[b].pad1 = 0;
        chunks += nc;
        e0 += nb * (long long)(nb - 1 < k ? (nb > 0 ? nb - 1 : 0) : k);
    }
    h->emb = emb;
    h->n_total = n_total;
    h->n_events = n_events;
    h->total_chunks = chunks;
    h->chunk = chunk;
    h->d = d;
    h->dp = (d + 3) & ~3;
    h->k = k;
    h->r = 0.f;
    h->r2 = inf;
    h->g_max = p->tuning.g_max;
    h->cell_scale = p->tuning.cell_scale;
    h->emit_d2 = (p->prm.flags & FRNN_EMIT_D2) ? 1 : 0;
    h->knn = 1;
    h->stall = p->stall_next ? 1 : 0;
    p->stall_next = false;
    h->edge_capacity = p->edge_cap;
    h->spill_capacity = 0;
    h->spill_max = 0;
    h->bbox_group = bbox_group(p, chunks);
    const size_t bytes = sizeof(CallHdr) + sizeof(EvDesc) * (size_t)n_events;
    if (cudaMemcpyAsync(p->d_call, p->h_call[slot], bytes, cudaMemcpyHostToDevice, s) != cudaSuccess)
        return FRNN_ERR_CUDA;
    if (cudaEventRecord(p->ring_ev[slot], s) != cudaSuccess) return FRNN_ERR_CUDA;
    const int cap = next_pow2((k > 32 ? k : 32) + 32);
    LaunchCfg cfg;
    rc = get_walk_cfg(p, h->dp / 4, cap, &cfg);
    if (rc != FRNN_OK) return rc;
    if (launch_knn(st, h->dp / 4, cfg, s) != 0) return FRNN_ERR_CUDA;
    p->last = *out;
    p->last_r2 = inf;
    p->last_d = d;
    p->has_last = true;
    if (p->prm.flags & FRNN_DEBUG) return run_checks(p, s);
    return FRNN_OK;
}

int frnn_build_graph_profiled(frnn_plan* p, const float* emb, const int64_t* ev_off, int n_events,
                              int d, float r, int k_max, void* stream, frnn_csr* out, float* stage_ms,
                              int n_stages)
{
    frnn::NvtxRange nvtx("frnn_build_graph_profiled");
    if (!p || !stage_ms || n_stages < kStages) return FRNN_ERR_INVALID_ARG;
    DeviceGuard dg(p->prm.device);
    if (!dg.ok) return FRNN_ERR_CUDA;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaEvent_t ev[kStages + 1] = {};
    int rc = FRNN_OK;
    for (int i = 0; i <= kStages && rc == FRNN_OK; ++i)
        if (cudaEventCreate(&ev[i]) != cudaSuccess) rc = FRNN_ERR_CUDA;
    if (rc == FRNN_OK) rc = build_batched(p, emb, ev_off, n_events, d, r, k_max, s, out, ev);
    for (int i = 0; i < kStages; ++i) stage_ms[i] = 0.f;
    if (rc == FRNN_OK && out->n_total > 0) {
        if (cudaEventSynchronize(ev[kStages]) != cudaSuccess) rc = FRNN_ERR_CUDA;
        for (int i = 0; rc == FRNN_OK && i < kStages; ++i)
            if (cudaEventElapsedTime(&stage_ms[i], ev[i], ev[i + 1]) != cudaSuccess) rc = FRNN_ERR_CUDA;
    }
    for (int i = 0; i <= kStages; ++i)
        if (ev[i]) cudaEventDestroy(ev[i]);
    return rc;
}

int frnn_plan_autotune(frnn_plan* p, const float* emb, const int64_t* ev_off, int n_events, int d, float r,
                       int k_max, void* stream, frnn_tuning* best, float* best_ms)
{
    frnn::NvtxRange nvtx("frnn_plan_autotune");
    if (!p) return FRNN_ERR_INVALID_ARG;
    DeviceGuard dg(p->prm.device);
    if (!dg.ok) return FRNN_ERR_CUDA;
    return autotune(p, emb, ev_off, n_events, d, r, k_max, static_cast<cudaStream_t>(stream), best, best_ms);
}

int frnn_plan_tuning_for(const frnn_plan* p, const int64_t* ev_off, int n_events, int d, float r, int k_max,
                         frnn_tuning* out, int* cached)
{
    if (!p || !ev_off || !out || n_events < 1) return FRNN_ERR_INVALID_ARG;
    bool c = false;
    *out = tuning_for(p, ev_off, n_events, d, r, k_max, &c);
    if (cached) *cached = c ? 1 : 0;
    return FRNN_OK;
}

int frnn_label_components(frnn_plan* p, float d2_max, void* stream, int32_t* labels)
{
    frnn::NvtxRange nvtx("frnn_label_components");
    if (!p || !labels || std::isnan(d2_max)) return FRNN_ERR_INVALID_ARG;
    if (!p->has_last) return FRNN_ERR_INVALID_ARG;
    const bool all = d2_max >= p->last_r2;
    if (!all && !(p->prm.flags & FRNN_EMIT_D2)) return FRNN_ERR_INVALID_ARG;
    DeviceGuard dg(p->prm.device);
    if (!dg.ok) return FRNN_ERR_CUDA;
    if (p->last.n_total == 0) return FRNN_OK;
    const int grid = p->n_sm * 8;
    return launch_label(p->st, reinterpret_cast<int*>(p->st.key), labels, d2_max, all ? 0 : 1, grid, stream) == 0
               ? FRNN_OK : FRNN_ERR_CUDA;
}

int frnn_edge_features(frnn_plan* p, const float* emb, int64_t e_begin, int64_t e_end, float* out, void* stream)
{
    frnn::NvtxRange nvtx("frnn_edge_features");
    if (!p || !p->has_last || e_begin < 0 || e_end < e_begin) return FRNN_ERR_INVALID_ARG;
    if (e_end > e_begin && (!emb || !out)) return FRNN_ERR_INVALID_ARG;
    if (e_end > p->edge_cap) return FRNN_ERR_INVALID_ARG;
    DeviceGuard dg(p->prm.device);
    if (!dg.ok) return FRNN_ERR_CUDA;
    if (e_end == e_begin || p->last.n_total == 0) return FRNN_OK;
    return launch_edge_features(p->st, emb, p->last_d, e_begin, e_end, out, p->n_sm, stream) == 0 ? FRNN_OK
                                                                                                : FRNN_ERR_CUDA;
}

int frnn_plan_test_stall_next_build(frnn_plan* p)
{
    if (!p) return FRNN_ERR_INVALID_ARG;
    p->stall_next = true;
    return FRNN_OK;
}

int frnn_get_last_status(frnn_plan* p, void* stream)
{
    frnn::NvtxRange nvtx("frnn_get_last_status");
    unsigned word = 0;
    const int rc = read_status_bits(p, stream, &word);
    if (rc != FRNN_OK) return rc;
    if (word & kStCheck) return FRNN_ERR_CHECK;
    if (word & kStTimeout) return FRNN_ERR_TIMEOUT;
    if (word & kStOverflow) return FRNN_ERR_OVERFLOW;
    if (word & kStNonfinite) return FRNN_ERR_NONFINITE_INPUT;
    return FRNN_OK;
}

int frnn_check_last_build(frnn_plan* p, void* stream)
{
    frnn::NvtxRange nvtx("frnn_check_last_build");
    if (!p || !p->has_last) return FRNN_ERR_INVALID_ARG;
    DeviceGuard dg(p->prm.device);
    if (!dg.ok) return FRNN_ERR_CUDA;
    return run_checks(p, static_cast<cudaStream_t>(stream));
}

int frnn_get_last_check(frnn_plan* p, void* stream, int* check, int64_t* index)
{
    if (!p || !check || !index) return FRNN_ERR_INVALID_ARG;
    DeviceGuard dg(p->prm.device);
    if (!dg.ok) return FRNN_ERR_CUDA;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    unsigned long long rec = ~0ull;
    if (cudaStreamSynchronize(s) != cudaSuccess ||
        cudaMemcpyAsync(&rec, p->chk_first, sizeof(rec), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaMemsetAsync(p->chk_first, 0xff, sizeof(rec), s) != cudaSuccess || cudaStreamSynchronize(s) != cudaSuccess) {
        cudaGetLastError();
        return FRNN_ERR_CUDA;
    }
    if (rec == ~0ull) {
        *check = FRNN_CHECK_NONE;
        *index = -1;
    } else {
        *check = (int)(rec >> 48);
        *index = (int64_t)(rec & 0xffffffffffffull);
    }
    return FRNN_OK;
}

int frnn_build_graph_host(frnn_plan* p, const float* h_emb, const int64_t* ev_off, int n_events,
                          int d, float r, int k_max, int32_t* h_row_ptr, int32_t* h_col,
                          int64_t col_capacity, int32_t* h_edge_off, int64_t* h_n_edges, void* stream)
{
    frnn::NvtxRange nvtx("frnn_build_graph_host");
    if (!p || !ev_off || !h_row_ptr || !h_n_edges || col_capacity < 0 || n_events < 1) return FRNN_ERR_INVALID_ARG;
    DeviceGuard dg(p->prm.device);
    if (!dg.ok) return FRNN_ERR_CUDA;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const long long n = ev_off[n_events];
    if (n < 0 || (n > 0 && !h_emb) || d < 1 || d > kMaxDims) return FRNN_ERR_INVALID_ARG;
    if (n > p->prm.n_max || d > p->prm.d_max) return FRNN_ERR_CAPACITY;
    const long long need = n * d;
    if (need > p->d_input_floats) return FRNN_ERR_CAPACITY;  // cannot happen: sized at creation for n_max x d_max
    if (n > 0 && cudaMemcpyAsync(p->d_input, h_emb, sizeof(float) * (size_t)need, cudaMemcpyHostToDevice, s) != cudaSuccess)
        return FRNN_ERR_CUDA;
    frnn_csr csr;
    int rc = build_batched(p, p->d_input, ev_off, n_events, d, r, k_max, s, &csr);
    if (rc != FRNN_OK) return rc;
    if (cudaMemcpyAsync(h_row_ptr, csr.row_ptr, sizeof(int32_t) * (size_t)(n + 1), cudaMemcpyDeviceToHost, s) != cudaSuccess)
        return FRNN_ERR_CUDA;
    if (h_edge_off && cudaMemcpyAsync(h_edge_off, csr.edge_off, sizeof(int32_t) * (size_t)(n_events + 1),
                                      cudaMemcpyDeviceToHost, s) != cudaSuccess)
        return FRNN_ERR_CUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return FRNN_ERR_CUDA;
    const long long e = h_row_ptr[n];
    *h_n_edges = e;
    rc = FRNN_OK;
    if (e > col_capacity || (e > 0 && !h_col)) {
        rc = FRNN_ERR_OVERFLOW;
    } else if (e > 0) {
        if (cudaMemcpyAsync(h_col, csr.col, sizeof(int32_t) * (size_t)e, cudaMemcpyDeviceToHost, s) != cudaSuccess)
            return FRNN_ERR_CUDA;
    }
    const int st = frnn_get_last_status(p, stream);
    return st != FRNN_OK ? st : rc;
}

}  // extern "C"

int frnn::read_status_bits(frnn_plan* p, void* stream, unsigned* bits)
{
    if (!p || !bits) return FRNN_ERR_INVALID_ARG;
    *bits = 0;
    DeviceGuard dg(p->prm.device);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (cudaStreamSynchronize(s) != cudaSuccess) {
        cudaGetLastError();
        return FRNN_ERR_CUDA;
    }
    unsigned word = 0;
    if (cudaMemcpyAsync(&word, p->st.status, sizeof(unsigned), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaMemsetAsync(p->st.status, 0, sizeof(unsigned), s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess) {
        cudaGetLastError();
        return FRNN_ERR_CUDA;
    }
    if (word & kStTimeout) recover_after_timeout(p, stream);
    *bits = word;
    return FRNN_OK;
}

int frnn::enqueue_status_read(frnn_plan* p, void* stream, unsigned* h_word)
{
    DeviceGuard dg(p->prm.device);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (cudaMemcpyAsync(h_word, p->st.status, sizeof(unsigned), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaMemsetAsync(p->st.status, 0, sizeof(unsigned), s) != cudaSuccess) {
        cudaGetLastError();
        return 1;
    }
    return 0;
}

int frnn::recover_after_timeout(frnn_plan* p, void* stream)
{
    // a wait gave up part-way: restore the between-builds state; the last
    // graph is not valid, so labeling and edge features refuse it
    DeviceGuard dg(p->prm.device);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int rc = reset_device_state(p, s);
    const bool ok = cudaStreamSynchronize(s) == cudaSuccess;
    p->has_last = false;
    return (rc == FRNN_OK && ok) ? FRNN_OK : FRNN_ERR_CUDA;
}
