// Internal data structures shared by the kernels and the host side of libfrnn.
#pragma once

#include <cstdint>

#include <nvtx3/nvToolsExt.h>

struct frnn_plan;

namespace frnn {

constexpr int kMaxG = 6;            // most gridded dimensions (3^(g-1) runs per cell)
constexpr int kMaxRuns = 243;       // 3^(kMaxG - 1)
constexpr int kMaxDims = 64;        // largest embedding dimension
constexpr int kChunk = 2048;        // points per chunk of the per-point kernels, at most
constexpr int kChunkMin = 256;      // ... and at least (small builds: more chunks than blocks)
constexpr int kPtThreads = 256;     // threads of the per-point kernels
constexpr int kScanThreads = 256;
constexpr int kScanItems = 8;                                  // cell scan: 2048 cells per tile
constexpr int kScanTile = kScanThreads * kScanItems;
constexpr int kRowScanItems = 2;                               // row scan: 512 points per tile (it also
constexpr int kRowScanTile = kScanThreads * kRowScanItems;     // copies their rows: more tiles, more warps)
constexpr int kWalkThreads = 128;   // collect walk: 4 warps, 32 queries per warp at a time
constexpr int kFillThreads = 128;   // fill walk: 4 warps (more shared memory per warp)
constexpr int kMaxDimCells = 32768; // cells along one hashed dimension (float32 key bound)
constexpr int kSpillSlots = 384;    // neighbour positions kept per long row in the spill area

// Bits of the device status word (1 << frnn_status).
constexpr unsigned kStNonfinite = 1u << 4;
constexpr unsigned kStTimeout = 1u << 5;
constexpr unsigned kStOverflow = 1u << 6;
constexpr unsigned kStCheck = 1u << 8;  // a debug check of the build's output failed

// Written by the host once per call and uploaded in front of the event table.
struct CallHdr {
    const float* emb;    // device [n_total][d], caller-owned
    long long n_total;   // points of the call
    int n_events;
    int total_chunks;    // sum over events of max(1, ceil(n_b / chunk))
    int chunk;           // points per chunk of the per-point kernels (kChunkMin .. kChunk)
    int d;
    int dp;              // row length of the sorted copy (d rounded up to 4)
    int k;               // neighbour cap
    float r;
    float r2;            // fl32(r * r)
    int g_max;           // tuning: most hashed dims
    float cell_scale;    // tuning: cell edge / r (>= 1)
    int emit_d2;
    int knn;             // 1: k nearest with no radius (cell edge from density; r unused)
    int stall;           // 1: the cell scan's first tile waits for a predecessor that never
                         // publishes, so its bounded waits run out (failure-detection tests)
    long long edge_capacity;
    long long spill_capacity;  // entries of the neighbour-position spill area (0: none)
    int spill_max;             // most hits a spilled row may have (0: rows are never spilled)
    int bbox_group;            // consecutive chunks the bounding-box kernel takes at a time (0: 1)
};

struct EvDesc {
    long long pt_off;    // first point of the event within the call
    int n;               // points
    int chunk_off;       // first chunk of the event
    int nchunk;          // chunks (>= 1, also for an empty event)
    int cell_budget;     // cell slots the event may use
    int edge0;           // kNN builds: first edge of the event (rows of fixed length)
    int pad1;
};

// Written on the device by the planning step (one per event).
struct EvPlan {
    float lo[kMaxG];     // lower corner of the grid along each hashed dim
    float s;             // cell edge
    float inv_s;         // fl32(1 / s)
    int g;               // hashed dims (>= 1)
    int skip;            // 1: the event holds a non-finite value, rows are left empty
    int dims[kMaxG];     // which embedding dims are hashed (widest first)
    int ncell[kMaxG];
    int stride[kMaxG];   // linear cell id = sum k_t * stride_t; dims[g-1] is fastest
    int n_cells;
    int cell_off;        // first global cell slot of the event
};

// Written on the device by the planning step (one per event): the
// candidate filter.  Every point gets a 4-byte key, one byte per filter dim,
// q_t = floor((x_t - lo_t) * inv_h) with a single step 1 / inv_h for the four
// dims (the widest dims the grid leaves out first).  For two points within r,
// sum_t |q_t - q'_t| <= thr, so a candidate whose keys fail that test is
// skipped without reading its coordinates (the bound is argued in plan_filter).
constexpr int kFiltDims = 4;
struct FiltPlan {
    int dim[kFiltDims];  // embedding dim of each key byte, or -1 (byte 0)
    float lo[kFiltDims];
    float inv_h;         // 0: every key is 0 (the filter passes everything)
    int thr;
    int pad[2];
};

// Counter slots (all return to zero at the end of every build).
enum { kCtrPlanned = 0, kCtrScanCellsTile, kCtrScanCellsExit, kCtrScanRowsTile,
       kCtrScanRowsExit, kCtrLongRows, kCtrWalkChunks, kCtrEmitRows, kCtrLabelCapped, kCtrKeptRows,
       kCtrCount = 16 };

// Device pointers owned by the plan.  Fixed for the plan's life, so a
// captured CUDA graph of the build stays valid for every call: everything
// that changes per call is read from *hdr and ev[].
struct DevState {
    const CallHdr* hdr;
    const EvDesc* ev;
    EvPlan* plan;
    int2* run_tab;           // [events_max * kMaxRuns] per event and run: cell offset, off-grid dim masks
    unsigned* bb_min;        // [events_max * kMaxDims] order-preserving encodings
    unsigned* bb_max;
    unsigned* chunk_done;    // [events_max]
    unsigned* nonfinite;     // [events_max]
    unsigned* counters;      // [kCtrCount]
    int* cells_total;
    unsigned* key;           // [n_max] cell id of each input point (event-local)
    unsigned* rank;          // [n_max] slot of the point inside its cell (until the scatter);
                             // then the list of long rows (collect walk -> emit walk)
    int* perm;               // [n_max] sorted position -> event-local point index
    unsigned* cell_s;        // [n_max] sorted position -> cell id
    float* xs;               // [n_max * dp_max] points in cell order, rows padded with 0
    unsigned* xq;            // [roundup(n_max, 8) + 8] filter key of each point, in cell order
    FiltPlan* fplan;         // [events_max]
    int* pool_off;           // [n_max] point -> first pool slot of its row, or -1
    int* cnt_o;              // [n_max] point -> min(|S_i|, k)
    int* row_ptr;            // [n_max + 1]
    unsigned* cell_count;    // [cells_max], zero between builds
    int* cell_start;         // [cells_max + 1]
    unsigned long long* scan_cells;  // [tiles], zero between builds
    unsigned long long* scan_rows;
    int* col;
    float* d2;
    int* pool;               // [edge_capacity] short rows, sorted, parked by the collect walk
    float* pool_d2;          // [edge_capacity] their d2 (FRNN_EMIT_D2 only)
    unsigned long long* pool_ctr;  // next free pool slot; zero between builds
    int* edge_off;           // [events_max + 1]
    unsigned* status;
    // Nonzero once the scatter has seen a coordinate off the exact fast
    // path's grid (cleared by the bounding-box pass of every build): while it
    // is zero, squared distances may be accumulated with fused multiply-adds.
    unsigned* offgrid;
    // Long rows (more than kFast neighbours) whose neighbours the collect walk
    // keeps: per chunk that has one, 32 x kSpillSlots positions taken from
    // spill_ctr; per entry of the emit walk's list, the row's first position
    // in spill (or -1: walk its candidates again) and its hit count.
    int* spill;              // [spill_capacity] sorted positions of a long row's neighbours (and itself)
    unsigned long long* spill_ctr;  // next free spill entry; zero between builds
    long long* spill_at;     // [n_max]
    int* spill_n;            // [n_max]
};

#ifdef __CUDACC__
// A bounded wait of this build, or of an earlier one whose status has not
// been read yet, ran out: cell and row offsets may be wrong, so the kernels
// that address memory through them skip their work.
__device__ __forceinline__ bool timed_out(const DevState& st)
{
    return (__ldcg(st.status) & kStTimeout) != 0u;
}
#endif

// A named NVTX range over a host call of the library: the kernels it launches
// fall inside it for timeline tools and for ncu's --nvtx filters.  Without an
// attached tool a push or pop costs one test of a function pointer.
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};

// Forms of the collect walk (frnn_tuning.walk).
constexpr int kWalkAuto = 0;
constexpr int kWalkCandMajor = 1;   // lanes hold candidates; a segment's queries in packed pairs
constexpr int kWalkQueryMajor = 2;  // a lane per query streams its segment's candidates (d <= 12)
constexpr int kMaxDp4QueryMajor = 3;

// The collect walk a build runs: the query-major form where it exists
// (rows of up to 12 floats) unless the tuning asks for the other.
inline int resolve_walk(int walk, int dp4)
{
    if (dp4 > kMaxDp4QueryMajor) return kWalkCandMajor;
    return walk == kWalkCandMajor ? kWalkCandMajor : kWalkQueryMajor;
}

struct LaunchCfg {
    int grid_pt;       // per-point kernels (persistent: blocks loop over chunks)
    int grid_scatter;  // scatter: as many blocks as are resident at once
    int grid_scan;     // scans (persistent: blocks take tiles from a counter)
    int grid_count;    // count walk (persistent: warps stride over queries)
    int grid_count_q;  // its query-major form
    int grid_fill;     // fill walk
    int fill_cap;      // per-warp key buffer of the fill walk (power of two, >= k + 32)
    int fill_smem;     // its dynamic shared memory in bytes
};

// Host-side launchers (frnn_kernels.cu).  All return a cudaError_t value.
// stage_events: NULL, or kStages + 1 cudaEvent_t recorded around the stages.
constexpr int kStages = 7;  // the last (emit) stage is two kernels: kept-hit rows, then rows walked again
// walk: kWalkCandMajor or kWalkQueryMajor (the latter for dp4 <= kMaxDp4QueryMajor only).
int launch_build(const DevState& st, int dp4, const LaunchCfg& cfg, int walk, void* stream, void* stage_events);
int config_walk(int dp4, int fill_cap, int n_sm, LaunchCfg* cfg);
// Weakly connected components of the last build (frnn_label.cu); parent is
// n_total ints of scratch, labels receives event-local component labels.
int launch_label(const DevState& st, int* parent, int* labels, float d2_max, int use_d2, int grid, void* stream);
// Edge features [x_i, x_j, d2] of edges [e_begin, e_end) of the last build (frnn_label.cu).
int launch_edge_features(const DevState& st, const float* emb, int d, long long e_begin, long long e_end,
                         float* out, int n_sm, void* stream);
int config_pt(int n_sm, LaunchCfg* cfg);
// Autotuner probe: stages 1-3 of a radius build on the current tuning, then
// out[0] = candidate tests a collect walk would make, out[1] = non-empty
// cells, out[2] = cell slots scanned (device, 3 x u64).  Leaves the plan's
// between-builds state as a build does.
int launch_probe(const DevState& st, const LaunchCfg& cfg, unsigned long long* out, void* stream);
// The k-nearest-neighbour build (no radius): grid, fixed-length rows, ring walk.
int launch_knn(const DevState& st, int dp4, const LaunchCfg& cfg, void* stream);

// Debug checks of the last build (frnn_debug.cu): kernels that only read the
// build's buffers and its input; a failure sets kStCheck in the status word
// and lowers *first to (check id << 48 | index).  bits: (n_max + 31) / 32
// words of scratch, cleared here.  n_total, n_events, d: those of the last
// build (nothing is checked for n_total = 0).  Returns 0 or 1 (a CUDA error).
int launch_checks(const DevState& st, unsigned long long* first, unsigned* bits, long long n_total,
                  int n_events, long long cells_max, int d, int n_sm, void* stream);

// Synchronise the stream, then return in *bits and clear the status bits the
// plan's kernels latched (kStNonfinite, kStTimeout, kStOverflow); after a
// timeout the plan's between-builds state is restored, as by
// frnn_get_last_status (frnn_api.cu).  Returns FRNN_OK or an error status.
int read_status_bits(struct ::frnn_plan* p, void* stream, unsigned* bits);

// Without a synchronisation: enqueue on the stream a copy of the plan's
// status word into *h_word (pinned host memory), then its reset; the word is
// valid once the stream has passed this point.  Returns 0 or 1 (a CUDA
// error).  A word holding kStTimeout must be followed by
// recover_after_timeout before the plan's next build.
int enqueue_status_read(struct ::frnn_plan* p, void* stream, unsigned* h_word);

// Restore the plan's between-builds state after a bounded wait ran out and
// forget its last build, as frnn_get_last_status does (synchronous).
int recover_after_timeout(struct ::frnn_plan* p, void* stream);

}  // namespace frnn
