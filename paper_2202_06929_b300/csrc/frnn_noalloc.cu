// frnn_build_graph_noalloc: the graph build of one event without any device
// allocation, for callers that cannot call cudaMalloc.
//
// Some callers of a graph builder cannot allocate device memory at the point
// where they need the graph: code that runs inside a framework which hands
// out all device memory from its own pool and forbids allocation after
// start-up (real-time trigger farms are built that way), code whose device
// memory budget is fixed once at initialisation, and code that must not
// perform the implicit device-wide synchronisation cudaMalloc can imply.
// They still own their inputs and outputs, so this entry point takes the
// points, row_ptr and col from the caller and keeps every other buffer of
// the build in one statically sized array in device memory, declared below.
//
// That array exists once per device that loads the library, for as long as
// the process lives, and every call on that device shares it: calls whose
// work overlaps on the GPU (two streams, or two host threads) race on it and
// must be serialised by the caller.  Each call clears the parts that must
// start at zero before it runs, so a call never depends on what the previous
// one left behind.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <mutex>

#include "frnn.h"
#include "frnn_internal.h"

using namespace frnn;

namespace {

// Limits of one call (the array below is sized for them).
constexpr long long kNoallocMaxPoints = 32768;
constexpr int kNoallocMaxDims = 16;
constexpr int kNoallocMaxK = 64;
constexpr long long kNoallocCells = 4 * kNoallocMaxPoints + 4096;  // 4 slots per point + 4096
constexpr long long kNoallocPool = kNoallocMaxPoints * kNoallocMaxK;

constexpr size_t align256(size_t v) { return (v + 255) & ~size_t(255); }

// Byte offsets of the buffers inside the static array.
constexpr size_t kOffHdr = 0;
constexpr size_t kOffEv = align256(kOffHdr + sizeof(CallHdr));
constexpr size_t kOffPlan = align256(kOffEv + sizeof(EvDesc));
constexpr size_t kOffRunOff = align256(kOffPlan + sizeof(EvPlan));
constexpr size_t kOffBbMin = align256(kOffRunOff + sizeof(int2) * kMaxRuns);
constexpr size_t kOffBbMax = align256(kOffBbMin + sizeof(unsigned) * kMaxDims);
constexpr size_t kOffChunkDone = align256(kOffBbMax + sizeof(unsigned) * kMaxDims);
constexpr size_t kOffNonfinite = align256(kOffChunkDone + sizeof(unsigned));
constexpr size_t kOffCounters = align256(kOffNonfinite + sizeof(unsigned));
constexpr size_t kOffCellsTotal = align256(kOffCounters + sizeof(unsigned) * kCtrCount);
constexpr size_t kOffPoolCtr = align256(kOffCellsTotal + sizeof(int));
constexpr size_t kOffEdgeOff = align256(kOffPoolCtr + sizeof(unsigned long long));
constexpr size_t kOffStatus = align256(kOffEdgeOff + 2 * sizeof(int));
constexpr size_t kOffOffgrid = align256(kOffStatus + sizeof(unsigned));
constexpr size_t kOffKey = align256(kOffOffgrid + sizeof(unsigned));
constexpr size_t kOffRank = align256(kOffKey + sizeof(unsigned) * kNoallocMaxPoints);
constexpr size_t kOffPerm = align256(kOffRank + sizeof(unsigned) * kNoallocMaxPoints);
constexpr size_t kOffCellS = align256(kOffPerm + sizeof(int) * kNoallocMaxPoints);
constexpr size_t kOffPoolOff = align256(kOffCellS + sizeof(unsigned) * kNoallocMaxPoints);
constexpr size_t kOffCntO = align256(kOffPoolOff + sizeof(int) * kNoallocMaxPoints);
constexpr size_t kOffXs = align256(kOffCntO + sizeof(int) * kNoallocMaxPoints);
constexpr size_t kOffXq = align256(kOffXs + sizeof(float) * kNoallocMaxPoints * kNoallocMaxDims);
constexpr size_t kOffFplan = align256(kOffXq + sizeof(unsigned) * (kNoallocMaxPoints + 8));
constexpr size_t kOffCellCount = align256(kOffFplan + sizeof(FiltPlan));
constexpr size_t kOffCellStart = align256(kOffCellCount + sizeof(unsigned) * kNoallocCells);
constexpr long long kTilesCells = kNoallocCells / kScanTile + 1;
constexpr long long kTilesRows = kNoallocMaxPoints / kRowScanTile + 1;
constexpr size_t kOffScanCells = align256(kOffCellStart + sizeof(int) * (kNoallocCells + 1));
constexpr size_t kOffScanRows = align256(kOffScanCells + sizeof(unsigned long long) * kTilesCells);
constexpr size_t kOffPool = align256(kOffScanRows + sizeof(unsigned long long) * kTilesRows);
constexpr size_t kArenaBytes = align256(kOffPool + sizeof(int) * kNoallocPool);  // about 12.5 MB

// The scratch of every call on this device (see the file comment).
static __device__ __align__(256) unsigned char g_noalloc_scratch[kArenaBytes];

// Per-device set-up, done by the first call on each device.
struct DeviceSetup {
    unsigned char* base = nullptr;  // device address of g_noalloc_scratch
    int n_sm = 0;
    bool cfg_ok[17] = {};
    LaunchCfg cfg[17];
};
constexpr int kMaxDevices = 64;
DeviceSetup g_setup[kMaxDevices];
std::mutex g_setup_mutex;

__global__ void k_noalloc_header(CallHdr h, EvDesc e, CallHdr* dst_h, EvDesc* dst_e)
{
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        *dst_h = h;
        *dst_e = e;
    }
}

// Device-side outcome of the build as an frnn_status, in the severity order
// of frnn_get_last_status().
__global__ void k_noalloc_status(const unsigned* word, int32_t* out)
{
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        const unsigned w = *word;
        *out = (w & kStTimeout) ? FRNN_ERR_TIMEOUT
             : (w & kStOverflow) ? FRNN_ERR_OVERFLOW
             : (w & kStNonfinite) ? FRNN_ERR_NONFINITE_INPUT : FRNN_OK;
    }
}

int next_pow2(int v)
{
    int p = 1;
    while (p < v) p <<= 1;
    return p;
}

}  // namespace

extern "C" int frnn_build_graph_noalloc(const float* emb, int64_t n, int d, float r, int k_max,
                                        int32_t* row_ptr, int32_t* col, int64_t col_capacity,
                                        int32_t* status, void* stream)
{
    frnn::NvtxRange nvtx("frnn_build_graph_noalloc");
    if (n < 0 || d < 1 || k_max < 1 || !row_ptr || !status || col_capacity < 0) return FRNN_ERR_INVALID_ARG;
    if (!(r > 0.0f) || !std::isfinite(r) || !(r * r > 0.0f) || !std::isfinite(r * r)) return FRNN_ERR_INVALID_ARG;
    if (n > 0 && (!emb || (reinterpret_cast<uintptr_t>(emb) & 3u))) return FRNN_ERR_INVALID_ARG;
    if (col_capacity > 0 && !col) return FRNN_ERR_INVALID_ARG;
    if (n > kNoallocMaxPoints || d > kNoallocMaxDims || k_max > kNoallocMaxK) return FRNN_ERR_CAPACITY;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        cudaGetLastError();
        return FRNN_ERR_CUDA;
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int dp4 = (d + 3) / 4;
    DeviceSetup* ds = &g_setup[dev];
    LaunchCfg cfg;
    {
        std::lock_guard<std::mutex> lock(g_setup_mutex);
        if (!ds->base || !ds->cfg_ok[dp4]) {
            // The set-up below makes calls that are not stream-ordered; under
            // stream capture they would fail or invalidate the capture, so a
            // set-up call on a capturing stream is refused before any of them.
            cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
            if (cudaStreamIsCapturing(s, &cap) != cudaSuccess || cap != cudaStreamCaptureStatusNone) {
                cudaGetLastError();
                return FRNN_ERR_INVALID_ARG;
            }
        }
        if (!ds->base) {
            // Host code must not use g_noalloc_scratch directly (its host-side
            // name is not a device address): fetch the address once per device.
            void* ptr = nullptr;
            if (cudaGetSymbolAddress(&ptr, g_noalloc_scratch) != cudaSuccess || !ptr) {
                cudaGetLastError();
                return FRNN_ERR_CUDA;
            }
            int n_sm = 0;
            if (cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
                cudaGetLastError();
                return FRNN_ERR_CUDA;
            }
            ds->n_sm = n_sm;
            ds->base = static_cast<unsigned char*>(ptr);
        }
        if (!ds->cfg_ok[dp4]) {
            LaunchCfg c{};
            if (config_pt(ds->n_sm, &c) != 0 || config_walk(dp4, next_pow2(kNoallocMaxK + 32), ds->n_sm, &c) != 0) {
                cudaGetLastError();
                return FRNN_ERR_CUDA;
            }
            ds->cfg[dp4] = c;
            ds->cfg_ok[dp4] = true;
        }
        cfg = ds->cfg[dp4];
    }
    unsigned char* b = ds->base;
    DevState st{};
    st.hdr = reinterpret_cast<const CallHdr*>(b + kOffHdr);
    st.ev = reinterpret_cast<const EvDesc*>(b + kOffEv);
    st.plan = reinterpret_cast<EvPlan*>(b + kOffPlan);
    st.run_tab = reinterpret_cast<int2*>(b + kOffRunOff);
    st.bb_min = reinterpret_cast<unsigned*>(b + kOffBbMin);
    st.bb_max = reinterpret_cast<unsigned*>(b + kOffBbMax);
    st.chunk_done = reinterpret_cast<unsigned*>(b + kOffChunkDone);
    st.nonfinite = reinterpret_cast<unsigned*>(b + kOffNonfinite);
    st.counters = reinterpret_cast<unsigned*>(b + kOffCounters);
    st.cells_total = reinterpret_cast<int*>(b + kOffCellsTotal);
    st.key = reinterpret_cast<unsigned*>(b + kOffKey);
    st.rank = reinterpret_cast<unsigned*>(b + kOffRank);
    st.perm = reinterpret_cast<int*>(b + kOffPerm);
    st.cell_s = reinterpret_cast<unsigned*>(b + kOffCellS);
    st.xs = reinterpret_cast<float*>(b + kOffXs);
    st.xq = reinterpret_cast<unsigned*>(b + kOffXq);
    st.fplan = reinterpret_cast<FiltPlan*>(b + kOffFplan);
    st.pool_off = reinterpret_cast<int*>(b + kOffPoolOff);
    st.cnt_o = reinterpret_cast<int*>(b + kOffCntO);
    st.row_ptr = row_ptr;
    st.cell_count = reinterpret_cast<unsigned*>(b + kOffCellCount);
    st.cell_start = reinterpret_cast<int*>(b + kOffCellStart);
    st.scan_cells = reinterpret_cast<unsigned long long*>(b + kOffScanCells);
    st.scan_rows = reinterpret_cast<unsigned long long*>(b + kOffScanRows);
    st.col = col;
    st.d2 = nullptr;
    st.pool = reinterpret_cast<int*>(b + kOffPool);
    st.pool_d2 = nullptr;
    st.pool_ctr = reinterpret_cast<unsigned long long*>(b + kOffPoolCtr);
    st.edge_off = reinterpret_cast<int*>(b + kOffEdgeOff);
    st.status = reinterpret_cast<unsigned*>(b + kOffStatus);
    st.offgrid = reinterpret_cast<unsigned*>(b + kOffOffgrid);

    // Everything that must start at zero (or at the empty bounding box) is
    // cleared here, on the caller's stream, before the build runs.
    bool ok = true;
    ok &= cudaMemsetAsync(st.bb_min, 0xff, sizeof(unsigned) * kMaxDims, s) == cudaSuccess;
    ok &= cudaMemsetAsync(st.bb_max, 0, sizeof(unsigned) * kMaxDims, s) == cudaSuccess;
    ok &= cudaMemsetAsync(st.chunk_done, 0, sizeof(unsigned), s) == cudaSuccess;
    ok &= cudaMemsetAsync(st.nonfinite, 0, sizeof(unsigned), s) == cudaSuccess;
    ok &= cudaMemsetAsync(st.counters, 0, sizeof(unsigned) * kCtrCount, s) == cudaSuccess;
    ok &= cudaMemsetAsync(st.pool_ctr, 0, sizeof(unsigned long long), s) == cudaSuccess;
    ok &= cudaMemsetAsync(st.status, 0, sizeof(unsigned), s) == cudaSuccess;
    ok &= cudaMemsetAsync(st.cell_count, 0, sizeof(unsigned) * kNoallocCells, s) == cudaSuccess;
    ok &= cudaMemsetAsync(st.scan_cells, 0, sizeof(unsigned long long) * kTilesCells, s) == cudaSuccess;
    ok &= cudaMemsetAsync(st.scan_rows, 0, sizeof(unsigned long long) * kTilesRows, s) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        return FRNN_ERR_CUDA;
    }
    if (n == 0) {
        if (cudaMemsetAsync(row_ptr, 0, sizeof(int32_t), s) != cudaSuccess ||
            cudaMemsetAsync(status, 0, sizeof(int32_t), s) != cudaSuccess) {
            cudaGetLastError();
            return FRNN_ERR_CUDA;
        }
        return FRNN_OK;
    }
    const long long cap_edges = n * (long long)k_max;
    // points per chunk of the per-point kernels: as for a plan's build, the
    // smallest power of two from kChunkMin that leaves at most about two
    // chunks per block, so that a small event still spreads over the SMs
    int chunk = kChunkMin;
    while (chunk < kChunk && (n + chunk - 1) / chunk > 2ll * cfg.grid_pt) chunk *= 2;
    CallHdr h{};
    h.emb = emb;
    h.n_total = n;
    h.n_events = 1;
    h.total_chunks = (int)((n + chunk - 1) / chunk);
    h.chunk = chunk;
    h.d = d;
    h.dp = dp4 * 4;
    h.k = k_max;
    h.r = r;
    h.r2 = r * r;
    h.g_max = 4;
    h.cell_scale = 1.0f;
    h.emit_d2 = 0;
    h.edge_capacity = col_capacity < cap_edges ? col_capacity : cap_edges;
    EvDesc e{};
    e.pt_off = 0;
    e.n = (int)n;
    e.chunk_off = 0;
    e.nchunk = h.total_chunks;
    e.cell_budget = (int)(4 * n + 4096);
    k_noalloc_header<<<1, 32, 0, s>>>(h, e, reinterpret_cast<CallHdr*>(b + kOffHdr),
                                      reinterpret_cast<EvDesc*>(b + kOffEv));
    if (cudaGetLastError() != cudaSuccess) return FRNN_ERR_CUDA;
    if (launch_build(st, dp4, cfg, resolve_walk(kWalkAuto, dp4), s, nullptr) != 0) {
        cudaGetLastError();
        return FRNN_ERR_CUDA;
    }
    k_noalloc_status<<<1, 32, 0, s>>>(st.status, status);
    return cudaGetLastError() == cudaSuccess ? FRNN_OK : FRNN_ERR_CUDA;
}
