// Debug checks of a build's output (FRNN_DEBUG, frnn_check_last_build).
//
// Each kernel re-derives what one stage of the build must have produced and
// compares: the per-event edge offsets, the cell table (the cell lists of
// Sec. 3.4), the scatter into cell order, the row offsets, every edge (its
// column, its distance against the radius, its emitted d2, the (d2, j) order
// of its row) and, by brute force over the event, that each row holds
// exactly the points it must (Sec. 3.1: the k nearest within the radius).
// The kernels only read the build's buffers and its input.  Every index
// taken from those buffers is range-checked before it addresses memory, so
// a corrupt buffer gives a recorded failure, never a fault.
#include <cuda_runtime.h>

#include <climits>

#include "frnn.h"
#include "frnn_internal.h"

namespace frnn {
namespace {

constexpr int kChkThreads = 128;
constexpr long long kBrutePairs = 1ll << 34;  // distance evaluations per event, at most

struct Chk {
    unsigned long long* first;  // lowest (check id << 48 | index) seen
    unsigned* status;
    unsigned* bits;             // one bit per point of the call: seen in the sorted order
    long long cells_max;        // slots of the cell table
};

__device__ void fail(const Chk& c, int id, long long where)
{
    const unsigned long long rec = ((unsigned long long)id << 48) | ((unsigned long long)where & 0xffffffffffffull);
    atomicMin(c.first, rec);
    atomicOr(c.status, kStCheck);
}

// The event holding position p of the call (an empty event starts where the
// next one does; the later, non-empty one is returned).
__device__ int event_at(const EvDesc* ev, int n_events, long long p)
{
    int lo = 0, hi = n_events - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (ev[mid].pt_off <= p) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// d2 as the build defines it: float32, dims summed in order, every
// subtraction, product and sum rounded once (no fused multiply-add).
__device__ float dist2(const float* a, const float* b, int d)
{
    float s = 0.f;
    for (int t = 0; t < d; ++t) {
        const float u = __fsub_rn(__ldg(a + t), __ldg(b + t));
        s = __fadd_rn(s, __fmul_rn(u, u));
    }
    return s;
}

// The same with the query's row held in registers (d <= DR).
template <int DR>
__device__ __forceinline__ float dist2_reg(const float (&x)[DR], const float* b, int d)
{
    float s = 0.f;
#pragma unroll
    for (int t = 0; t < DR; ++t) {
        if (t < d) {
            const float u = __fsub_rn(x[t], __ldg(b + t));
            s = __fadd_rn(s, __fmul_rn(u, u));
        }
    }
    return s;
}

// Per-event offsets and the cell table: an event's cells cover its sorted
// positions pt_off .. pt_off + n - 1 in ascending order.
__global__ void __launch_bounds__(kChkThreads) k_check_events(DevState st, Chk c)
{
    if (timed_out(st)) return;
    const CallHdr h = *st.hdr;
    for (int b = blockIdx.x; b < h.n_events; b += gridDim.x) {
        const EvDesc e = st.ev[b];
        if (threadIdx.x == 0) {
            if (st.edge_off[b] != st.row_ptr[e.pt_off]) fail(c, FRNN_CHECK_EVENT_OFFSETS, b);
            if (b == h.n_events - 1 && st.edge_off[h.n_events] != st.row_ptr[h.n_total])
                fail(c, FRNN_CHECK_EVENT_OFFSETS, h.n_events);
        }
        if (e.n == 0) continue;
        const long long c0 = st.plan[b].cell_off, nc = st.plan[b].n_cells;
        if (c0 < 0 || nc < 1 || c0 + nc > c.cells_max) {
            if (threadIdx.x == 0) fail(c, FRNN_CHECK_CELL_TABLE, c0 < 0 ? 0 : c0);
            continue;
        }
        if (threadIdx.x == 0) {
            if (st.cell_start[c0] != e.pt_off) fail(c, FRNN_CHECK_CELL_TABLE, c0);
            if (st.cell_start[c0 + nc] != e.pt_off + e.n) fail(c, FRNN_CHECK_CELL_TABLE, c0 + nc);
        }
        for (long long q = threadIdx.x; q < nc; q += blockDim.x)
            if (st.cell_start[c0 + q + 1] < st.cell_start[c0 + q]) fail(c, FRNN_CHECK_CELL_TABLE, c0 + q + 1);
    }
}

// The scatter: sorted position pos holds a point of its event that no other
// position holds, inside the range of the cell it is listed under, and its
// sorted row is the input row bit for bit, padded with zeros.
__global__ void __launch_bounds__(kChkThreads) k_check_sorted(DevState st, Chk c)
{
    if (timed_out(st)) return;
    const CallHdr h = *st.hdr;
    const long long step = (long long)gridDim.x * blockDim.x;
    for (long long pos = blockIdx.x * (long long)blockDim.x + threadIdx.x; pos < h.n_total; pos += step) {
        const int b = event_at(st.ev, h.n_events, pos);
        const EvDesc e = st.ev[b];
        const int pi = st.perm[pos];
        if (pi < 0 || pi >= e.n) {
            fail(c, FRNN_CHECK_SCATTER, pos);
            continue;
        }
        const long long p = e.pt_off + pi;
        const unsigned m = 1u << (p & 31);
        if (atomicOr(c.bits + (p >> 5), m) & m) fail(c, FRNN_CHECK_SCATTER, pos);
        const long long c0 = st.plan[b].cell_off, nc = st.plan[b].n_cells;
        const unsigned cell = st.cell_s[pos];
        if (c0 < 0 || nc < 1 || c0 + nc > c.cells_max || (long long)cell >= nc) {
            fail(c, FRNN_CHECK_SCATTER, pos);
            continue;
        }
        if (!(st.cell_start[c0 + cell] <= pos && pos < st.cell_start[c0 + cell + 1])) fail(c, FRNN_CHECK_SCATTER, pos);
        const float* x = h.emb + p * h.d;
        const float* y = st.xs + pos * h.dp;
        for (int t = 0; t < h.dp; ++t) {
            const unsigned want = t < h.d ? __float_as_uint(__ldg(x + t)) : 0u;
            if (__float_as_uint(y[t]) != want) {
                fail(c, FRNN_CHECK_SCATTER, pos);
                break;
            }
        }
    }
}

// Whether row p's entries must come in (d2, j) order: every row but those
// longer than 32 of a build without a cap.
__device__ __forceinline__ bool row_sorted(const CallHdr& h, long long len)
{
    return h.knn || h.k != INT_MAX || len <= 32;
}

// Row offsets and every edge of the row.
__global__ void __launch_bounds__(kChkThreads) k_check_rows(DevState st, Chk c)
{
    if (timed_out(st)) return;
    const CallHdr h = *st.hdr;
    const long long total = st.row_ptr[h.n_total];
    const bool cols = total >= 0 && total <= h.edge_capacity;  // else the edges overflowed: columns unchecked
    const long long step = (long long)gridDim.x * blockDim.x;
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < h.n_total; p += step) {
        const int b = event_at(st.ev, h.n_events, p);
        const EvDesc e = st.ev[b];
        const long long i = p - e.pt_off;
        const bool skip = st.plan[b].skip != 0;
        const long long s0 = st.row_ptr[p], s1 = st.row_ptr[p + 1];
        if (p == 0 && s0 != 0) fail(c, FRNN_CHECK_ROW_PTR, 0);
        if (s0 < 0 || s1 < s0) {
            fail(c, FRNN_CHECK_ROW_PTR, p);
            continue;
        }
        const long long len = s1 - s0;
        if (h.knn) {
            const long long kb = min((long long)h.k, (long long)e.n - 1);
            if (len != kb) {
                fail(c, FRNN_CHECK_ROW_PTR, p);
                continue;
            }
        } else if (len > (skip ? 0ll : (long long)h.k)) {
            fail(c, FRNN_CHECK_ROW_PTR, p);
            continue;
        }
        if (!cols || s1 > h.edge_capacity) continue;
        if (h.knn && skip) {  // rows of an event with NaN or Inf: column -1, d2 +Inf
            for (long long t = s0; t < s1; ++t) {
                if (st.col[t] != -1) {
                    fail(c, FRNN_CHECK_COLUMN, t);
                    break;
                }
                if (h.emit_d2 && __float_as_uint(st.d2[t]) != 0x7f800000u) {
                    fail(c, FRNN_CHECK_D2, t);
                    break;
                }
            }
            continue;
        }
        const float* xi = h.emb + p * h.d;
        const bool sorted = row_sorted(h, len);
        float pd = 0.f;
        int pj = -1;
        for (long long t = s0; t < s1; ++t) {
            const int j = st.col[t];
            if (j < 0 || j >= e.n || j == i) {
                fail(c, FRNN_CHECK_COLUMN, t);
                break;
            }
            const float d2 = dist2(xi, h.emb + (e.pt_off + j) * h.d, h.d);
            if (!h.knn && !(d2 <= h.r2)) fail(c, FRNN_CHECK_RADIUS, t);
            if (h.emit_d2 && __float_as_uint(st.d2[t]) != __float_as_uint(d2)) fail(c, FRNN_CHECK_D2, t);
            if (sorted && t > s0 && !(pd < d2 || (pd == d2 && pj < j))) fail(c, FRNN_CHECK_ORDER, t);
            pd = d2;
            pj = j;
        }
    }
}

// Brute force: row i of an event must hold min(k, |S_i|) entries (kNN:
// min(k, n - 1)), and exactly the points of the event that are in reach
// (within r, or any point for kNN) and no larger by (d2, j) than its last
// entry; the sums of the columns and of their squares are compared with
// those of the points found.  Rows without an order (no cap, longer than 32)
// must hold every point within r.  Rows of an event of n points are taken
// every ceil(n^2 / 2^34)-th, so an event costs at most 2^34 distances; the
// rows taken go to consecutive threads (thread u of the event: row u x step).
// Four candidates at a time (independent sums).  DR > 0: the query's row is
// held in DR registers (d <= DR).
template <int DR>
__global__ void __launch_bounds__(kChkThreads) k_check_complete(DevState st, Chk c)
{
    if (timed_out(st)) return;
    const CallHdr h = *st.hdr;
    const long long total = st.row_ptr[h.n_total];
    if (total < 0 || total > h.edge_capacity) return;
    const int d = h.d;
    const long long step = (long long)gridDim.x * blockDim.x;
    for (long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x; g < h.n_total; g += step) {
        const int b = event_at(st.ev, h.n_events, g);
        const EvDesc e = st.ev[b];
        if (st.plan[b].skip) continue;
        const long long n = e.n;
        const long long every = (n * n + kBrutePairs - 1) / kBrutePairs;
        const long long i = (g - e.pt_off) * every;
        if (i >= n) continue;
        const long long p = e.pt_off + i;
        const long long s0 = st.row_ptr[p], s1 = st.row_ptr[p + 1];
        if (s0 < 0 || s1 < s0 || s1 > h.edge_capacity) continue;  // reported by k_check_rows
        const long long len = s1 - s0;
        const bool sorted = row_sorted(h, len);
        const float* xe = h.emb + e.pt_off * d;
        float xr[DR > 0 ? DR : 1];
#pragma unroll
        for (int t = 0; t < (DR > 0 ? DR : 1); ++t) xr[t] = (DR > 0 && t < d) ? __ldg(xe + i * d + t) : 0.f;
        auto dist = [&](long long j) {
            if constexpr (DR > 0) return dist2_reg<DR>(xr, xe + j * d, d);
            else return dist2(xe + i * d, xe + j * d, d);
        };
        long long last_j = -1;
        float last_d = 0.f;
        if (sorted && len > 0) {
            last_j = st.col[s1 - 1];
            if (last_j < 0 || last_j >= n || last_j == i) continue;  // reported by k_check_rows
            last_d = dist(last_j);
        }
        long long found = 0, below = 0;
        unsigned long long sum1 = 0, sum2 = 0;
        for (long long j0 = 0; j0 < n; j0 += 4) {
            float dd[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) dd[u] = dist(j0 + u < n ? j0 + u : j0);
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const long long j = j0 + u;
                if (j >= n || j == i) continue;
                if (!h.knn && !(dd[u] <= h.r2)) continue;
                ++found;
                if (!sorted || dd[u] < last_d || (dd[u] == last_d && j <= last_j)) {
                    ++below;
                    sum1 += (unsigned long long)j;
                    sum2 += (unsigned long long)(j * j);
                }
            }
        }
        const long long want = h.knn ? min((long long)h.k, n - 1) : min((long long)h.k, found);
        unsigned long long row1 = 0, row2 = 0;
        for (long long t = s0; t < s1; ++t) {
            const long long j = st.col[t];
            row1 += (unsigned long long)j;
            row2 += (unsigned long long)(j * j);
        }
        if (len != want || below != len || row1 != sum1 || row2 != sum2) fail(c, FRNN_CHECK_COMPLETE, p);
    }
}

}  // namespace

int launch_checks(const DevState& st, unsigned long long* first, unsigned* bits, long long n_total, int n_events,
                  long long cells_max, int d, int n_sm, void* stream)
{
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (n_total <= 0) return 0;
    if (cudaMemsetAsync(bits, 0, sizeof(unsigned) * (size_t)((n_total + 31) / 32), s) != cudaSuccess) return 1;
    const Chk c{first, st.status, bits, cells_max};
    const int grid = n_sm * 8;
    // the brute-force pass: a thread per row (its rows take long and vary)
    const long long blocks = (n_total + kChkThreads - 1) / kChkThreads;
    const int grid_rows = blocks < (1 << 24) ? (int)blocks : (1 << 24);
    k_check_events<<<n_events < 1024 ? n_events : 1024, kChkThreads, 0, s>>>(st, c);
    k_check_sorted<<<grid, kChkThreads, 0, s>>>(st, c);
    k_check_rows<<<grid, kChkThreads, 0, s>>>(st, c);
    if (d <= 4) k_check_complete<4><<<grid_rows, kChkThreads, 0, s>>>(st, c);
    else if (d <= 8) k_check_complete<8><<<grid_rows, kChkThreads, 0, s>>>(st, c);
    else if (d <= 12) k_check_complete<12><<<grid_rows, kChkThreads, 0, s>>>(st, c);
    else if (d <= 16) k_check_complete<16><<<grid_rows, kChkThreads, 0, s>>>(st, c);
    else k_check_complete<0><<<grid_rows, kChkThreads, 0, s>>>(st, c);
    return cudaGetLastError() == cudaSuccess ? 0 : 1;
}

}  // namespace frnn
