// Track labeling over a built graph: weakly connected components.
//
// The step after graph building in the paper's pipeline (Sec. 2): edges that
// pass a score cut are grouped into weakly connected components, each one a
// track candidate; the paper runs cuGraph's lock-free WCC on the GPU
// (Sec. 3.2).  Here the score of an edge is its squared distance (no trained
// network is involved): an edge i -> j is kept when d2 <= d2_max, its
// direction is ignored, and every point gets the smallest index of its
// component as its label, so labels are unique and independent of timing.
//
// Lock-free union-find over a parent array of call-wide point indices, in
// four passes: every point starts under its smallest kept neighbour; paths
// are compressed (each point then hangs directly under its root, and on
// clustered data almost every edge already lies inside one tree); each edge
// whose ends hang under different roots joins the trees, a root only ever
// being attached (by compare-and-swap) under a smaller root; the labels are
// read off.  Every parent pointer is a smaller point of the same component
// (or the point itself), so finds end, and the root of a component is its
// minimum.
#include <cuda_runtime.h>

#include "frnn_internal.h"

namespace frnn {
namespace {

constexpr int kLabelThreads = 256;
constexpr int kUnionLimit = 1 << 20;  // retries of one union (each failure means another thread progressed)

// Parent reads that see other threads' updates (volatile: never cached in a
// register or in L1).
__device__ __forceinline__ int ld_parent(const int* p)
{
    return *reinterpret_cast<const volatile int*>(p);
}

__device__ __forceinline__ int find_root(int* parent, int x)
{
    for (;;) {
        const int px = ld_parent(parent + x);
        if (px == x) return x;
        const int ppx = ld_parent(parent + px);
        if (ppx != px) parent[x] = ppx;  // path halving: ppx is an ancestor of x
        x = ppx;
    }
}

__device__ __forceinline__ bool unite(int* parent, int a, int b)
{
    for (int it = 0; it < kUnionLimit; ++it) {
        a = find_root(parent, a);
        b = find_root(parent, b);
        if (a == b) return true;
        if (a > b) {
            const int t = a;
            a = b;
            b = t;
        }
        const int old = atomicCAS(parent + b, b, a);  // attach the larger root under the smaller
        if (old == b) return true;
        b = old;
    }
    return false;
}

__device__ __forceinline__ int event_of(const EvDesc* ev, int n_events, long long p)
{
    int lo = 0, hi = n_events - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (ev[mid].pt_off <= p) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// Start of the forest: every point points at its smallest kept neighbour (or
// at itself).  A parent is a smaller point of the same component, so this is
// a valid union-find state, and a cluster whose points are all neighbours of
// one another is already a one-level tree.
__global__ void __launch_bounds__(kLabelThreads) k_label_init(DevState st, int* parent, float d2_max, int use_d2)
{
    unsigned* capped = &st.counters[kCtrLabelCapped];
    const int K = st.hdr->k;
    const long long P = st.hdr->n_total;
    const int B = st.hdr->n_events;
    const long long ecap = st.hdr->edge_capacity;
    const bool dead = timed_out(st);  // the build's edges are not valid: every point alone
    long long lo = 1, hi = 0, off = 0;
    for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < P; p += (long long)gridDim.x * blockDim.x) {
        if (p < lo || p >= hi) {
            const int b = event_of(st.ev, B, p);
            off = st.ev[b].pt_off;
            lo = off;
            hi = off + st.ev[b].n;
        }
        const int rs = st.row_ptr[p], re = st.row_ptr[p + 1];
        long long m = p;
        if (!dead && (long long)re <= ecap) {
            for (int e = rs; e < re; ++e) {
                if (use_d2 && !(st.d2[e] <= d2_max)) continue;
                const int c = st.col[e];
                if (c >= 0) m = min(m, off + c);  // -1: entry of an event with non-finite input
            }
        }
        parent[p] = (int)m;
        // a row of k entries may have been cut at k: note it for the union pass
        if (re - rs >= K) atomicOr(capped, 1u);
    }
}

// Full path compression after the start: every point is made to point at its
// root (reads along the chain; the one write only shortens a path, which is
// safe while other threads walk it).
__global__ void __launch_bounds__(kLabelThreads) k_label_compress(DevState st, int* parent)
{
    const long long P = st.hdr->n_total;
    for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < P; p += (long long)gridDim.x * blockDim.x) {
        int x = parent[p];
        if (x == (int)p) continue;
        int px = ld_parent(parent + x);
        while (px != x) {
            x = px;
            px = ld_parent(parent + x);
        }
        parent[p] = x;
    }
}

// Every kept edge joins its two trees.  An edge p -> q with q < p is left to
// q's row when that row holds all of q's neighbours (it was not cut at k),
// since q -> p is then processed from there (when no row of the build was
// cut, that holds for every such edge).  p's root is carried from edge to
// edge (a root that was hooked meanwhile is still an ancestor of p), and an
// edge whose far end already hangs directly under it costs one load.
__global__ void __launch_bounds__(kLabelThreads) k_label_union(DevState st, int* parent, float d2_max, int use_d2)
{
    if (timed_out(st)) return;
    const bool any_capped = __ldcg(&st.counters[kCtrLabelCapped]) != 0u;
    const long long P = st.hdr->n_total;
    const int B = st.hdr->n_events;
    const int K = st.hdr->k;
    const long long ecap = st.hdr->edge_capacity;
    long long lo = 1, hi = 0, off = 0;
    for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < P; p += (long long)gridDim.x * blockDim.x) {
        if (p < lo || p >= hi) {
            const int b = event_of(st.ev, B, p);
            off = st.ev[b].pt_off;
            lo = off;
            hi = off + st.ev[b].n;
        }
        const int rs = st.row_ptr[p], re = st.row_ptr[p + 1];
        if ((long long)re > ecap) continue;  // rows past the edge capacity were never written
        int rp = -1;
        for (int e = rs; e < re; ++e) {
            if (use_d2 && !(st.d2[e] <= d2_max)) continue;
            const int c = st.col[e];
            if (c < 0) continue;  // entry of an event with non-finite input (kNN builds)
            const long long q = off + c;
            if (q < p && (!any_capped || st.cnt_o[q] < K)) continue;
            if (rp < 0) rp = __ldcg(parent + p);  // an ancestor of p (its root after compression)
            const int pq = __ldcg(parent + q);
            if (pq == rp) continue;  // q's parent is p's root (trees only merge)
            const int rq = find_root(parent, pq);
            if (rq == rp) continue;
            if (!unite(parent, rp, rq)) atomicOr(st.status, kStTimeout);
            rp = find_root(parent, rp);
        }
    }
}

__global__ void __launch_bounds__(kLabelThreads) k_label_final(DevState st, int* parent, int* labels)
{
    const long long P = st.hdr->n_total;
    const int B = st.hdr->n_events;
    long long lo = 1, hi = 0, off = 0;
    for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < P; p += (long long)gridDim.x * blockDim.x) {
        if (p < lo || p >= hi) {
            const int b = event_of(st.ev, B, p);
            off = st.ev[b].pt_off;
            lo = off;
            hi = off + st.ev[b].n;
        }
        labels[p] = (int)(find_root(parent, (int)p) - off);
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) st.counters[kCtrLabelCapped] = 0u;  // read by the union pass only
}

}  // namespace

int launch_label(const DevState& st, int* parent, int* labels, float d2_max, int use_d2, int grid, void* stream)
{
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    k_label_init<<<grid, kLabelThreads, 0, s>>>(st, parent, d2_max, use_d2);
    k_label_compress<<<grid, kLabelThreads, 0, s>>>(st, parent);
    k_label_union<<<grid, kLabelThreads, 0, s>>>(st, parent, d2_max, use_d2);
    k_label_final<<<grid, kLabelThreads, 0, s>>>(st, parent, labels);
    return (int)cudaGetLastError();
}

}  // namespace frnn

// ---------------------------------------------------------------------------
// Edge features for the filter stage (Sec. 3: the filter network reads the
// graph's edges in fixed-size batches): for every edge e in [e_begin, e_end)
// of the last build, out[(e - e_begin) * (2d + 1) + ...] = x_i[0..d), x_j[0..d),
// d2(i, j), with d2 summed in dimension order, one rounding per operation (the
// same value the build tested).
namespace frnn {
namespace {

__device__ __forceinline__ long long row_of_edge(const int* row_ptr, long long n, long long e)
{
    // largest p with row_ptr[p] <= e
    long long lo = 0, hi = n - 1;
    while (lo < hi) {
        const long long mid = (lo + hi + 1) >> 1;
        if ((long long)row_ptr[mid] <= e) lo = mid; else hi = mid - 1;
    }
    return lo;
}

constexpr int kEfWarps = 4;  // warps per block of the edge-feature kernel
constexpr int kEfPer = 1;    // edges per lane of a chunk (2 measured no faster)
constexpr int kEfChunk = 32 * kEfPer;
constexpr unsigned kAllLanes = 0xffffffffu;

// row_of_edge by a whole warp: 32 probes per step narrow the range 32-fold,
// so a search over millions of rows takes about five dependent loads.
__device__ __forceinline__ long long warp_row_of_edge(const int* row_ptr, long long n, long long e, int lane)
{
    long long lo = 0, hi = n - 1;  // the answer lies in [lo, hi]; row_ptr[lo] <= e
    while (hi - lo >= 32) {
        const long long span = hi - lo + 1;
        const long long pos = lo + (span * lane) / 32;  // pos of lane 0 is lo
        const unsigned m = __ballot_sync(kAllLanes, (long long)row_ptr[pos] <= e);
        const int k = __popc(m);  // probes 0 .. k-1 hold, the rest do not
        const long long nlo = lo + (span * (k - 1)) / 32;
        const long long nhi = k < 32 ? lo + (span * k) / 32 - 1 : hi;
        lo = nlo;
        hi = nhi;
    }
    const long long pos = lo + lane;
    const unsigned m = __ballot_sync(kAllLanes, pos <= hi && (long long)row_ptr[pos] <= e);
    return lo + __popc(m) - 1;
}

// A warp takes a contiguous range of chunks of kEfChunk edges, kEfPer per
// lane.  The row of its first edge comes from one warp-wide search; after that
// the row of every edge follows by binary lifting over the 32 row starts after
// the previous chunk's last row (a per-edge search when a chunk reaches past
// them, i.e. many empty rows).  Each lane assembles its edges' 2d + 1 values in
// shared memory (record stride 2d + 1 is odd, so the lanes' writes hit
// distinct banks) and the warp stores the chunk's records with consecutive
// 4-byte writes.
__global__ void __launch_bounds__(kEfWarps * 32) k_edge_features(DevState st, const float* emb, long long e_begin,
                                                                 long long e_end, float* out)
{
    extern __shared__ float s_ef[];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const long long P = st.hdr->n_total;
    const int B = st.hdr->n_events;
    const int D = st.hdr->d;
    const int W = 2 * D + 1;
    float* buf = s_ef + (size_t)wib * kEfChunk * W;
    if (P == 0 || e_end <= e_begin || timed_out(st)) return;
    const long long nchunk = (e_end - e_begin + kEfChunk - 1) / kEfChunk;
    const long long nwarps = (long long)gridDim.x * kEfWarps;
    const long long per = (nchunk + nwarps - 1) / nwarps;
    const long long c_begin = ((long long)blockIdx.x * kEfWarps + wib) * per;
    const long long c_end = min(c_begin + per, nchunk);
    if (c_begin >= c_end) return;
    // a row at or before the chunk's first edge
    long long p0 = warp_row_of_edge(st.row_ptr, P, e_begin + c_begin * kEfChunk, lane);
    long long lo = 1, hi = 0, off = 0;  // this lane's event: points [lo, hi), first point off
    for (long long c = c_begin; c < c_end; ++c) {
        const long long e0 = e_begin + c * kEfChunk;
        const long long e_last = min(e0 + kEfChunk - 1, e_end - 1);
        long long e[kEfPer];
        int cj[kEfPer];
#pragma unroll
        for (int u = 0; u < kEfPer; ++u) {
            e[u] = e0 + 32 * u + lane;
            cj[u] = e[u] < e_end ? st.col[e[u]] : 0;  // issued first: they do not depend on the rows
        }
        const long long pi = p0 + 1 + lane;
        const int rs = pi <= P ? st.row_ptr[pi] : 0x7fffffff;  // starts of rows p0 + 1 ..
        const bool lift = (long long)__shfl_sync(kAllLanes, rs, 31) > e_last;
        long long p[kEfPer];
#pragma unroll
        for (int u = 0; u < kEfPer; ++u) {
            if (lift) {
                int r = 0;
                for (int step = 16; step >= 1; step >>= 1) {
                    const int v = __shfl_sync(kAllLanes, rs, r + step - 1);
                    if ((long long)v <= e[u]) r += step;
                }
                p[u] = p0 + r;
            } else {
                p[u] = e[u] < e_end ? row_of_edge(st.row_ptr, P, e[u]) : p0;
            }
        }
        {
            // carry the row of the chunk's last edge to the next chunk
            const int li = (int)(e_last - e0);
            long long pl = p[0];
#pragma unroll
            for (int u = 1; u < kEfPer; ++u)
                if ((li >> 5) == u) pl = p[u];
            p0 = __shfl_sync(kAllLanes, pl, li & 31);
        }
#pragma unroll
        for (int u = 0; u < kEfPer; ++u) {
            if (e[u] >= e_end) continue;
            if (p[u] < lo || p[u] >= hi) {
                const int b = event_of(st.ev, B, p[u]);
                off = st.ev[b].pt_off;
                lo = off;
                hi = off + st.ev[b].n;
            }
            float* rec = buf + (32 * u + lane) * W;
            if (cj[u] < 0) {
                // entry of an event with non-finite input: NaN features
                for (int f = 0; f < W; ++f) rec[f] = __int_as_float(0x7fc00000);
            } else {
                const float* xi = emb + p[u] * D;
                const float* xj = emb + (off + cj[u]) * D;
                float sum = 0.f;
                for (int t = 0; t < D; ++t) {
                    const float a = __ldg(xi + t), b = __ldg(xj + t);
                    rec[t] = a;
                    rec[D + t] = b;
                    const float dd = __fsub_rn(a, b);
                    sum = __fadd_rn(sum, __fmul_rn(dd, dd));  // the build's d2: dims in order, one rounding each
                }
                rec[2 * D] = sum;
            }
        }
        __syncwarp();
        const int nrec = (int)(e_last - e0 + 1);
        float* dst = out + (e0 - e_begin) * W;
        for (int i = lane; i < nrec * W; i += 32) dst[i] = buf[i];
        __syncwarp();  // buf is rewritten by the next chunk
    }
}

}  // namespace

int launch_edge_features(const DevState& st, const float* emb, int d, long long e_begin, long long e_end,
                         float* out, int n_sm, void* stream)
{
    // one chunk's records staged per warp; the attribute (set on the current
    // device at every call, a host-side update) covers the largest d
    constexpr int kMaxSmem = kEfWarps * kEfChunk * (2 * kMaxDims + 1) * (int)sizeof(float);
    const cudaError_t attr =
        cudaFuncSetAttribute(k_edge_features, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxSmem);
    if (attr != cudaSuccess) return (int)attr;
    if (d < 1 || d > kMaxDims) return (int)cudaErrorInvalidValue;
    const int smem = kEfWarps * kEfChunk * (2 * d + 1) * (int)sizeof(float);
    int nb = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_edge_features, kEfWarps * 32, smem);
    if (e != cudaSuccess) return (int)e;
    const long long chunks = (e_end - e_begin + kEfChunk - 1) / kEfChunk;
    long long grid = (long long)n_sm * (nb > 0 ? nb : 1);
    const long long need = (chunks + kEfWarps - 1) / kEfWarps;
    if (grid > need) grid = need > 0 ? need : 1;
    k_edge_features<<<(unsigned)grid, kEfWarps * 32, smem, static_cast<cudaStream_t>(stream)>>>(st, emb, e_begin,
                                                                                               e_end, out);
    return (int)cudaGetLastError();
}

}  // namespace frnn
