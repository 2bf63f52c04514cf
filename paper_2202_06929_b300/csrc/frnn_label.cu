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
// same value the build tested).  One warp per row: its records are contiguous.
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

__global__ void __launch_bounds__(kLabelThreads) k_edge_features(DevState st, const float* emb, long long e_begin,
                                                                 long long e_end, float* out)
{
    const int lane = threadIdx.x & 31;
    const long long P = st.hdr->n_total;
    const int B = st.hdr->n_events;
    const int D = st.hdr->d;
    const int W = 2 * D + 1;
    if (P == 0 || e_end <= e_begin || timed_out(st)) return;
    const long long p_lo = row_of_edge(st.row_ptr, P, e_begin);
    const long long p_hi = row_of_edge(st.row_ptr, P, e_end - 1);
    const long long nwarps = (long long)gridDim.x * (blockDim.x >> 5);
    long long lo = 1, hi = 0, off = 0;
    for (long long p = p_lo + (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); p <= p_hi; p += nwarps) {
        if (p < lo || p >= hi) {
            const int b = event_of(st.ev, B, p);
            off = st.ev[b].pt_off;
            lo = off;
            hi = off + st.ev[b].n;
        }
        const long long a = max((long long)st.row_ptr[p], e_begin);
        const long long z = min((long long)st.row_ptr[p + 1], e_end);
        const float* xi = emb + p * D;
        const long long nel = (z - a) * W;
        for (long long t = lane; t < nel; t += 32) {
            const long long e = a + t / W;
            const int f = (int)(t % W);
            const int c = st.col[e];
            const float* xj = emb + (off + (c >= 0 ? c : 0)) * D;
            float v;
            if (c < 0) {
                v = __int_as_float(0x7fc00000);  // entry of an event with non-finite input: NaN features
            } else if (f < D) {
                v = xi[f];
            } else if (f < 2 * D) {
                v = xj[f - D];
            } else {
                float s = 0.f;
                for (int u = 0; u < D; ++u) {
                    const float dd = __fsub_rn(xi[u], xj[u]);
                    s = __fadd_rn(s, __fmul_rn(dd, dd));
                }
                v = s;
            }
            out[(e - e_begin) * W + f] = v;
        }
    }
}

}  // namespace

int launch_edge_features(const DevState& st, const float* emb, long long e_begin, long long e_end, float* out,
                         int grid, void* stream)
{
    k_edge_features<<<grid, kLabelThreads, 0, static_cast<cudaStream_t>(stream)>>>(st, emb, e_begin, e_end, out);
    return (int)cudaGetLastError();
}

}  // namespace frnn
