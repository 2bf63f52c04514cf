/*
 * CPU oracle for the fixed-radius nearest-neighbour (FRNN) graph build.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * CPU-baseline leg of the benchmark may load this library.  The CUDA library
 * never calls it, and the two share no source, header or helper.
 *
 * What it computes (Sec. 2 of the paper: the graph joins every spacepoint to
 * the others within a constant radius in the embedding space; Sec. 3.4: the
 * FRNN problem; Sec. 3.1: exact kNN followed by a radius cut).  For every
 * query i of an event with n points x[n][d] (float32, row-major):
 *
 *   1. d2(i,j) = sum over t = 0..d-1 of (x[i][t] - x[j][t])^2 for every j != i,
 *      in float32, one rounding per subtraction, product and addition, the
 *      terms added in order t = 0, 1, ..., d-1 (built with -ffp-contract=off,
 *      so no fused multiply-add);
 *   2. S_i = { j != i : d2(i,j) <= r2 } with r2 = fl32(r * r);
 *   3. keep the min(|S_i|, k) members of S_i that are smallest by the pair
 *      (d2, j) in lexicographic order (k <= 0 keeps all of S_i);
 *   4. row i of the CSR lists them in that order.
 *
 * The integer-grid variant takes coordinates as integers m (x = m / 256) and
 * decides an edge by q(i,j) = sum (m_i - m_j)^2 <= thr in int64, ordering by
 * (q, j).  With thr = floor(r2 * 65536) it gives the same graph as the float
 * path on grid inputs, through arithmetic that shares nothing with it.
 *
 * Track labeling (the step after graph building, Sec. 2: edges that pass a
 * score cut are grouped into weakly connected components, each one a track
 * candidate; Sec. 3.2): fo_components treats every edge i -> j of a CSR
 * whose weight is <= w_max as undirected and labels each point with the
 * smallest point index of its component (sequential union-find).
 *
 * Plain brute force, O(n^2 d) per pass, parallel over queries with OpenMP.
 * Every function returns 0 on success and -1 on a bad argument or a failed
 * allocation.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
    float d2;
    int32_t j;
} fo_hit;

typedef struct {
    int64_t q;
    int32_t j;
} fo_hit_grid;

static int fo_cmp_hit(const void* a, const void* b)
{
    const fo_hit* u = (const fo_hit*)a;
    const fo_hit* v = (const fo_hit*)b;
    if (u->d2 < v->d2) return -1;
    if (u->d2 > v->d2) return 1;
    return (u->j > v->j) - (u->j < v->j);
}

static int fo_cmp_hit_grid(const void* a, const void* b)
{
    const fo_hit_grid* u = (const fo_hit_grid*)a;
    const fo_hit_grid* v = (const fo_hit_grid*)b;
    if (u->q < v->q) return -1;
    if (u->q > v->q) return 1;
    return (u->j > v->j) - (u->j < v->j);
}

/* Step 1: squared distance in float32, sequential over t. */
static float fo_dist2(const float* a, const float* b, int d)
{
    float s = 0.0f;
    for (int t = 0; t < d; ++t) {
        float diff = a[t] - b[t];
        float sq = diff * diff;
        s = s + sq;
    }
    return s;
}

static int64_t fo_dist2_grid(const int32_t* a, const int32_t* b, int d)
{
    int64_t s = 0;
    for (int t = 0; t < d; ++t) {
        int64_t diff = (int64_t)a[t] - (int64_t)b[t];
        s += diff * diff;
    }
    return s;
}

static int64_t fo_query(const int64_t* queries, int64_t qi)
{
    return queries ? queries[qi] : qi;
}

/*
 * |S_i| for each listed query (queries == NULL means all n points, in order).
 * deg[qi] receives the uncapped size of S_{queries[qi]}.
 */
int fo_degree(const float* x, int64_t n, int d, float r, const int64_t* queries,
              int64_t nq, int64_t* deg)
{
    if (n < 0 || d < 1 || nq < 0 || (n > 0 && !x) || !deg) return -1;
    const float r2 = r * r;
    int bad = 0;
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t qi = 0; qi < nq; ++qi) {
        int64_t i = fo_query(queries, qi);
        if (i < 0 || i >= n) {
#pragma omp atomic write
            bad = 1;
            continue;
        }
        int64_t c = 0;
        for (int64_t j = 0; j < n; ++j) {
            if (j == i) continue;
            if (fo_dist2(x + i * d, x + j * d, d) <= r2) ++c;
        }
        deg[qi] = c;
    }
    return bad ? -1 : 0;
}

/*
 * Rows of the capped graph for each listed query.  row_ptr[qi] .. row_ptr[qi+1]
 * is the slot range of query qi in col (and d2_out if not NULL); the caller
 * sizes it as min(|S_i|, k) (k <= 0: |S_i|), normally from fo_degree.
 */
int fo_fill(const float* x, int64_t n, int d, float r, int k, const int64_t* queries,
            int64_t nq, const int64_t* row_ptr, int32_t* col, float* d2_out)
{
    if (n < 0 || d < 1 || nq < 0 || (n > 0 && !x) || !row_ptr || !col) return -1;
    const float r2 = r * r;
    int bad = 0;
#pragma omp parallel
    {
        fo_hit* buf = (fo_hit*)malloc(sizeof(fo_hit) * (size_t)(n > 0 ? n : 1));
        if (!buf) {
#pragma omp atomic write
            bad = 1;
        }
#pragma omp for schedule(dynamic, 16)
        for (int64_t qi = 0; qi < nq; ++qi) {
            if (!buf) continue;
            int64_t i = fo_query(queries, qi);
            if (i < 0 || i >= n) {
#pragma omp atomic write
                bad = 1;
                continue;
            }
            int64_t m = 0;
            for (int64_t j = 0; j < n; ++j) {
                if (j == i) continue;
                float v = fo_dist2(x + i * d, x + j * d, d);
                if (v <= r2) {
                    buf[m].d2 = v;
                    buf[m].j = (int32_t)j;
                    ++m;
                }
            }
            qsort(buf, (size_t)m, sizeof(fo_hit), fo_cmp_hit);
            int64_t keep = (k > 0 && m > k) ? k : m;
            if (row_ptr[qi + 1] - row_ptr[qi] != keep) {
#pragma omp atomic write
                bad = 1;
                continue;
            }
            for (int64_t e = 0; e < keep; ++e) {
                col[row_ptr[qi] + e] = buf[e].j;
                if (d2_out) d2_out[row_ptr[qi] + e] = buf[e].d2;
            }
        }
        free(buf);
    }
    return bad ? -1 : 0;
}

/* Integer-grid variant of fo_degree: edge iff sum (m_i - m_j)^2 <= thr. */
int fo_degree_grid(const int32_t* m, int64_t n, int d, int64_t thr, const int64_t* queries,
                   int64_t nq, int64_t* deg)
{
    if (n < 0 || d < 1 || nq < 0 || (n > 0 && !m) || !deg) return -1;
    int bad = 0;
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t qi = 0; qi < nq; ++qi) {
        int64_t i = fo_query(queries, qi);
        if (i < 0 || i >= n) {
#pragma omp atomic write
            bad = 1;
            continue;
        }
        int64_t c = 0;
        for (int64_t j = 0; j < n; ++j) {
            if (j == i) continue;
            if (fo_dist2_grid(m + i * d, m + j * d, d) <= thr) ++c;
        }
        deg[qi] = c;
    }
    return bad ? -1 : 0;
}

/* Integer-grid variant of fo_fill; q_out (optional) receives the integer q. */
int fo_fill_grid(const int32_t* m, int64_t n, int d, int64_t thr, int k,
                 const int64_t* queries, int64_t nq, const int64_t* row_ptr,
                 int32_t* col, int64_t* q_out)
{
    if (n < 0 || d < 1 || nq < 0 || (n > 0 && !m) || !row_ptr || !col) return -1;
    int bad = 0;
#pragma omp parallel
    {
        fo_hit_grid* buf = (fo_hit_grid*)malloc(sizeof(fo_hit_grid) * (size_t)(n > 0 ? n : 1));
        if (!buf) {
#pragma omp atomic write
            bad = 1;
        }
#pragma omp for schedule(dynamic, 16)
        for (int64_t qi = 0; qi < nq; ++qi) {
            if (!buf) continue;
            int64_t i = fo_query(queries, qi);
            if (i < 0 || i >= n) {
#pragma omp atomic write
                bad = 1;
                continue;
            }
            int64_t c = 0;
            for (int64_t j = 0; j < n; ++j) {
                if (j == i) continue;
                int64_t q = fo_dist2_grid(m + i * d, m + j * d, d);
                if (q <= thr) {
                    buf[c].q = q;
                    buf[c].j = (int32_t)j;
                    ++c;
                }
            }
            qsort(buf, (size_t)c, sizeof(fo_hit_grid), fo_cmp_hit_grid);
            int64_t keep = (k > 0 && c > k) ? k : c;
            if (row_ptr[qi + 1] - row_ptr[qi] != keep) {
#pragma omp atomic write
                bad = 1;
                continue;
            }
            for (int64_t e = 0; e < keep; ++e) {
                col[row_ptr[qi] + e] = buf[e].j;
                if (q_out) q_out[row_ptr[qi] + e] = buf[e].q;
            }
        }
        free(buf);
    }
    return bad ? -1 : 0;
}

/* Number of OpenMP threads a parallel region of this library uses. */
int fo_num_threads(void)
{
    int t = 1;
#pragma omp parallel
    {
#pragma omp single
        {
#ifdef _OPENMP
            extern int omp_get_num_threads(void);
            t = omp_get_num_threads();
#endif
        }
    }
    return t;
}

static int64_t fo_find(int64_t* parent, int64_t x)
{
    while (parent[x] != x) x = parent[x];
    return x;
}

/*
 * Weakly connected components of the graph whose edges are the CSR entries
 * (row i, col[e]) with w[e] <= w_max (w == NULL keeps every edge).  labels[i]
 * receives the smallest index of i's component.  Sequential union-find: the
 * larger root is attached under the smaller, so every root is the minimum of
 * its component.
 */
int fo_components(const int64_t* row_ptr, const int32_t* col, const float* w, float w_max, int64_t n,
                  int32_t* labels)
{
    if (n < 0 || (n > 0 && (!row_ptr || !labels))) return -1;
    int64_t* parent = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    if (!parent) return -1;
    for (int64_t i = 0; i < n; ++i) parent[i] = i;
    for (int64_t i = 0; i < n; ++i) {
        for (int64_t e = row_ptr[i]; e < row_ptr[i + 1]; ++e) {
            if (w && !(w[e] <= w_max)) continue;
            int64_t j = col[e];
            if (j < 0 || j >= n) { free(parent); return -1; }
            int64_t a = fo_find(parent, i), b = fo_find(parent, j);
            if (a == b) continue;
            if (a < b) parent[b] = a; else parent[a] = b;
        }
    }
    for (int64_t i = 0; i < n; ++i) labels[i] = (int32_t)fo_find(parent, i);
    free(parent);
    return 0;
}
