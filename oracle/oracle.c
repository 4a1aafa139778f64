/*
 * oracle.c -- plain, slow-but-obviously-correct CPU reference for load-balanced CSR SpMV.
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, the smoke check and the benchmark's CPU-baseline
 * leg may load this library.  It shares no code, header, table or helper with the CUDA
 * path under paper_2212_08964_gb300/.
 *
 * Floating-point inputs are FP64 (FP32 data is widened exactly by the caller), so the
 * finite-difference pins can perturb x and v freely.
 *
 * Every function computes a plain definition from the dissertation ("GPU Load Balancing",
 * Osama 2022), Ch.3 and Ch.4, in FP64 where floating point is involved:
 *
 *   - SpMV y = A x over CSR (Sec. "Compressed Sparse Data Structures"; Listing lst:spmv):
 *     y_i = sum_{k = ro[i]}^{ro[i+1]-1} v_k * x[ci_k], summed sequentially in k.
 *   - The merge-path split of a diagonal d (Sec. "Work-Oriented", Alg. alg:work-oriented,
 *     the "2DSearch"; Sec. "Merge-path load balancing"): the row-end list
 *     R_r (key ro[r+1]) is merged with the nonzero indices N_k (key k); a row end is taken
 *     before nonzero k exactly when ro[r+1] <= k, which is the loop bound of the algorithm
 *     (a row's nonzeros are consumed while k < ro[r+1], then its output is written).
 *     In that merge R_r sits at position r + ro[r+1], so split(d) = (i, d - i) with
 *     i = #{ r : r + ro[r+1] < d }.
 *   - Tile boundaries d_c = min(c * T, W), c = 0..G, G = ceil(W / T), W = m + nnz
 *     (Alg. alg:work-oriented: total_work = rows + nonzeros, an equal share per worker;
 *     a fixed share T so that the split does not depend on the processor count).
 *   - CSC plan: a stable transpose (counting sort by column; entries of one column keep
 *     increasing original index k, hence increasing row).  The framework ships CSR, CSC
 *     and COO views (Sec. "Implementing Sparse Data Structures").
 *   - Backward of L = 1/2 ||A x - t||^2: dx = A^T g with dx_j = sum over nonzeros of column
 *     j, in increasing k, of v_k g[row(k)]; dv_k = g[row(k)] * x[ci_k].
 *   - SpMM C = A B with B dense n x kc, row-major (Sec. "Application Space", the SpMM
 *     listing: SpMV with an extra loop over the columns of B):
 *     C[i][j] = sum_{k = ro[i]}^{ro[i+1]-1} v_k * B[ci_k][j], summed sequentially in k.
 *   - Single-source shortest paths over a CSR graph with non-negative edge weights (Sec.
 *     "Application Space", the SSSP listing): dist[v] = min over paths from the source of the
 *     sum of edge weights, +inf if unreachable.  The oracle is Dijkstra's algorithm with a
 *     binary heap (any correct method gives the same minimum); sums in FP64.
 *
 * OpenMP only splits independent outputs (rows or columns); each output is summed in its
 * stated order, so results do not depend on the thread count.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>

#ifdef _OPENMP
#include <omp.h>
#endif

static int oracle_threads(int requested) {
#ifdef _OPENMP
    return requested > 0 ? requested : omp_get_max_threads();
#else
    (void)requested;
    return 1;
#endif
}

int oracle_max_threads(void) { return oracle_threads(0); }

/* y_i = sum_k v_k x[ci_k], FP64, sequential in k.  Listing lst:spmv. */
void oracle_spmv_f64(int64_t m, const int32_t *ro, const int32_t *ci, const double *v,
                     const double *x, double *y, int threads) {
    int nt = oracle_threads(threads);
    (void)nt;
#pragma omp parallel for schedule(dynamic, 256) num_threads(nt)
    for (int64_t i = 0; i < m; ++i) {
        double s = 0.0;
        for (int64_t k = ro[i]; k < ro[i + 1]; ++k) s += v[k] * x[ci[k]];
        y[i] = s;
    }
}

/* C = A B, B dense n x kc row-major; C m x kc row-major. */
void oracle_spmm_f64(int64_t m, int64_t kc, const int32_t *ro, const int32_t *ci, const double *v,
                     const double *B, double *C, int threads) {
    int nt = oracle_threads(threads);
    (void)nt;
#pragma omp parallel for schedule(dynamic, 64) num_threads(nt)
    for (int64_t i = 0; i < m; ++i) {
        for (int64_t j = 0; j < kc; ++j) {
            double s = 0.0;
            for (int64_t k = ro[i]; k < ro[i + 1]; ++k) s += v[k] * B[(int64_t)ci[k] * kc + j];
            C[i * kc + j] = s;
        }
    }
}

/* sum_k |v_k| |B[ci_k][j]| per entry of C: the scale of the per-entry error bound. */
void oracle_spmm_absdot(int64_t m, int64_t kc, const int32_t *ro, const int32_t *ci, const double *v,
                        const double *B, double *S, int threads) {
    int nt = oracle_threads(threads);
    (void)nt;
#pragma omp parallel for schedule(dynamic, 64) num_threads(nt)
    for (int64_t i = 0; i < m; ++i) {
        for (int64_t j = 0; j < kc; ++j) {
            double s = 0.0;
            for (int64_t k = ro[i]; k < ro[i + 1]; ++k) s += fabs(v[k]) * fabs(B[(int64_t)ci[k] * kc + j]);
            S[i * kc + j] = s;
        }
    }
}

/* sum_j |a_ij| |x_j| per row: the scale of the per-row error bound. */
void oracle_row_absdot(int64_t m, const int32_t *ro, const int32_t *ci, const double *v,
                       const double *x, double *s_out, int threads) {
    int nt = oracle_threads(threads);
    (void)nt;
#pragma omp parallel for schedule(dynamic, 256) num_threads(nt)
    for (int64_t i = 0; i < m; ++i) {
        double s = 0.0;
        for (int64_t k = ro[i]; k < ro[i + 1]; ++k) s += fabs(v[k]) * fabs(x[ci[k]]);
        s_out[i] = s;
    }
}

/* split(d) = (i, d - i), i = #{r : r + ro[r+1] < d}: counted directly, O(m). */
void oracle_merge_split(int64_t m, const int32_t *ro, int64_t d, int64_t *i_out, int64_t *j_out) {
    int64_t i = 0;
    for (int64_t r = 0; r < m; ++r)
        if (r + (int64_t)ro[r + 1] < d) ++i;
    *i_out = i;
    *j_out = d - i;
}

/* Number of tiles G = ceil(W / T) for W = m + nnz work items. */
int64_t oracle_num_tiles(int64_t m, int64_t nnz, int64_t T) {
    int64_t W = m + nnz;
    return (W + T - 1) / T;
}

/*
 * Tile boundaries (tile_row[c], tile_nz[c]) = split(min(c T, W)) for c = 0..G.
 * Same count as oracle_merge_split, taken for all boundaries in one sweep: the row-end
 * positions r + ro[r+1] increase strictly with r, so the number below a boundary only
 * grows as the boundary moves right.  Returns G.
 */
int64_t oracle_partition(int64_t m, const int32_t *ro, int64_t T, int32_t *tile_row, int32_t *tile_nz) {
    int64_t nnz = m > 0 ? ro[m] : 0;
    int64_t W = m + nnz;
    int64_t G = (W + T - 1) / T;
    int64_t i = 0; /* #{r : r + ro[r+1] < d} for the current d */
    for (int64_t c = 0; c <= G; ++c) {
        int64_t d = c * T < W ? c * T : W;
        while (i < m && i + (int64_t)ro[i + 1] < d) ++i;
        tile_row[c] = (int32_t)i;
        tile_nz[c] = (int32_t)(d - i);
    }
    return G;
}

/* Stable transpose: co = exclusive scan of column counts; entries of a column in increasing k. */
void oracle_transpose(int64_t m, int64_t n, const int32_t *ro, const int32_t *ci, int32_t *co,
                      int32_t *ri, int32_t *perm) {
    int64_t nnz = m > 0 ? ro[m] : 0;
    int64_t *next = (int64_t *)calloc((size_t)(n + 1), sizeof(int64_t));
    for (int64_t k = 0; k < nnz; ++k) next[ci[k] + 1]++;
    for (int64_t j = 0; j < n; ++j) next[j + 1] += next[j];
    for (int64_t j = 0; j <= n; ++j) co[j] = (int32_t)next[j];
    for (int64_t r = 0; r < m; ++r) {
        for (int64_t k = ro[r]; k < ro[r + 1]; ++k) {
            int64_t p = next[ci[k]]++;
            ri[p] = (int32_t)r;
            perm[p] = (int32_t)k;
        }
    }
    free(next);
}

/* dx_j = sum over column j's entries (increasing k) of v_k g[row(k)], FP64. */
void oracle_spmv_t_f64(int64_t m, int64_t n, const int32_t *ro, const int32_t *ci, const double *v,
                       const double *g, double *dx, int threads) {
    int64_t nnz = m > 0 ? ro[m] : 0;
    int32_t *co = (int32_t *)malloc((size_t)(n + 1) * sizeof(int32_t));
    int32_t *ri = (int32_t *)malloc((size_t)(nnz > 0 ? nnz : 1) * sizeof(int32_t));
    int32_t *perm = (int32_t *)malloc((size_t)(nnz > 0 ? nnz : 1) * sizeof(int32_t));
    oracle_transpose(m, n, ro, ci, co, ri, perm);
    int nt = oracle_threads(threads);
    (void)nt;
#pragma omp parallel for schedule(dynamic, 256) num_threads(nt)
    for (int64_t j = 0; j < n; ++j) {
        double s = 0.0;
        for (int64_t p = co[j]; p < co[j + 1]; ++p) s += v[perm[p]] * g[ri[p]];
        dx[j] = s;
    }
    free(co);
    free(ri);
    free(perm);
}

/* sum_i |a_ij| |g_i| per column: the scale of the per-column error bound of dx. */
void oracle_col_absdot(int64_t m, int64_t n, const int32_t *ro, const int32_t *ci, const double *v,
                       const double *g, double *s_out) {
    for (int64_t j = 0; j < n; ++j) s_out[j] = 0.0;
    for (int64_t r = 0; r < m; ++r)
        for (int64_t k = ro[r]; k < ro[r + 1]; ++k) s_out[ci[k]] += fabs(v[k]) * fabs(g[r]);
}

/* dv_k = g[row(k)] * x[ci_k], FP64. */
void oracle_dvalues_f64(int64_t m, const int32_t *ro, const int32_t *ci, const double *g,
                        const double *x, double *dv, int threads) {
    int nt = oracle_threads(threads);
    (void)nt;
#pragma omp parallel for schedule(dynamic, 256) num_threads(nt)
    for (int64_t r = 0; r < m; ++r)
        for (int64_t k = ro[r]; k < ro[r + 1]; ++k) dv[k] = g[r] * x[ci[k]];
}

/* ----------------------------------------------------------------------------------------
 * Single-source shortest paths: Dijkstra with a binary heap of (distance, vertex) pairs and
 * lazy deletion.  Edges u -> ci[k] for k in [ro[u], ro[u+1]) with weight w[k] >= 0 (w == NULL:
 * every weight 1, so dist is the BFS level).  dist[v] = INFINITY when v is unreachable. */
typedef struct {
    double d;
    int64_t v;
} heap_item;

static void heap_push(heap_item *h, int64_t *size, heap_item it) {
    int64_t i = (*size)++;
    while (i > 0) {
        int64_t p = (i - 1) / 2;
        if (h[p].d <= it.d) break;
        h[i] = h[p];
        i = p;
    }
    h[i] = it;
}

static heap_item heap_pop(heap_item *h, int64_t *size) {
    heap_item top = h[0];
    heap_item last = h[--(*size)];
    int64_t i = 0;
    for (;;) {
        int64_t c = 2 * i + 1;
        if (c >= *size) break;
        if (c + 1 < *size && h[c + 1].d < h[c].d) ++c;
        if (last.d <= h[c].d) break;
        h[i] = h[c];
        i = c;
    }
    if (*size > 0) h[i] = last;
    return top;
}

int oracle_sssp_f64(int64_t n, const int32_t *ro, const int32_t *ci, const double *w, int64_t source,
                    double *dist) {
    for (int64_t v = 0; v < n; ++v) dist[v] = INFINITY;
    if (source < 0 || source >= n) return -1;
    int64_t cap = (int64_t)ro[n] + 1;
    heap_item *h = (heap_item *)malloc((size_t)cap * sizeof(heap_item));
    if (!h) return -2;
    int64_t size = 0;
    dist[source] = 0.0;
    heap_item s0 = {0.0, source};
    heap_push(h, &size, s0);
    while (size > 0) {
        heap_item it = heap_pop(h, &size);
        if (it.d > dist[it.v]) continue; /* stale entry */
        for (int64_t k = ro[it.v]; k < ro[it.v + 1]; ++k) {
            double nd = it.d + (w ? w[k] : 1.0);
            int64_t u = ci[k];
            if (nd < dist[u]) {
                dist[u] = nd;
                heap_item e = {nd, u};
                heap_push(h, &size, e); /* at most one push per edge: fits cap */
            }
        }
    }
    free(h);
    return 0;
}
