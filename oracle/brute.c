/*
 * FP64 brute-force tree field integration — ORACLE, test infrastructure only.
 *
 * Plain definition (paper Eq. "integration", specialised to trees in
 * Eq. "stad-target", on the quantised metric of Appendix "Distance
 * quantization"):
 *
 *     out[u, c] = sum_v ftab[dhat(u, v)] * F[v, c]
 *
 * where dhat(u, v) is the sum of the integer edge lengths q_e on the tree path
 * and ftab[k] = f(k * delta) is supplied by the caller (evaluated in FP64).
 * Vertices in other trees of a forest are unreachable and contribute nothing.
 * One depth-first traversal per target vertex; accumulation in FP64.
 *
 * Build: gcc -O2 -fopenmp -shared -fPIC brute.c -o _brute.so
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <omp.h>

/* Grid distances from s to every vertex of its tree. dist[] must hold -1 on
 * entry for all vertices; on return, dist[v] >= 0 for the visited set, which
 * is listed in order[0..*count). */
static void traverse(const int64_t *ptr, const int32_t *adj, const int64_t *len,
                     int32_t s, int64_t *dist, int32_t *order, int64_t *count)
{
    int64_t head = 0, tail = 0;
    dist[s] = 0;
    order[tail++] = s;
    while (head < tail) {
        int32_t a = order[head++];
        for (int64_t e = ptr[a]; e < ptr[a + 1]; ++e) {
            int32_t b = adj[e];
            if (dist[b] < 0) {
                dist[b] = dist[a] + len[e];
                order[tail++] = b;
            }
        }
    }
    *count = tail;
}

/* Largest grid distance between two vertices of the same tree (the maximum
 * diameter over the forest's trees), found with two traversals per tree. */
int64_t tfi_oracle_max_dist(int32_t n, const int64_t *ptr, const int32_t *adj, const int64_t *len)
{
    int64_t *dist = (int64_t *)malloc(sizeof(int64_t) * (size_t)n);
    int32_t *order = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    char *seen = (char *)calloc((size_t)n, 1);
    int64_t best = 0;
    for (int32_t i = 0; i < n; ++i) dist[i] = -1;
    for (int32_t s = 0; s < n; ++s) {
        if (seen[s]) continue;
        int64_t cnt;
        traverse(ptr, adj, len, s, dist, order, &cnt);
        int32_t far = s;
        for (int64_t k = 0; k < cnt; ++k) {
            seen[order[k]] = 1;
            if (dist[order[k]] > dist[far]) far = order[k];
        }
        for (int64_t k = 0; k < cnt; ++k) dist[order[k]] = -1;
        traverse(ptr, adj, len, far, dist, order, &cnt);
        for (int64_t k = 0; k < cnt; ++k) {
            if (dist[order[k]] > best) best = dist[order[k]];
        }
        for (int64_t k = 0; k < cnt; ++k) dist[order[k]] = -1;
    }
    free(dist);
    free(order);
    free(seen);
    return best;
}

/* out[t, :] for each target t = targets[i] (row i of out, nt x d).
 * Returns 0, or 1 if some distance is beyond the table. */
int tfi_oracle_apply(int32_t n, const int64_t *ptr, const int32_t *adj, const int64_t *len,
                     const double *ftab, int64_t tlen, const double *F, int32_t d,
                     const int32_t *targets, int64_t nt, double *out, int32_t nthreads)
{
    int bad = 0;
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel reduction(| : bad)
    {
        int64_t *dist = (int64_t *)malloc(sizeof(int64_t) * (size_t)n);
        int32_t *order = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
        double *acc = (double *)malloc(sizeof(double) * (size_t)d);
        for (int32_t i = 0; i < n; ++i) dist[i] = -1;
#pragma omp for schedule(dynamic, 1)
        for (int64_t i = 0; i < nt; ++i) {
            int64_t cnt;
            traverse(ptr, adj, len, targets[i], dist, order, &cnt);
            for (int32_t c = 0; c < d; ++c) acc[c] = 0.0;
            for (int64_t k = 0; k < cnt; ++k) {
                int32_t v = order[k];
                int64_t g = dist[v];
                if (g >= tlen) { bad = 1; continue; }
                double fv = ftab[g];
                const double *row = F + (size_t)v * (size_t)d;
                for (int32_t c = 0; c < d; ++c) acc[c] += fv * row[c];
            }
            memcpy(out + (size_t)i * (size_t)d, acc, sizeof(double) * (size_t)d);
            for (int64_t k = 0; k < cnt; ++k) dist[order[k]] = -1;
        }
        free(dist);
        free(order);
        free(acc);
    }
    return bad;
}

/* Distance-binned correlation hist[k] = sum over targets u, and all v with
 * dhat(u, v) = k, of <Gr[u, :], F[v, :]>. With Gr = dL/dout this gives the
 * gradient with respect to kernel parameters theta:
 *     dL/dtheta = sum_k (d f(k delta)/d theta) * hist[k].
 * Per-thread histograms are summed in thread order. */
int tfi_oracle_corr_hist(int32_t n, const int64_t *ptr, const int32_t *adj, const int64_t *len,
                         const double *Gr, const double *F, int32_t d,
                         const int32_t *targets, int64_t nt, double *hist, int64_t tlen, int32_t nthreads)
{
    int bad = 0;
    if (nthreads <= 0) nthreads = omp_get_max_threads();
    double *parts = (double *)calloc((size_t)nthreads * (size_t)tlen, sizeof(double));
#pragma omp parallel num_threads(nthreads) reduction(| : bad)
    {
        int tid = omp_get_thread_num();
        double *h = parts + (size_t)tid * (size_t)tlen;
        int64_t *dist = (int64_t *)malloc(sizeof(int64_t) * (size_t)n);
        int32_t *order = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
        for (int32_t i = 0; i < n; ++i) dist[i] = -1;
#pragma omp for schedule(dynamic, 1)
        for (int64_t i = 0; i < nt; ++i) {
            int64_t cnt;
            int32_t u = targets[i];
            traverse(ptr, adj, len, u, dist, order, &cnt);
            const double *gu = Gr + (size_t)u * (size_t)d;
            for (int64_t k = 0; k < cnt; ++k) {
                int32_t v = order[k];
                int64_t g = dist[v];
                if (g >= tlen) { bad = 1; continue; }
                const double *fv = F + (size_t)v * (size_t)d;
                double s = 0.0;
                for (int32_t c = 0; c < d; ++c) s += gu[c] * fv[c];
                h[g] += s;
            }
            for (int64_t k = 0; k < cnt; ++k) dist[order[k]] = -1;
        }
        free(dist);
        free(order);
    }
    for (int64_t k = 0; k < tlen; ++k) {
        double s = 0.0;
        for (int t = 0; t < nthreads; ++t) s += parts[(size_t)t * (size_t)tlen + (size_t)k];
        hist[k] = s;
    }
    free(parts);
    return bad;
}

/* All grid distances from each listed source (row i = source sources[i]),
 * -1 where unreachable. For small trees only (nt x n int64). */
void tfi_oracle_dist_rows(int32_t n, const int64_t *ptr, const int32_t *adj, const int64_t *len,
                          const int32_t *sources, int64_t nt, int64_t *rows)
{
    int32_t *order = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    for (int64_t i = 0; i < nt; ++i) {
        int64_t *dist = rows + (size_t)i * (size_t)n;
        int64_t cnt;
        for (int32_t v = 0; v < n; ++v) dist[v] = -1;
        traverse(ptr, adj, len, sources[i], dist, order, &cnt);
    }
    free(order);
}
