/* ORACLE -- test infrastructure, not part of the library.
 *
 * Weighted betweenness centrality (positive integer arc weights): Brandes'
 * accumulation over a shortest-path DAG whose distances come from Dijkstra's
 * algorithm instead of a BFS.  Per source s:
 *   1. dist by Dijkstra (binary heap, lazy deletion), 64-bit integer sums;
 *   2. the reached vertices sorted by (dist, id): every DAG predecessor of v
 *      (an arc u -> v with dist[u] + w(u, v) == dist[v]) comes before v, as
 *      weights are positive;
 *   3. sigma pushed along DAG arcs in that order (sigma[s] = 1);
 *   4. delta pulled from DAG successors in reverse order,
 *      delta[v] = sum over arcs v -> x with dist[v] + w == dist[x] of
 *      sigma[v] / sigma[x] * (1 + delta[x]), and BC[v] += delta[v] for v != s.
 * This is the same recurrence as the unweighted listing (Appendix A, BC
 * listing; Section 2.3.2 iterateInBFS / iterateInReverse) with BFS levels
 * replaced by weighted distances.  Plain double arithmetic, no reordering.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
    int64_t d;
    int32_t v;
} HeapItem;

static void heap_push(HeapItem* h, int64_t* size, int64_t d, int32_t v) {
    int64_t i = (*size)++;
    while (i > 0) {
        int64_t p = (i - 1) / 2;
        if (h[p].d < d || (h[p].d == d && h[p].v <= v)) break;
        h[i] = h[p];
        i = p;
    }
    h[i].d = d;
    h[i].v = v;
}

static HeapItem heap_pop(HeapItem* h, int64_t* size) {
    HeapItem top = h[0];
    HeapItem last = h[--(*size)];
    int64_t i = 0;
    for (;;) {
        int64_t c = 2 * i + 1;
        if (c >= *size) break;
        if (c + 1 < *size && (h[c + 1].d < h[c].d || (h[c + 1].d == h[c].d && h[c + 1].v < h[c].v))) c++;
        if (last.d < h[c].d || (last.d == h[c].d && last.v <= h[c].v)) break;
        h[i] = h[c];
        i = c;
    }
    h[i] = last;
    return top;
}

static int64_t* g_sort_dist;
static int cmp_dist_id(const void* a, const void* b) {
    int32_t x = *(const int32_t*)a, y = *(const int32_t*)b;
    if (g_sort_dist[x] != g_sort_dist[y]) return g_sort_dist[x] < g_sort_dist[y] ? -1 : 1;
    return x < y ? -1 : (x > y);
}

/* One source: dist (-1 = unreached), sigma, delta, and the reached order.
 * Returns the number of reached vertices, or -1 on a non-positive weight or
 * allocation failure. */
static int64_t wsource(int32_t n, const int32_t* off, const int32_t* adj, const int32_t* wt, int32_t s,
                       int64_t* dist, double* sigma, double* delta, int32_t* order) {
    for (int32_t v = 0; v < n; ++v) {
        dist[v] = -1;
        sigma[v] = 0.0;
        delta[v] = 0.0;
    }
    int64_t m = off[n];
    HeapItem* h = (HeapItem*)malloc(sizeof(HeapItem) * (size_t)(m + 1));
    char* done = (char*)calloc((size_t)n, 1);
    if (!h || !done) {
        free(h);
        free(done);
        return -1;
    }
    int64_t hs = 0, nr = 0;
    dist[s] = 0;
    heap_push(h, &hs, 0, s);
    while (hs > 0) {
        HeapItem it = heap_pop(h, &hs);
        if (done[it.v] || it.d != dist[it.v]) continue;
        done[it.v] = 1;
        order[nr++] = it.v;
        for (int32_t e = off[it.v]; e < off[it.v + 1]; ++e) {
            if (wt[e] <= 0) {
                free(h);
                free(done);
                return -1;
            }
            const int32_t x = adj[e];
            const int64_t nd = it.d + wt[e];
            if (dist[x] < 0 || nd < dist[x]) {
                dist[x] = nd;
                heap_push(h, &hs, nd, x);
            }
        }
    }
    free(h);
    free(done);
    g_sort_dist = dist;
    qsort(order, (size_t)nr, sizeof(int32_t), cmp_dist_id);
    sigma[s] = 1.0;
    for (int64_t i = 0; i < nr; ++i) {
        const int32_t v = order[i];
        for (int32_t e = off[v]; e < off[v + 1]; ++e) {
            const int32_t x = adj[e];
            if (dist[v] + wt[e] == dist[x]) sigma[x] += sigma[v];
        }
    }
    for (int64_t i = nr - 1; i >= 0; --i) {
        const int32_t v = order[i];
        double d = 0.0;
        for (int32_t e = off[v]; e < off[v + 1]; ++e) {
            const int32_t x = adj[e];
            if (dist[v] + wt[e] == dist[x]) d += sigma[v] / sigma[x] * (1.0 + delta[x]);
        }
        delta[v] = d;
    }
    return nr;
}

/* Raw weighted BC over the listed sources (one term per occurrence). */
int oracle_wbc_f64(int32_t n, const int32_t* off, const int32_t* adj, const int32_t* wt, int32_t nsrc,
                   const int32_t* src, double* bc) {
    for (int32_t v = 0; v < n; ++v) bc[v] = 0.0;
    if (n == 0) return 0;
    int64_t* dist = (int64_t*)malloc(sizeof(int64_t) * (size_t)n);
    double* sigma = (double*)malloc(sizeof(double) * (size_t)n);
    double* delta = (double*)malloc(sizeof(double) * (size_t)n);
    int32_t* order = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
    int rc = 0;
    if (!dist || !sigma || !delta || !order) rc = 2;
    for (int32_t i = 0; rc == 0 && i < nsrc; ++i) {
        const int32_t s = src[i];
        if (s < 0 || s >= n) {
            rc = 1;
            break;
        }
        if (wsource(n, off, adj, wt, s, dist, sigma, delta, order) < 0) {
            rc = 3;
            break;
        }
        for (int32_t v = 0; v < n; ++v)
            if (v != s) bc[v] += delta[v];
    }
    free(dist);
    free(sigma);
    free(delta);
    free(order);
    return rc;
}

/* One source's dist (-1 unreached), sigma and delta. */
int oracle_wsource(int32_t n, const int32_t* off, const int32_t* adj, const int32_t* wt, int32_t s, int64_t* dist,
                   double* sigma, double* delta) {
    if (s < 0 || s >= n) return 1;
    int32_t* order = (int32_t*)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    if (!order) return 2;
    int64_t r = wsource(n, off, adj, wt, s, dist, sigma, delta, order);
    free(order);
    return r < 0 ? 3 : 0;
}
