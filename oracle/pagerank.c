/*
 * ORACLE -- test infrastructure, not part of the library.
 *
 * PageRank as the paper's computePR program (Appendix A, PR listing) states
 * it, in double precision: every rank starts at 1/n; each sweep computes for
 * every vertex v the sum of rank(u) / outdeg(u) over the vertices u with an
 * arc u -> v (ascending u), the new rank (1 - delta)/n + delta * sum, and the
 * change diff = sum over v of |new - old|; the sweeps repeat while
 * diff > beta and fewer than max_iter sweeps have run.  Ranks are replaced
 * all at once after a sweep (pageRank = pageRank_nxt).  No redistribution of
 * the rank of vertices without out-arcs (the listing has none).
 * off/adj: out-adjacency (for an undirected graph, either direction).
 */
#include <stdint.h>
#include <stdlib.h>
#include <math.h>

int oracle_pagerank(int32_t n, const int32_t* off, const int32_t* adj, double delta, double beta, int32_t max_iter,
                    double* pr, double* diff_out) {
    if (n <= 0) {
        if (diff_out) *diff_out = 0.0;
        return 0;
    }
    const int64_t m = off[n];
    /* in-adjacency by counting sort over the arcs, sources in ascending order */
    int64_t* ioff = (int64_t*)calloc((size_t)n + 1, sizeof(int64_t));
    int32_t* isrc = (int32_t*)malloc(sizeof(int32_t) * (size_t)(m > 0 ? m : 1));
    int64_t* fill = (int64_t*)malloc(sizeof(int64_t) * (size_t)n);
    double* nxt = (double*)malloc(sizeof(double) * (size_t)n);
    if (!ioff || !isrc || !fill || !nxt) {
        free(ioff); free(isrc); free(fill); free(nxt);
        return -1;
    }
    for (int64_t e = 0; e < m; ++e) ioff[adj[e] + 1]++;
    for (int32_t v = 0; v < n; ++v) ioff[v + 1] += ioff[v];
    for (int32_t v = 0; v < n; ++v) fill[v] = ioff[v];
    for (int32_t u = 0; u < n; ++u)
        for (int32_t e = off[u]; e < off[u + 1]; ++e) isrc[fill[adj[e]]++] = u;
    for (int32_t v = 0; v < n; ++v) pr[v] = 1.0 / (double)n;
    int32_t it = 0;
    double diff = 0.0;
    do {
        diff = 0.0;
        for (int32_t v = 0; v < n; ++v) {
            double sum = 0.0;
            for (int64_t e = ioff[v]; e < ioff[v + 1]; ++e) {
                const int32_t u = isrc[e];
                sum += pr[u] / (double)(off[u + 1] - off[u]);
            }
            const double val = (1.0 - delta) / (double)n + delta * sum;
            diff += fabs(val - pr[v]);
            nxt[v] = val;
        }
        for (int32_t v = 0; v < n; ++v) pr[v] = nxt[v];
        ++it;
    } while (diff > beta && it < max_iter);
    if (diff_out) *diff_out = diff;
    free(ioff); free(isrc); free(fill); free(nxt);
    return it;
}
