/*
 * ORACLE -- test infrastructure, not part of the library.
 *
 * PageRank by its definition: the fixed point of
 *     x = (1 - delta)/n * 1 + delta * P^T x,   P = D^-1 A,
 * where A is the adjacency matrix of the arcs (A[u][v] = number of arcs u -> v)
 * and D the diagonal of out-degrees, found by power iteration from x0 = 1/n.
 * A row of P whose vertex has no out-arcs is all zero: that vertex's rank is
 * not passed on (no dangling-mass correction), so the total can fall below 1.
 * Parameters and stopping rule as the paper's computePR (Appendix A, PR
 * program): damping delta, tolerance beta and an iteration cap; iterate while
 * the L1 change ||x_{k+1} - x_k||_1 exceeds beta and fewer than max_iter
 * iterations have run.  Double precision.
 *
 * The product P^T x is formed by scattering each vertex's share x[u]/outdeg(u)
 * along its arcs, vertices u in ascending order, so every y[v] adds its
 * in-neighbours' shares in ascending u.
 * off/adj: out-adjacency (for an undirected graph, either direction).
 * Returns the number of iterations run; *diff_out = the last L1 change.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* y = P^T x  (y zeroed first) */
static void transpose_apply(int32_t n, const int32_t* off, const int32_t* adj, const double* x, double* y) {
    memset(y, 0, sizeof(double) * (size_t)n);
    for (int32_t u = 0; u < n; ++u) {
        const int32_t outdeg = off[u + 1] - off[u];
        if (outdeg == 0) continue;
        const double share = x[u] / (double)outdeg;
        for (int32_t e = off[u]; e < off[u + 1]; ++e) y[adj[e]] += share;
    }
}

int oracle_pagerank(int32_t n, const int32_t* off, const int32_t* adj, double delta, double beta, int32_t max_iter,
                    double* pr, double* diff_out) {
    if (n <= 0) {
        if (diff_out) *diff_out = 0.0;
        return 0;
    }
    double* y = (double*)malloc(sizeof(double) * (size_t)n);
    if (!y) return -1;
    const double teleport = (1.0 - delta) / (double)n;
    for (int32_t v = 0; v < n; ++v) pr[v] = 1.0 / (double)n;
    int32_t k = 0;
    double change = 0.0;
    for (;;) {
        transpose_apply(n, off, adj, pr, y);
        change = 0.0;
        for (int32_t v = 0; v < n; ++v) {
            const double next = teleport + delta * y[v];
            change += fabs(next - pr[v]);
            y[v] = next;
        }
        memcpy(pr, y, sizeof(double) * (size_t)n);
        ++k;
        if (!(change > beta) || k >= max_iter) break;
    }
    if (diff_out) *diff_out = change;
    free(y);
    return k;
}
