/*
 * ORACLE -- test infrastructure, not part of the library.
 *
 * Plain, slow, single-threaded reference for the betweenness-centrality path.
 * Only the tests, the smoke check and the benchmark's CPU-baseline leg may
 * call it.  It shares no code, header, table or helper with the CUDA library.
 *
 * What it computes (the paper's computeBC, Appendix A, BC listing; Section 2.3.2,
 * iterateInBFS / iterateInReverse):
 *   for every source s in the given list (duplicates counted once per entry):
 *     sigma = 0, delta = 0, sigma[s] = 1, level[s] = 0
 *     forward: breadth-first from s; for each vertex v in BFS order and each
 *       neighbour w: an unseen w gets level[v] + 1; if level[w] == level[v]+1
 *       then sigma[w] += sigma[v]            (w is a BFS-DAG successor of v)
 *     backward: vertices in reverse BFS order; for each v != s and each DAG
 *       successor w:  delta[v] += (sigma[v] / sigma[w]) * (1 + delta[w]);
 *       then BC[v] += delta[v]
 * The result is the raw sum over the listed sources: no halving for
 * undirected graphs, no normalisation (the paper's listing has neither).
 *
 * Two precisions are built from one body: double, and long double (x86-64
 * 80-bit extended: 64-bit significand, exponent range to 2^16383) for graphs
 * whose path counts leave the double range.
 *
 * Also here: the degree-descending relabelling the library applies on ingest
 * (its plain definition: stable sort by degree, descending, ties by id) and
 * the CSR validity rules the library enforces.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* Per-source detail record (pointers may be NULL when not wanted). */
typedef struct {
    int32_t* level;       /* [n], -1 when unreachable */
    void* sigma;          /* [n] REAL */
    void* delta;          /* [n] REAL */
    int64_t edag;         /* #arcs (v,w) with level[w] == level[v] + 1 */
    int64_t reached;      /* #vertices with level >= 0 (includes s) */
    int64_t sum_dm1;      /* sum over reached t != s of (level[t] - 1) */
    int32_t max_level;
} oracle_detail;

#define BRANDES_BODY(REAL)                                                                  \
    int32_t* level = (int32_t*)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));           \
    int32_t* order = (int32_t*)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));           \
    REAL* sigma = (REAL*)malloc(sizeof(REAL) * (size_t)(n > 0 ? n : 1));                    \
    REAL* delta = (REAL*)malloc(sizeof(REAL) * (size_t)(n > 0 ? n : 1));                    \
    if (!level || !order || !sigma || !delta) {                                             \
        free(level); free(order); free(sigma); free(delta);                                 \
        return -4;                                                                          \
    }                                                                                       \
    for (int32_t v = 0; v < n; ++v) bc[v] = 0;                                              \
    for (int32_t si = 0; si < nsrc; ++si) {                                                 \
        const int32_t s = src[si];                                                          \
        if (s < 0 || s >= n) { free(level); free(order); free(sigma); free(delta); return -3; } \
        for (int32_t v = 0; v < n; ++v) { level[v] = -1; sigma[v] = 0; delta[v] = 0; }     \
        level[s] = 0;                                                                       \
        sigma[s] = 1;                                                                       \
        /* forward: FIFO queue; 'order' doubles as the queue and the stack */              \
        int32_t head = 0, tail = 0;                                                         \
        order[tail++] = s;                                                                  \
        int64_t edag = 0;                                                                   \
        while (head < tail) {                                                               \
            const int32_t v = order[head++];                                                \
            for (int32_t e = off[v]; e < off[v + 1]; ++e) {                                 \
                const int32_t w = adj[e];                                                   \
                if (level[w] < 0) { level[w] = level[v] + 1; order[tail++] = w; }           \
                if (level[w] == level[v] + 1) { sigma[w] += sigma[v]; ++edag; }             \
            }                                                                               \
        }                                                                                   \
        /* backward: reverse BFS order, DAG successors pulled */                           \
        for (int32_t i = tail - 1; i >= 0; --i) {                                           \
            const int32_t v = order[i];                                                     \
            if (v == s) continue;                                                           \
            for (int32_t e = off[v]; e < off[v + 1]; ++e) {                                 \
                const int32_t w = adj[e];                                                   \
                if (level[w] == level[v] + 1)                                               \
                    delta[v] += (sigma[v] / sigma[w]) * (1 + delta[w]);                     \
            }                                                                               \
            bc[v] += delta[v];                                                              \
        }                                                                                   \
        if (detail) {                                                                       \
            oracle_detail* d = &detail[si];                                                 \
            int64_t sdm1 = 0; int32_t ml = 0;                                               \
            for (int32_t i = 1; i < tail; ++i) {                                            \
                int32_t lv = level[order[i]];                                               \
                sdm1 += lv - 1;                                                             \
                if (lv > ml) ml = lv;                                                       \
            }                                                                               \
            d->edag = edag; d->reached = tail; d->sum_dm1 = sdm1; d->max_level = ml;        \
            if (d->level) memcpy(d->level, level, sizeof(int32_t) * (size_t)n);             \
            if (d->sigma) memcpy(d->sigma, sigma, sizeof(REAL) * (size_t)n);                \
            if (d->delta) memcpy(d->delta, delta, sizeof(REAL) * (size_t)n);                \
        }                                                                                   \
    }                                                                                       \
    free(level); free(order); free(sigma); free(delta);                                     \
    return 0;

/* Returns 0, -3 for a source out of range, -4 when host memory runs out. */
int oracle_bc_f64(int32_t n, const int32_t* off, const int32_t* adj, int32_t nsrc,
                  const int32_t* src, double* bc, oracle_detail* detail) {
    BRANDES_BODY(double)
}

int oracle_bc_ld(int32_t n, const int32_t* off, const int32_t* adj, int32_t nsrc,
                 const int32_t* src, long double* bc, oracle_detail* detail) {
    BRANDES_BODY(long double)
}

/* long double results narrowed to double for callers without an 80-bit type. */
int oracle_bc_ld_out_f64(int32_t n, const int32_t* off, const int32_t* adj, int32_t nsrc,
                         const int32_t* src, double* bc_out) {
    long double* bc = (long double*)malloc(sizeof(long double) * (size_t)(n > 0 ? n : 1));
    if (!bc) return -4;
    int rc = oracle_bc_ld(n, off, adj, nsrc, src, bc, NULL);
    for (int32_t v = 0; v < n; ++v) bc_out[v] = (double)bc[v];
    free(bc);
    return rc;
}

/* One source in long double, with sigma/delta returned as doubles plus the
 * sigma value split as mantissa * 2^exponent so values beyond 2^1024 survive. */
int oracle_source_ld(int32_t n, const int32_t* off, const int32_t* adj, int32_t s,
                     int32_t* level, double* sigma_mant, int32_t* sigma_exp, double* delta) {
    long double* sg = (long double*)malloc(sizeof(long double) * (size_t)(n > 0 ? n : 1));
    long double* dl = (long double*)malloc(sizeof(long double) * (size_t)(n > 0 ? n : 1));
    long double* bc = (long double*)malloc(sizeof(long double) * (size_t)(n > 0 ? n : 1));
    oracle_detail d;
    memset(&d, 0, sizeof d);
    d.level = level; d.sigma = sg; d.delta = dl;
    int rc = oracle_bc_ld(n, off, adj, 1, &s, bc, &d);
    for (int32_t v = 0; rc == 0 && v < n; ++v) {
        int e = 0;
        /* exact power-of-two split: sigma = mant * 2^e with mant in [0.5, 1) */
        long double x = frexpl(sg[v], &e);
        sigma_mant[v] = (double)x;
        sigma_exp[v] = e;
        delta[v] = (double)dl[v];
    }
    free(sg); free(dl); free(bc);
    return rc;
}

/* ---------------- source-parallel timing wrapper ---------------- */
/* One independent oracle instance per thread over a contiguous slice of the
 * sources; slices' results are summed afterwards in thread order. */
typedef struct {
    int32_t n; const int32_t* off; const int32_t* adj;
    int32_t nsrc; const int32_t* src; double* bc; int rc;
} oracle_slice;

static void* oracle_slice_run(void* p) {
    oracle_slice* t = (oracle_slice*)p;
    t->rc = oracle_bc_f64(t->n, t->off, t->adj, t->nsrc, t->src, t->bc, NULL);
    return NULL;
}

int oracle_bc_f64_threads(int32_t n, const int32_t* off, const int32_t* adj, int32_t nsrc,
                          const int32_t* src, double* bc, int nthreads) {
    if (nthreads < 1) nthreads = 1;
    if (nthreads > nsrc) nthreads = nsrc > 0 ? nsrc : 1;
    oracle_slice* sl = (oracle_slice*)calloc((size_t)nthreads, sizeof(oracle_slice));
    pthread_t* th = (pthread_t*)calloc((size_t)nthreads, sizeof(pthread_t));
    int32_t base = 0;
    for (int t = 0; t < nthreads; ++t) {
        int32_t cnt = nsrc / nthreads + (t < nsrc % nthreads ? 1 : 0);
        sl[t].n = n; sl[t].off = off; sl[t].adj = adj; sl[t].nsrc = cnt; sl[t].src = src + base;
        sl[t].bc = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
        base += cnt;
        pthread_create(&th[t], NULL, oracle_slice_run, &sl[t]);
    }
    int rc = 0;
    for (int32_t v = 0; v < n; ++v) bc[v] = 0;
    for (int t = 0; t < nthreads; ++t) {
        pthread_join(th[t], NULL);
        if (sl[t].rc) rc = sl[t].rc;
        for (int32_t v = 0; v < n; ++v) bc[v] += sl[t].bc[v];
        free(sl[t].bc);
    }
    free(sl); free(th);
    return rc;
}

/* ---------------- per-source path-length sums (breadth-first search only) ----------------
 * For each source s: the sum over the vertices t != s reached from s of
 * (d(s,t) - 1).  A shortest s-t path has d(s,t) - 1 interior vertices, and
 * delta_s(v) is v's share of them over all t, so this equals the sum over
 * v != s of delta_s(v): summed over a source list it is the sum of the raw BC
 * over all vertices.  Distances only (no path counts), so it is cheap enough
 * to check a full-size call; sources are split over threads. */
typedef struct {
    int32_t n;
    const int32_t* off;
    const int32_t* adj;
    int32_t nsrc;
    const int32_t* src;
    int64_t* out;
    int rc;
} dsum_slice;

static void* dsum_run(void* arg) {
    dsum_slice* d = (dsum_slice*)arg;
    const int32_t n = d->n;
    int32_t* dist = (int32_t*)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    int32_t* queue = (int32_t*)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    if (!dist || !queue) { d->rc = -4; free(dist); free(queue); return NULL; }
    for (int32_t i = 0; i < d->nsrc; ++i) {
        const int32_t s = d->src[i];
        if (s < 0 || s >= n) { d->rc = -3; break; }
        for (int32_t v = 0; v < n; ++v) dist[v] = -1;
        int32_t head = 0, tail = 0;
        dist[s] = 0;
        queue[tail++] = s;
        int64_t sum = 0;
        while (head < tail) {
            const int32_t v = queue[head++];
            if (v != s) sum += dist[v] - 1;
            for (int32_t e = d->off[v]; e < d->off[v + 1]; ++e) {
                const int32_t w = d->adj[e];
                if (dist[w] < 0) { dist[w] = dist[v] + 1; queue[tail++] = w; }
            }
        }
        d->out[i] = sum;
    }
    free(dist); free(queue);
    return NULL;
}

/* out[i] for src[i]; returns 0, -3 for a source out of range, -4 when memory runs out. */
int oracle_sum_dm1_threads(int32_t n, const int32_t* off, const int32_t* adj, int32_t nsrc, const int32_t* src,
                           int64_t* out, int nthreads) {
    if (nthreads < 1) nthreads = 1;
    if (nthreads > nsrc) nthreads = nsrc > 0 ? nsrc : 1;
    dsum_slice* sl = (dsum_slice*)calloc((size_t)nthreads, sizeof(dsum_slice));
    pthread_t* th = (pthread_t*)calloc((size_t)nthreads, sizeof(pthread_t));
    if (!sl || !th) { free(sl); free(th); return -4; }
    int32_t base = 0;
    for (int t = 0; t < nthreads; ++t) {
        const int32_t cnt = nsrc / nthreads + (t < nsrc % nthreads ? 1 : 0);
        sl[t].n = n; sl[t].off = off; sl[t].adj = adj; sl[t].nsrc = cnt; sl[t].src = src + base;
        sl[t].out = out + base;
        base += cnt;
        pthread_create(&th[t], NULL, dsum_run, &sl[t]);
    }
    int rc = 0;
    for (int t = 0; t < nthreads; ++t) {
        pthread_join(th[t], NULL);
        if (sl[t].rc) rc = sl[t].rc;
    }
    free(sl); free(th);
    return rc;
}

/* The same sums, 64 sources per breadth-first pass: bit j of a vertex's word
 * marks source j of the group.  Each level pushes the frontier words along
 * every arc; a vertex's bits that are new at level L add L - 1 to their
 * sources' sums.  Groups of sources are split over threads, each with its
 * own words. */
typedef struct {
    int32_t n;
    const int32_t* off;
    const int32_t* adj;
    int32_t nsrc;
    const int32_t* src;
    int64_t* out;
    int rc;
} dsum64_slice;

static void* dsum64_run(void* arg) {
    dsum64_slice* d = (dsum64_slice*)arg;
    const int32_t n = d->n;
    uint64_t* seen = (uint64_t*)malloc(sizeof(uint64_t) * (size_t)(n > 0 ? n : 1));
    uint64_t* front = (uint64_t*)malloc(sizeof(uint64_t) * (size_t)(n > 0 ? n : 1));
    uint64_t* next = (uint64_t*)malloc(sizeof(uint64_t) * (size_t)(n > 0 ? n : 1));
    if (!seen || !front || !next) { d->rc = -4; free(seen); free(front); free(next); return NULL; }
    for (int32_t g0 = 0; g0 < d->nsrc; g0 += 64) {
        const int32_t gs = d->nsrc - g0 < 64 ? d->nsrc - g0 : 64;
        memset(seen, 0, sizeof(uint64_t) * (size_t)n);
        memset(front, 0, sizeof(uint64_t) * (size_t)n);
        for (int32_t j = 0; j < gs; ++j) {
            const int32_t s = d->src[g0 + j];
            if (s < 0 || s >= n) { d->rc = -3; goto done; }
            seen[s] |= 1ull << j;
            front[s] |= 1ull << j;
            d->out[g0 + j] = 0;
        }
        for (int32_t level = 1;; ++level) {
            memset(next, 0, sizeof(uint64_t) * (size_t)n);
            int any = 0;
            for (int32_t v = 0; v < n; ++v) {
                const uint64_t f = front[v];
                if (!f) continue;
                for (int32_t e = d->off[v]; e < d->off[v + 1]; ++e) next[d->adj[e]] |= f;
            }
            for (int32_t w = 0; w < n; ++w) {
                uint64_t nw = next[w] & ~seen[w];
                front[w] = nw;
                if (!nw) continue;
                any = 1;
                seen[w] |= nw;
                while (nw) {
                    const int j = __builtin_ctzll(nw);
                    nw &= nw - 1;
                    d->out[g0 + j] += level - 1;
                }
            }
            if (!any) break;
        }
    }
done:
    free(seen); free(front); free(next);
    return NULL;
}

int oracle_sum_dm1_bits(int32_t n, const int32_t* off, const int32_t* adj, int32_t nsrc, const int32_t* src,
                        int64_t* out, int nthreads) {
    const int32_t groups = (nsrc + 63) / 64;
    if (nthreads < 1) nthreads = 1;
    if (nthreads > groups) nthreads = groups > 0 ? groups : 1;
    dsum64_slice* sl = (dsum64_slice*)calloc((size_t)nthreads, sizeof(dsum64_slice));
    pthread_t* th = (pthread_t*)calloc((size_t)nthreads, sizeof(pthread_t));
    if (!sl || !th) { free(sl); free(th); return -4; }
    int32_t gbase = 0;
    for (int t = 0; t < nthreads; ++t) {
        const int32_t cnt = groups / nthreads + (t < groups % nthreads ? 1 : 0);
        const int32_t b = gbase * 64, e = (gbase + cnt) * 64 < nsrc ? (gbase + cnt) * 64 : nsrc;
        sl[t].n = n; sl[t].off = off; sl[t].adj = adj; sl[t].nsrc = e - b; sl[t].src = src + b; sl[t].out = out + b;
        gbase += cnt;
        pthread_create(&th[t], NULL, dsum64_run, &sl[t]);
    }
    int rc = 0;
    for (int t = 0; t < nthreads; ++t) {
        pthread_join(th[t], NULL);
        if (sl[t].rc) rc = sl[t].rc;
    }
    free(sl); free(th);
    return rc;
}

/* ---------------- ingest: relabelling and validation ---------------- */

static const int32_t* g_deg_for_cmp;
static int cmp_deg_desc(const void* a, const void* b) {
    int32_t x = *(const int32_t*)a, y = *(const int32_t*)b;
    int32_t dx = g_deg_for_cmp[x], dy = g_deg_for_cmp[y];
    if (dx != dy) return dx > dy ? -1 : 1;   /* larger degree first */
    return (x > y) - (x < y);                /* then smaller id first */
}

static int cmp_i32(const void* a, const void* b) {
    int32_t x = *(const int32_t*)a, y = *(const int32_t*)b;
    return (x > y) - (x < y);
}

/*
 * perm[r] = original id of the vertex given new id r, ordering vertices by
 * degree descending with ties by original id ascending; inv[perm[r]] = r.
 * The relabelled CSR has row r = the neighbours of perm[r] mapped through
 * inv and sorted ascending.  new_off: n+1, new_adj: m.
 */
void oracle_relabel(int32_t n, const int32_t* off, const int32_t* adj, int32_t* perm, int32_t* inv,
                    int32_t* new_off, int32_t* new_adj) {
    int32_t* deg = (int32_t*)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    for (int32_t v = 0; v < n; ++v) { deg[v] = off[v + 1] - off[v]; perm[v] = v; }
    g_deg_for_cmp = deg;
    qsort(perm, (size_t)n, sizeof(int32_t), cmp_deg_desc);
    for (int32_t r = 0; r < n; ++r) inv[perm[r]] = r;
    new_off[0] = 0;
    for (int32_t r = 0; r < n; ++r) {
        const int32_t v = perm[r];
        int32_t base = new_off[r];
        for (int32_t e = off[v]; e < off[v + 1]; ++e) new_adj[base + (e - off[v])] = inv[adj[e]];
        qsort(new_adj + base, (size_t)deg[v], sizeof(int32_t), cmp_i32);
        new_off[r + 1] = base + deg[v];
    }
    free(deg);
}

/*
 * CSR validity: 0 when valid, else a reason code.
 *  1 offsets[0] != 0, not non-decreasing, or offsets[n] != m
 *  2 an index outside [0, n)
 *  3 a self-loop
 *  4 a duplicate arc (same neighbour twice in one row)
 *  5 (undirected only) an arc (v,w) without its reverse (w,v)
 * Rows need not be sorted.
 */
int oracle_validate_csr(int32_t n, int64_t m, const int32_t* off, const int32_t* adj, int undirected) {
    if (n < 0 || m < 0) return 1;
    if (off[0] != 0 || (int64_t)off[n] != m) return 1;
    for (int32_t v = 0; v < n; ++v)
        if (off[v + 1] < off[v]) return 1;
    for (int64_t e = 0; e < m; ++e)
        if (adj[e] < 0 || adj[e] >= n) return 2;
    for (int32_t v = 0; v < n; ++v)
        for (int32_t e = off[v]; e < off[v + 1]; ++e)
            if (adj[e] == v) return 3;
    int32_t* row = (int32_t*)malloc(sizeof(int32_t) * (size_t)(m > 0 ? m : 1));
    memcpy(row, adj, sizeof(int32_t) * (size_t)m);
    for (int32_t v = 0; v < n; ++v) qsort(row + off[v], (size_t)(off[v + 1] - off[v]), sizeof(int32_t), cmp_i32);
    int rc = 0;
    for (int32_t v = 0; v < n && !rc; ++v)
        for (int32_t e = off[v] + 1; e < off[v + 1]; ++e)
            if (row[e] == row[e - 1]) { rc = 4; break; }
    if (!rc && undirected) {
        for (int32_t v = 0; v < n && !rc; ++v)
            for (int32_t e = off[v]; e < off[v + 1]; ++e) {
                int32_t w = adj[e];
                if (!bsearch(&v, row + off[w], (size_t)(off[w + 1] - off[w]), sizeof(int32_t), cmp_i32)) { rc = 5; break; }
            }
    }
    free(row);
    return rc;
}
