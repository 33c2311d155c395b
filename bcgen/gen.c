/*
 * Seeded synthetic graph inputs for betweenness-centrality workloads.
 *
 * This module holds no part of the centrality computation: it only produces
 * graphs (int32 CSR), source lists and request streams.  Both the CPU oracle
 * and the CUDA library consume what it writes; neither is linked into it.
 *
 * Random numbers come from one counter-based generator:
 *   mix64(z)          = the SplitMix64 output finaliser (Steele, Lea, Flood,
 *                       "Fast splittable pseudorandom number generators",
 *                       OOPSLA 2014; constants as published by Vigna);
 *   draw(seed,st,t)   = mix64( mix64(seed ^ (st * PHI)) + (t + 1) * PHI ),
 *                       PHI = 0x9E3779B97F4A7C15 (the SplitMix64 increment);
 *   unit(seed,st,t)   = (draw >> 11) * 2^-53, uniform on [0, 1).
 * Streams (st) separate independent uses of one seed.
 *
 * R-MAT follows Chakrabarti, Zhan, Faloutsos (SDM 2004): each edge picks one
 * quadrant per bit level with probabilities (a, b, c, d); no noise is added.
 * The paper this library follows uses R-MAT with a=.57 b=.19 c=.19 d=.05 for
 * its synthetic input (Section 5, input graphs table).
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define PHI 0x9E3779B97F4A7C15ULL

enum { ST_RMAT = 1, ST_PERM = 2, ST_GRID = 3, ST_SRC = 4, ST_ER = 5, ST_TREE = 6 };

uint64_t bcg_mix64(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

uint64_t bcg_draw(uint64_t seed, uint64_t stream, uint64_t t) {
    return bcg_mix64(bcg_mix64(seed ^ (stream * PHI)) + (t + 1) * PHI);
}

static inline uint64_t draw_k(uint64_t key, uint64_t t) { return bcg_mix64(key + (t + 1) * PHI); }
static inline uint64_t stream_key(uint64_t seed, uint64_t stream) { return bcg_mix64(seed ^ (stream * PHI)); }
static inline double unit_k(uint64_t key, uint64_t t) { return (double)(draw_k(key, t) >> 11) * 0x1.0p-53; }
/* uniform integer in [0, bound) by Lemire's multiply-shift (bias < bound/2^64). */
static inline uint64_t below_k(uint64_t key, uint64_t t, uint64_t bound) {
    return (uint64_t)(((__uint128_t)draw_k(key, t) * bound) >> 64);
}

double bcg_unit(uint64_t seed, uint64_t stream, uint64_t t) { return unit_k(stream_key(seed, stream), t); }

/* out[i] = unit(seed, stream, t0 + i) for i < count */
void bcg_units(uint64_t seed, uint64_t stream, int64_t t0, int64_t count, double* out) {
    const uint64_t key = stream_key(seed, stream);
    for (int64_t i = 0; i < count; ++i) out[i] = unit_k(key, (uint64_t)(t0 + i));
}

/* R-MAT edge endpoints (raw: may contain self-loops and duplicates). */
void bcg_rmat_edges(int scale, int64_t nedges, double a, double b, double c, uint64_t seed,
                    int32_t* u, int32_t* v) {
    const uint64_t key = stream_key(seed, ST_RMAT);
    const double ab = a + b, abc = a + b + c;
#pragma omp parallel for schedule(static)
    for (int64_t e = 0; e < nedges; ++e) {
        uint32_t uu = 0, vv = 0;
        for (int lv = 0; lv < scale; ++lv) {
            double r = unit_k(key, (uint64_t)e * (uint64_t)scale + (uint64_t)lv);
            uint32_t bu, bv;
            if (r < a) { bu = 0; bv = 0; }
            else if (r < ab) { bu = 0; bv = 1; }
            else if (r < abc) { bu = 1; bv = 0; }
            else { bu = 1; bv = 1; }
            uu = (uu << 1) | bu;
            vv = (vv << 1) | bv;
        }
        u[e] = (int32_t)uu;
        v[e] = (int32_t)vv;
    }
}

/* Seeded uniform random permutation of [0, n) (Fisher-Yates, Durstenfeld form). */
void bcg_random_perm(int64_t n, uint64_t seed, uint64_t stream, int32_t* perm) {
    const uint64_t key = stream_key(seed, stream);
    for (int64_t i = 0; i < n; ++i) perm[i] = (int32_t)i;
    for (int64_t i = n - 1; i > 0; --i) {
        int64_t j = (int64_t)below_k(key, (uint64_t)i, (uint64_t)(i + 1));
        int32_t t = perm[i]; perm[i] = perm[j]; perm[j] = t;
    }
}

void bcg_apply_perm(int64_t ne, const int32_t* perm, int32_t* u, int32_t* v) {
#pragma omp parallel for schedule(static)
    for (int64_t e = 0; e < ne; ++e) { u[e] = perm[u[e]]; v[e] = perm[v[e]]; }
}

static int cmp_i32(const void* x, const void* y) {
    int32_t a = *(const int32_t*)x, b = *(const int32_t*)y;
    return (a > b) - (a < b);
}

static void sort_row(int32_t* r, int64_t len) {
    if (len < 24) {
        for (int64_t i = 1; i < len; ++i) {
            int32_t x = r[i]; int64_t j = i - 1;
            while (j >= 0 && r[j] > x) { r[j + 1] = r[j]; --j; }
            r[j + 1] = x;
        }
    } else {
        qsort(r, (size_t)len, sizeof(int32_t), cmp_i32);
    }
}

/*
 * Undirected simple CSR from an edge list: both directions of every edge,
 * self-loops dropped, duplicates merged, rows sorted ascending.
 * off: n+1 entries.  adj: capacity 2*ne.  scratch: n+1 int64 (caller-owned).
 * Returns the number of arcs m (= off[n]).
 */
int64_t bcg_edges_to_csr(int32_t n, int64_t ne, const int32_t* u, const int32_t* v,
                         int32_t* off, int32_t* adj, int64_t* pos) {
    memset(pos, 0, sizeof(int64_t) * ((size_t)n + 1));
    for (int64_t e = 0; e < ne; ++e) {
        if (u[e] == v[e]) continue;
        pos[u[e] + 1]++;
        pos[v[e] + 1]++;
    }
    for (int32_t i = 0; i < n; ++i) pos[i + 1] += pos[i];
    /* pos[i] is now the start of row i in the raw (duplicated) layout. */
    int64_t* fill = (int64_t*)malloc(sizeof(int64_t) * (size_t)n);
    for (int32_t i = 0; i < n; ++i) fill[i] = pos[i];
    for (int64_t e = 0; e < ne; ++e) {
        if (u[e] == v[e]) continue;
        adj[fill[u[e]]++] = v[e];
        adj[fill[v[e]]++] = u[e];
    }
    free(fill);
    /* sort + dedup each row, recording the unique length in fill-free way */
    int64_t* ulen = (int64_t*)malloc(sizeof(int64_t) * (size_t)n);
#pragma omp parallel for schedule(dynamic, 1024)
    for (int32_t i = 0; i < n; ++i) {
        int32_t* r = adj + pos[i];
        int64_t len = pos[i + 1] - pos[i];
        sort_row(r, len);
        int64_t w = 0;
        for (int64_t j = 0; j < len; ++j)
            if (w == 0 || r[j] != r[w - 1]) r[w++] = r[j];
        ulen[i] = w;
    }
    /* compact rows to the front, in order */
    int64_t m = 0;
    off[0] = 0;
    for (int32_t i = 0; i < n; ++i) {
        int64_t s = pos[i];
        if (s != m) memmove(adj + m, adj + s, sizeof(int32_t) * (size_t)ulen[i]);
        m += ulen[i];
        off[i + 1] = (int32_t)m;
    }
    free(ulen);
    return m;
}

/*
 * R x C 4-neighbour grid, vertex id = r*C + c.  Of its E = R(C-1) + (R-1)C
 * edges exactly round(remove_frac * E) are removed, chosen by a seeded partial
 * Fisher-Yates shuffle of the edge indices (horizontal edges first, row-major,
 * then vertical edges, row-major).  Returns m; off has R*C+1 entries, adj
 * capacity 2E.
 */
int64_t bcg_grid(int32_t R, int32_t C, double remove_frac, uint64_t seed, int32_t* off, int32_t* adj) {
    const int64_t EH = (int64_t)R * (C - 1), E = EH + (int64_t)(R - 1) * C;
    int64_t nrem = (int64_t)(remove_frac * (double)E + 0.5);
    if (nrem > E) nrem = E;
    int32_t* idx = (int32_t*)malloc(sizeof(int32_t) * (size_t)E);
    uint8_t* gone = (uint8_t*)calloc((size_t)E, 1);
    for (int64_t i = 0; i < E; ++i) idx[i] = (int32_t)i;
    const uint64_t key = stream_key(seed, ST_GRID);
    for (int64_t i = 0; i < nrem; ++i) {
        int64_t j = i + (int64_t)below_k(key, (uint64_t)i, (uint64_t)(E - i));
        int32_t t = idx[i]; idx[i] = idx[j]; idx[j] = t;
        gone[idx[i]] = 1;
    }
    free(idx);
    int64_t m = 0;
    off[0] = 0;
    for (int32_t r = 0; r < R; ++r) {
        for (int32_t c = 0; c < C; ++c) {
            /* neighbours in ascending id order: up, left, right, down */
            if (r > 0 && !gone[EH + (int64_t)(r - 1) * C + c]) adj[m++] = (r - 1) * C + c;
            if (c > 0 && !gone[(int64_t)r * (C - 1) + (c - 1)]) adj[m++] = r * C + c - 1;
            if (c < C - 1 && !gone[(int64_t)r * (C - 1) + c]) adj[m++] = r * C + c + 1;
            if (r < R - 1 && !gone[EH + (int64_t)r * C + c]) adj[m++] = (r + 1) * C + c;
            off[(int64_t)r * C + c + 1] = (int32_t)m;
        }
    }
    free(gone);
    return m;
}

/*
 * k sources drawn uniformly without replacement from the vertices of degree
 * >= 1 (partial Fisher-Yates over that candidate list).  Returns the number
 * written (min(k, #candidates)).
 */
int32_t bcg_sample_sources(int32_t n, const int32_t* off, int32_t k, uint64_t seed, int32_t* out) {
    int32_t* cand = (int32_t*)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    int32_t nc = 0;
    for (int32_t i = 0; i < n; ++i)
        if (off[i + 1] > off[i]) cand[nc++] = i;
    if (k > nc) k = nc;
    const uint64_t key = stream_key(seed, ST_SRC);
    for (int32_t i = 0; i < k; ++i) {
        int32_t j = i + (int32_t)below_k(key, (uint64_t)i, (uint64_t)(nc - i));
        int32_t t = cand[i]; cand[i] = cand[j]; cand[j] = t;
        out[i] = cand[i];
    }
    free(cand);
    return k;
}

/* Erdos-Renyi G(n, p) edge list (i < j); returns the number of edges written (<= cap). */
int64_t bcg_gnp_edges(int32_t n, double p, uint64_t seed, int32_t* u, int32_t* v, int64_t cap) {
    const uint64_t key = stream_key(seed, ST_ER);
    int64_t ne = 0, t = 0;
    for (int32_t i = 0; i < n; ++i)
        for (int32_t j = i + 1; j < n; ++j, ++t)
            if (unit_k(key, (uint64_t)t) < p && ne < cap) { u[ne] = i; v[ne] = j; ++ne; }
    return ne;
}

/* Uniform random labelled tree on n >= 2 vertices from a random Pruefer sequence; writes n-1 edges. */
void bcg_random_tree(int32_t n, uint64_t seed, int32_t* u, int32_t* v) {
    const uint64_t key = stream_key(seed, ST_TREE);
    if (n < 2) return;
    int32_t L = n - 2;
    int32_t* seq = (int32_t*)malloc(sizeof(int32_t) * (size_t)(L > 0 ? L : 1));
    int32_t* deg = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
    for (int32_t i = 0; i < n; ++i) deg[i] = 1;
    for (int32_t i = 0; i < L; ++i) { seq[i] = (int32_t)below_k(key, (uint64_t)i, (uint64_t)n); deg[seq[i]]++; }
    /* linear-time decoding: ptr walks the smallest leaf */
    int32_t ptr = 0;
    while (deg[ptr] != 1) ++ptr;
    int32_t leaf = ptr, ne = 0;
    for (int32_t i = 0; i < L; ++i) {
        int32_t x = seq[i];
        u[ne] = leaf; v[ne] = x; ++ne;
        if (--deg[x] == 1 && x < ptr) {
            leaf = x;
        } else {
            ++ptr;
            while (deg[ptr] != 1) ++ptr;
            leaf = ptr;
        }
    }
    /* last edge joins the remaining leaf to n-1 */
    u[ne] = leaf; v[ne] = n - 1;
    free(seq); free(deg);
}
