// Weighted betweenness centrality (positive integer arc weights) on the
// resident graph: Brandes' accumulation over the shortest-path DAG of
// weighted distances.  The paper's BC program (Appendix A, BC listing) walks
// BFS levels; with weights the levels become distances, and the paper's own
// SSSP program (Section 2.3, the Min construct inside a fixed-point loop)
// gives them by Bellman-Ford relaxation.  Per batch of 32 sources (lane =
// column), one cooperative persistent launch runs three fixed-point loops,
// all in place:
//   dist:  d(v) = min(d(v), min over arcs u -> v of d(u) + w), pushed: the
//          rows that changed relax their out-arcs with an atomic min;
//   sigma: s(v) = [v = source] + sum over arcs u -> v with d(u) + w = d(v) of s(u),
//          pulled over in-arcs;
//   delta: t(v) = s(v) * sum over arcs v -> x with d(v) + w = d(x) of rho(x),
//          rho(x) = (1 + t(x)) / s(x), rewritten with each new t(x), pulled
//          over out-arcs.
// Pushes run along out-arcs, so only the dependency loop's stamps (a changed
// row stamps its in-neighbours) read in-arcs: on a directed graph the rows and
// indices of the in-CSR built at ingest, on an undirected one the CSR.  Each
// loop runs until a pass changes nothing; then BC(v) += t(v) for every
// non-source column, columns in order.  Distances only fall and counts and dependencies
// only grow towards the DAG values, so a read of a neighbour another warp is
// rewriting is always a valid bound and the fixed point is the unique one,
// whatever the timing.  After a loop's first pass, a pass recomputes only the
// rows that read a row that changed, or pushes only from the rows that
// changed (stamps).  Distance mins and integer path
// counts do not depend on the order of their terms; every double sum runs in
// CSR order (long rows: per chunk, chunks combined in order), so results
// repeat bit for bit.  Every task is one warp: a row of at most 1024 arcs, or
// a 1024-arc chunk of a longer row (heavy rows: the relabelled prefix
// [0, n_heavy)), whose partials (dependency loop) the row's last chunk
// combines.  Grid barriers are bounded by
// a cycle budget like the traversal kernel's.
#include <climits>
#include <cstdint>
#include <cuda_runtime.h>

#include "bc_internal.cuh"

namespace bcx {
namespace {

constexpr int kWThreads = 256;
constexpr int KW = 32;  // sources per batch
constexpr long long kInf = LLONG_MAX;
constexpr unsigned int kAll = 0xffffffffu;
constexpr int kBuckets = 4096;  // distance buckets of the row order
static_assert(kWbcHistWords == kBuckets + 2, "bucket counts and an 8-byte largest key");
static_assert(kBuckets % kWThreads == 0, "the prefix gives each thread whole buckets");

struct WParams {
    int n;
    WCsr out;                  // out-arcs with their weights
    WCsr in;                   // in-arcs (the same CSR when undirected): rows and indices only,
                               // for the dependency loop's stamps
    int* arr;                  // [heavy rows] chunk arrival counters, by heavy index
    void* scratch;             // [chunk tasks][32] partials (24 bytes each at most); in the
                               // path-count loop, the heavy rows' increments [heavy rows][32]
    const int* src;            // [32] relabelled sources, -1 = unused column
    long long* dist;           // [n][32]
    unsigned long long* sig;   // [n][32] path counts
    double* inv;               // [n][32] 1 / sigma
    double* del;               // [n][32] dependencies
    double* rho;               // [n][32] (1 + delta) / sigma, kept with delta
    int* mark;                 // [2][n] pass stamps: the rows the next pass visits (rows that
                               // changed, in push form; rows that read one, in pull form)
    int* ord;                  // [n] rows by mean distance (dependency passes)
    unsigned int* dag;         // [m] out-arc DAG masks of the batch (bit c: a DAG arc of column c)
    unsigned int* hist;        // [kBuckets] bucket counts, then cursors
    unsigned long long* keymax;  // [1] largest mean distance
    double* bc;                // [n] relabelled
    Ctl* ctl;
    int* changed;              // [3] rotating "a pass changed something" flags
    int* passes;               // [3] passes run by each loop, summed over launches (out)
    unsigned long long* visited;  // [4] arcs and rows the passes read, arcs read through DAG masks and
                                  // the (arc, column) pairs those select, summed over launches (out)
    long long budget;
    int max_passes;
};

__device__ __forceinline__ size_t at(int v, int lane) { return (size_t)v * KW + lane; }

// Reads another warp's partial from L2 (its writer fenced before arriving).
template <class T>
__device__ __forceinline__ T load_cg(const T* q) {
    static_assert(sizeof(T) % 8 == 0, "partials are whole 8-byte words");
    T x;
    long long* d = reinterpret_cast<long long*>(&x);
    const long long* s = reinterpret_cast<const long long*>(q);
#pragma unroll
    for (int i = 0; i < (int)(sizeof(T) / 8); ++i) d[i] = __ldcg(s + i);
    return x;
}

// The light rows a pass visits, in the same warp-interleaved order as one row
// per warp step (slot i goes to warp i mod nw): each lane of a warp reads the
// row and stamp of one of the warp's next 32 slots, so 32 stamp reads are in
// flight together, and the warp runs `body` on the stamped rows in slot order.
// Light slots are the rows [n_heavy, n) of `g` in id order, or the `ord` list
// (reversed when `rev`).
template <class Body>
__device__ __forceinline__ void stamped_light_rows(const WParams& p, const WCsr& g, const int* ord, bool rev,
                                                   int pass, bool all, Body body) {
    const int* mprev = p.mark + (size_t)(pass & 1) * p.n;
    const int lane = threadIdx.x & 31;
    const long long wid = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
    const long long nl = ord ? p.n : p.n - g.n_heavy;
    for (long long s0 = 0; wid + s0 * nw < nl; s0 += 32) {
        const long long i = wid + (s0 + lane) * nw;
        int r = -1;
        if (i < nl) r = ord ? ord[rev ? p.n - 1 - i : i] : g.n_heavy + (int)i;
        unsigned int bits = __ballot_sync(kAll, r >= 0 && (all || mprev[r] == pass));
        while (bits) {
            const int j = __ffs(bits) - 1;
            bits &= bits - 1;
            body(__shfl_sync(kAll, r, j));
        }
    }
}

// One pass over every row of `rd`, one warp per task: a light row, or a
// 1024-arc chunk of a heavy row (chunk slots hcum[k] .. hcum[k+1] of heavy
// row k).  A chunk's partial goes to its scratch slot; the warp that finishes
// a row's last chunk (arrival counter) combines the partials in chunk order
// and finishes the row.
//
// Active rows: a pass recomputes only the rows stamped by the previous pass
// (every row when `all`): a row whose value changed stamps the rows that read
// it (its row in `sc`, the transpose of `rd`) for the next pass, in the other
// of two stamp arrays, so no stamp a pass reads changes during it.
//
// Light rows run in id order, or, given `ord`, in that order (reversed when
// `rev`), every row listed and the heavy ones skipped there.
template <class Arc, class Finish, class T>
__device__ __forceinline__ void row_pass(const WParams& p, const WCsr& rd, const WCsr& sc, T init, Arc arc,
                                         Finish finish, int pass, bool all, const int* ord = nullptr,
                                         bool rev = false) {
    const int* mprev = p.mark + (size_t)(pass & 1) * p.n;
    int* mnext = p.mark + (size_t)((pass + 1) & 1) * p.n;
    auto stamp = [&](int r) {
        for (int j = sc.off[r] + (threadIdx.x & 31); j < sc.off[r + 1]; j += 32) mnext[__ldg(sc.adj + j)] = pass + 1;
    };
    const int lane = threadIdx.x & 31;
    const long long wid = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
    T* scratch = reinterpret_cast<T*>(p.scratch);
    unsigned long long arcs = 0, rows = 0;  // read by this warp (lane 0 reports)
    unsigned long long marcs = 0, lanes = 0;  // of those, arcs read through masks; the columns they select
    for (long long t = wid; t < rd.hchunks; t += nw) {
        {
            int lo = 0, hi = rd.n_heavy;  // hcum[lo] <= t < hcum[hi]
            while (hi - lo > 1) {
                const int mid = (lo + hi) >> 1;
                if (rd.hcum[mid] <= t) lo = mid;
                else hi = mid;
            }
            const int k = lo, r = k, c0 = rd.hcum[k], nch = rd.hcum[k + 1] - c0;
            if (!all && mprev[r] != pass) continue;  // the same answer for every chunk of the row
            const int b = rd.off[r] + (int)(t - c0) * kChunk, e = min(rd.off[r + 1], b + kChunk);
            T acc = arc.start(r, init);
            if (__any_sync(kAll, arc.live(acc))) {
                int j = b;
                for (; j + 4 <= e; j += 4) arc.quad(j, rd.adj, rd.w, acc, lanes);
                for (; j < e; ++j) arc(j, rd.adj, rd.w, acc, lanes);
                arcs += e - b;
                if (Arc::kMasked) marcs += e - b;
            }
            scratch[(size_t)t * KW + lane] = acc;
            __threadfence();
            __syncwarp();
            int last = 0;
            if (lane == 0) last = atomicAdd(&p.arr[k], 1) == nch - 1;
            last = __shfl_sync(kAll, last, 0);
            if (last) {
                __threadfence();
                T tot = load_cg(&scratch[(size_t)c0 * KW + lane]);
                for (int q = 1; q < nch; ++q) tot = Arc::combine(tot, load_cg(&scratch[(size_t)(c0 + q) * KW + lane]));
                ++rows;
                if (__any_sync(kAll, finish(r, tot))) stamp(r);
                if (lane == 0) p.arr[k] = 0;  // ready for the next pass (after its barrier)
            }
        }
    }
    stamped_light_rows(p, rd, ord, rev, pass, all, [&](int r) {
        const int b = rd.off[r], e = rd.off[r + 1];
        if (ord && e - b > kChunk) return;  // a heavy row: its chunk tasks ran it
        T acc = arc.start(r, init);
        ++rows;
        if (__any_sync(kAll, arc.live(acc))) {
            int j = b;
            for (; j + 4 <= e; j += 4) arc.quad(j, rd.adj, rd.w, acc, lanes);
            for (; j < e; ++j) arc(j, rd.adj, rd.w, acc, lanes);
            arcs += e - b;
            if (Arc::kMasked) marcs += e - b;
        }
        if (__any_sync(kAll, finish(r, acc))) stamp(r);
    });
    if (lane == 0 && arcs) atomicAdd(&p.visited[0], arcs);
    if (lane == 0 && rows) atomicAdd(&p.visited[1], rows);
    if (lane == 0 && marcs) atomicAdd(&p.visited[2], marcs);
    if (lane == 0 && lanes) atomicAdd(&p.visited[3], lanes);
}

// Arc functors: start(v, init) gives a row's running state, live(state)
// whether the lane's column needs the row's arcs at all (a warp skips a row
// no lane needs), operator()(j, adj, w, state, lanes) takes arc j of the CSR
// the pass reads, combine joins the partials of a heavy row in order.
struct DeltaAcc {
    double sum;
    long long dv;
};

// The dependency loop's arcs, read through the batch's DAG masks (dag_masks):
// x's index only when some column has the arc, x's rho in those columns.
// `lanes` counts the (arc, column) pairs the masks select.
struct DeltaArc {
    static constexpr bool kMasked = true;
    const WParams* p;
    int lane;
    __device__ DeltaAcc start(int v, DeltaAcc init) const {
        init.dv = p->dist[at(v, lane)];
        return init;
    }
    __device__ bool live(const DeltaAcc& a) const { return a.dv != kInf; }
    __device__ void operator()(int j, const int* adj, const int*, DeltaAcc& a, unsigned long long& lanes) const {
        const unsigned int m = p->dag[j];
        lanes += __popc(m);
        if ((m >> lane) & 1u) a.sum += p->rho[at(__ldg(adj + j), lane)];
    }
    // arcs j..j+3, their loads issued together
    __device__ void quad(int j, const int* adj, const int*, DeltaAcc& a, unsigned long long& lanes) const {
        unsigned int m[4];
        double r[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) m[q] = p->dag[j + q];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const bool s = (m[q] >> lane) & 1u;
            lanes += __popc(m[q]);
            r[q] = s ? p->rho[at(__ldg(adj + j + q), lane)] : 0.0;
        }
#pragma unroll
        for (int q = 0; q < 4; ++q)
            if ((m[q] >> lane) & 1u) a.sum += r[q];  // CSR order
    }
    __device__ static DeltaAcc combine(DeltaAcc a, DeltaAcc b) { return DeltaAcc{a.sum + b.sum, a.dv}; }
};

// The batch's DAG masks, once the distances are final: for every out-arc
// v -> x, bit c set when d_c(v) + w = d_c(x) (a shortest-path DAG arc of
// column c).  One warp per task as in the passes (lane = column, a ballot per
// arc); rows no column reaches keep stale words, which nothing reads (their
// counts never grow and the dependency loop skips them).
__device__ __forceinline__ void dag_masks(const WParams& p) {
    const WCsr& g = p.out;
    const int lane = threadIdx.x & 31;
    const long long wid = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
    const long long tasks = g.hchunks + (p.n - g.n_heavy);
    unsigned long long arcs = 0;
    for (long long t = wid; t < tasks; t += nw) {
        int r, b, e;
        if (t < g.hchunks) {
            int lo = 0, hi = g.n_heavy;  // hcum[lo] <= t < hcum[hi]
            while (hi - lo > 1) {
                const int mid = (lo + hi) >> 1;
                if (g.hcum[mid] <= t) lo = mid;
                else hi = mid;
            }
            r = lo;
            b = g.off[r] + (int)(t - g.hcum[lo]) * kChunk;
            e = min(g.off[r + 1], b + kChunk);
        } else {
            const int i = (int)(t - g.hchunks);
            r = g.n_heavy + i;
            b = g.off[r];
            e = g.off[r + 1];
        }
        const long long dv = p.dist[at(r, lane)];
        if (!__any_sync(kAll, dv != kInf)) continue;
        arcs += e - b;
        int j = b;
        for (; j + 4 <= e; j += 4) {
            int x[4], wq[4];
            long long dx[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                x[q] = __ldg(g.adj + j + q);
                wq[q] = __ldg(g.w + j + q);
            }
#pragma unroll
            for (int q = 0; q < 4; ++q) dx[q] = p.dist[at(x[q], lane)];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const unsigned int m = __ballot_sync(kAll, dv != kInf && dx[q] != kInf && dv + wq[q] == dx[q]);
                if (lane == 0) p.dag[j + q] = m;
            }
        }
        for (; j < e; ++j) {
            const int x = __ldg(g.adj + j);
            const long long dx = p.dist[at(x, lane)];
            const unsigned int m = __ballot_sync(kAll, dv != kInf && dx != kInf && dv + __ldg(g.w + j) == dx);
            if (lane == 0) p.dag[j] = m;
        }
    }
    if (lane == 0 && arcs) atomicAdd(&p.visited[0], arcs);
}

// One pass of the distance loop in push form: every row whose distance changed
// in the previous pass (every reached row on the first pass) relaxes its
// out-arcs, d(v) = min(d(v), d(u) + w) by a 64-bit atomic min per column, and
// a row it lowers is stamped for the next pass.  The min of a set does not
// depend on the order of its terms, so the fixed point is the pull form's;
// a row is read when its own distance changed, not whenever a neighbour's
// did (hubs change rarely and have the longest rows).  Tasks as in row_pass
// (heavy out-rows in kChunk-arc chunks, which need no combining here).
__device__ __forceinline__ bool push_min_pass(const WParams& p, int pass, bool all) {
    const WCsr& g = p.out;
    const int* mprev = p.mark + (size_t)(pass & 1) * p.n;
    int* mnext = p.mark + (size_t)((pass + 1) & 1) * p.n;
    const int lane = threadIdx.x & 31;
    const long long wid = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
    unsigned long long arcs = 0, rows = 0;
    bool ch = false;
    auto work = [&](int r, int b, int e) {
        const long long du = p.dist[at(r, lane)];
        if (!__any_sync(kAll, du != kInf)) return;
        ++rows;
        arcs += e - b;
        if (du == kInf) return;  // this column has nothing to push
        auto relax = [&](int v, long long c, long long dv) {
            if (c < dv && atomicMin(&p.dist[at(v, lane)], c) > c) {
                mnext[v] = pass + 1;
                ch = true;
            }
        };
        int j = b;
        for (; j + 4 <= e; j += 4) {
            int v[4];
            long long c[4], dv[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                v[q] = __ldg(g.adj + j + q);
                c[q] = du + __ldg(g.w + j + q);
            }
#pragma unroll
            for (int q = 0; q < 4; ++q) dv[q] = p.dist[at(v[q], lane)];
#pragma unroll
            for (int q = 0; q < 4; ++q) relax(v[q], c[q], dv[q]);
        }
        for (; j < e; ++j) {
            const int v = __ldg(g.adj + j);
            relax(v, du + __ldg(g.w + j), p.dist[at(v, lane)]);
        }
    };
    for (long long t = wid; t < g.hchunks; t += nw) {
        int lo = 0, hi = g.n_heavy;  // hcum[lo] <= t < hcum[hi]
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (g.hcum[mid] <= t) lo = mid;
            else hi = mid;
        }
        const int r = lo;
        if (!all && mprev[r] != pass) continue;
        const int b = g.off[r] + (int)(t - g.hcum[lo]) * kChunk;
        work(r, b, min(g.off[r + 1], b + kChunk));
    }
    stamped_light_rows(p, g, nullptr, false, pass, all, [&](int r) { work(r, g.off[r], g.off[r + 1]); });
    if (lane == 0 && arcs) atomicAdd(&p.visited[0], arcs);
    if (lane == 0 && rows) atomicAdd(&p.visited[1], rows);
    return ch;
}

// Path counts in push form, one pass: every row stamped by the previous pass
// (every row on the first) adds the growth of its count since its last push,
// inc = sigma(u) - pushed(u), to each DAG successor v (d(u) + w = d(v)) with a
// 64-bit integer atomic add, and stamps v.  Integer sums do not depend on the
// order of their terms, so the counts are the pull form's, bit for bit; a
// wrap of an add (a count reaching 2^64) sets `ovf`.  A heavy row's chunks
// must push the same increment: `hinc` holds the heavy rows' increments,
// taken before the pass (heavy_increments) behind a grid barrier; a light row
// takes its own inline, as one warp owns it.  Adds that land on a row after
// it took its increment are pushed in a later pass (the add stamps it).
__device__ __forceinline__ void heavy_increments(const WParams& p, int pass, bool all,
                                                 unsigned long long* pushed, unsigned long long* hinc) {
    const WCsr& g = p.out;
    const int* mprev = p.mark + (size_t)(pass & 1) * p.n;
    const int lane = threadIdx.x & 31;
    const long long wid = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
    for (long long k = wid; k < g.n_heavy; k += nw) {
        const int r = (int)k;
        if (!all && mprev[r] != pass) continue;
        const unsigned long long s = p.sig[at(r, lane)];
        hinc[(size_t)k * KW + lane] = s - pushed[at(r, lane)];
        pushed[at(r, lane)] = s;
    }
}

__device__ __forceinline__ bool push_sigma_pass(const WParams& p, int pass, bool all, unsigned long long* pushed,
                                                const unsigned long long* hinc, bool& ovf) {
    unsigned long long adds = 0;  // this lane's (arc, column) adds
    const WCsr& g = p.out;
    const int* mprev = p.mark + (size_t)(pass & 1) * p.n;
    int* mnext = p.mark + (size_t)((pass + 1) & 1) * p.n;
    const int lane = threadIdx.x & 31;
    const long long wid = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
    unsigned long long arcs = 0, rows = 0;
    bool ch = false;
    auto work = [&](int b, int e, unsigned long long inc) {
        if (!__any_sync(kAll, inc != 0ull)) return;
        ++rows;
        arcs += e - b;
        if (inc == 0ull) return;  // this column has nothing to push
        auto add = [&](int v, unsigned int m) {
            if ((m >> lane) & 1u) {
                const unsigned long long old = atomicAdd(&p.sig[at(v, lane)], inc);
                ovf |= old + inc < old;
                mnext[v] = pass + 1;
                ch = true;
                ++adds;
            }
        };
        int j = b;
        for (; j + 4 <= e; j += 4) {
            unsigned int m[4];
            int v[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) m[q] = p.dag[j + q];
#pragma unroll
            for (int q = 0; q < 4; ++q) v[q] = m[q] ? __ldg(g.adj + j + q) : 0;
#pragma unroll
            for (int q = 0; q < 4; ++q) add(v[q], m[q]);
        }
        for (; j < e; ++j) {
            const unsigned int m = p.dag[j];
            add(m ? __ldg(g.adj + j) : 0, m);
        }
    };
    for (long long t = wid; t < g.hchunks; t += nw) {
        int lo = 0, hi = g.n_heavy;  // hcum[lo] <= t < hcum[hi]
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (g.hcum[mid] <= t) lo = mid;
            else hi = mid;
        }
        const int r = lo;
        if (!all && mprev[r] != pass) continue;
        const int b = g.off[r] + (int)(t - g.hcum[lo]) * kChunk;
        work(b, min(g.off[r + 1], b + kChunk), hinc[(size_t)lo * KW + lane]);
    }
    stamped_light_rows(p, g, nullptr, false, pass, all, [&](int r) {
        const unsigned long long s = p.sig[at(r, lane)];
        const unsigned long long inc = s - pushed[at(r, lane)];
        pushed[at(r, lane)] = s;
        work(g.off[r], g.off[r + 1], inc);
    });
    if (lane == 0 && arcs) atomicAdd(&p.visited[0], arcs);
    if (lane == 0 && rows) atomicAdd(&p.visited[1], rows);
    if (lane == 0 && arcs) atomicAdd(&p.visited[2], arcs);  // every arc here is read through its mask
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) adds += __shfl_xor_sync(kAll, adds, o);
    if (lane == 0 && adds) atomicAdd(&p.visited[3], adds);
    return ch;
}

__global__ void __launch_bounds__(kWThreads, 5) k_wbc(WParams p) {
    GridTeam team{p.ctl, p.ctl, (int)gridDim.x, p.budget};
    const int lane = threadIdx.x & 31;
    const long long nthr = (long long)gridDim.x * blockDim.x;
    const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long cells = (long long)p.n * KW;
    int pass = 0;
    // true when the pass just ended changed something; false (and an error
    // word) when the pass budget ran out or a barrier failed
    bool fail = false;
    auto end_pass = [&](bool mine) -> bool {
        if (__any_sync(kAll, mine) && lane == 0) p.changed[pass % 3] = 1;
        if (blockIdx.x == 0 && threadIdx.x == 0) p.changed[(pass + 1) % 3] = 0;
        if (!team.sync()) {
            fail = true;
            return false;
        }
        const int c = *(volatile int*)&p.changed[pass % 3];
        ++pass;
        return c != 0;
    };
    for (long long i = tid; i < cells; i += nthr) {
        p.dist[i] = kInf;
        p.sig[i] = 0ull;
        p.del[i] = 0.0;
        p.rho[i] = 0.0;  // all-zero bits: the pushed path counts start at 0
    }
    for (long long i = tid; i < kBuckets; i += nthr) p.hist[i] = 0u;
    if (tid == 0) *p.keymax = 0ull;
    if (!team.sync()) return;
    if (tid < KW && p.src[tid] >= 0) {
        p.dist[at(p.src[tid], (int)tid)] = 0;
        p.sig[at(p.src[tid], (int)tid)] = 1ull;  // the path of length 0
    }
    if (!team.sync()) return;

    // distances, pushed from the rows that changed (stale reads are valid
    // upper bounds: a read below the truth never happens, one above it only
    // costs an atomic that lowers nothing)
    int np = 0;
    for (bool more = true; more;) {
        if (++np > p.max_passes) {
            if (tid == 0) atomicOr(&p.ctl->err, ERR_INTERNAL);
            return;
        }
        more = end_pass(push_min_pass(p, pass, np == 1));
        if (fail) return;
    }
    const int pass_dist = np;
    dag_masks(p);  // read after the row-order barriers below

    // Row order for the next two loops: rows by the mean of their finite
    // distances over the batch's columns, in kBuckets buckets.  A DAG
    // predecessor is closer in its column, so in this order (reversed for the
    // dependencies) an in-place pass mostly meets a row's inputs already
    // updated.  The order within a bucket follows the scatter's timing; it
    // changes pass counts only, never the values.
    {
        long long* key = reinterpret_cast<long long*>(p.inv);  // free until the counts are final
        const long long wid = tid >> 5, nw = nthr >> 5;
        unsigned long long kmax = 0;
        for (long long v = wid; v < p.n; v += nw) {
            const long long d = p.dist[at((int)v, lane)];
            long long sum = d != kInf ? d : 0;
            const int cnt = __popc(__ballot_sync(kAll, d != kInf));
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(kAll, sum, o);
            const long long k = cnt ? sum / cnt : 0;
            if (lane == 0) key[v] = k;
            kmax = (unsigned long long)k > kmax ? (unsigned long long)k : kmax;
        }
        if (lane == 0 && kmax) atomicMax(p.keymax, kmax);
        if (!team.sync()) return;
        const unsigned long long km = *(volatile unsigned long long*)p.keymax;
        auto bucket = [&](long long k) {  // k <= km, so the ratio is at most 1
            return km ? (int)((double)k / (double)km * (kBuckets - 1)) : 0;
        };
        for (long long v = tid; v < p.n; v += nthr) atomicAdd(&p.hist[bucket(key[v])], 1u);
        if (!team.sync()) return;
        if (blockIdx.x == 0) {  // exclusive prefix of the bucket counts, in place
            __shared__ unsigned int part[kWThreads];
            constexpr int per = kBuckets / kWThreads;
            unsigned int loc[per], run = 0;
#pragma unroll
            for (int q = 0; q < per; ++q) {
                loc[q] = *(volatile unsigned int*)&p.hist[threadIdx.x * per + q];
                run += loc[q];
            }
            part[threadIdx.x] = run;
            __syncthreads();
            unsigned int base = 0;
            for (int q = 0; q < (int)threadIdx.x; ++q) base += part[q];
#pragma unroll
            for (int q = 0; q < per; ++q) {
                p.hist[threadIdx.x * per + q] = base;
                base += loc[q];
            }
        }
        if (!team.sync()) return;
        for (long long v = tid; v < p.n; v += nthr) p.ord[atomicAdd(&p.hist[bucket(key[v])], 1u)] = (int)v;
        if (!team.sync()) return;
    }

    // path counts, pushed along the DAG arcs in exact integer increments
    // (pushed counts in the rho array, the heavy rows' increments in the
    // chunk scratch, both free until the dependencies)
    np = 0;
    {
        unsigned long long* pushed = reinterpret_cast<unsigned long long*>(p.rho);
        unsigned long long* hinc = reinterpret_cast<unsigned long long*>(p.scratch);
        for (bool more = true; more;) {
            if (++np > p.max_passes) {
                if (tid == 0) atomicOr(&p.ctl->err, ERR_INTERNAL);
                return;
            }
            heavy_increments(p, pass, np == 1, pushed, hinc);
            if (!team.sync()) return;
            bool ovf = false;
            const bool ch = push_sigma_pass(p, pass, np == 1, pushed, hinc, ovf);
            if (ovf) atomicOr(&p.ctl->err, ERR_SIGMA_RANGE);
            more = end_pass(ch);
            if (fail) return;
        }
    }
    const int pass_sigma = np;
    bool big = false;
    for (long long i = tid; i < cells; i += nthr) {
        big |= p.sig[i] >= (1ull << 53);
        const double iv = p.sig[i] ? 1.0 / (double)p.sig[i] : 0.0;
        p.inv[i] = iv;
        p.rho[i] = iv;  // delta = 0
    }
    if (__any_sync(kAll, big) && lane == 0) atomicOr(&p.ctl->flags, BST_INEXACT);
    if (!team.sync()) return;

    // dependencies, in place, rho rewritten with each new delta
    np = 0;
    for (bool more = true; more;) {
        if (++np > p.max_passes) {
            if (tid == 0) atomicOr(&p.ctl->err, ERR_INTERNAL);
            return;
        }
        bool ch = false;
        auto finish = [&](int v, DeltaAcc a) {
            const double d = (double)p.sig[at(v, lane)] * a.sum;
            if (__double_as_longlong(d) != __double_as_longlong(p.del[at(v, lane)])) {
                p.del[at(v, lane)] = d;
                p.rho[at(v, lane)] = (1.0 + d) * p.inv[at(v, lane)];
                ch = true;
                return true;
            }
            return false;
        };
        DeltaArc arc{&p, lane};
        row_pass<DeltaArc>(p, p.out, p.in, DeltaAcc{0.0, kInf}, arc, finish, pass, np == 1, p.ord, true);
        more = end_pass(ch);
        if (fail) return;
    }
    const int pass_delta = np;

    // BC += delta of every non-source column, columns in order
    for (long long v = tid; v < p.n; v += nthr) {
        double acc = p.bc[v];
        for (int c = 0; c < KW; ++c)
            if (p.src[c] >= 0 && p.src[c] != v) acc += p.del[at((int)v, c)];
        p.bc[v] = acc;
    }
    if (tid == 0) {  // batches run one after another: plain sums
        p.passes[0] += pass_dist;
        p.passes[1] += pass_sigma;
        p.passes[2] += pass_delta;
    }
}

// Weights of the relabelled arcs, looked up in the original CSR (rows sorted
// ascending): relabelled arc (r, c) is original (perm[r], perm[c]).
__global__ void k_weight_lookup(const int* __restrict__ ooff, const int* __restrict__ oadj,
                                const int* __restrict__ ow, const int* __restrict__ perm, const int* __restrict__ noff,
                                const int* __restrict__ nadj, int n, int* nw, int* err) {
    const long long nthr = (long long)gridDim.x * blockDim.x;
    for (long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x; r < n; r += nthr) {
        const int u = perm[r];
        const int b = ooff[u], e = ooff[u + 1];
        for (int j = noff[r]; j < noff[r + 1]; ++j) {
            const int v = perm[nadj[j]];
            int lo = b, hi = e;  // first position with oadj >= v
            while (lo < hi) {
                const int mid = (lo + hi) >> 1;
                if (oadj[mid] < v) lo = mid + 1;
                else hi = mid;
            }
            if (lo < e && oadj[lo] == v) {
                nw[j] = ow[lo];
                if (ow[lo] <= 0) atomicOr(err, 2);
            } else {
                nw[j] = 1;
                atomicOr(err, 1);  // rows not sorted
            }
        }
    }
}

// Both arcs of an undirected edge must carry the same weight.
__global__ void k_weight_symmetry(const int* __restrict__ noff, const int* __restrict__ nadj,
                                  const int* __restrict__ nw, int n, int* err) {
    const long long nthr = (long long)gridDim.x * blockDim.x;
    for (long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x; r < n; r += nthr) {
        for (int j = noff[r]; j < noff[r + 1]; ++j) {
            const int c = nadj[j];
            int lo = noff[c], hi = noff[c + 1];
            while (lo < hi) {
                const int mid = (lo + hi) >> 1;
                if (nadj[mid] < (int)r) lo = mid + 1;
                else hi = mid;
            }
            if (lo >= noff[c + 1] || nadj[lo] != (int)r || nw[lo] != nw[j]) atomicOr(err, 4);
        }
    }
}

}  // namespace

int wbc_blocks() {
    int dev = 0, sms = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_wbc, kWThreads, 0);
    if (per > 5) per = 5;
    return sms * per;
}

cudaError_t launch_wbc(int n, const WCsr& out, const WCsr& in, int* arr, void* scratch, const int* src,
                       long long* dist, unsigned long long* sig, double* inv, double* del, double* rho, int* mark,
                       int* ord, unsigned int* hist, unsigned int* dag, double* bc, Ctl* ctl, int* changed,
                       int* passes, unsigned long long* visited, long long budget, int blocks, cudaStream_t st) {
    WParams p;
    p.n = n;
    p.out = out;
    p.in = in;
    p.arr = arr;
    p.scratch = scratch;
    p.src = src;
    p.dist = dist;
    p.sig = sig;
    p.inv = inv;
    p.del = del;
    p.rho = rho;
    p.mark = mark;
    p.ord = ord;
    p.dag = dag;
    p.hist = hist;
    p.keymax = reinterpret_cast<unsigned long long*>(hist + kBuckets);
    p.bc = bc;
    p.ctl = ctl;
    p.changed = changed;
    p.passes = passes;
    p.visited = visited;
    p.budget = budget;
    p.max_passes = n + 2;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(blocks);
    cfg.blockDim = dim3(kWThreads);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k_wbc, p);
}

cudaError_t launch_weight_ingest(const int* ooff, const int* oadj, const int* ow, const int* perm, const int* noff,
                                 const int* nadj, int n, int* nw, int* err, bool check_symmetry, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    const int blocks = (n + 255) / 256 < 4096 ? (n + 255) / 256 : 4096;
    k_weight_lookup<<<blocks, 256, 0, st>>>(ooff, oadj, ow, perm, noff, nadj, n, nw, err);
    if (check_symmetry) k_weight_symmetry<<<blocks, 256, 0, st>>>(noff, nadj, nw, n, err);
    return cudaGetLastError();
}

}  // namespace bcx
