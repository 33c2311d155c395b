// Batched Brandes betweenness centrality: the persistent sm_103a kernel.
//
// One cooperative launch runs every batch of a bc_compute call.  A batch is
// K sources (K = 1, 32, 64 or 128) traversed together: column c of every
// per-vertex array belongs to source c of the batch, and all columns advance
// one BFS level per iteration (the paper's iterateInBFS, Section 2.2, run for
// K roots at once).  Per iteration:
//   * discovery, either top-down (push: frontier rows claim unseen neighbours
//     with atomicOr on their column masks, warp-aggregated list appends) or
//     bottom-up (pull: every not-yet-complete vertex scans its row against the
//     frontier masks), switched by frontier size;
//   * the path-count sum sigma_c(w) = sum of sigma_c(v) over frontier
//     neighbours v (the BFS body w.sigma += v.sigma of the BC listing), pulled
//     over each new vertex's row: no atomics.
// Then the reverse sweep (iterateInReverse) walks the kept level lists from
// the deepest level up, pulling rho_c(w) = (1 + delta_c(w)) / sigma_c(w) from
// DAG successors:  delta_c(v) = sigma_c(v) * sum_w rho_c(w).  This equals the
// listing's per-arc (sigma_v / sigma_w)(1 + delta_w) summed over w, with one
// division per vertex and column instead of one per arc.  Finally each vertex
// adds its columns' delta into BC (source columns excluded), in column order.
//
// Lanes map to columns (K >= 32: lane l owns columns [W*l, W*l + W), W = K/32)
// so that a neighbour's per-column values are one coalesced row read; with
// K == 1 lanes map to neighbours instead.  Every floating-point sum runs in
// CSR order within fixed 1024-arc chunks, chunks combined in order, so each
// column's arithmetic is independent of K, of the other columns and of the
// push/pull choice: results are bitwise reproducible across batch widths.
//
// Grid-wide phases are separated by a software barrier whose wait is bounded
// by a cycle budget; on expiry it raises ERR_TIMEOUT and every block returns.
#include <cstdint>
#include <cuda_runtime.h>

#include "bc_internal.cuh"

namespace bcx {

#define FULL_MASK 0xffffffffu

__device__ __forceinline__ int lane_id() { return threadIdx.x & 31; }
__device__ __forceinline__ int warp_id() { return threadIdx.x >> 5; }

// ------------------------------------------------------------------ barrier
struct GridTeam {
    Ctl* ctl;
    long long budget;

    // Returns false when the launch has failed (timeout or a fatal error).
    __device__ bool sync() {
        __shared__ int s_bad;
        __syncthreads();
        if (threadIdx.x == 0) {
            int bad = 0;
            volatile unsigned int* genp = &ctl->bar_gen;
            volatile int* errp = &ctl->err;
            unsigned int g = *genp;
            __threadfence();
            unsigned int arrived = atomicAdd(&ctl->bar_count, 1u);
            if (arrived == gridDim.x - 1) {
                atomicExch(&ctl->bar_count, 0u);
                __threadfence();
                atomicAdd(&ctl->bar_gen, 1u);
            } else {
                long long t0 = clock64();
                while (*genp == g) {
                    if (*errp) { bad = 1; break; }
                    if (clock64() - t0 > budget) { atomicOr(&ctl->err, ERR_TIMEOUT); bad = 1; break; }
                    __nanosleep(64);
                }
            }
            __threadfence();
            if (*errp) bad = 1;
            s_bad = bad;
        }
        __syncthreads();
        return !s_bad;
    }
};

// ------------------------------------------------------------------ work distribution
__device__ __forceinline__ int block_grab(unsigned int* ctr, long long total) {
    __shared__ int s_item;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned int i = atomicAdd(ctr, 1u);
        s_item = ((long long)i < total) ? (int)i : -1;
    }
    __syncthreads();
    return s_item;
}

__device__ __forceinline__ long long warp_grab(unsigned int* ctr, long long total, int G, int& cnt) {
    unsigned int i = 0;
    if (lane_id() == 0) i = atomicAdd(ctr, (unsigned int)G);
    i = __shfl_sync(FULL_MASK, i, 0);
    if ((long long)i >= total) { cnt = 0; return -1; }
    long long rem = total - (long long)i;
    cnt = rem < G ? (int)rem : G;
    return (long long)i;
}

// ------------------------------------------------------------------ masks
template <int W>
struct Mask {
    uint32_t w[W];
};

template <int W>
__device__ __forceinline__ void load_mask(const uint32_t* base, int v, uint32_t (&m)[W]) {
    const uint32_t* p = base + (size_t)v * W;
    if constexpr (W == 1) {
        m[0] = p[0];
    } else if constexpr (W == 2) {
        uint2 x = *reinterpret_cast<const uint2*>(p);
        m[0] = x.x; m[1] = x.y;
    } else {
        uint4 x = *reinterpret_cast<const uint4*>(p);
        m[0] = x.x; m[1] = x.y; m[2] = x.z; m[3] = x.w;
    }
}

template <int W>
__device__ __forceinline__ bool mask_any(const uint32_t (&m)[W]) {
    uint32_t a = 0;
#pragma unroll
    for (int t = 0; t < W; ++t) a |= m[t];
    return a != 0;
}

// bits of column group [W*lane, W*lane+W) taken from word `word` of the mask
template <int W>
__device__ __forceinline__ uint32_t lane_field(uint32_t word, int lane) {
    return (word >> ((W * lane) & 31)) & ((1u << W) - 1u);
}

// ------------------------------------------------------------------ extended-range arithmetic
// Path count as m * 2^e with a 64-bit integer mantissa; values below 2^64 keep
// e == 0 and are exact.  A nonzero e implies the top mantissa bit is set.
__device__ __forceinline__ void xu_add(unsigned long long& am, int& ae, unsigned long long xm, int xe) {
    if (xm == 0) return;
    if (am == 0) { am = xm; ae = xe; return; }
    if (xe > ae) {
        int d = xe - ae;
        am = d >= 64 ? 0ull : (am >> d);
        ae = xe;
    } else if (xe < ae) {
        int d = ae - xe;
        xm = d >= 64 ? 0ull : (xm >> d);
    }
    unsigned long long s = am + xm;
    if (s < am) {  // carry out of bit 63
        s = (s >> 1) | (1ull << 63);
        ae += 1;
    }
    am = s;
}

// Real value r * 2^e (r a double) summed with alignment to the larger exponent.
__device__ __forceinline__ void xd_add(double& ar, int& ae, double xr, int xe) {
    if (xr == 0.0) return;
    if (ar == 0.0) { ar = xr; ae = xe; return; }
    if (xe > ae) {
        ar = scalbn(ar, ae - xe);
        ae = xe;
        ar += xr;
    } else {
        ar += scalbn(xr, xe - ae);
    }
}

// ------------------------------------------------------------------ accumulators
// Per lane, W columns.  FWD: path counts.  BWD: sums of rho.
enum { FWD = 0, BWD = 1 };

template <int W, bool EXT, int DIR>
struct Acc {
    unsigned long long m[W];  // FWD mantissa
    double r[W];              // BWD value
    int e[W];                 // exponent (EXT)
    __device__ __forceinline__ void zero() {
#pragma unroll
        for (int t = 0; t < W; ++t) { m[t] = 0ull; r[t] = 0.0; e[t] = 0; }
    }
    // add column t of another accumulator / term
    __device__ __forceinline__ void add1(int t, unsigned long long xm, double xr, int xe, bool& carry) {
        if constexpr (DIR == FWD) {
            if constexpr (EXT) {
                xu_add(m[t], e[t], xm, xe);
            } else {
                unsigned long long s = m[t] + xm;
                carry |= (s < xm);
                m[t] = s;
            }
        } else {
            if constexpr (EXT) xd_add(r[t], e[t], xr, xe);
            else r[t] += xr;
        }
    }
    __device__ __forceinline__ void add_acc(const Acc& o, bool& carry) {
#pragma unroll
        for (int t = 0; t < W; ++t) add1(t, o.m[t], o.r[t], o.e[t], carry);
    }
};

// ------------------------------------------------------------------ gathers
// Load the per-column term of neighbour v for this lane's columns selected by `my`.
template <int K, int W, bool EXT, int DIR>
__device__ __forceinline__ void load_term(const KParams& p, int v, uint32_t my, Acc<W, EXT, DIR>& tm) {
    tm.zero();
    if (!my) return;
    const int lane = lane_id();
    const size_t base = (size_t)v * K + (K == 1 ? 0 : (size_t)W * lane);
    if constexpr (DIR == FWD) {
        const unsigned long long* s = p.sig + base;
        if constexpr (W == 1) {
            tm.m[0] = s[0];
        } else if constexpr (W == 2) {
            ulonglong2 x = *reinterpret_cast<const ulonglong2*>(s);
            tm.m[0] = x.x; tm.m[1] = x.y;
        } else {
            ulonglong2 x = *reinterpret_cast<const ulonglong2*>(s);
            ulonglong2 y = *reinterpret_cast<const ulonglong2*>(s + 2);
            tm.m[0] = x.x; tm.m[1] = x.y; tm.m[2] = y.x; tm.m[3] = y.y;
        }
        if constexpr (EXT) {
#pragma unroll
            for (int t = 0; t < W; ++t) tm.e[t] = p.sig_e[base + t];
        }
    } else {
        const double* s = p.rho + base;
        if constexpr (W == 1) {
            tm.r[0] = s[0];
        } else if constexpr (W == 2) {
            double2 x = *reinterpret_cast<const double2*>(s);
            tm.r[0] = x.x; tm.r[1] = x.y;
        } else {
            double2 x = *reinterpret_cast<const double2*>(s);
            double2 y = *reinterpret_cast<const double2*>(s + 2);
            tm.r[0] = x.x; tm.r[1] = x.y; tm.r[2] = y.x; tm.r[3] = y.y;
        }
        if constexpr (EXT) {
#pragma unroll
            for (int t = 0; t < W; ++t) tm.e[t] = p.rho_e[base + t];
        }
    }
#pragma unroll
    for (int t = 0; t < W; ++t)
        if (!((my >> t) & 1u)) { tm.m[t] = 0ull; tm.r[t] = 0.0; tm.e[t] = 0; }
}

// One chunk [cb, ce) of a row, in CSR order, into `part` (zeroed by the caller).
// Fm: neighbour masks; want: the columns of interest (uniform across the warp);
// orm: per-lane OR of the matched masks (reduced by the caller).
template <int K, int W, bool EXT, int DIR>
__device__ __forceinline__ void gather_chunk(const KParams& p, long long cb, long long ce, const uint32_t* Fm,
                                             const uint32_t (&want)[W], Acc<W, EXT, DIR>& part,
                                             uint32_t (&orm)[W], bool& carry) {
    const int lane = lane_id();
    const int myword = (W * lane) >> 5;
    for (long long base = cb; base < ce; base += 32) {
        const long long e = base + lane;
        int v = 0;
        uint32_t f[W];
#pragma unroll
        for (int t = 0; t < W; ++t) f[t] = 0;
        if (e < ce) {
            v = __ldg(p.adj + e);
            load_mask<W>(Fm, v, f);
#pragma unroll
            for (int t = 0; t < W; ++t) f[t] &= want[t];
        }
#pragma unroll
        for (int t = 0; t < W; ++t) orm[t] |= f[t];
        unsigned int bal = __ballot_sync(FULL_MASK, mask_any<W>(f));
        if constexpr (K == 1) {
            // lanes own neighbours: each matching lane loads its own term, then the
            // terms are added in lane (= CSR) order by every lane.
            Acc<W, EXT, DIR> mine;
            load_term<K, W, EXT, DIR>(p, v, f[0] & 1u, mine);
            while (bal) {
                const int j = __ffs(bal) - 1;
                bal &= bal - 1;
                unsigned long long xm = __shfl_sync(FULL_MASK, mine.m[0], j);
                double xr = __shfl_sync(FULL_MASK, mine.r[0], j);
                int xe = __shfl_sync(FULL_MASK, mine.e[0], j);
                part.add1(0, xm, xr, xe, carry);
            }
        } else {
            while (bal) {
                int js[4];
                int nj = 0;
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    if (bal) { js[q] = __ffs(bal) - 1; bal &= bal - 1; nj = q + 1; }
                    else js[q] = 0;
                }
                Acc<W, EXT, DIR> tm[4];
                uint32_t my[4];
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const int vj = __shfl_sync(FULL_MASK, v, js[q]);
                    uint32_t word = 0;
#pragma unroll
                    for (int t = 0; t < W; ++t) {
                        uint32_t x = __shfl_sync(FULL_MASK, f[t], js[q]);
                        if (t == myword) word = x;
                    }
                    my[q] = (q < nj) ? lane_field<W>(word, lane) : 0u;
                    load_term<K, W, EXT, DIR>(p, vj, my[q], tm[q]);
                }
#pragma unroll
                for (int q = 0; q < 4; ++q)
                    if (q < nj) part.add_acc(tm[q], carry);
            }
        }
    }
}

// Whole row by one warp: chunks of kChunk arcs, each summed in order from zero,
// combined in order into `total` (zeroed here).
template <int K, int W, bool EXT, int DIR>
__device__ __forceinline__ void warp_row(const KParams& p, long long beg, long long end, const uint32_t* Fm,
                                         const uint32_t (&want)[W], Acc<W, EXT, DIR>& total, uint32_t (&orm)[W],
                                         bool& carry) {
    total.zero();
    for (long long cb = beg; cb < end; cb += kChunk) {
        Acc<W, EXT, DIR> part;
        part.zero();
        const long long ce = (end < cb + kChunk) ? end : cb + kChunk;
        gather_chunk<K, W, EXT, DIR>(p, cb, ce, Fm, want, part, orm, carry);
        total.add_acc(part, carry);
    }
}

template <int W>
__device__ __forceinline__ void warp_or_reduce(uint32_t (&m)[W]) {
#pragma unroll
    for (int t = 0; t < W; ++t) m[t] = __reduce_or_sync(FULL_MASK, m[t]);
}

// Shared scratch for block-level (heavy) rows.
template <int W>
struct HeavySmem {
    unsigned long long m[kWarps][32 * W];
    double r[kWarps][32 * W];
    int e[kWarps][32 * W];
    uint32_t orm[W];
    int carry;
};

// Whole row by the block: warp w takes chunks w, w + kWarps, ...; partials are
// combined in chunk order by warp 0, which returns the total.  The OR of the
// matched masks is returned to every warp.
template <int K, int W, bool EXT, int DIR>
__device__ void block_row(const KParams& p, long long beg, long long end, const uint32_t* Fm,
                          const uint32_t (&want)[W], Acc<W, EXT, DIR>& total, uint32_t (&orm)[W], bool& carry,
                          HeavySmem<W>& sh) {
    const int lane = lane_id(), wid = warp_id();
    total.zero();
    if (threadIdx.x < W) sh.orm[threadIdx.x] = 0;
    if (threadIdx.x == 0) sh.carry = 0;
    const long long nch = (end - beg + kChunk - 1) / kChunk;
    for (long long r0 = 0; r0 < nch; r0 += kWarps) {
        Acc<W, EXT, DIR> part;
        part.zero();
        const long long c = r0 + wid;
        if (c < nch) {
            const long long cb = beg + c * kChunk;
            const long long ce = (end < cb + kChunk) ? end : cb + kChunk;
            gather_chunk<K, W, EXT, DIR>(p, cb, ce, Fm, want, part, orm, carry);
        }
        // K == 1: every lane holds the same partial; lane-indexed slots keep the code uniform
#pragma unroll
        for (int t = 0; t < W; ++t) {
            sh.m[wid][lane * W + t] = part.m[t];
            sh.r[wid][lane * W + t] = part.r[t];
            sh.e[wid][lane * W + t] = part.e[t];
        }
        __syncthreads();
        if (wid == 0) {
            const long long lim = (nch - r0 < kWarps) ? (nch - r0) : kWarps;
            for (int w2 = 0; w2 < lim; ++w2) {
#pragma unroll
                for (int t = 0; t < W; ++t)
                    total.add1(t, sh.m[w2][lane * W + t], sh.r[w2][lane * W + t], sh.e[w2][lane * W + t], carry);
            }
        }
        __syncthreads();
    }
    warp_or_reduce<W>(orm);
    if (lane == 0) {
#pragma unroll
        for (int t = 0; t < W; ++t) atomicOr(&sh.orm[t], orm[t]);
        if (carry) atomicOr(&sh.carry, 1);
    }
    __syncthreads();
#pragma unroll
    for (int t = 0; t < W; ++t) orm[t] = sh.orm[t];
    carry = sh.carry != 0;
    __syncthreads();
}

// ------------------------------------------------------------------ appends
// Per-warp staging of discovered vertices; flushed 32 at a time.
struct AppendBuf {
    int v[kWarps][32];
    long long dsum[kWarps];
};

__device__ __forceinline__ void flush_append(const KParams& p, int lev, AppendBuf& ab, int& cnt) {
    const int lane = lane_id(), wid = warp_id();
    if (cnt == 0) return;
    __syncwarp();
    int base = 0;
    if (lane == 0) {
        base = atomicAdd(&p.la.cnt[lev], cnt);
        atomicAdd((unsigned long long*)&p.la.dsum[lev], (unsigned long long)ab.dsum[wid]);
        ab.dsum[wid] = 0;
    }
    base = __shfl_sync(FULL_MASK, base, 0);
    const long long pos = (long long)p.la.start[lev] + base + lane;
    if (lane < cnt) {
        if (pos < p.cap) p.ent[pos] = ab.v[wid][lane];
        else atomicOr(&p.ctl->err, ERR_CAPACITY);
    }
    __syncwarp();
    cnt = 0;
}

// append one vertex (called by the whole warp, uniform)
__device__ __forceinline__ void warp_append(const KParams& p, int lev, int w, long long deg, AppendBuf& ab, int& cnt) {
    const int lane = lane_id(), wid = warp_id();
    if (lane == 0) { ab.v[wid][cnt] = w; ab.dsum[wid] += deg; }
    __syncwarp();
    ++cnt;
    if (cnt == 32) flush_append(p, lev, ab, cnt);
}

__device__ __forceinline__ void heavy_append(const KParams& p, int lev, int w, long long deg) {
    int i = atomicAdd(&p.la.hcnt[lev], 1);
    atomicAdd((unsigned long long*)&p.la.dsum[lev], (unsigned long long)deg);
    long long pos = (long long)p.la.hstart[lev] + i;
    if (pos < p.hcap) p.hent[pos] = w;
    else atomicOr(&p.ctl->err, ERR_CAPACITY);
}

// ------------------------------------------------------------------ vertex finalisation
// Forward: write path counts and levels of the newly reached columns `nm` of w.
template <int K, int W, bool EXT>
__device__ __forceinline__ void fwd_finish(const KParams& p, int w, const uint32_t (&nm)[W], int lev,
                                           const uint32_t (&active)[W], const Acc<W, EXT, FWD>& tot) {
    const int lane = lane_id();
    if constexpr (K == 1) {
        if (lane == 0) {
            p.sig[w] = tot.m[0];
            if constexpr (EXT) p.sig_e[w] = tot.e[0];
            p.lvl[w] = (uint16_t)lev;
            p.V[w] |= nm[0];
            bool inexact = EXT ? (tot.e[0] > 0 || tot.m[0] >= (1ull << 53)) : (tot.m[0] >= (1ull << 53));
            if (inexact) atomicOr(&p.ctl->flags, BST_INEXACT);
            if ((p.V[w] & active[0]) == active[0])
                atomicAdd((unsigned long long*)&p.la.fulldeg[lev], (unsigned long long)(p.off[w + 1] - p.off[w]));
        }
    } else {
        const int myword = (W * lane) >> 5;
        uint32_t word = 0;
#pragma unroll
        for (int t = 0; t < W; ++t)
            if (t == myword) word = nm[t];
        const uint32_t my = lane_field<W>(word, lane);
        bool inexact = false;
#pragma unroll
        for (int t = 0; t < W; ++t) {
            if ((my >> t) & 1u) {
                const size_t idx = (size_t)w * K + W * lane + t;
                p.sig[idx] = tot.m[t];
                if constexpr (EXT) p.sig_e[idx] = tot.e[t];
                p.lvl[idx] = (uint16_t)lev;
                inexact |= EXT ? (tot.e[t] > 0 || tot.m[t] >= (1ull << 53)) : (tot.m[t] >= (1ull << 53));
            }
        }
        if (__any_sync(FULL_MASK, inexact) && lane == 0) atomicOr(&p.ctl->flags, BST_INEXACT);
        bool full = true;
        if (lane < W) {
            uint32_t nv = p.V[(size_t)w * W + lane] | nm[0];
            // select nm[lane] without dynamic register indexing
#pragma unroll
            for (int t = 0; t < W; ++t)
                if (t == lane) nv = p.V[(size_t)w * W + lane] | nm[t];
            p.V[(size_t)w * W + lane] = nv;
            uint32_t act = active[0];
#pragma unroll
            for (int t = 0; t < W; ++t)
                if (t == lane) act = active[t];
            full = (nv & act) == act;
        }
        full = __all_sync(FULL_MASK, full);
        if (full && lane == 0)
            atomicAdd((unsigned long long*)&p.la.fulldeg[lev], (unsigned long long)(p.off[w + 1] - p.off[w]));
    }
}

// Backward: from the rho sums, delta and rho of v for its columns `mk` at level l.
template <int K, int W, bool EXT>
__device__ __forceinline__ void bwd_finish(const KParams& p, int v, const uint32_t (&mk)[W],
                                           const Acc<W, EXT, BWD>& tot) {
    const int lane = lane_id();
    uint32_t my;
    if constexpr (K == 1) {
        my = (lane == 0) ? (mk[0] & 1u) : 0u;
    } else {
        const int myword = (W * lane) >> 5;
        uint32_t word = 0;
#pragma unroll
        for (int t = 0; t < W; ++t)
            if (t == myword) word = mk[t];
        my = lane_field<W>(word, lane);
    }
#pragma unroll
    for (int t = 0; t < W; ++t) {
        if ((my >> t) & 1u) {
            const size_t idx = (size_t)v * K + (K == 1 ? 0 : W * lane + t);
            const unsigned long long sm = p.sig[idx];
            const double sd = (double)sm;  // rounds only when the count is >= 2^53
            double delta, rho;
            int rho_e = 0;
            if constexpr (EXT) {
                const int se = p.sig_e[idx];
                delta = scalbn(sd * tot.r[t], se + tot.e[t]);
                rho = (1.0 + delta) / sd;
                rho_e = -se;
            } else {
                delta = sd * tot.r[t];
                rho = (1.0 + delta) / sd;
            }
            p.sig[idx] = (unsigned long long)__double_as_longlong(delta);
            p.rho[idx] = rho;
            if constexpr (EXT) p.rho_e[idx] = rho_e;
        }
    }
}

// ------------------------------------------------------------------ phases
template <int K>
struct Cfg {
    static constexpr int W = K >= 32 ? K / 32 : 1;
};

// Level-`lev` column mask of v from the stored levels (K >= 32: every lane
// tests its W columns; the words are assembled with OR reductions).
template <int K, int W>
__device__ __forceinline__ void level_mask(const KParams& p, int v, int lev, uint32_t (&mk)[W]) {
    const int lane = lane_id();
    uint32_t vm[W];
    load_mask<W>(p.V, v, vm);
    if constexpr (K == 1) {
        mk[0] = (vm[0] & 1u) && p.lvl[v] == (uint16_t)lev ? 1u : 0u;
    } else {
        uint32_t field = 0;
#pragma unroll
        for (int t = 0; t < W; ++t)
            if (p.lvl[(size_t)v * K + W * lane + t] == (uint16_t)lev) field |= 1u << t;
        const int myword = (W * lane) >> 5;
#pragma unroll
        for (int t = 0; t < W; ++t) {
            uint32_t contrib = (t == myword) ? (field << ((W * lane) & 31)) : 0u;
            mk[t] = __reduce_or_sync(FULL_MASK, contrib) & vm[t];
        }
    }
}

template <int W>
__device__ __forceinline__ void store_mask(uint32_t* base, int v, const uint32_t (&m)[W]) {
    const int lane = lane_id();
    if (lane < W) {
        uint32_t x = m[0];
#pragma unroll
        for (int t = 0; t < W; ++t)
            if (t == lane) x = m[t];
        base[(size_t)v * W + lane] = x;
    }
}

// Per-phase counters: slot = ph & 3; the slot two phases ahead is cleared here.
__device__ __forceinline__ unsigned int* wq_heavy(const KParams& p, int ph) { return &p.ctl->wq[(ph & 3) * 2]; }
__device__ __forceinline__ unsigned int* wq_light(const KParams& p, int ph) { return &p.ctl->wq[(ph & 3) * 2 + 1]; }
__device__ __forceinline__ void phase_prologue(const KParams& p, int ph) {
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        p.ctl->wq[((ph + 2) & 3) * 2] = 0;
        p.ctl->wq[((ph + 2) & 3) * 2 + 1] = 0;
    }
}

// Clear the dense masks of level `lev` (entries of that level) in buffer F.
template <int W>
__device__ void clear_level_masks(const KParams& p, uint32_t* F, int lev) {
    const long long s = p.la.start[lev], c = p.la.cnt[lev], hs = p.la.hstart[lev], hc = p.la.hcnt[lev];
    const long long nthr = (long long)gridDim.x * blockDim.x;
    const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    for (long long i = tid; i < (c + hc) * W; i += nthr) {
        long long j = i / W;
        int t = (int)(i % W);
        int v = j < c ? p.ent[s + j] : p.hent[hs + (j - c)];
        F[(size_t)v * W + t] = 0;
    }
}

template <int K>
__device__ void active_mask(const KParams& p, int b, uint32_t (&act)[Cfg<K>::W]) {
    constexpr int W = Cfg<K>::W;
#pragma unroll
    for (int t = 0; t < W; ++t) act[t] = 0;
    for (int c = 0; c < K; ++c)
        if (p.src[(size_t)b * K + c] >= 0) act[c >> 5] |= 1u << (c & 31);
}

// Pull (bottom-up) discovery fused with the path-count sum, iteration `it`
// (frontier = level it, new vertices get level it + 1).
template <int K, bool EXT>
__device__ void phase_pull(const KParams& p, int it, int ph, const uint32_t (&act)[Cfg<K>::W], AppendBuf& ab,
                           HeavySmem<Cfg<K>::W>& hs) {
    constexpr int W = Cfg<K>::W;
    const int lane = lane_id();
    const uint32_t* Fc = p.F[it % 3];
    uint32_t* Fn = p.F[(it + 1) % 3];
    const int lev = it + 1;
    bool carry = false;
    phase_prologue(p, ph);
    // heavy rows: whole blocks
    for (;;) {
        int w = block_grab(wq_heavy(p, ph), p.n_heavy);
        if (w < 0) break;
        uint32_t vm[W], um[W];
        load_mask<W>(p.V, w, vm);
#pragma unroll
        for (int t = 0; t < W; ++t) um[t] = act[t] & ~vm[t];
        if (!mask_any<W>(um)) continue;
        Acc<W, EXT, FWD> tot;
        uint32_t nm[W];
#pragma unroll
        for (int t = 0; t < W; ++t) nm[t] = 0;
        block_row<K, W, EXT, FWD>(p, p.off[w], p.off[w + 1], Fc, um, tot, nm, carry, hs);
        if (mask_any<W>(nm) && warp_id() == 0) {
            store_mask<W>(Fn, w, nm);
            fwd_finish<K, W, EXT>(p, w, nm, lev, act, tot);
            if (lane == 0) heavy_append(p, lev, w, p.off[w + 1] - p.off[w]);
        }
    }
    // light rows: one warp each
    int acnt = 0;
    const long long nlight = (long long)p.n_nz - p.n_heavy;
    for (;;) {
        int cnt;
        long long i0 = warp_grab(wq_light(p, ph), nlight, 32, cnt);
        if (i0 < 0) break;
        for (int q = 0; q < cnt; ++q) {
            const int w = p.n_heavy + (int)(i0 + q);
            uint32_t vm[W], um[W];
            load_mask<W>(p.V, w, vm);
#pragma unroll
            for (int t = 0; t < W; ++t) um[t] = act[t] & ~vm[t];
            if (!mask_any<W>(um)) continue;
            Acc<W, EXT, FWD> tot;
            uint32_t nm[W];
#pragma unroll
            for (int t = 0; t < W; ++t) nm[t] = 0;
            warp_row<K, W, EXT, FWD>(p, p.off[w], p.off[w + 1], Fc, um, tot, nm, carry);
            warp_or_reduce<W>(nm);
            if (mask_any<W>(nm)) {
                store_mask<W>(Fn, w, nm);
                fwd_finish<K, W, EXT>(p, w, nm, lev, act, tot);
                warp_append(p, lev, w, p.off[w + 1] - p.off[w], ab, acnt);
            }
        }
    }
    flush_append(p, lev, ab, acnt);
    if (__any_sync(FULL_MASK, carry) && lane_id() == 0) atomicOr(&p.ctl->flags, BST_NEED_EXT);
    if (it >= 1) clear_level_masks<W>(p, p.F[(it + 2) % 3], it - 1);
}

// Push (top-down) discovery over the frontier entries of level `it`.
template <int K>
__device__ void phase_push(const KParams& p, int it, int ph, const uint32_t (&act)[Cfg<K>::W]) {
    constexpr int W = Cfg<K>::W;
    const int lane = lane_id();
    const uint32_t* Fc = p.F[it % 3];
    uint32_t* Fn = p.F[(it + 1) % 3];
    const int lev = it + 1;
    const int stampv = lev;
    phase_prologue(p, ph);
    auto visit = [&](int v, long long e0, long long e1, long long step) {
        uint32_t fm[W];
        load_mask<W>(Fc, v, fm);
        for (long long base = e0; base < e1; base += step) {
            const long long e = base + lane;
            bool light_claim = false, heavy_claim = false;
            int w = 0;
            long long deg = 0;
            if (e < e1) {
                w = __ldg(p.adj + e);
                uint32_t vw[W], nb[W];
                load_mask<W>(p.V, w, vw);
                bool any = false;
#pragma unroll
                for (int t = 0; t < W; ++t) { nb[t] = fm[t] & ~vw[t]; any |= nb[t] != 0; }
                if (any) {
#pragma unroll
                    for (int t = 0; t < W; ++t)
                        if (nb[t]) atomicOr(&Fn[(size_t)w * W + t], nb[t]);
                    if (*(volatile int*)&p.stamp[w] != stampv && atomicExch(&p.stamp[w], stampv) != stampv) {
                        deg = p.off[w + 1] - p.off[w];
                        if (w < p.n_heavy) heavy_claim = true;
                        else light_claim = true;
                    }
                }
            }
            const unsigned int lb = __ballot_sync(FULL_MASK, light_claim);
            if (lb) {
                long long ds = light_claim ? deg : 0;
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) ds += __shfl_xor_sync(FULL_MASK, ds, o);
                int base0 = 0;
                const int leader = __ffs(lb) - 1;
                if (lane == leader) {
                    base0 = atomicAdd(&p.la.cnt[lev], __popc(lb));
                    atomicAdd((unsigned long long*)&p.la.dsum[lev], (unsigned long long)ds);
                }
                base0 = __shfl_sync(FULL_MASK, base0, leader);
                if (light_claim) {
                    const long long pos = (long long)p.la.start[lev] + base0 + __popc(lb & ((1u << lane) - 1u));
                    if (pos < p.cap) p.ent[pos] = w;
                    else atomicOr(&p.ctl->err, ERR_CAPACITY);
                }
            }
            if (heavy_claim) heavy_append(p, lev, w, deg);
        }
    };
    // heavy frontier rows: whole blocks, warps interleaved over the row
    const int hs = p.la.hstart[it], hc = p.la.hcnt[it];
    for (;;) {
        int i = block_grab(wq_heavy(p, ph), hc);
        if (i < 0) break;
        const int v = p.hent[hs + i];
        visit(v, (long long)p.off[v] + warp_id() * 32, p.off[v + 1], (long long)kThreads);
    }
    const int ls = p.la.start[it], lc = p.la.cnt[it];
    for (;;) {
        int cnt;
        long long i0 = warp_grab(wq_light(p, ph), lc, 4, cnt);
        if (i0 < 0) break;
        for (int q = 0; q < cnt; ++q) {
            const int v = p.ent[ls + i0 + q];
            visit(v, p.off[v], p.off[v + 1], 32);
        }
    }
    (void)act;
}

// Path counts of the vertices claimed by the push phase (entries of level it+1).
template <int K, bool EXT>
__device__ void phase_sigma(const KParams& p, int it, int ph, const uint32_t (&act)[Cfg<K>::W],
                            HeavySmem<Cfg<K>::W>& hs) {
    constexpr int W = Cfg<K>::W;
    const uint32_t* Fc = p.F[it % 3];
    const uint32_t* Fn = p.F[(it + 1) % 3];
    const int lev = it + 1;
    bool carry = false;
    phase_prologue(p, ph);
    const int hst = p.la.hstart[lev], hc = p.la.hcnt[lev];
    for (;;) {
        int i = block_grab(wq_heavy(p, ph), hc);
        if (i < 0) break;
        const int w = p.hent[hst + i];
        uint32_t nm[W], orm[W];
        load_mask<W>(Fn, w, nm);
#pragma unroll
        for (int t = 0; t < W; ++t) orm[t] = 0;
        Acc<W, EXT, FWD> tot;
        block_row<K, W, EXT, FWD>(p, p.off[w], p.off[w + 1], Fc, nm, tot, orm, carry, hs);
        if (warp_id() == 0) fwd_finish<K, W, EXT>(p, w, nm, lev, act, tot);
    }
    const int ls = p.la.start[lev], lc = p.la.cnt[lev];
    for (;;) {
        int cnt;
        long long i0 = warp_grab(wq_light(p, ph), lc, 4, cnt);
        if (i0 < 0) break;
        for (int q = 0; q < cnt; ++q) {
            const int w = p.ent[ls + i0 + q];
            uint32_t nm[W], orm[W];
            load_mask<W>(Fn, w, nm);
#pragma unroll
            for (int t = 0; t < W; ++t) orm[t] = 0;
            Acc<W, EXT, FWD> tot;
            warp_row<K, W, EXT, FWD>(p, p.off[w], p.off[w + 1], Fc, nm, tot, orm, carry);
            fwd_finish<K, W, EXT>(p, w, nm, lev, act, tot);
        }
    }
    if (__any_sync(FULL_MASK, carry) && lane_id() == 0) atomicOr(&p.ctl->flags, BST_NEED_EXT);
    if (it >= 1) clear_level_masks<W>(p, p.F[(it + 2) % 3], it - 1);
}

// Reverse sweep over level l: delta and rho of its entries from level l+1.
template <int K, bool EXT>
__device__ void phase_back(const KParams& p, int l, int ph, HeavySmem<Cfg<K>::W>& hs) {
    constexpr int W = Cfg<K>::W;
    const uint32_t* Fd = p.F[(l + 1) % 3];  // level l+1 masks
    uint32_t* Fl = p.F[l % 3];              // level l masks (written for level l-1)
    bool carry = false;
    phase_prologue(p, ph);
    const int hst = p.la.hstart[l], hc = p.la.hcnt[l];
    for (;;) {
        int i = block_grab(wq_heavy(p, ph), hc);
        if (i < 0) break;
        const int v = p.hent[hst + i];
        uint32_t mk[W], orm[W];
        level_mask<K, W>(p, v, l, mk);
#pragma unroll
        for (int t = 0; t < W; ++t) orm[t] = 0;
        Acc<W, EXT, BWD> tot;
        block_row<K, W, EXT, BWD>(p, p.off[v], p.off[v + 1], Fd, mk, tot, orm, carry, hs);
        if (warp_id() == 0) {
            bwd_finish<K, W, EXT>(p, v, mk, tot);
            store_mask<W>(Fl, v, mk);
        }
    }
    const int ls = p.la.start[l], lc = p.la.cnt[l];
    for (;;) {
        int cnt;
        long long i0 = warp_grab(wq_light(p, ph), lc, 4, cnt);
        if (i0 < 0) break;
        for (int q = 0; q < cnt; ++q) {
            const int v = p.ent[ls + i0 + q];
            uint32_t mk[W], orm[W];
            level_mask<K, W>(p, v, l, mk);
#pragma unroll
            for (int t = 0; t < W; ++t) orm[t] = 0;
            Acc<W, EXT, BWD> tot;
            warp_row<K, W, EXT, BWD>(p, p.off[v], p.off[v + 1], Fd, mk, tot, orm, carry);
            bwd_finish<K, W, EXT>(p, v, mk, tot);
            store_mask<W>(Fl, v, mk);
        }
    }
    clear_level_masks<W>(p, p.F[(l + 2) % 3], l + 2);
}

// BC[v] += delta of every reached, non-source column, in column order.  Each
// column belongs to a job (col_job; all job 0 when absent) whose columns are
// contiguous; a job's sum is carried sequentially across its columns and its
// batches, so the additions happen in the job's source-list order whatever
// else shares the batch.
template <int K>
__device__ void phase_bc(const KParams& p, int b) {
    constexpr int W = Cfg<K>::W;
    const long long nthr = (long long)gridDim.x * blockDim.x;
    const int* src = p.src + (size_t)b * K;
    const int* cj = p.col_job ? p.col_job + (size_t)b * K : nullptr;
    for (long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x; v < p.n_nz; v += nthr) {
        uint32_t vm[W];
        load_mask<W>(p.V, (int)v, vm);
        if (!mask_any<W>(vm)) continue;
        int cur = -1;
        double acc = 0.0;
        for (int c = 0; c < K; ++c) {
            if (!((vm[c >> 5] >> (c & 31)) & 1u)) continue;
            const int s = __ldg(src + c);
            if (s == (int)v) continue;
            const int j = cj ? __ldg(cj + c) : 0;
            if (j != cur) {
                if (cur >= 0) p.job_bc[cur][v] = acc;
                cur = j;
                acc = p.job_bc[j][v];
            }
            acc += __longlong_as_double((long long)p.sig[(size_t)v * K + c]);
        }
        if (cur >= 0) p.job_bc[cur][v] = acc;
    }
}

// ------------------------------------------------------------------ one batch
template <int K, bool EXT>
__device__ bool run_batch(const KParams& p, int b, GridTeam& team, int& ph, AppendBuf& ab,
                          HeavySmem<Cfg<K>::W>& hs) {
    constexpr int W = Cfg<K>::W;
    const long long nthr = (long long)gridDim.x * blockDim.x;
    const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    uint32_t act[W];
    active_mask<K>(p, b, act);

    // init A: clear masks and stamps, zero the first level slots and the batch flags
    for (long long i = tid; i < (long long)p.n * W; i += nthr) {
        p.V[i] = 0; p.F[0][i] = 0; p.F[1][i] = 0; p.F[2][i] = 0;
    }
    for (long long i = tid; i < p.n; i += nthr) p.stamp[i] = -1;
    if (tid < 3) {
        p.la.cnt[tid] = 0; p.la.hcnt[tid] = 0; p.la.dsum[tid] = 0; p.la.fulldeg[tid] = 0;
    }
    if (tid == 0) { p.ctl->flags = 0; p.la.start[0] = 0; p.la.hstart[0] = 0; }
    if (!team.sync()) return false;
    // init B: sources (block 0): level 0 entries, unique vertices
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        const int* src = p.src + (size_t)b * K;
        for (int c = 0; c < K; ++c) {
            const int s = src[c];
            if (s < 0) continue;
            const uint32_t bit = 1u << (c & 31);
            p.V[(size_t)s * W + (c >> 5)] |= bit;
            p.F[0][(size_t)s * W + (c >> 5)] |= bit;
            p.sig[(size_t)s * K + c] = 1ull;
            if (EXT) p.sig_e[(size_t)s * K + c] = 0;
            p.lvl[(size_t)s * K + c] = 0;
            bool first = true;
            for (int c2 = 0; c2 < c; ++c2)
                if (src[c2] == s) { first = false; break; }
            if (!first) continue;
            const long long deg = p.off[s + 1] - p.off[s];
            if (s < p.n_heavy) { p.hent[p.la.hcnt[0]++] = s; }
            else { p.ent[p.la.cnt[0]++] = s; }
            p.la.dsum[0] += deg;
        }
    }
    if (!team.sync()) return false;

    // forward sweep
    long long full_arcs = 0;
    bool pull = false;
    int it = 0;
    for (;; ++it) {
        const int nf = p.la.cnt[it] + p.la.hcnt[it];
        if (nf == 0) break;
        if (it + 1 > kMaxLevel) {
            if (tid == 0) atomicOr(&p.ctl->err, ERR_LIMIT);
            return false;
        }
        full_arcs += p.la.fulldeg[it];
        const long long mf = p.la.dsum[it];
        const long long mu = p.m_nz - full_arcs;
        if (p.direction == 1) pull = false;
        else if (p.direction == 2) pull = true;
        else if (!pull) pull = (double)mf * p.alpha > (double)mu;
        else pull = !((double)nf * p.beta < (double)p.n_nz && (double)mf * p.alpha < (double)mu);
        // next level's start offsets: every block writes the same values itself, so
        // its own warps (ordered by the phase's first __syncthreads) read them
        // without a grid barrier; counters two levels ahead are cleared here.
        if (threadIdx.x == 0) {
            p.la.start[it + 1] = p.la.start[it] + p.la.cnt[it];
            p.la.hstart[it + 1] = p.la.hstart[it] + p.la.hcnt[it];
        }
        if (tid == 0) {
            if (pull) p.ctl->pull_levels++;
            else p.ctl->push_levels++;
        }
        if (tid == 1 && it + 2 < kLevelSlots) {
            p.la.cnt[it + 2] = 0; p.la.hcnt[it + 2] = 0; p.la.dsum[it + 2] = 0; p.la.fulldeg[it + 2] = 0;
        }
        if (pull) {
            phase_pull<K, EXT>(p, it, ph++, act, ab, hs);
        } else {
            phase_push<K>(p, it, ph++, act);
            if (!team.sync()) return false;
            phase_sigma<K, EXT>(p, it, ph++, act, hs);
        }
        if (!team.sync()) return false;
        if (*(volatile int*)&p.ctl->flags & BST_NEED_EXT) break;
    }
    const int L = it - 1;  // deepest nonempty level
    if (!EXT && (*(volatile int*)&p.ctl->flags & BST_NEED_EXT)) {
        if (tid == 0) p.batch_status[b] = BST_NEED_EXT;
        return team.sync();
    }
    if (tid == 0 && L + 1 > p.ctl->max_levels) p.ctl->max_levels = L + 1;
    if (p.forward_only) {
        if (tid == 0) p.batch_status[b] = BST_DONE | (p.ctl->flags & BST_INEXACT);
        return team.sync();
    }
    // the forward sweep leaves buffer L%3 = level L masks, the others zero
    for (int l = L; l >= 1; --l) {
        phase_back<K, EXT>(p, l, ph++, hs);
        if (!team.sync()) return false;
    }
    phase_bc<K>(p, b);
    if (tid == 0) p.batch_status[b] = BST_DONE | (p.ctl->flags & BST_INEXACT);
    return team.sync();
}

template <int K>
__global__ void __launch_bounds__(kThreads) bc_persistent(KParams p) {
    __shared__ AppendBuf ab;
    __shared__ HeavySmem<Cfg<K>::W> hs;
    if (threadIdx.x < kWarps) ab.dsum[threadIdx.x] = 0;
    __syncthreads();
    GridTeam team{p.ctl, p.budget};
    int ph = 0;
    for (int b = 0; b < p.nbatch; ++b) {
        bool ok = p.ext ? run_batch<K, true>(p, b, team, ph, ab, hs) : run_batch<K, false>(p, b, team, ph, ab, hs);
        if (!ok) return;
    }
}

// ------------------------------------------------------------------ small kernels
__global__ void k_unpermute(const double* __restrict__ bc_rel, const int* __restrict__ inv, double* out, int n) {
    int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v < n) out[v] = bc_rel[inv[v]];
}

__global__ void k_map_sources(const int* __restrict__ src, int nsrc, const int* __restrict__ inv, int n, int K,
                              int* dst, int total, int* bad) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= total) return;
    if (i < nsrc) {
        int s = src[i];
        if (s < 0 || s >= n) { atomicOr(bad, 1); dst[i] = -1; }
        else dst[i] = inv[s];
    } else {
        dst[i] = -1;
    }
}

__global__ void k_debug_extract(KParams p, int K, int* level_rel, unsigned long long* sig_rel, int* sige_rel) {
    int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= p.n) return;
    const int W = K >= 32 ? K / 32 : 1;
    bool reached = (p.V[(size_t)v * W] & 1u) != 0;
    level_rel[v] = reached ? (int)p.lvl[(size_t)v * K] : -1;
    sig_rel[v] = reached ? p.sig[(size_t)v * K] : 0ull;
    sige_rel[v] = (reached && p.ext) ? p.sig_e[(size_t)v * K] : 0;
}

// ------------------------------------------------------------------ host launchers
template <int K>
static cudaError_t launch_k(const KParams& p, int blocks, cudaStream_t st) {
    KParams q = p;
    void* args[] = {&q};
    return cudaLaunchCooperativeKernel((const void*)bc_persistent<K>, dim3(blocks), dim3(kThreads), args, 0, st);
}

cudaError_t launch_batches(int K, const KParams& p, int blocks, cudaStream_t st) {
    switch (K) {
        case 1: return launch_k<1>(p, blocks, st);
        case 32: return launch_k<32>(p, blocks, st);
        case 64: return launch_k<64>(p, blocks, st);
        case 128: return launch_k<128>(p, blocks, st);
        default: return cudaErrorInvalidValue;
    }
}

template <int K>
static int occ() {
    int nb = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, bc_persistent<K>, kThreads, 0);
    return nb;
}

int max_coop_blocks(int K, int* per_sm) {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    int nb = 0;
    switch (K) {
        case 1: nb = occ<1>(); break;
        case 32: nb = occ<32>(); break;
        case 64: nb = occ<64>(); break;
        case 128: nb = occ<128>(); break;
    }
    if (per_sm) *per_sm = nb;
    return nb * sms;
}

cudaError_t launch_unpermute(const double* bc_rel, const int* inv, double* out, int n, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    k_unpermute<<<(n + 255) / 256, 256, 0, st>>>(bc_rel, inv, out, n);
    return cudaGetLastError();
}

cudaError_t launch_map_sources(const int* src_orig, int nsrc, const int* inv, int n, int K, int* dst, int nbatch,
                               int* bad, cudaStream_t st) {
    int total = nbatch * K;
    if (total <= 0) return cudaSuccess;
    k_map_sources<<<(total + 255) / 256, 256, 0, st>>>(src_orig, nsrc, inv, n, K, dst, total, bad);
    return cudaGetLastError();
}

cudaError_t launch_debug_extract(const KParams& p, int K, int* level_rel, unsigned long long* sig_rel, int* sige_rel,
                                 cudaStream_t st) {
    if (p.n <= 0) return cudaSuccess;
    k_debug_extract<<<(p.n + 255) / 256, 256, 0, st>>>(p, K, level_rel, sig_rel, sige_rel);
    return cudaGetLastError();
}

}  // namespace bcx
