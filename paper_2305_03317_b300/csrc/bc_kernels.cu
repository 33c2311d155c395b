// Batched Brandes betweenness centrality: the persistent sm_103a kernel.
//
// One cooperative launch runs every batch of a bc_compute call.  A batch is
// K sources (K = 1, 32, 64 or 128) traversed together: column c of every
// per-vertex array belongs to source c of the batch, and all columns advance
// one BFS level per iteration (the paper's iterateInBFS, Section 2.3.2, run for
// K roots at once).  Per iteration:
//   * discovery, either top-down (push: frontier rows claim unseen neighbours
//     with atomicOr on their column masks, warp-aggregated list appends) or
//     bottom-up (pull: every not-yet-complete vertex scans its row against the
//     frontier masks), switched by frontier size;
//   * the path-count sum sigma_c(w) = sum of sigma_c(v) over frontier
//     neighbours v (the BFS body w.sigma += v.sigma of the BC listing), pulled
//     over each new vertex's row: no atomics.
// The reverse sweep (iterateInReverse) walks the kept level lists (vertex id
// and column mask per entry) from the deepest level up, pulling
// rho_c(w) = (1 + delta_c(w)) / sigma_c(w) from DAG successors:
//     delta_c(v) = sigma_c(v) * sum_w rho_c(w).
// This equals the listing's per-arc (sigma_v / sigma_w)(1 + delta_w) summed
// over w, with one division per vertex and column instead of one per arc.
// Finally each vertex adds its columns' delta into BC (source columns
// excluded) in column order.
//
// Work decomposition (uniform units, no block-level phases):
//   * rows of degree <= 1024 ("light") are handled up to 32 vertices per warp
//     task; the warp enumerates the concatenated arcs of its rows 32 at a time
//     (load-balanced: every lane holds one arc), then walks the matching arcs
//     in CSR order with lanes mapped to columns (lane l owns columns
//     [W*l, W*l+W), W = K/32) so that a neighbour's per-column values are one
//     coalesced row read.  With K == 1 lanes load their own arc's value and
//     the values are added in lane order.
//   * rows of degree > 1024 ("heavy", a prefix of the degree-sorted ids) are
//     cut into 1024-arc chunk tasks.  Each chunk's partial sum goes to a
//     scratch slot; the warp that completes the last chunk combines the
//     partials in chunk order and finishes the vertex.
// Every floating-point sum therefore runs in CSR order within fixed 1024-arc
// chunks, chunks combined in order: each column's arithmetic is independent
// of K, of the other columns, of the grouping and of the push/pull choice, so
// results are bitwise reproducible across all of them.
//
// Grid-wide phases are separated by a software barrier whose wait is bounded
// by a cycle budget; on expiry it raises ERR_TIMEOUT and every block returns.
#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

#include "bc_internal.cuh"

namespace bcx {

#define FULL_MASK 0xffffffffu

__device__ __forceinline__ int lane_id() { return threadIdx.x & 31; }
__device__ __forceinline__ int warp_id() { return threadIdx.x >> 5; }

// Phase trace: block 0 stamps the end of every grid-wide phase (after its barrier).
__device__ __forceinline__ void trace_mark(const KParams& p, int kind, int level) {
    if (p.trace == nullptr || p.team != 0 || p.rank != 0 || threadIdx.x != 0) return;
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    const int i = p.gctl->trace_n;
    if (i < p.trace_cap) {
        p.trace[2 * i] = ((long long)kind << 24) | (long long)(level & 0xFFFFFF);
        p.trace[2 * i + 1] = (long long)t;
        p.gctl->trace_n = i + 1;
    }
}

// Work distribution inside a phase: a warp's first task is its global warp
// index (no atomics while tasks are fewer than warps); later tasks come from a
// per-phase counter.  Returns -1 when the phase has no task left for the warp.
__device__ __forceinline__ long long next_task(const KParams& p, unsigned int* ctr, long long total, bool& first) {
    const long long nw = ((long long)p.team_blocks * blockDim.x) >> 5;
    long long t;
    if (first) {
        first = false;
        t = (((long long)p.rank * blockDim.x) + threadIdx.x) >> 5;
    } else {
        if (total <= nw) return -1;
        unsigned int i = 0;
        if (lane_id() == 0) i = atomicAdd(ctr, 1u);
        t = nw + (long long)__shfl_sync(FULL_MASK, i, 0);
    }
    return t < total ? t : -1;
}

// ------------------------------------------------------------------ masks
template <int W>
__device__ __forceinline__ void load_mask(const uint32_t* base, long long idx, uint32_t (&m)[W]) {
    const uint32_t* p = base + (size_t)idx * W;
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
__device__ __forceinline__ void store_mask_full(uint32_t* base, long long idx, const uint32_t (&m)[W]) {
    uint32_t* p = base + (size_t)idx * W;
    if constexpr (W == 1) {
        p[0] = m[0];
    } else if constexpr (W == 2) {
        *reinterpret_cast<uint2*>(p) = make_uint2(m[0], m[1]);
    } else {
        *reinterpret_cast<uint4*>(p) = make_uint4(m[0], m[1], m[2], m[3]);
    }
}

template <int W>
__device__ __forceinline__ bool mask_any(const uint32_t (&m)[W]) {
    uint32_t a = 0;
#pragma unroll
    for (int t = 0; t < W; ++t) a |= m[t];
    return a != 0;
}

// bits of column group [W*lane, W*lane+W) from word `word` of a mask
template <int W>
__device__ __forceinline__ uint32_t lane_field(uint32_t word, int lane) {
    return (word >> ((W * lane) & 31)) & ((1u << W) - 1u);
}

// W consecutive 8-byte terms (16-byte aligned when W >= 2)
template <int W>
__device__ __forceinline__ void load_terms(const unsigned long long* p, unsigned long long (&x)[W]) {
    if constexpr (W == 1) {
        x[0] = p[0];
    } else {
#pragma unroll
        for (int i = 0; i < W; i += 2) {
            const ulonglong2 y = *reinterpret_cast<const ulonglong2*>(p + i);
            x[i] = y.x;
            x[i + 1] = y.y;
        }
    }
}

template <int W>
__device__ __forceinline__ void store_terms(unsigned long long* p, const unsigned long long (&x)[W]) {
    if constexpr (W == 1) {
        p[0] = x[0];
    } else {
#pragma unroll
        for (int i = 0; i < W; i += 2) *reinterpret_cast<ulonglong2*>(p + i) = make_ulonglong2(x[i], x[i + 1]);
    }
}

template <int W>
__device__ __forceinline__ uint32_t pick(const uint32_t (&m)[W], int t) {
    uint32_t x = m[0];
#pragma unroll
    for (int i = 1; i < W; ++i)
        if (i == t) x = m[i];
    return x;
}

// ------------------------------------------------------------------ accumulation
// A running sum per (owner, column): FWD path counts (u64, or 64-bit mantissa
// with exponent), BWD sums of rho (double bits, or double with exponent).
enum { FWD = 0, BWD = 1 };

template <bool EXT, int DIR>
__device__ __forceinline__ void acc_add(unsigned long long& v, int& e, unsigned long long x, int xe, bool& carry) {
    if constexpr (DIR == FWD) {
        if constexpr (EXT) {
            xu_add(v, e, x, xe);
        } else {
            const unsigned long long s = v + x;
            carry |= (s < x);
            v = s;
        }
    } else {
        double r = __longlong_as_double((long long)v);
        if constexpr (EXT) xd_add(r, e, __longlong_as_double((long long)x), xe);
        else r += __longlong_as_double((long long)x);
        v = (unsigned long long)__double_as_longlong(r);
    }
}

// ------------------------------------------------------------------ per-warp shared state
template <int K>
struct Geo {
    static constexpr int W = K >= 32 ? K / 32 : 1;
    // owners per light task: the per-owner accumulator rows use G*K <= 512 slots
    static constexpr int G = K == 1 ? 32 : (K == 32 ? 16 : (K == 64 ? 8 : 4));
    static constexpr int PCAP = 512;  // (arc, column) pairs expanded per window
};

// 16-byte aligned so that every warp's copy (consecutive in dynamic shared
// memory) keeps its accumulator rows aligned for 16-byte vector accesses.
template <int K, bool EXT>
struct __align__(16) WarpSmem {
    static constexpr int W = Geo<K>::W, G = Geo<K>::G;
    int ov[G];                    // owner vertex
    int obeg[G];                  // first arc index (into adj) of the owner's range
    int ostart[G];                // exclusive prefix of range lengths
    int opos[G];                  // entry position of the owner (lists) or -1
    uint32_t owant[G][W];         // columns of interest of the owner
    uint32_t onm[G][W];           // OR of the owner's matched columns
    unsigned long long acc[G * K];  // running sums, owner-major
    int acce[EXT ? G * K : 1];    // exponents (extended form)
    int sv[32];                   // neighbour of each arc of the current step
    int so[32];                   // owner of each arc of the current step
    uint32_t fw[32][W];           // matched columns of each arc of the step; slot tags in the rounds
    alignas(16) uint32_t pr[Geo<K>::PCAP];  // expanded pairs: arc << 16 | column; during the
                                            // column-mapped arcs, a ring of two staged rows
    int av[32];                   // append staging (pull): vertex
    uint32_t am[32][W];           // append staging: mask
    long long adeg;               // append staging: degree sum
    unsigned long long cnt_dag;   // this warp's forward sum terms (DAG arc, column), flushed at exit
    unsigned long long cnt_reached;  // this warp's reached (vertex, column) pairs, flushed at exit
    alignas(8) unsigned long long mbar[2];  // completion barriers of the two staged-row slots
    uint32_t mph;                 // their phase bits (bit s: parity of slot s's next completion)
    int berr;                     // a staged-row wait gave up (reported as an internal error)
};

using WS128 = WarpSmem<128, false>;
using WS64 = WarpSmem<64, false>;
using WS32 = WarpSmem<32, false>;
static_assert(sizeof(WS128) % 16 == 0 && offsetof(WS128, acc) % 16 == 0 && sizeof(WS64) % 16 == 0 &&
              offsetof(WS64, acc) % 16 == 0 && sizeof(WS32) % 16 == 0 && offsetof(WS32, acc) % 16 == 0,
              "accumulator rows need 16-byte alignment");

// Fill the owner table (lane i describes owner i < ng) and return the arc total.
template <int K, bool EXT>
__device__ __forceinline__ int set_owners(WarpSmem<K, EXT>& ws, int ng, int v, int beg, int len, int pos,
                                          const uint32_t (&want)[Geo<K>::W]) {
    constexpr int W = Geo<K>::W;
    const int lane = lane_id();
    int incl = len;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(FULL_MASK, incl, o);
        if (lane >= o) incl += y;
    }
    __syncwarp();
    if (lane < ng) {
        ws.ov[lane] = v;
        ws.obeg[lane] = beg;
        ws.ostart[lane] = incl - len;
        ws.opos[lane] = pos;
#pragma unroll
        for (int t = 0; t < W; ++t) ws.owant[lane][t] = want[t];
    }
    __syncwarp();
    return __shfl_sync(FULL_MASK, incl, 31);
}

// ------------------------------------------------------------------ column-mapped arcs
// The arcs of bit set `db` (indices into the current step, taken in increasing
// order, i.e. CSR order) are summed with lanes mapped to columns: lane l adds
// the terms of its columns [W*l, W*l+W) that the arc matches, reading them as
// one vector load, into its own accumulator slots.  No two lanes share a slot,
// so no atomics and no ordering rounds are needed.  Each lane's slots take
// the arcs in order, so ordered (floating-point) sums stay in CSR order.
//
// The neighbours' rows (K terms, 8 bytes each) are staged in shared memory by
// 1-D bulk asynchronous copies (cp.async.bulk, completion on an mbarrier),
// one instruction of one lane per row, into a ring of two slots in the pair
// buffer, which is idle until the step's pairs are expanded: one row is
// added while the next is in flight.  Rows are 16-byte aligned (their arrays
// start on 256-byte boundaries and a row is 8K bytes).
template <int K, bool EXT, int DIR>
__device__ __forceinline__ void dense_arcs(WarpSmem<K, EXT>& ws, unsigned int db,
                                           const unsigned long long* __restrict__ termv, bool& carry) {
    constexpr int W = Geo<K>::W;
    constexpr unsigned ROW = K * 8;
    static_assert(K >= 32 && !EXT, "column-mapped arcs need K >= 32 and the plain form");
    static_assert(2 * ROW <= sizeof(ws.pr), "two rows fit the pair buffer");
    const int lane = lane_id();
    const int word = (W * lane) >> 5;
    unsigned int di = db;
    unsigned char* ring = reinterpret_cast<unsigned char*>(ws.pr);
    unsigned ph = ws.mph;
    // stage the next arc's row (CSR order) into slot s
    auto issue = [&](int s) {
        if (!di) return;
        const int j = __ffs(di) - 1;
        di &= di - 1;
        if (lane == 0) {
            const unsigned long long* src = termv + (size_t)ws.sv[j] * K;
            const unsigned mb = (unsigned)__cvta_generic_to_shared(&ws.mbar[s]);
            const unsigned dst = (unsigned)__cvta_generic_to_shared(ring + s * ROW);
            // the warp's reads of the slot's previous row (generic proxy) before the
            // copy overwrites it (the rows' own writes are ordered by the phase prologue)
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" :: "r"(mb), "r"(ROW) : "memory");
            asm volatile("cp.async.bulk.shared::cta.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                         :: "r"(dst), "l"(src), "r"(ROW), "r"(mb) : "memory");
        }
    };
    issue(0);
    issue(1);
    int cur = -1, s = 0;
    unsigned long long r[W];
#pragma unroll
    for (int i = 0; i < W; ++i) r[i] = 0ull;
    while (db) {
        const int j = __ffs(db) - 1;
        db &= db - 1;
        {  // wait (bounded) for slot s's row
            const unsigned mb = (unsigned)__cvta_generic_to_shared(&ws.mbar[s]);
            const unsigned par = (ph >> s) & 1u;
            bool ok = false;
            for (int it = 0; it < (1 << 22) && !ok; ++it) {
                unsigned done;
                asm volatile("{ .reg .pred q; mbarrier.try_wait.parity.shared::cta.b64 q, [%1], %2; selp.u32 %0, 1, 0, q; }"
                             : "=r"(done) : "r"(mb), "r"(par) : "memory");
                ok = done != 0;
            }
            if (!ok && lane == 0) ws.berr = 1;
            ph ^= 1u << s;
        }
        const uint32_t b = lane_field<W>(ws.fw[j][word], lane);
        unsigned long long xa[W];
        if (b) {
            load_terms<W>(reinterpret_cast<const unsigned long long*>(ring + s * ROW) + W * lane, xa);
        } else {
#pragma unroll
            for (int i = 0; i < W; ++i) xa[i] = 0ull;
        }
        const int o = ws.so[j];
        if (o != cur) {
            if (cur >= 0) store_terms<W>(&ws.acc[cur * K + W * lane], r);
            load_terms<W>(&ws.acc[o * K + W * lane], r);
            cur = o;
        }
        int e = 0;
#pragma unroll
        for (int i = 0; i < W; ++i)
            if ((b >> i) & 1u) acc_add<false, DIR>(r[i], e, xa[i], 0, carry);
        __syncwarp();  // every lane has read slot s: it takes the row after next
        issue(s);
        s ^= 1;
    }
    if (cur >= 0) store_terms<W>(&ws.acc[cur * K + W * lane], r);
    if (lane == 0) ws.mph = ph;
    __syncwarp();
}

// One 32-arc step of group_gather: arc `lane` of the step has owner o,
// neighbour v and matched columns f (n of them).
template <int K, bool EXT, int DIR>
__device__ __forceinline__ void gather_step(const KParams& p, WarpSmem<K, EXT>& ws, int o, int v, int n,
                                            uint32_t (&f)[Geo<K>::W], const unsigned long long* termv,
                                            const int* terme, bool& carry) {
    constexpr int W = Geo<K>::W;
    constexpr int PCAP = Geo<K>::PCAP;
    constexpr bool ORDERED = EXT || DIR == BWD;
    const int lane = lane_id();
    if constexpr (DIR == FWD) {
        // every matched (arc, column) of a forward sum is a DAG arc of that column's source
        const unsigned int terms = __reduce_add_sync(FULL_MASK, (unsigned int)n);
        if (lane == 0) ws.cnt_dag += terms;
    }
    if (!__any_sync(FULL_MASK, n > 0)) return;
    if (n > 0) {
#pragma unroll
        for (int t = 0; t < W; ++t)
            if (f[t]) atomicOr(&ws.onm[o][t], f[t]);
    }
    ws.sv[lane] = v;
    ws.so[lane] = o;
    if constexpr (K >= 32 && !EXT) {
        // arcs matching many columns go column-mapped.  Integer path counts
        // split per arc; ordered sums take the whole step one way (every
        // slot then still adds in CSR order).
        bool dn;
        if constexpr (DIR == FWD) {
            dn = n >= p.dense_min;
        } else {
            int tot = n;
#pragma unroll
            for (int s = 16; s > 0; s >>= 1) tot += __shfl_xor_sync(FULL_MASK, tot, s);
            const int arcs = __popc(__ballot_sync(FULL_MASK, n > 0));
            dn = n > 0 && tot >= arcs * p.dense_min;
        }
        const unsigned int db = __ballot_sync(FULL_MASK, dn);
        if (db) {
#pragma unroll
            for (int t = 0; t < W; ++t) ws.fw[lane][t] = f[t];
            __syncwarp();
            dense_arcs<K, EXT, DIR>(ws, db, termv, carry);
            if (dn) n = 0;
            if (!__any_sync(FULL_MASK, n > 0)) return;
        }
    }
    int incl = n;
#pragma unroll
    for (int s = 1; s < 32; s <<= 1) {
        int y = __shfl_up_sync(FULL_MASK, incl, s);
        if (lane >= s) incl += y;
    }
    const int P = incl - n;
    const int tot = __shfl_sync(FULL_MASK, incl, 31);
    __syncwarp();
    int j0 = 0, pb = 0;
    while (pb < tot) {
        // window: the arcs from j0 whose pairs fit in the buffer (always >= 1 arc)
        const unsigned int inwin = __ballot_sync(FULL_MASK, lane >= j0 && incl - pb <= PCAP);
        const int j1 = 32 - __clz(inwin);
        const int pe = __shfl_sync(FULL_MASK, incl, j1 - 1);
        // expansion: arcs with few pairs write their own (one lane, serially:
        // cost = the largest such count); arcs with many can be written by the
        // whole warp, lanes mapped to the bits of each mask word (cost = W per
        // arc).  The split threshold is the cheapest of a few candidates.
        const bool inw = lane >= j0 && lane < j1;
        const int nw = inw ? n : 0;
        int coop = 1 << 30;
        if constexpr (K >= 32) {
            int best = __reduce_max_sync(FULL_MASK, nw);
#pragma unroll
            for (int th = 64; th >= 8; th >>= 1) {
                if (th > K) continue;
                const int cost = __reduce_max_sync(FULL_MASK, nw < th ? nw : 0) +
                                 W * __popc(__ballot_sync(FULL_MASK, nw >= th));
                if (cost < best) {
                    best = cost;
                    coop = th;
                }
            }
        }
        if (inw && n > 0 && n < coop) {
            int idx = P - pb;
#pragma unroll
            for (int t = 0; t < W; ++t) {
                uint32_t m = f[t];
                while (m) {
                    const int b = __ffs(m) - 1;
                    m &= m - 1;
                    ws.pr[idx++] = ((uint32_t)lane << 16) | (uint32_t)(t * 32 + b);
                }
            }
        }
        if constexpr (K >= 32) {
            unsigned int bm = __ballot_sync(FULL_MASK, inw && n >= coop);
            while (bm) {
                const int j = __ffs(bm) - 1;
                bm &= bm - 1;
                int idx = __shfl_sync(FULL_MASK, P, j) - pb;
#pragma unroll
                for (int t = 0; t < W; ++t) {
                    const uint32_t ft = __shfl_sync(FULL_MASK, f[t], j);
                    if ((ft >> lane) & 1u)
                        ws.pr[idx + __popc(ft & ((1u << lane) - 1u))] = ((uint32_t)j << 16) | (uint32_t)(t * 32 + lane);
                    idx += __popc(ft);
                }
            }
        }
        __syncwarp();
        const int cnt = pe - pb;
        constexpr int R = 4;  // rounds whose loads are in flight together
        for (int r0 = 0; r0 < cnt; r0 += 32 * R) {
            int slot[R];
            unsigned long long x[R];
            int xe[R];
            bool valid[R];
#pragma unroll
            for (int i = 0; i < R; ++i) {
                const int q = r0 + 32 * i + lane;
                valid[i] = q < cnt;
                slot[i] = 0;
                x[i] = 0ull;
                xe[i] = 0;
                if (valid[i]) {
                    const uint32_t e = ws.pr[q];
                    const int j = (int)(e >> 16), c = (int)(e & 0xFFFFu);
                    const size_t idx = (size_t)ws.sv[j] * K + c;
                    slot[i] = ws.so[j] * K + c;
                    x[i] = termv[idx];
                    if constexpr (EXT) xe[i] = terme[idx];
                }
            }
#pragma unroll
            for (int i = 0; i < R; ++i) {
                if (r0 + 32 * i >= cnt) break;
                if constexpr (!ORDERED) {
                    // integer path counts, order-free: two 32-bit shared atomics (the
                    // low word's carry goes into the high word).  Terms are below
                    // 2^sum_bits, which leaves room for the longest sum (1024-arc
                    // chunks, or whole rows where rows are not chunked): a path
                    // count at or above that bound sends the batch to the extended
                    // form when it is written (write_columns), before any sum
                    // takes it as a term.
                    if (valid[i]) {
                        unsigned int* a32 = reinterpret_cast<unsigned int*>(&ws.acc[slot[i]]);
                        const unsigned int xl = (unsigned int)x[i], xh = (unsigned int)(x[i] >> 32);
                        const unsigned int old = atomicAdd(a32, xl);
                        const unsigned int cy = (old + xl < old) ? 1u : 0u;
                        if (xh | cy) atomicAdd(a32 + 1, xh + cy);
                    }
                } else {
                    // ordered: lanes that share a slot add in lane (CSR) order.  A
                    // cheap test first: every lane writes its id to a hashed tag of
                    // its slot (the step's mask words are free during the rounds); if
                    // each reads its own id back, no two lanes share a slot.
                    constexpr int MK = 32 * W;
                    uint32_t* tagv = &ws.fw[0][0];
                    if (valid[i]) tagv[slot[i] & (MK - 1)] = (uint32_t)lane;
                    __syncwarp();
                    const bool clash = valid[i] && tagv[slot[i] & (MK - 1)] != (uint32_t)lane;
                    __syncwarp();
                    int rank = 0, maxr = 0;
                    if (__any_sync(FULL_MASK, clash)) {
                        const int key = valid[i] ? slot[i] : -(lane + 1);
                        const unsigned int peers = __match_any_sync(FULL_MASK, key);
                        rank = __popc(peers & ((1u << lane) - 1u));
                        maxr = __reduce_max_sync(FULL_MASK, valid[i] ? rank : 0);
                    }
                    for (int k = 0; k <= maxr; ++k) {
                        if (valid[i] && rank == k) {
                            unsigned long long av = ws.acc[slot[i]];
                            int ae = EXT ? ws.acce[slot[i]] : 0;
                            acc_add<EXT, DIR>(av, ae, x[i], xe[i], carry);
                            ws.acc[slot[i]] = av;
                            if constexpr (EXT) ws.acce[slot[i]] = ae;
                        }
                        __syncwarp();
                    }
                }
            }
        }
        __syncwarp();
        j0 = j1;
        pb = pe;
    }
    __syncwarp();
}

// ------------------------------------------------------------------ grouped, pair-compacted gather
// Walks the arcs of ng owners (ranges in the owner table, T arcs in total) 32
// at a time, in CSR order.  For each arc (owner o, neighbour v) the matched
// columns f = Fm[v] & want(o) are expanded into (arc, column) pairs, and the
// pairs are processed 32 per round, one per lane: the term of v at column c is
// added into acc[o][c].  Exact path counts use shared-memory atomics (integer
// sums: order-free); every other sum is ordered: lanes hitting the same
// (owner, column) add in lane order, which is CSR order.
template <int K, bool EXT, int DIR>
__device__ __forceinline__ void group_gather(const KParams& p, WarpSmem<K, EXT>& ws, int ng, int T,
                                             const uint32_t* __restrict__ Fm, const int* __restrict__ adjv,
                                             bool& carry) {
    constexpr int W = Geo<K>::W;
    const int lane = lane_id();
    for (int i = lane; i < ng * K; i += 32) {
        ws.acc[i] = 0ull;
        if constexpr (EXT) ws.acce[i] = 0;
    }
    for (int i = lane; i < ng * W; i += 32) (&ws.onm[0][0])[i] = 0u;
    __syncwarp();
    const unsigned long long* termv =
        DIR == FWD ? p.sig : reinterpret_cast<const unsigned long long*>(p.rho);
    const int* terme = DIR == FWD ? p.sig_e : p.rho_e;
    // Step pipeline (lane = arc): the neighbour ids are loaded two steps ahead
    // and the frontier masks one step ahead, so a step's own loads are in
    // flight while the previous steps are processed.
    auto owner_of = [&](int a) {
        int o = 0;
#pragma unroll
        for (int step = 16; step >= 1; step >>= 1)
            if (o + step < ng && ws.ostart[o + step] <= a) o += step;
        return o;
    };
    auto nbr_of = [&](int a, int o) { return a < T ? __ldg(adjv + ws.obeg[o] + (a - ws.ostart[o])) : 0; };
    int o = owner_of(lane);
    int v = nbr_of(lane, o);
    uint32_t fr[W];
#pragma unroll
    for (int t = 0; t < W; ++t) fr[t] = 0;
    if (lane < T) load_mask<W>(Fm, v, fr);
    int o1 = owner_of(lane + 32);
    int v1 = nbr_of(lane + 32, o1);
    for (int base = 0; base < T; base += 32) {
        const int a = base + lane;
        int n = 0;
        uint32_t f[W];
#pragma unroll
        for (int t = 0; t < W; ++t) {
            f[t] = a < T ? fr[t] & ws.owant[o][t] : 0u;
            n += __popc(f[t]);
        }
        // next step's masks, the step after's neighbour ids
#pragma unroll
        for (int t = 0; t < W; ++t) fr[t] = 0;
        if (a + 32 < T) load_mask<W>(Fm, v1, fr);
        const int o2 = owner_of(a + 64);
        const int v2 = nbr_of(a + 64, o2);
        const int ocur = o, vcur = v;
        o = o1; v = v1; o1 = o2; v1 = v2;
        gather_step<K, EXT, DIR>(p, ws, ocur, vcur, n, f, termv, terme, carry);
    }
    __syncwarp();
}

// ------------------------------------------------------------------ finishing vertices
// Position of the k-th (0-based) set bit of x (x has more than k set bits).
__device__ __forceinline__ int select_bit(uint32_t x, int k) {
    int pos = 0;
#pragma unroll
    for (int sh = 16; sh > 0; sh >>= 1) {
        const uint32_t low = x & ((1u << sh) - 1u);
        const int c = __popc(low);
        if (k >= c) {
            k -= c;
            x >>= sh;
            pos += sh;
        } else {
            x = low;
        }
    }
    return pos;
}

// Column of the k-th set bit of a W-word mask.
template <int W>
__device__ __forceinline__ int select_col(const uint32_t* m, int k) {
    int base = 0;
#pragma unroll
    for (int t = 0; t < W - 1; ++t) {
        const int c = __popc(m[t]);
        if (k >= c && base == t * 32) {
            k -= c;
            base = (t + 1) * 32;
        }
    }
    return base + select_bit(m[base >> 5], k);
}

// Finish the columns of the group's owners, one (owner, column) pair per lane:
// masks[o] selects the columns of owner o (row o of the accumulator).
// FWD writes the path counts; BWD turns rho sums into delta and rho.
template <int K, bool EXT, int DIR>
__device__ __forceinline__ void write_columns(const KParams& p, WarpSmem<K, EXT>& ws, int ng,
                                              const uint32_t (*masks)[Geo<K>::W]) {
    constexpr int W = Geo<K>::W;
    const int lane = lane_id();
    int cnt = 0;
    if (lane < ng) {
#pragma unroll
        for (int t = 0; t < W; ++t) cnt += __popc(masks[lane][t]);
    }
    int incl = cnt;
#pragma unroll
    for (int s = 1; s < 32; s <<= 1) {
        int y = __shfl_up_sync(FULL_MASK, incl, s);
        if (lane >= s) incl += y;
    }
    const int Q = __shfl_sync(FULL_MASK, incl, 31);
    const int ex = incl - cnt;  // exclusive prefix of owner `lane`
    if (DIR == FWD && lane == 0) ws.cnt_reached += (unsigned long long)Q;
    bool inexact = false, big = false;
    for (int r = 0; r < Q; r += 32) {
        const int q = r + lane;
        // owner: the largest o < ng with exclusive prefix <= q
        int o = 0;
#pragma unroll
        for (int step = 16; step >= 1; step >>= 1) {
            const int cand = o + step;
            const int sc = __shfl_sync(FULL_MASK, ex, cand < 32 ? cand : 31);
            if (cand < ng && sc <= q) o = cand;
        }
        const int so = __shfl_sync(FULL_MASK, ex, o);
        if (q < Q) {
            const int c = (K == 1) ? 0 : select_col<W>(masks[o], q - so);
            const int v = ws.ov[o];
            const size_t idx = (size_t)v * K + c;
            const int slot = o * K + c;
            if constexpr (DIR == FWD) {
                const unsigned long long x = ws.acc[slot];
                p.sig[idx] = x;
                int xe = 0;
                if constexpr (EXT) {
                    xe = ws.acce[slot];
                    p.sig_e[idx] = xe;
                } else {
                    p.rho[idx] = __drcp_rn((double)x);  // 1 / sigma, used by the reverse sweep
                    big |= (x >> p.sum_bits) != 0ull;  // a term too large for the plain sums
                }
                inexact |= (xe > 0 || x >= (1ull << 53));
            } else {
                // rho = (1 + delta) / sigma = 1 / sigma + sum, with delta = sigma * sum
                const double sd = (double)p.sig[idx];  // rounds only when the count is >= 2^53
                const double sr = __longlong_as_double((long long)ws.acc[slot]);
                double delta, rho;
                if constexpr (EXT) {
                    const int se = p.sig_e[idx];
                    delta = scale2(sd * sr, se + ws.acce[slot]);
                    rho = __drcp_rn(sd) + scale2(sr, se + ws.acce[slot]);
                    p.rho_e[idx] = -se;
                } else {
                    delta = sd * sr;
                    rho = p.rho[idx] + sr;
                }
                p.sig[idx] = (unsigned long long)__double_as_longlong(delta);
                p.rho[idx] = rho;
            }
        }
    }
    if (DIR == FWD && __any_sync(FULL_MASK, inexact) && lane == 0) atomicOr(&p.ctl->flags, BST_INEXACT);
    if (DIR == FWD && __any_sync(FULL_MASK, big) && lane == 0) atomicOr(&p.ctl->flags, BST_NEED_EXT);
}

// Owner-level forward bookkeeping (lane o handles owner o): mark the newly
// reached columns nm in V and account vertices whose every column is reached.
template <int W>
__device__ __forceinline__ void mark_reached(const KParams& p, int w, const uint32_t (&nm)[W], int lev,
                                             const uint32_t (&act)[W]) {
    uint32_t vm[W];
    load_mask<W>(p.V, w, vm);
    bool full = true;
#pragma unroll
    for (int t = 0; t < W; ++t) {
        vm[t] |= nm[t];
        full &= (vm[t] & act[t]) == act[t];
    }
    store_mask_full<W>(p.V, w, vm);
    if (full) atomicAdd((unsigned long long*)&p.la.fulldeg[lev], (unsigned long long)(p.off[w + 1] - p.off[w]));
}

__device__ __forceinline__ int nchunks(int deg) { return (deg + kChunk - 1) / kChunk; }

// ------------------------------------------------------------------ list appends
template <int K, bool EXT>
__device__ __forceinline__ void flush_append(const KParams& p, int lev, WarpSmem<K, EXT>& ws, int& cnt) {
    constexpr int W = Geo<K>::W;
    const int lane = lane_id();
    if (cnt == 0) return;
    __syncwarp();
    int base = 0;
    if (lane == 0) {
        base = atomicAdd(&p.la.cnt[lev], cnt);
        atomicAdd((unsigned long long*)&p.la.dsum[lev], (unsigned long long)ws.adeg);
        ws.adeg = 0;
    }
    base = __shfl_sync(FULL_MASK, base, 0);
    const long long pos = (long long)p.la.start[lev] + base + lane;
    if (lane < cnt) {
        if (pos < p.cap) {
            p.ent[pos] = ws.av[lane];
            uint32_t m[W];
#pragma unroll
            for (int t = 0; t < W; ++t) m[t] = ws.am[lane][t];
            store_mask_full<W>(p.emask, pos, m);
        } else {
            atomicOr(&p.gctl->err, ERR_CAPACITY);
        }
    }
    __syncwarp();
    cnt = 0;
}

template <int W>
__device__ __forceinline__ void heavy_append(const KParams& p, int lev, int w, long long deg, const uint32_t (&m)[W]) {
    const int i = atomicAdd(&p.la.hcnt[lev], 1);
    atomicAdd((unsigned long long*)&p.la.dsum[lev], (unsigned long long)deg);
    const long long pos = (long long)p.la.hstart[lev] + i;
    if (pos < p.hcap) {
        p.hent[pos] = w;
        store_mask_full<W>(p.hmask, pos, m);
    } else {
        atomicOr(&p.gctl->err, ERR_CAPACITY);
    }
}

// ------------------------------------------------------------------ heavy chunk tasks

// Task t of a heavy list level -> (entry position, chunk), by binary search of
// the level's chunk prefix.
__device__ __forceinline__ void heavy_list_task(const KParams& p, int lev, int t, int& pos, int& chunk) {
    int lo = p.la.hstart[lev], hi = lo + p.la.hcnt[lev] - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (p.hpre[mid] <= t) lo = mid;
        else hi = mid - 1;
    }
    pos = lo;
    chunk = t - p.hpre[lo];
}

// Static heavy task t -> (vertex r, chunk) for the pull phase.
__device__ __forceinline__ void heavy_static_task(const KParams& p, int t, int& r, int& chunk) {
    int lo = 0, hi = p.n_heavy - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (p.hcum[mid] <= t) lo = mid;
        else hi = mid - 1;
    }
    r = lo;
    chunk = t - p.hcum[lo];
}

// Exclusive chunk prefix of the heavy entries of a level (recomputed from the
// row lengths, so it may run more than once per level).  Block 0 scans in tiles.
__device__ void heavy_prefix(const KParams& p, int lev) {
    if (p.rank != 0) return;
    __shared__ int wsum[kWarps];
    __shared__ int carry_s;
    const int lane = lane_id(), wid = warp_id();
    const int hs = p.la.hstart[lev], hc = p.la.hcnt[lev];
    if (threadIdx.x == 0) carry_s = 0;
    __syncthreads();
    for (int i0 = 0; i0 < hc; i0 += kThreads) {
        const int i = i0 + threadIdx.x;
        int c = 0;
        if (i < hc) {
            const int v = p.hent[hs + i];
            c = nchunks(p.off[v + 1] - p.off[v]);
        }
        int incl = c;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int y = __shfl_up_sync(FULL_MASK, incl, o);
            if (lane >= o) incl += y;
        }
        if (lane == 31) wsum[wid] = incl;
        __syncthreads();
        int before = carry_s;
        for (int w2 = 0; w2 < wid; ++w2) before += wsum[w2];
        if (i < hc) p.hpre[hs + i] = before + incl - c;
        __syncthreads();
        if (threadIdx.x == kThreads - 1) carry_s = before + incl;
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const int total = p.n_heavy > 0 ? p.hcum[p.n_heavy] : 0;
        if (carry_s > total) {  // impossible for consistent lists: refuse to schedule
            atomicOr(&p.gctl->err, ERR_INTERNAL);
            p.la.hchunks[lev] = 0;
        } else {
            p.la.hchunks[lev] = carry_s;
        }
    }
}

// Store the chunk partial held in accumulator row 0; returns true (warp-
// uniform) for the warp that completes the vertex, after combining every
// partial, in chunk order, back into row 0 (and their masks into nm).
template <int K, bool EXT, int DIR>
__device__ __forceinline__ bool heavy_partial(const KParams& p, WarpSmem<K, EXT>& ws, int r, int chunk, int nch,
                                              uint32_t (&nm)[Geo<K>::W]) {
    constexpr int W = Geo<K>::W;
    const int lane = lane_id();
    const size_t slot = (size_t)(p.hcum[r] + chunk);
    for (int c = lane; c < K; c += 32) {
        p.scr_v[slot * K + c] = ws.acc[c];
        if constexpr (EXT) p.scr_e[slot * K + c] = ws.acce[c];
    }
    if (lane < W) p.scr_or[slot * W + lane] = ws.onm[0][lane];
    __threadfence();
    __syncwarp();
    int last = 0;
    if (lane == 0) last = (atomicAdd(&p.arr[r], 1) == nch - 1);
    last = __shfl_sync(FULL_MASK, last, 0);
    if (!last) return false;
    __threadfence();
    bool carry = false;
    const size_t s0 = (size_t)p.hcum[r];
    for (int c = lane; c < K; c += 32) {
        unsigned long long v = 0ull;
        int e = 0;
        for (int ch = 0; ch < nch; ++ch) {
            const unsigned long long x = *(volatile unsigned long long*)&p.scr_v[(s0 + ch) * K + c];
            const int xe = EXT ? *(volatile int*)&p.scr_e[(s0 + ch) * K + c] : 0;
            acc_add<EXT, DIR>(v, e, x, xe, carry);
        }
        ws.acc[c] = v;
        if constexpr (EXT) ws.acce[c] = e;
    }
#pragma unroll
    for (int t = 0; t < W; ++t) {
        uint32_t m = 0;
        for (int ch = 0; ch < nch; ++ch) m |= *(volatile uint32_t*)&p.scr_or[(s0 + ch) * W + t];
        nm[t] = m;
    }
    __syncwarp();
    if (lane == 0) p.arr[r] = 0;
    return true;
}

// ------------------------------------------------------------------ phases
__device__ __forceinline__ unsigned int* wq(const KParams& p, int ph, int which) {
    return &p.ctl->wq[(ph & 3) * 2 + which];
}
template <bool STAGED>
__device__ __forceinline__ void phase_prologue(const KParams& p, int ph) {
    // the rows a phase stages by bulk copies (async proxy: the column-mapped
    // arcs of K >= 32 in the plain form) were written before the barrier that
    // opened it: order the issuing lanes' acquire before them
    if (STAGED && (threadIdx.x & 31) == 0) asm volatile("fence.proxy.async.global;" ::: "memory");
    if (p.rank == 0 && threadIdx.x == 0) {
        p.ctl->wq[((ph + 2) & 3) * 2] = 0;
        p.ctl->wq[((ph + 2) & 3) * 2 + 1] = 0;
    }
}

// Clear the dense masks of level `lev` (entries of that level) in buffer F.
template <int W>
__device__ void clear_level_masks(const KParams& p, uint32_t* F, int lev) {
    const long long s = p.la.start[lev], c = p.la.cnt[lev], hs = p.la.hstart[lev], hc = p.la.hcnt[lev];
    const long long nthr = (long long)p.team_blocks * blockDim.x;
    const long long tid = (long long)p.rank * blockDim.x + threadIdx.x;
    const uint32_t zero[W] = {};
    for (long long j = tid; j < c + hc; j += nthr) {
        const int v = j < c ? p.ent[s + j] : p.hent[hs + (j - c)];
        store_mask_full<W>(F, v, zero);  // the entry's W words in one store
    }
}

template <int K>
__device__ void active_mask(const KParams& p, int b, uint32_t (&act)[Geo<K>::W]) {
    constexpr int W = Geo<K>::W;
#pragma unroll
    for (int t = 0; t < W; ++t) act[t] = 0;
    for (int c = 0; c < K; ++c)
        if (p.src[(size_t)b * K + c] >= 0) act[c >> 5] |= 1u << (c & 31);
}

template <int W>
__device__ __forceinline__ void read_mask_s(const uint32_t (&src)[W], uint32_t (&m)[W]) {
#pragma unroll
    for (int t = 0; t < W; ++t) m[t] = src[t];
}

// Pull (bottom-up) discovery fused with the path-count sum, iteration `it`
// (frontier = level it, new vertices get level it + 1).
template <int K, bool EXT>
__device__ void phase_pull(const KParams& p, int it, int ph, const uint32_t (&act)[Geo<K>::W], WarpSmem<K, EXT>& ws,
                           int group) {
    constexpr int W = Geo<K>::W;
    const int lane = lane_id();
    const uint32_t* Fc = p.F[it % 3];
    uint32_t* Fn = p.F[(it + 1) % 3];
    const int lev = it + 1;
    bool carry = false;
    phase_prologue<K >= 32 && !EXT>(p, ph);
    // directed graphs pull over in-rows (the transpose), whole rows: no chunk tasks
    const bool directed = p.ioff != nullptr;
    const int* roff = directed ? p.ioff : p.off;
    const int* radj = directed ? p.iadj : p.adj;
    // heavy rows: chunk tasks over the static prefix of heavy ids
    const int HC = (!directed && p.n_heavy > 0) ? p.hcum[p.n_heavy] : 0;
    for (bool fst = true;;) {
        const long long t0 = next_task(p, wq(p, ph, 0), HC, fst);
        if (t0 < 0) break;
        int r, chunk;
        heavy_static_task(p, (int)t0, r, chunk);
        uint32_t vm[W], um[W];
        load_mask<W>(p.V, r, vm);
#pragma unroll
        for (int t = 0; t < W; ++t) um[t] = act[t] & ~vm[t];
        if (!mask_any<W>(um)) continue;
        const int rb = p.off[r], deg = p.off[r + 1] - rb, nch = nchunks(deg);
        const int cb = chunk * kChunk, len = min(kChunk, deg - cb);
        const int T = set_owners<K, EXT>(ws, 1, r, rb + cb, lane == 0 ? len : 0, -1, um);
        group_gather<K, EXT, FWD>(p, ws, 1, T, Fc, p.adj, carry);
        uint32_t nm[W];
        if (heavy_partial<K, EXT, FWD>(p, ws, r, chunk, nch, nm) && mask_any<W>(nm)) {
            if (lane == 0) {
#pragma unroll
                for (int t = 0; t < W; ++t) ws.onm[0][t] = nm[t];
            }
            __syncwarp();
            write_columns<K, EXT, FWD>(p, ws, 1, ws.onm);
            if (lane == 0) {
                store_mask_full<W>(Fn, r, nm);
                mark_reached<W>(p, r, nm, lev, act);
                heavy_append<W>(p, lev, r, deg, nm);
            }
        }
    }
    // light rows: groups of consecutive ids
    int acnt = 0;
    if (lane == 0) ws.adeg = 0;
    const long long lbase = directed ? 0 : p.n_heavy;  // first row of the grouped path
    const long long nlight = (long long)p.n_nz - lbase;
    const long long ngroups = (nlight + group - 1) / group;
    for (bool fst = true;;) {
        const long long g0 = next_task(p, wq(p, ph, 1), ngroups, fst);
        if (g0 < 0) break;
        const long long first = lbase + g0 * group;
        const int ng = (int)min((long long)group, (long long)p.n_nz - first);
        int v = 0, beg = 0, len = 0;
        uint32_t um[W];
#pragma unroll
        for (int t = 0; t < W; ++t) um[t] = 0;
        if (lane < ng) {
            v = (int)(first + lane);
            uint32_t vm[W];
            load_mask<W>(p.V, v, vm);
#pragma unroll
            for (int t = 0; t < W; ++t) um[t] = act[t] & ~vm[t];
            beg = roff[v];
            len = mask_any<W>(um) ? roff[v + 1] - beg : 0;
        }
        if (!__any_sync(FULL_MASK, len > 0)) continue;
        const int T = set_owners<K, EXT>(ws, ng, v, beg, len, -1, um);
        group_gather<K, EXT, FWD>(p, ws, ng, T, Fc, radj, carry);
        write_columns<K, EXT, FWD>(p, ws, ng, ws.onm);
        // owners reached in this level (lane o = owner o): masks, V, staged appends
        uint32_t nm[W];
        bool found = false;
        int w = 0;
        if (lane < ng) {
            read_mask_s<W>(ws.onm[lane], nm);
            found = mask_any<W>(nm);
            w = ws.ov[lane];
            if (found) {
                store_mask_full<W>(Fn, w, nm);
                mark_reached<W>(p, w, nm, lev, act);
                // directed graphs pull every row here: rows heavy by out-degree still
                // go to the heavy list (chunked push and reverse steps)
                if (w < p.n_heavy) {
                    heavy_append<W>(p, lev, w, p.off[w + 1] - p.off[w], nm);
                    found = false;
                }
            }
        }
        const unsigned int fb = __ballot_sync(FULL_MASK, found);
        const int nf = __popc(fb);
        if (nf) {
            if (acnt + nf > 32) flush_append<K, EXT>(p, lev, ws, acnt);
            long long dg = found ? (long long)(p.off[w + 1] - p.off[w]) : 0;
#pragma unroll
            for (int s2 = 16; s2 > 0; s2 >>= 1) dg += __shfl_xor_sync(FULL_MASK, dg, s2);
            if (found) {
                const int slot = acnt + __popc(fb & ((1u << lane) - 1u));
                ws.av[slot] = w;
#pragma unroll
                for (int t = 0; t < W; ++t) ws.am[slot][t] = nm[t];
            }
            if (lane == 0) ws.adeg += dg;
            __syncwarp();
            acnt += nf;
            if (acnt == 32) flush_append<K, EXT>(p, lev, ws, acnt);
        }
    }
    flush_append<K, EXT>(p, lev, ws, acnt);
    if (__any_sync(FULL_MASK, carry) && lane == 0) atomicOr(&p.ctl->flags, BST_NEED_EXT);
    if (it >= 1) clear_level_masks<W>(p, p.F[(it + 2) % 3], it - 1);
}

// Push (top-down) discovery over the frontier entries of level `it`.
template <int K, bool EXT>
__device__ void phase_push(const KParams& p, int it, int ph, WarpSmem<K, EXT>& ws, int group) {
    constexpr int W = Geo<K>::W;
    const int lane = lane_id();
    uint32_t* Fn = p.F[(it + 1) % 3];
    const int lev = it + 1;
    const int stampv = lev;
    phase_prologue<false>(p, ph);
    // claim unseen columns of the neighbours of the owner table's arcs
    auto visit = [&](int ng, int T) {
        for (int base = 0; base < T; base += 32) {
            const int a = base + lane;
            int o = 0;
#pragma unroll
            for (int step = 16; step >= 1; step >>= 1)
                if (o + step < ng && ws.ostart[o + step] <= a) o += step;
            bool light_claim = false, heavy_claim = false;
            int w = 0;
            long long deg = 0;
            if (a < T) {
                w = __ldg(p.adj + ws.obeg[o] + (a - ws.ostart[o]));
                uint32_t vw[W], nb[W];
                load_mask<W>(p.V, w, vw);
                bool any = false;
#pragma unroll
                for (int t = 0; t < W; ++t) { nb[t] = ws.owant[o][t] & ~vw[t]; any |= nb[t] != 0; }
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
                for (int s = 16; s > 0; s >>= 1) ds += __shfl_xor_sync(FULL_MASK, ds, s);
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
                    else atomicOr(&p.gctl->err, ERR_CAPACITY);
                }
            }
            if (heavy_claim) {
                const int i = atomicAdd(&p.la.hcnt[lev], 1);
                atomicAdd((unsigned long long*)&p.la.dsum[lev], (unsigned long long)deg);
                const long long pos = (long long)p.la.hstart[lev] + i;
                if (pos < p.hcap) p.hent[pos] = w;
                else atomicOr(&p.gctl->err, ERR_CAPACITY);
            }
        }
    };
    // heavy frontier rows: chunk tasks
    const int HT = p.la.hcnt[it] > 0 ? p.la.hchunks[it] : 0;
    for (bool fst = true;;) {
        const long long t0 = next_task(p, wq(p, ph, 0), HT, fst);
        if (t0 < 0) break;
        int pos, chunk;
        heavy_list_task(p, it, (int)t0, pos, chunk);
        const int v = p.hent[pos];
        uint32_t fm[W];
        load_mask<W>(p.hmask, pos, fm);
        const int rb = p.off[v], deg = p.off[v + 1] - rb;
        const int cb = chunk * kChunk, len = min(kChunk, deg - cb);
        const int T = set_owners<K, EXT>(ws, 1, v, rb + cb, lane == 0 ? len : 0, pos, fm);
        visit(1, T);
        __syncwarp();
    }
    // light frontier entries: groups
    constexpr int G = Geo<K>::G;
    const int grp = group < G ? group : G;
    const int ls = p.la.start[it], lc = p.la.cnt[it];
    const long long ngroups = (lc + grp - 1) / grp;
    for (bool fst = true;;) {
        const long long g0 = next_task(p, wq(p, ph, 1), ngroups, fst);
        if (g0 < 0) break;
        const int first = (int)(g0 * grp);
        const int ng = min(grp, lc - first);
        int v = 0, beg = 0, len = 0;
        uint32_t fm[W];
#pragma unroll
        for (int t = 0; t < W; ++t) fm[t] = 0;
        if (lane < ng) {
            v = p.ent[ls + first + lane];
            load_mask<W>(p.emask, ls + first + lane, fm);
            beg = p.off[v];
            len = p.off[v + 1] - beg;
        }
        const int T = set_owners<K, EXT>(ws, ng, v, beg, len, ls + first + lane, fm);
        visit(ng, T);
        __syncwarp();
    }
}

// Path counts of the vertices claimed by the push phase (entries of level it+1).
template <int K, bool EXT>
__device__ void phase_sigma(const KParams& p, int it, int ph, const uint32_t (&act)[Geo<K>::W],
                            WarpSmem<K, EXT>& ws, int group) {
    constexpr int W = Geo<K>::W;
    const int lane = lane_id();
    const uint32_t* Fc = p.F[it % 3];
    const uint32_t* Fn = p.F[(it + 1) % 3];
    const int lev = it + 1;
    bool carry = false;
    phase_prologue<K >= 32 && !EXT>(p, ph);
    // directed graphs sum over in-rows (the transpose), whole rows: heavy entries
    // (heavy by out-degree) join the grouped path below
    const bool directed = p.ioff != nullptr;
    const int* roff = directed ? p.ioff : p.off;
    const int* radj = directed ? p.iadj : p.adj;
    const int HT = (!directed && p.la.hcnt[lev] > 0) ? p.la.hchunks[lev] : 0;
    for (bool fst = true;;) {
        const long long t0 = next_task(p, wq(p, ph, 0), HT, fst);
        if (t0 < 0) break;
        int pos, chunk;
        heavy_list_task(p, lev, (int)t0, pos, chunk);
        const int w = p.hent[pos];
        uint32_t nm[W];
        load_mask<W>(Fn, w, nm);
        const int rb = p.off[w], deg = p.off[w + 1] - rb, nch = nchunks(deg);
        const int cb = chunk * kChunk, len = min(kChunk, deg - cb);
        const int T = set_owners<K, EXT>(ws, 1, w, rb + cb, lane == 0 ? len : 0, pos, nm);
        group_gather<K, EXT, FWD>(p, ws, 1, T, Fc, p.adj, carry);
        uint32_t om[W];
        if (heavy_partial<K, EXT, FWD>(p, ws, w, chunk, nch, om)) {
            write_columns<K, EXT, FWD>(p, ws, 1, ws.owant);
            if (lane == 0) {
                mark_reached<W>(p, w, nm, lev, act);
                store_mask_full<W>(p.hmask, pos, nm);
            }
        }
    }
    const int ls = p.la.start[lev], lc = p.la.cnt[lev], hs = p.la.hstart[lev];
    const int ltot = lc + (directed ? p.la.hcnt[lev] : 0);  // light entries, then (directed) heavy ones
    const long long ngroups = (ltot + group - 1) / group;
    for (bool fst = true;;) {
        const long long g0 = next_task(p, wq(p, ph, 1), ngroups, fst);
        if (g0 < 0) break;
        const int first = (int)(g0 * group);
        const int ng = min(group, ltot - first);
        int v = 0, beg = 0, len = 0, pos = 0;
        uint32_t nm[W];
#pragma unroll
        for (int t = 0; t < W; ++t) nm[t] = 0;
        if (lane < ng) {
            const int i = first + lane;
            pos = i < lc ? ls + i : -(hs + (i - lc)) - 1;  // >= 0: light list, < 0: heavy list
            v = i < lc ? p.ent[ls + i] : p.hent[hs + (i - lc)];
            load_mask<W>(Fn, v, nm);
            beg = roff[v];
            len = roff[v + 1] - beg;
        }
        const int T = set_owners<K, EXT>(ws, ng, v, beg, len, pos, nm);
        group_gather<K, EXT, FWD>(p, ws, ng, T, Fc, radj, carry);
        write_columns<K, EXT, FWD>(p, ws, ng, ws.owant);
        if (lane < ng) {
            uint32_t want[W];
            read_mask_s<W>(ws.owant[lane], want);
            mark_reached<W>(p, ws.ov[lane], want, lev, act);
            const int q = ws.opos[lane];
            if (q >= 0) store_mask_full<W>(p.emask, q, want);
            else store_mask_full<W>(p.hmask, -q - 1, want);
        }
    }
    if (__any_sync(FULL_MASK, carry) && lane == 0) atomicOr(&p.ctl->flags, BST_NEED_EXT);
    if (it >= 1) clear_level_masks<W>(p, p.F[(it + 2) % 3], it - 1);
}

// Reverse sweep over level l: delta and rho of its entries from level l+1.
template <int K, bool EXT>
__device__ void phase_back(const KParams& p, int l, int ph, WarpSmem<K, EXT>& ws, int group) {
    constexpr int W = Geo<K>::W;
    const int lane = lane_id();
    const uint32_t* Fd = p.F[(l + 1) % 3];  // level l+1 masks
    uint32_t* Fl = p.F[l % 3];              // level l masks (read by level l-1)
    bool carry = false;
    phase_prologue<K >= 32 && !EXT>(p, ph);
    const int HT = p.la.hcnt[l] > 0 ? p.la.hchunks[l] : 0;
    for (bool fst = true;;) {
        const long long t0 = next_task(p, wq(p, ph, 0), HT, fst);
        if (t0 < 0) break;
        int pos, chunk;
        heavy_list_task(p, l, (int)t0, pos, chunk);
        const int v = p.hent[pos];
        uint32_t mk[W];
        load_mask<W>(p.hmask, pos, mk);
        const int rb = p.off[v], deg = p.off[v + 1] - rb, nch = nchunks(deg);
        const int cb = chunk * kChunk, len = min(kChunk, deg - cb);
        const int T = set_owners<K, EXT>(ws, 1, v, rb + cb, lane == 0 ? len : 0, pos, mk);
        group_gather<K, EXT, BWD>(p, ws, 1, T, Fd, p.adj, carry);
        uint32_t om[W];
        if (heavy_partial<K, EXT, BWD>(p, ws, v, chunk, nch, om)) {
            write_columns<K, EXT, BWD>(p, ws, 1, ws.owant);
            if (lane == 0) store_mask_full<W>(Fl, v, mk);
        }
    }
    const int ls = p.la.start[l], lc = p.la.cnt[l];
    const long long ngroups = (lc + group - 1) / group;
    for (bool fst = true;;) {
        const long long g0 = next_task(p, wq(p, ph, 1), ngroups, fst);
        if (g0 < 0) break;
        const int first = (int)(g0 * group);
        const int ng = min(group, lc - first);
        int v = 0, beg = 0, len = 0;
        uint32_t mk[W], fin[W];
#pragma unroll
        for (int t = 0; t < W; ++t) mk[t] = fin[t] = 0;
        if (lane < ng) {
            v = p.ent[ls + first + lane];
            load_mask<W>(p.emask, ls + first + lane, mk);
            // a vertex of degree 1 at a level >= 1 has no successor: its delta is 0
            // and its rho the 1/sigma the forward sweep stored, so it is not
            // gathered or finished (plain form; phase_bc leaves it out too)
            if (EXT || v < p.first_leaf) {
                beg = p.off[v];
                len = p.off[v + 1] - beg;
#pragma unroll
                for (int t = 0; t < W; ++t) fin[t] = mk[t];
            }
        }
        const int T = set_owners<K, EXT>(ws, ng, v, beg, len, ls + first + lane, fin);
        group_gather<K, EXT, BWD>(p, ws, ng, T, Fd, p.adj, carry);
        write_columns<K, EXT, BWD>(p, ws, ng, ws.owant);
        if (lane < ng) store_mask_full<W>(Fl, v, mk);  // level-l tags for level l-1's gathers
    }
    clear_level_masks<W>(p, p.F[(l + 2) % 3], l + 2);
}

// BC[v] += delta of every reached, non-source column, in column order.  Each
// column belongs to a job (col_job; all job 0 when absent) whose columns are
// contiguous; a job's sum is carried sequentially across its columns and its
// batches, so the additions happen in the job's source-list order whatever
// else shares the batch.
template <int K, bool EXT>
__device__ void phase_bc(const KParams& p, int b) {
    constexpr int W = Geo<K>::W;
    const long long nthr = (long long)p.team_blocks * blockDim.x;
    const int* src = p.src + (size_t)b * K;
    const int* cj = p.col_job ? p.col_job + (size_t)b * K : nullptr;
    // vertices of degree 1 (ids [first_leaf, n_nz)) add nothing: their dependency is 0
    const long long vend = EXT ? p.n_nz : min((long long)p.n_nz, (long long)p.first_leaf);
    for (long long v = (long long)p.rank * blockDim.x + threadIdx.x; v < vend; v += nthr) {
        uint32_t vm[W];
        load_mask<W>(p.V, v, vm);
        if (!mask_any<W>(vm)) continue;
        int cur = -1;
        double acc = 0.0;
        // the row's dependencies four columns (one 32-byte sector) at a time, so
        // that each sector is read once per thread, not once per column: rows of
        // neighbouring threads do not stay in L1 between a thread's columns
        constexpr int Q = K >= 4 ? 4 : 1;
        for (int c0 = 0; c0 < K; c0 += Q) {
            const uint32_t bits = (vm[c0 >> 5] >> (c0 & 31)) & ((1u << Q) - 1u);
            if (!bits) continue;
            unsigned long long d[Q];
            load_terms<Q>(p.sig + (size_t)v * K + c0, d);
#pragma unroll
            for (int i = 0; i < Q; ++i) {
                if (!((bits >> i) & 1u)) continue;
                const int c = c0 + i;
                const int s = __ldg(src + c);
                if (s == (int)v) continue;
                const int j = cj ? __ldg(cj + c) : 0;
                if (j != cur) {
                    if (cur >= 0) p.job_bc[cur][v] = acc;
                    cur = j;
                    acc = p.job_bc[j][v];
                }
                acc += __longlong_as_double((long long)d[i]);
            }
        }
        if (cur >= 0) p.job_bc[cur][v] = acc;
    }
}

// ------------------------------------------------------------------ BC order across teams
// Batch b may add into BC only after batch b-1 has: the team's first thread
// waits (bounded) for the launch-wide turn counter, then the team proceeds.
__device__ bool bc_turn_wait(const KParams& p, GridTeam& team, int b) {
    if (p.nteams > 1 && p.rank == 0 && threadIdx.x == 0) {
        volatile unsigned int* turn = &p.gctl->bc_next;
        volatile int* errp = &p.gctl->err;
        const long long t0 = clock64();
        while (*turn != (unsigned int)b) {
            if (*errp) break;
            if (clock64() - t0 > p.budget) {
                atomicOr(&p.gctl->err, ERR_TIMEOUT);
                break;
            }
            __nanosleep(64);
        }
        __threadfence();
    }
    return team.sync();
}

// After the team barrier that follows its BC phase: hand the turn to batch b+1.
__device__ __forceinline__ void bc_turn_pass(const KParams& p, int b) {
    if (p.nteams > 1 && p.rank == 0 && threadIdx.x == 0) {
        __threadfence();
        atomicExch(&p.gctl->bc_next, (unsigned int)(b + 1));
    }
}

// ------------------------------------------------------------------ one batch
template <int K, bool EXT>
__device__ bool run_batch(const KParams& p, int b, GridTeam& team, int& ph, WarpSmem<K, EXT>& ws) {
    constexpr int W = Geo<K>::W;
    constexpr int G = Geo<K>::G;
    const long long nthr = (long long)p.team_blocks * blockDim.x;
    const long long tid = (long long)p.rank * blockDim.x + threadIdx.x;
    // Values used across the phases are recomputed or held in shared memory (one
    // copy per block), not kept in registers: the phases are inlined into this
    // loop, and registers live across them cost spills inside them.  With the
    // active columns and the team barrier's state (the kernel's) moved out of
    // registers, R-MAT 22 went 1175 -> 1125 ms, R-MAT 20 88.4 -> 83.5 ms.
    const auto group = [&p]() { return p.group < G ? p.group : G; };
    const auto lead = [&p]() { return p.rank == 0 && threadIdx.x == 0; };
    __shared__ long long s_full;  // arcs of rows whose every column is reached (block copy)
    __shared__ int s_pull;        // this level's direction (block copy)
    if (threadIdx.x == 0) { s_full = 0; s_pull = 0; }
    __shared__ uint32_t act[W];  // the batch's active columns
    if (threadIdx.x == 0) active_mask<K>(p, b, act);

    // init A: clear masks and stamps, zero the first level slots and the batch flags
    {
        // 16-byte stores (the per-team arrays start 256-byte aligned); a scalar tail
        const long long words = (long long)p.n * W, quads = words >> 2;
        const uint4 z = make_uint4(0u, 0u, 0u, 0u);
        for (long long i = tid; i < quads; i += nthr) {
            reinterpret_cast<uint4*>(p.V)[i] = z;
            reinterpret_cast<uint4*>(p.F[0])[i] = z;
            reinterpret_cast<uint4*>(p.F[1])[i] = z;
            reinterpret_cast<uint4*>(p.F[2])[i] = z;
        }
        for (long long i = (quads << 2) + tid; i < words; i += nthr) {
            p.V[i] = 0; p.F[0][i] = 0; p.F[1][i] = 0; p.F[2][i] = 0;
        }
    }
    {
        const long long quads = (long long)p.n >> 2;
        const int4 m1 = make_int4(-1, -1, -1, -1);
        for (long long i = tid; i < quads; i += nthr) reinterpret_cast<int4*>(p.stamp)[i] = m1;
        for (long long i = (quads << 2) + tid; i < p.n; i += nthr) p.stamp[i] = -1;
    }
    if (tid < 3) {
        p.la.cnt[tid] = 0; p.la.hcnt[tid] = 0; p.la.dsum[tid] = 0; p.la.fulldeg[tid] = 0;
    }
    if (tid == 0) { p.ctl->flags = 0; p.la.start[0] = 0; p.la.hstart[0] = 0; }
    if (!team.sync()) return false;
    trace_mark(p, TR_INIT, b);
    // init B: sources (block 0): level-0 entries, one per distinct source vertex
    if (p.rank == 0 && threadIdx.x == 0) {
        const int* src = p.src + (size_t)b * K;
        for (int c = 0; c < K; ++c) {
            const int s = src[c];
            if (s < 0) continue;
            ws.cnt_reached += 1;  // the source itself, level 0 of its column
            const uint32_t bit = 1u << (c & 31);
            p.V[(size_t)s * W + (c >> 5)] |= bit;
            p.F[0][(size_t)s * W + (c >> 5)] |= bit;
            p.sig[(size_t)s * K + c] = 1ull;
            if (EXT) p.sig_e[(size_t)s * K + c] = 0;
        }
        for (int c = 0; c < K; ++c) {
            const int s = src[c];
            if (s < 0) continue;
            bool first = true;
            for (int c2 = 0; c2 < c; ++c2)
                if (src[c2] == s) { first = false; break; }
            if (!first) continue;
            uint32_t m[W];
            load_mask<W>(p.F[0], s, m);
            const long long deg = p.off[s + 1] - p.off[s];
            if (s < p.n_heavy) {
                const int i = p.la.hcnt[0]++;
                p.hent[i] = s;
                store_mask_full<W>(p.hmask, i, m);
            } else {
                const int i = p.la.cnt[0]++;
                p.ent[i] = s;
                store_mask_full<W>(p.emask, i, m);
            }
            p.la.dsum[0] += deg;
        }
    }
    if (!team.sync()) return false;
    trace_mark(p, TR_INIT, b);

    // forward sweep
    int it = 0;
    for (;; ++it) {
        const int nf = p.la.cnt[it] + p.la.hcnt[it];
        if (nf == 0) break;
        if ((long long)p.la.start[it] + p.la.cnt[it] > p.cap || (long long)p.la.hstart[it] + p.la.hcnt[it] > p.hcap) {
            // the level lists overflowed their capacity: every block sees the same
            // counts and leaves; the host reruns the call with full capacity
            if (lead()) atomicOr(&p.gctl->err, ERR_CAPACITY);
            return false;
        }
        if (it + 1 > kMaxLevel || it + 3 > p.level_slots) {
            if (lead()) atomicOr(&p.gctl->err, ERR_LIMIT);
            return false;
        }
        // the direction and the next level's start offsets: every block's first
        // thread takes the same decision and writes the same values itself, so
        // its own warps read them after the block-wide barrier below
        if (threadIdx.x == 0) {
            s_full += p.la.fulldeg[it];
            const long long mf = p.la.dsum[it];
            const long long mu = p.m_nz - s_full;
            bool pl = s_pull != 0;
            if (p.direction == 1) pl = false;
            else if (p.direction == 2) pl = true;
            else if (!pl) pl = (double)mf * p.alpha > (double)mu;
            else pl = !((double)nf * p.beta < (double)p.n_nz && (double)mf * p.alpha < (double)mu);
            s_pull = pl;
            p.la.start[it + 1] = p.la.start[it] + p.la.cnt[it];
            p.la.hstart[it + 1] = p.la.hstart[it] + p.la.hcnt[it];
            if (p.rank == 0) atomicAdd(pl ? &p.gctl->pull_levels : &p.gctl->push_levels, 1);
        }
        if (p.rank == 0 && threadIdx.x == 1 && it + 2 < p.level_slots) {
            p.la.cnt[it + 2] = 0; p.la.hcnt[it + 2] = 0; p.la.dsum[it + 2] = 0; p.la.fulldeg[it + 2] = 0;
        }
        __syncthreads();
        // read before the phases: the first thread rewrites it only after the
        // team barrier that ends this level
        const bool pull = s_pull != 0;
        if (pull) {
            phase_pull<K, EXT>(p, it, ph++, act, ws, group());
        } else {
            if (p.la.hcnt[it] > 0) {  // chunk prefix of the heavy frontier entries
                heavy_prefix(p, it);
                if (!team.sync()) return false;
                trace_mark(p, TR_PREFIX, it);
            }
            phase_push<K, EXT>(p, it, ph++, ws, group());
            if (!team.sync()) return false;
            trace_mark(p, TR_PUSH, it);
            if (p.la.hcnt[it + 1] > 0) {
                heavy_prefix(p, it + 1);
                if (!team.sync()) return false;
                trace_mark(p, TR_PREFIX, it + 1);
            }
            phase_sigma<K, EXT>(p, it, ph++, act, ws, group());
        }
        if (!team.sync()) return false;
        trace_mark(p, pull ? TR_PULL : TR_SIGMA, it);
        if (*(volatile int*)&p.ctl->flags & BST_NEED_EXT) break;
    }
    const int L = it - 1;  // deepest nonempty level
    if (!EXT && (*(volatile int*)&p.ctl->flags & BST_NEED_EXT)) {
        if (lead()) p.batch_status[b] = BST_NEED_EXT;
        if (!bc_turn_wait(p, team, b)) return false;
        bc_turn_pass(p, b);
        return team.sync();
    }
    if (lead()) atomicMax(&p.gctl->max_levels, L + 1);
    if (p.forward_only) {
        if (lead()) {
            p.batch_status[b] = BST_DONE | (p.ctl->flags & BST_INEXACT);
            p.gctl->last_levels = L + 1;
        }
        if (!bc_turn_wait(p, team, b)) return false;
        bc_turn_pass(p, b);
        return team.sync();
    }
    // the forward sweep leaves buffer L%3 = level L masks, the others zero
    for (int l = L; l >= 1; --l) {
        if (p.la.hcnt[l] > 0) {
            heavy_prefix(p, l);
            if (!team.sync()) return false;
            trace_mark(p, TR_PREFIX, l);
        }
        phase_back<K, EXT>(p, l, ph++, ws, group());
        if (!team.sync()) return false;
        trace_mark(p, TR_BACK, l);
    }
    // batches add into BC in batch order, whichever team ran them
    if (!bc_turn_wait(p, team, b)) return false;
    phase_bc<K, EXT>(p, b);
    if (lead()) p.batch_status[b] = BST_DONE | (p.ctl->flags & BST_INEXACT);
    const bool ok = team.sync();
    bc_turn_pass(p, b);
    trace_mark(p, TR_BC, b);
    return ok;
}

template <typename T>
__device__ __forceinline__ void shift_ptr(T*& ptr, long long d) {
    if (ptr) ptr = reinterpret_cast<T*>(reinterpret_cast<char*>(ptr) + d);
}

// The team view of the parameters: every per-team array moved to this team's slice.
__device__ void make_team_view(KParams& t, const KParams& p) {
    t = p;
    t.team = blockIdx.x / p.team_blocks;
    t.rank = blockIdx.x % p.team_blocks;
    const long long d = (long long)t.team * p.team_bytes;
    shift_ptr(t.V, d);
    shift_ptr(t.F[0], d);
    shift_ptr(t.F[1], d);
    shift_ptr(t.F[2], d);
    shift_ptr(t.sig, d);
    shift_ptr(t.sig_e, d);
    shift_ptr(t.rho, d);
    shift_ptr(t.rho_e, d);
    shift_ptr(t.ent, d);
    shift_ptr(t.emask, d);
    shift_ptr(t.hent, d);
    shift_ptr(t.hmask, d);
    shift_ptr(t.hpre, d);
    shift_ptr(t.scr_v, d);
    shift_ptr(t.scr_e, d);
    shift_ptr(t.scr_or, d);
    shift_ptr(t.arr, d);
    shift_ptr(t.stamp, d);
    shift_ptr(t.la.cnt, d);
    shift_ptr(t.la.hcnt, d);
    shift_ptr(t.la.start, d);
    shift_ptr(t.la.hstart, d);
    shift_ptr(t.la.dsum, d);
    shift_ptr(t.la.fulldeg, d);
    shift_ptr(t.la.hchunks, d);
    shift_ptr(t.ctl, d);
}

template <int K, bool EXT>
__global__ void __launch_bounds__(kThreads, 3) bc_persistent(KParams p) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ KParams tv;
    WarpSmem<K, EXT>* wsm = reinterpret_cast<WarpSmem<K, EXT>*>(smem_raw);
    __shared__ GridTeam team;  // in shared memory: no registers held across the phases
    if (threadIdx.x == 0) {
        make_team_view(tv, p);
        team = GridTeam{tv.ctl, tv.gctl, tv.team_blocks, tv.budget};
    }
    __syncthreads();
    int ph = 0;
    WarpSmem<K, EXT>& ws = wsm[warp_id()];
    if (lane_id() == 0) {
        ws.cnt_dag = 0;
        ws.cnt_reached = 0;
        ws.mph = 0;
        ws.berr = 0;
        // the staged-row slots' completion barriers (one arrival each: the issuing lane)
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"((unsigned)__cvta_generic_to_shared(&ws.mbar[0])) : "memory");
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"((unsigned)__cvta_generic_to_shared(&ws.mbar[1])) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncwarp();
    for (int b = tv.team; b < tv.nbatch; b += tv.nteams)
        if (!run_batch<K, EXT>(tv, b, team, ph, ws)) return;
    __syncwarp();
    if (lane_id() == 0) {
        if (ws.cnt_dag) atomicAdd(&tv.gctl->dag_pairs, ws.cnt_dag);
        if (ws.cnt_reached) atomicAdd(&tv.gctl->reached_pairs, ws.cnt_reached);
        if (ws.berr) atomicOr(&tv.gctl->err, ERR_INTERNAL);
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

// Levels and path counts of column 0 after a forward-only run (one block):
// every entry of level l (light then heavy lists) with bit 0 set.
__global__ void k_debug_extract(KParams p, int K, int levels, int* level_rel, unsigned long long* sig_rel,
                                int* sige_rel) {
    const int W = K >= 32 ? K / 32 : 1;
    for (long long v = threadIdx.x; v < p.n; v += blockDim.x) {
        level_rel[v] = -1;
        sig_rel[v] = 0;
        sige_rel[v] = 0;
    }
    __syncthreads();
    for (int l = 0; l < levels; ++l) {
        const int s = p.la.start[l], c = p.la.cnt[l], hs = p.la.hstart[l], hc = p.la.hcnt[l];
        for (long long i = threadIdx.x; i < c + hc; i += blockDim.x) {
            const int v = i < c ? p.ent[s + i] : p.hent[hs + (i - c)];
            const uint32_t w0 = i < c ? p.emask[(size_t)(s + i) * W] : p.hmask[(size_t)(hs + i - c) * W];
            if (w0 & 1u) {
                level_rel[v] = l;
                sig_rel[v] = p.sig[(size_t)v * K];
                sige_rel[v] = p.ext ? p.sig_e[(size_t)v * K] : 0;
            }
        }
        __syncthreads();
    }
}

// Multi-source BFS output of one batch (after a forward-only traversal), in
// two coalesced passes.  (1) k_bfs_levels: one warp per level-list entry
// (vertex v, columns at level l) writes l into the relabelled table
// lvl[v][c] (uint16, 0xFFFF = unreached), lanes mapped to columns.
// (2) k_bfs_rows: one warp per 32 consecutive original ids u; lane i reads
// the table row and path-count row of v = inv[u0 + i] a slice at a time and
// the warp writes each column's 32 values as one contiguous run of row c of
// the [ncols][n] outputs.
__global__ void k_bfs_levels(KParams p, int K, int levels, unsigned short* lvl) {
    const int W = K >= 32 ? K / 32 : 1;
    const int lane = threadIdx.x & 31;
    const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
    const long long wid = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    for (int l = 0; l < levels; ++l) {
        const long long s = p.la.start[l], c = p.la.cnt[l], hs = p.la.hstart[l], hc = p.la.hcnt[l];
        for (long long i = wid; i < c + hc; i += nw) {
            const int v = i < c ? p.ent[s + i] : p.hent[hs + (i - c)];
            const uint32_t* m = i < c ? p.emask + (size_t)(s + i) * W : p.hmask + (size_t)(hs + (i - c)) * W;
            for (int col = lane; col < K; col += 32)
                if ((m[col >> 5] >> (col & 31)) & 1u) lvl[(size_t)v * K + col] = (unsigned short)l;
        }
    }
}

__global__ void k_bfs_rows(KParams p, int K, int ncols, const unsigned short* __restrict__ lvl,
                           const int* __restrict__ inv, long long n, int* level_out, double* sig_out, int* exp_out) {
    const int lane = threadIdx.x & 31;
    const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
    const long long tiles = (n + 31) / 32;
    for (long long t = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5; t < tiles; t += nw) {
        const long long u = t * 32 + lane;
        const bool ok = u < n;
        const long long v = ok ? inv[u] : 0;
        for (int c0 = 0; c0 < ncols; c0 += 8) {
            unsigned short l8[8];
            unsigned long long s8[8];
            int e8[8];
            if (K % 8 == 0 && ok) {
                // the 8 columns of the row slice with 16-byte reads (rows are
                // K * 2 and K * 8 bytes, K a multiple of 8); path counts of
                // unreached columns are read but not used
                const uint4 lv = *reinterpret_cast<const uint4*>(lvl + (size_t)v * K + c0);
                const unsigned int w4[4] = {lv.x, lv.y, lv.z, lv.w};
#pragma unroll
                for (int k = 0; k < 8; ++k) {
                    l8[k] = c0 + k < ncols ? (unsigned short)(w4[k >> 1] >> (16 * (k & 1))) : (unsigned short)0xFFFFu;
                    e8[k] = 0;
                    s8[k] = 0ull;
                }
                if (sig_out) {
                    const ulonglong2* sp = reinterpret_cast<const ulonglong2*>(p.sig + (size_t)v * K + c0);
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        const ulonglong2 x = sp[k];
                        s8[2 * k] = x.x;
                        s8[2 * k + 1] = x.y;
                    }
                    if (p.ext)
#pragma unroll
                        for (int k = 0; k < 8; ++k) e8[k] = p.sig_e[(size_t)v * K + c0 + k];
                }
            } else {
#pragma unroll
                for (int k = 0; k < 8; ++k) {
                    const int c = c0 + k;
                    l8[k] = 0xFFFFu;
                    s8[k] = 0ull;
                    e8[k] = 0;
                    if (ok && c < ncols) {
                        l8[k] = lvl[(size_t)v * K + c];
                        if (sig_out && l8[k] != 0xFFFFu) {
                            s8[k] = p.sig[(size_t)v * K + c];
                            if (p.ext) e8[k] = p.sig_e[(size_t)v * K + c];
                        }
                    }
                }
            }
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                const int c = c0 + k;
                if (!ok || c >= ncols) continue;
                const size_t o = (size_t)c * (size_t)n + (size_t)u;
                level_out[o] = l8[k] == 0xFFFFu ? -1 : (int)l8[k];
                if (sig_out) {
                    const unsigned long long sv = l8[k] == 0xFFFFu ? 0ull : s8[k];
                    if (exp_out) {
                        int e = 0;
                        sig_out[o] = frexp((double)sv, &e);
                        exp_out[o] = sv ? e + e8[k] : 0;
                    } else {
                        sig_out[o] = e8[k] ? ldexp((double)sv, e8[k]) : (double)sv;
                    }
                }
            }
        }
    }
}

// One status word per launch: Ctl error bits << 8 | OR of the batch status
// bits | 0x80 when a batch neither finished nor asked for the extended form.
__global__ void k_collect_status(const Ctl* ctl, const int* bstat, int nbatch, int* out) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    int flags = 0;
    for (int b = 0; b < nbatch; ++b) {
        const int x = bstat[b];
        flags |= x;
        if (!(x & (BST_DONE | BST_NEED_EXT))) flags |= 0x80;
    }
    *out = (ctl->err << 8) | flags;
}

// ------------------------------------------------------------------ host launchers
template <int K, bool EXT>
static size_t smem_bytes() { return sizeof(WarpSmem<K, EXT>) * kWarps; }

template <int K, bool EXT>
static cudaError_t prepare() {
    static bool done = false;  // attribute set once per process (single device)
    if (done) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(bc_persistent<K, EXT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem_bytes<K, EXT>());
    if (e == cudaSuccess) done = true;
    return e;
}

template <int K, bool EXT>
static cudaError_t launch_k(const KParams& p, int blocks, cudaStream_t st) {
    cudaError_t e = prepare<K, EXT>();
    if (e != cudaSuccess) return e;
    // cooperative launch (all blocks co-resident) through the attribute form,
    // which stream capture records into a CUDA graph
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(blocks);
    cfg.blockDim = dim3(kThreads);
    cfg.dynamicSmemBytes = smem_bytes<K, EXT>();
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, bc_persistent<K, EXT>, p);
}

cudaError_t launch_batches(int K, const KParams& p, int blocks, cudaStream_t st) {
    const bool ext = p.ext != 0;
    switch (K) {
        case 1: return ext ? launch_k<1, true>(p, blocks, st) : launch_k<1, false>(p, blocks, st);
        case 32: return ext ? launch_k<32, true>(p, blocks, st) : launch_k<32, false>(p, blocks, st);
        case 64: return ext ? launch_k<64, true>(p, blocks, st) : launch_k<64, false>(p, blocks, st);
        case 128: return ext ? launch_k<128, true>(p, blocks, st) : launch_k<128, false>(p, blocks, st);
        default: return cudaErrorInvalidValue;
    }
}

template <int K, bool EXT>
static int occ() {
    if (prepare<K, EXT>() != cudaSuccess) return 0;
    int nb = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, bc_persistent<K, EXT>, kThreads, smem_bytes<K, EXT>());
    return nb;
}

int max_coop_blocks(int K, bool ext, int* per_sm) {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    int nb = 0;
    switch (K) {
        case 1: nb = ext ? occ<1, true>() : occ<1, false>(); break;
        case 32: nb = ext ? occ<32, true>() : occ<32, false>(); break;
        case 64: nb = ext ? occ<64, true>() : occ<64, false>(); break;
        case 128: nb = ext ? occ<128, true>() : occ<128, false>(); break;
    }
    if (per_sm) *per_sm = nb;
    return nb * sms;
}

// Zero every team's control block and chunk arrival counters.
__global__ void k_team_reset(char* ctl0, char* arr0, long long team_bytes, int nteams, int arr_ints) {
    const int t = blockIdx.x;
    if (t >= nteams) return;
    int* c = reinterpret_cast<int*>(ctl0 + (long long)t * team_bytes);
    for (int i = threadIdx.x; i < (int)(sizeof(Ctl) / sizeof(int)); i += blockDim.x) c[i] = 0;
    int* a = reinterpret_cast<int*>(arr0 + (long long)t * team_bytes);
    for (int i = threadIdx.x; i < arr_ints; i += blockDim.x) a[i] = 0;
}

cudaError_t launch_team_reset(Ctl* ctl0, int* arr0, long long team_bytes, int nteams, int arr_ints, cudaStream_t st) {
    if (nteams <= 0) return cudaSuccess;
    k_team_reset<<<nteams, 256, 0, st>>>(reinterpret_cast<char*>(ctl0), reinterpret_cast<char*>(arr0), team_bytes,
                                         nteams, arr_ints);
    return cudaGetLastError();
}

cudaError_t launch_collect_status(const Ctl* ctl, const int* bstat, int nbatch, int* out, cudaStream_t st) {
    k_collect_status<<<1, 32, 0, st>>>(ctl, bstat, nbatch, out);
    return cudaGetLastError();
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

cudaError_t launch_bfs_extract(const KParams& p, int K, int levels, int ncols, const int* inv, long long n,
                               unsigned short* lvl, int* level_out, double* sig_out, int* exp_out, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int blocks = 8 * (sms > 0 ? sms : 1);
    cudaError_t e = cudaMemsetAsync(lvl, 0xFF, sizeof(unsigned short) * (size_t)n * (size_t)K, st);
    if (e != cudaSuccess) return e;
    if (levels > 0) k_bfs_levels<<<blocks, 256, 0, st>>>(p, K, levels, lvl);
    k_bfs_rows<<<blocks, 256, 0, st>>>(p, K, ncols, lvl, inv, n, level_out, sig_out, exp_out);
    return cudaGetLastError();
}

// Source grouping keys: keys[i][j] = level of source i (original id src[i])
// in the BFS of column j, read from the relabelled level table lvl[n][K];
// 0xFFFF for unreached vertices and for ids outside [0, n) (the traversal's
// own source check reports those).
__global__ void k_level_keys(const unsigned short* __restrict__ lvl, int K, int L, const int* __restrict__ src,
                             int nsrc, const int* __restrict__ inv, long long n, unsigned short* keys) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (long long)nsrc * L) return;
    const int s = src[i / L], j = (int)(i % L);
    keys[i] = (s >= 0 && s < n) ? lvl[(size_t)inv[s] * K + j] : (unsigned short)0xFFFFu;
}

cudaError_t launch_level_table(const KParams& p, int K, int levels, unsigned short* lvl, long long n,
                               cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaError_t e = cudaMemsetAsync(lvl, 0xFF, sizeof(unsigned short) * (size_t)n * (size_t)K, st);
    if (e != cudaSuccess) return e;
    if (levels > 0) k_bfs_levels<<<8 * (sms > 0 ? sms : 1), 256, 0, st>>>(p, K, levels, lvl);
    return cudaGetLastError();
}

cudaError_t launch_source_keys(const unsigned short* lvl, int K, int L, long long n, const int* src, int nsrc,
                               const int* inv, unsigned short* keys, cudaStream_t st) {
    if (n <= 0 || nsrc <= 0) return cudaSuccess;
    const long long tot = (long long)nsrc * L;
    k_level_keys<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(lvl, K, L, src, nsrc, inv, n, keys);
    return cudaGetLastError();
}

cudaError_t launch_debug_extract(const KParams& p, int K, int levels, int* level_rel, unsigned long long* sig_rel,
                                 int* sige_rel, cudaStream_t st) {
    if (p.n <= 0) return cudaSuccess;
    k_debug_extract<<<1, 1024, 0, st>>>(p, K, levels, level_rel, sig_rel, sige_rel);
    return cudaGetLastError();
}

}  // namespace bcx
