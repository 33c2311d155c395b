// Graphs of large diameter: one source per block.
//
// The same computation as the batched traversal: per source a level-
// synchronous BFS counting shortest paths, then the dependencies accumulated
// level by level in reverse (the BFS and reverse-BFS constructs of Section
// 2.3.2, as the BC program of Appendix A uses them).
//
// A graph like a road network or a grid runs thousands of BFS levels with a
// few thousand vertices each.  The batched traversal (bc_kernels.cu) then
// spends each level on grid-wide phases whose work is a handful of warp tasks
// per warp, so its time is levels x (dependent memory accesses + grid
// barriers).  Here every block runs whole sources on its own, level by level,
// with block barriers only: the levels of all sources in flight advance
// independently, and nothing waits on another block.
//
// State per block and vertex is one 32-byte record (path count, rho, their
// exponents and the level tag), so the neighbour test and the term it selects
// come from one sector, and the records of kWin arcs of a row are loaded
// together before they are used, in CSR order.  Level tags carry an epoch:
// a new source needs no clearing of its block's slice.  The forward sweep
// is one pass per level: each vertex of level l + 1 sums its count over its
// level-l neighbours and, in the same sweep of its row, claims its unseen
// neighbours for level l + 2.
//
// The arithmetic is the batched traversal's, in the same order, so results
// are bit for bit those of bc_compute's batched form:
//   * path counts in the extended form (64-bit mantissa x 2^e, exact and equal
//     to the plain 64-bit counts while below 2^64), summed over the
//     in-neighbours one level up in CSR order; an undirected row above kChunk
//     arcs is summed per kChunk-arc chunk and the chunk sums combined in chunk
//     order (directed graphs sum whole in-rows);
//   * rho = 1/sigma + S, S summed over the out-neighbours one level down in
//     CSR order (chunked the same way for rows above kChunk arcs), and
//     delta = sigma * S, in the extended form's scaling;
//   * BC adds the sources' dependencies in the order of the source list
//     (k_sum_dependency_rows, one thread per vertex).
// Run forward only, the kernel writes each source's levels and path counts
// instead (bc_bfs on deep graphs), converted as the batched extraction does.
#include <cstdint>
#include <cuda_runtime.h>

#include "bc_internal.cuh"

namespace bcx {
namespace {

constexpr int kDeepMaxThreads = 1024;
constexpr int kWin = 4;  // arcs of a row whose records are loaded together (divides kChunk)
static_assert(kChunk % kWin == 0, "windows must not straddle chunks");

__device__ __forceinline__ bool unseen(unsigned tag, unsigned E) { return (tag & 0xFFFF0000u) != E; }

// Path-count view of a record: {tag, se} and sm (one sector).
__device__ __forceinline__ void rec_fwd(const DeepRec* r, unsigned& tag, int& se, unsigned long long& sm) {
    const uint2 q = *reinterpret_cast<const uint2*>(&r->tag);
    tag = q.x;
    se = (int)q.y;
    sm = r->sm;
}

// Claim the vertices u[j] whose tags t[j] read as unseen for level `lv`: the
// compare-and-swaps are issued together, then the winners append themselves
// (with their out-row bounds ob[j]) to the level list.
__device__ __forceinline__ void claim_win(const int (&u)[kWin], const unsigned (&t)[kWin], const int2 (&ob)[kWin],
                                          DeepRec* rec, unsigned E, int lv, int* order, int2* orow, int base,
                                          int* rel) {
    bool won[kWin];
#pragma unroll
    for (int j = 0; j < kWin; ++j)
        won[j] = unseen(t[j], E) && atomicCAS(&rec[u[j]].tag, t[j], E | (unsigned)lv) == t[j];
#pragma unroll
    for (int j = 0; j < kWin; ++j) {
        if (won[j]) {
            const int k = base + atomicAdd(rel, 1);
            order[k] = u[j];
            orow[k] = ob[j];
        }
    }
}

__global__ void __launch_bounds__(kDeepMaxThreads) k_deep(DeepParams p) {
    __shared__ int s_rel[3];  // appends of pass l count in s_rel[l % 3]
    __shared__ int s_flags;
    __shared__ unsigned long long s_dag, s_reached;
    const int tid = threadIdx.x, bd = blockDim.x;
    const long long b = blockIdx.x;
    DeepRec* rec = p.rec + b * p.stride;
    int* order = p.order + b * p.stride;
    int2* orow = p.orow + b * p.stride;
    int* lvl = p.lvl + b * (long long)p.level_slots;
    const bool directed = p.ioff != nullptr;
    if (tid == 0) { s_dag = 0; s_reached = 0; }
    for (int i = blockIdx.x, j = 0; i < p.nsrc; i += gridDim.x, ++j) {
        const unsigned E = (p.epoch0 + (unsigned)j) << 16;
        const int s = p.src[i];
        double* dl = p.delta ? p.delta + (size_t)i * (size_t)p.n : nullptr;
        if (tid == 0) {
            s_rel[0] = s_rel[1] = s_rel[2] = 0;
            s_flags = 0;
            order[0] = s;
            orow[0] = make_int2(p.off[s], p.off[s + 1]);
            rec[s].sm = 1ull;
            rec[s].se = 0;
            rec[s].tag = E;  // level 0
            lvl[0] = 0;
            lvl[1] = 1;
        }
        __syncthreads();
        // level 1: the out-neighbours of the source, one arc per thread
        for (int e = p.off[s] + tid; e < p.off[s + 1]; e += bd) {
            const int w = p.adj[e];
            const unsigned t = rec[w].tag;
            const int2 ob = make_int2(p.off[w], p.off[w + 1]);
            if (unseen(t, E) && atomicCAS(&rec[w].tag, t, E | 1u) == t) {
                const int k = 1 + atomicAdd(&s_rel[2], 1);
                order[k] = w;
                orow[k] = ob;
            }
        }
        __syncthreads();
        int beg = 1, end = 1 + s_rel[2], L = 0;
        if (tid == 0) lvl[2] = end;
        unsigned long long dag = 0;
        bool inexact = false;
        // pass l: the path counts of level l + 1 = order[beg, end), and the
        // claims of level l + 2 among their unseen out-neighbours
        for (int l = 0;; ++l) {
            if (beg == end) {  // level l + 1 is empty: level l is the deepest
                L = l;
                break;
            }
            if (l + 1 >= kMaxLevel) {  // a level beyond kMaxLevel would follow
                if (tid == 0) s_flags = ERR_LIMIT;
                break;
            }
            int* rel = &s_rel[l % 3];
            if (tid == 0) s_rel[(l + 1) % 3] = 0;  // last read after the barrier ending pass l - 2
            const unsigned want = E | (unsigned)l;
            for (int k = beg + tid; k < end; k += bd) {
                const int w = order[k];
                const int2 orw = orow[k];
                const int* __restrict__ radj = directed ? p.iadj : p.adj;
                const int rb = directed ? p.ioff[w] : orw.x;
                const int rend = directed ? p.ioff[w + 1] : orw.y;
                const int step = (!directed && w < p.n_heavy) ? kChunk : (rend - rb);
                unsigned long long am = 0ull;
                int ae = 0;
                for (int c0 = rb; c0 < rend; c0 += step) {
                    const int c1 = c0 + step < rend ? c0 + step : rend;
                    unsigned long long cm = 0ull;
                    int ce = 0;
                    for (int e = c0; e < c1; e += kWin) {
                        int u[kWin];
                        unsigned t[kWin];
                        int se[kWin];
                        unsigned long long sm[kWin];
                        int2 ob[kWin];
#pragma unroll
                        for (int jj = 0; jj < kWin; ++jj) u[jj] = e + jj < c1 ? radj[e + jj] : -1;
#pragma unroll
                        for (int jj = 0; jj < kWin; ++jj) {
                            if (u[jj] >= 0) {
                                rec_fwd(rec + u[jj], t[jj], se[jj], sm[jj]);
                                // out-row bounds, ready in case this arc claims u (undirected rows)
                                ob[jj] = directed ? make_int2(0, 0) : make_int2(p.off[u[jj]], p.off[u[jj] + 1]);
                            } else {
                                t[jj] = E | 0xFFFFu;  // reads as seen, at no level in use
                                se[jj] = 0;
                                sm[jj] = 0ull;
                                ob[jj] = make_int2(0, 0);
                            }
                        }
                        // in CSR order: level-l neighbours add to the count
#pragma unroll
                        for (int jj = 0; jj < kWin; ++jj) {
                            if (t[jj] == want) {
                                xu_add(cm, ce, sm[jj], se[jj]);
                                ++dag;
                            }
                        }
                        // undirected rows are also the out-rows: claim their unseen neighbours
                        if (!directed) claim_win(u, t, ob, rec, E, l + 2, order, orow, end, rel);
                    }
                    xu_add(am, ae, cm, ce);
                }
                if (directed) {
                    for (int e = orw.x; e < orw.y; e += kWin) {
                        int u[kWin];
                        unsigned t[kWin];
                        int2 ob[kWin];
#pragma unroll
                        for (int jj = 0; jj < kWin; ++jj) u[jj] = e + jj < orw.y ? p.adj[e + jj] : -1;
#pragma unroll
                        for (int jj = 0; jj < kWin; ++jj) {
                            t[jj] = u[jj] >= 0 ? rec[u[jj]].tag : E;
                            ob[jj] = u[jj] >= 0 ? make_int2(p.off[u[jj]], p.off[u[jj] + 1]) : make_int2(0, 0);
                        }
                        claim_win(u, t, ob, rec, E, l + 2, order, orow, end, rel);
                    }
                }
                rec[w].sm = am;
                rec[w].se = ae;
                inexact |= (ae > 0 || am >= (1ull << 53));
            }
            __syncthreads();
            const int nend = end + *rel;
            if (tid == 0) lvl[l + 3] = nend;
            beg = end;
            end = nend;
        }
        __syncthreads();  // s_flags and the level starts, for every thread
        if (p.level_out && s_flags == 0) {
            // forward only: the source's row of levels and path counts, in original ids
            const size_t row = (size_t)i * (size_t)p.n;
            for (int u = tid; u < p.n; u += bd) {
                const int v = p.inv[u];
                const unsigned t = rec[v].tag;
                const bool reached = !unseen(t, E);
                p.level_out[row + u] = reached ? (int)(t & 0xFFFFu) : -1;
                if (p.sig_out) {
                    const unsigned long long sv = reached ? rec[v].sm : 0ull;
                    const int ev = reached ? rec[v].se : 0;
                    if (p.exp_out) {
                        int e = 0;
                        p.sig_out[row + u] = frexp((double)sv, &e);
                        p.exp_out[row + u] = sv ? e + ev : 0;
                    } else {
                        p.sig_out[row + u] = ev ? ldexp((double)sv, ev) : (double)sv;
                    }
                }
            }
        }
        // reverse: levels L .. 1
        for (int l = L; l >= 1 && s_flags == 0 && !p.level_out; --l) {
            const int lb = lvl[l], le = lvl[l + 1];
            const unsigned want = E | (unsigned)(l + 1);
            for (int k = lb + tid; k < le; k += bd) {
                const int v = order[k];
                const int2 orv = orow[k];
                const int rb = orv.x, rend = orv.y;
                const unsigned long long smv = rec[v].sm;
                const int sv = rec[v].se;
                double sr = 0.0;
                int sx = 0;
                const int step = v < p.n_heavy ? kChunk : (rend - rb);
                for (int c0 = rb; c0 < rend; c0 += step) {
                    const int c1 = c0 + step < rend ? c0 + step : rend;
                    double cr = 0.0;
                    int cx = 0;
                    for (int e = c0; e < c1; e += kWin) {
                        int w[kWin];
                        unsigned t[kWin];
                        int re[kWin];
                        double rh[kWin];
#pragma unroll
                        for (int jj = 0; jj < kWin; ++jj) w[jj] = e + jj < c1 ? p.adj[e + jj] : -1;
#pragma unroll
                        for (int jj = 0; jj < kWin; ++jj) {
                            if (w[jj] >= 0) {
                                t[jj] = rec[w[jj]].tag;
                                re[jj] = rec[w[jj]].re;
                                rh[jj] = rec[w[jj]].rho;
                            } else {
                                t[jj] = 0u;
                                re[jj] = 0;
                                rh[jj] = 0.0;
                            }
                        }
#pragma unroll
                        for (int jj = 0; jj < kWin; ++jj)
                            if (w[jj] >= 0 && t[jj] == want) xd_add(cr, cx, rh[jj], re[jj]);
                    }
                    xd_add(sr, sx, cr, cx);
                }
                const double sd = (double)smv;  // rounds only when the mantissa is >= 2^53
                dl[v] = scale2(sd * sr, sv + sx);
                rec[v].rho = __drcp_rn(sd) + scale2(sr, sv + sx);
                rec[v].re = -sv;
            }
            __syncthreads();
        }
        if (inexact) atomicOr(&s_flags, BST_INEXACT);
        atomicAdd(&s_dag, dag);
        __syncthreads();
        if (tid == 0) {
            const int f = s_flags;
            p.status[i] = (f & ERR_LIMIT) ? (ERR_LIMIT << 8) : (BST_DONE | (f & BST_INEXACT));
            p.depth[i] = L + 1;
            s_reached += (unsigned long long)end;  // vertices reached, the source included
        }
        __syncthreads();
    }
    if (tid == 0) {
        atomicAdd(p.dag_pairs, s_dag);
        atomicAdd(p.reached_pairs, s_reached);
    }
}

// bc[v] += delta[0][v] + delta[1][v] + ..., added one source at a time in list order.
__global__ void k_sum_dependency_rows(const double* __restrict__ delta, int nsrc, long long n, double* bc) {
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride) {
        double acc = bc[v];
        for (int i = 0; i < nsrc; ++i) acc += delta[(size_t)i * (size_t)n + (size_t)v];
        bc[v] = acc;
    }
}

}  // namespace

cudaError_t launch_deep(const DeepParams& p, int blocks, int threads, cudaStream_t st) {
    if (p.nsrc <= 0) return cudaSuccess;
    if (blocks < 1 || threads < 32 || threads > kDeepMaxThreads || threads % 32) return cudaErrorInvalidValue;
    k_deep<<<blocks, threads, 0, st>>>(p);
    return cudaGetLastError();
}

int deep_blocks_per_sm(int threads) {
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_deep, threads, 0) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return nb;
}

cudaError_t launch_deep_accumulate(const double* delta, int nsrc, long long n, double* bc, cudaStream_t st) {
    if (n <= 0 || nsrc <= 0) return cudaSuccess;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const long long want = (n + 255) / 256, cap = 8LL * (sms > 0 ? sms : 1);
    k_sum_dependency_rows<<<(unsigned)(want < cap ? want : cap), 256, 0, st>>>(delta, nsrc, n, bc);
    return cudaGetLastError();
}

}  // namespace bcx
