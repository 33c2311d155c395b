// Graphs of large diameter: one source per block.
//
// A graph like a road network or a grid runs thousands of BFS levels with a
// few thousand vertices each.  The batched traversal (bc_kernels.cu) then
// spends each level on grid-wide phases whose work is a handful of warp tasks
// per warp, so its time is levels x (dependent memory accesses + grid
// barriers).  Here every block runs whole sources on its own, level by level,
// with block barriers only: the levels of all sources in flight advance
// independently, and nothing waits on another block.
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
//     (k_deep_accumulate, one thread per vertex).
#include <cstdint>
#include <cuda_runtime.h>

#include "bc_internal.cuh"

namespace bcx {
namespace {

constexpr int kDeepMaxThreads = 1024;

// Path count of w (level l + 1): the extended-form sum over the in-row of w
// of the counts at level l, per kChunk-arc chunk when `chunked`.
__device__ __forceinline__ void deep_sigma(const int* __restrict__ rowp, int rb, int rend, bool chunked,
                                           const int* dist, const unsigned long long* sm, const int* se, int l,
                                           unsigned long long& am, int& ae, unsigned long long& dag) {
    const int step = chunked ? kChunk : (rend - rb);
    for (int c0 = rb; c0 < rend; c0 += step) {
        const int c1 = c0 + step < rend ? c0 + step : rend;
        unsigned long long cm = 0ull;
        int ce = 0;
        for (int e = c0; e < c1; ++e) {
            const int u = rowp[e];
            if (dist[u] == l) {
                xu_add(cm, ce, sm[u], se[u]);
                ++dag;
            }
        }
        xu_add(am, ae, cm, ce);
    }
}

__global__ void __launch_bounds__(kDeepMaxThreads) k_deep(DeepParams p) {
    __shared__ int s_rel[3];  // appends of pass l count in s_rel[l % 3]
    __shared__ int s_flags;
    __shared__ unsigned long long s_dag, s_reached;
    const int tid = threadIdx.x, bd = blockDim.x;
    const long long b = blockIdx.x;
    int* dist = p.dist + b * p.stride;
    int* order = p.order + b * p.stride;
    unsigned long long* sm = p.sm + b * p.stride;
    int* se = p.se + b * p.stride;
    double* rho = p.rho + b * p.stride;
    int* re = p.re + b * p.stride;
    int* lvl = p.lvl + b * (long long)p.level_slots;
    const bool directed = p.ioff != nullptr;
    if (tid == 0) { s_dag = 0; s_reached = 0; }
    for (int i = blockIdx.x; i < p.nsrc; i += gridDim.x) {
        const int s = p.src[i];
        double* dl = p.delta + (size_t)i * (size_t)p.n;
        for (int v = tid; v < p.n; v += bd) {
            dist[v] = -1;
            dl[v] = 0.0;
        }
        if (tid == 0) {
            s_rel[0] = s_rel[1] = s_rel[2] = 0;
            s_flags = 0;
        }
        __syncthreads();
        if (tid == 0) {
            order[0] = s;
            dist[s] = 0;
            sm[s] = 1ull;
            se[s] = 0;
            lvl[0] = 0;
            lvl[1] = 1;
        }
        __syncthreads();
        // level 1: the out-neighbours of the source
        for (int e = p.off[s] + tid; e < p.off[s + 1]; e += bd) {
            const int w = p.adj[e];
            if (dist[w] < 0 && atomicCAS(&dist[w], -1, 1) == -1) order[1 + atomicAdd(&s_rel[2], 1)] = w;
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
            for (int k = beg + tid; k < end; k += bd) {
                const int w = order[k];
                const bool chunked = !directed && w < p.n_heavy;
                unsigned long long am = 0ull;
                int ae = 0;
                if (directed) {
                    deep_sigma(p.iadj, p.ioff[w], p.ioff[w + 1], false, dist, sm, se, l, am, ae, dag);
                    for (int e = p.off[w]; e < p.off[w + 1]; ++e) {
                        const int u = p.adj[e];
                        if (dist[u] < 0 && atomicCAS(&dist[u], -1, l + 2) == -1) order[end + atomicAdd(rel, 1)] = u;
                    }
                } else {
                    // one sweep of the row: level-l neighbours add to the count,
                    // unseen ones are claimed for level l + 2
                    const int rb = p.off[w], rend = p.off[w + 1];
                    const int step = chunked ? kChunk : (rend - rb);
                    for (int c0 = rb; c0 < rend; c0 += step) {
                        const int c1 = c0 + step < rend ? c0 + step : rend;
                        unsigned long long cm = 0ull;
                        int ce = 0;
                        for (int e = c0; e < c1; ++e) {
                            const int u = p.adj[e];
                            const int du = dist[u];
                            if (du == l) {
                                xu_add(cm, ce, sm[u], se[u]);
                                ++dag;
                            } else if (du < 0 && atomicCAS(&dist[u], -1, l + 2) == -1) {
                                order[end + atomicAdd(rel, 1)] = u;
                            }
                        }
                        xu_add(am, ae, cm, ce);
                    }
                }
                sm[w] = am;
                se[w] = ae;
                inexact |= (ae > 0 || am >= (1ull << 53));
            }
            __syncthreads();
            const int nend = end + *rel;
            if (tid == 0) lvl[l + 3] = nend;
            beg = end;
            end = nend;
        }
        __syncthreads();  // s_flags and the level starts, for every thread
        // reverse: levels L .. 1
        for (int l = L; l >= 1 && s_flags == 0; --l) {
            const int lb = lvl[l], le = lvl[l + 1];
            for (int k = lb + tid; k < le; k += bd) {
                const int v = order[k];
                const int rb = p.off[v], rend = p.off[v + 1];
                double sr = 0.0;
                int sx = 0;
                const int step = v < p.n_heavy ? kChunk : (rend - rb);
                for (int c0 = rb; c0 < rend; c0 += step) {
                    const int c1 = c0 + step < rend ? c0 + step : rend;
                    double cr = 0.0;
                    int cx = 0;
                    for (int e = c0; e < c1; ++e) {
                        const int w = p.adj[e];
                        if (dist[w] == l + 1) xd_add(cr, cx, rho[w], re[w]);
                    }
                    xd_add(sr, sx, cr, cx);
                }
                const double sd = (double)sm[v];  // rounds only when the mantissa is >= 2^53
                const int sv = se[v];
                dl[v] = scalbn(sd * sr, sv + sx);
                rho[v] = __drcp_rn(sd) + scalbn(sr, sv + sx);
                re[v] = -sv;
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
__global__ void k_deep_accumulate(const double* __restrict__ delta, int nsrc, long long n, double* bc) {
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
    k_deep_accumulate<<<(unsigned)(want < cap ? want : cap), 256, 0, st>>>(delta, nsrc, n, bc);
    return cudaGetLastError();
}

}  // namespace bcx
