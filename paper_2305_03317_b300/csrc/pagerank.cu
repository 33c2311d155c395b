// PageRank on the resident graph: the paper's computePR program (Appendix A,
// PR listing).  Every rank starts at 1/n; a sweep forms for each vertex v
//     val(v) = (1 - delta)/n + delta * sum over arcs u -> v of rank(u) / outdeg(u)
// and the change diff = sum over v of |val(v) - rank(v)|; ranks are replaced
// after the sweep, and sweeps repeat while diff > beta and fewer than
// max_iter have run.
//
// One cooperative persistent launch runs every sweep: (1) contributions
// c(u) = rank(u) / outdeg(u); (2) a pull over in-rows (the CSR itself for an
// undirected graph, the transpose for a directed one).  The relabelled rows
// of an undirected graph are sorted by length, so they split into a prefix of
// rows of at least 8192 arcs (2048-arc warp tasks whose sums the row's last
// task adds in chunk order), then rows of at least 32
// (one warp per row) and the rest (one thread per row, CSR order; measured
// faster than 16/8/4/2-lane groups per row); in-rows of
// a directed graph are taken 32 at a time per warp, the long ones summed by
// the whole warp.  Block and warp sums use fixed trees, and each row's
// |change| is added by a fixed thread; block partials go to a slot per block;
// (3) block 0 sums the partials in block order and decides whether to go on.
// Every sum has a fixed order, so results repeat bit for bit.  Grid barriers
// are bounded by the same cycle budget as the traversal kernel.
#include <cstdint>
#include <cuda_runtime.h>

#include "bc_internal.cuh"

namespace bcx {
namespace {

constexpr int kPrThreads = 256;
constexpr unsigned int kAllLanes = 0xffffffffu;

struct PrParams {
    int n;
    const int* off;    // out-adjacency offsets (out-degrees)
    const int* roff;   // in-rows: offsets and sources
    const int* radj;
    double delta, beta;
    int max_iter;
    double* rank;      // [n] current ranks (relabelled ids)
    double* nxt;       // [n]
    double* contrib;   // [n]
    double* partial;   // [gridDim.x]
    Ctl* ctl;          // barrier and error word
    int* iters;        // sweeps run
    double* diff_out;  // last change
    int* go;           // 1 while another sweep follows
    long long budget;
    int n_block_rows;  // sorted rows: [0, n_block_rows) in chunks,
    int n_warp_rows;   // [n_block_rows, n_warp_rows) one warp each, the rest one thread each; -1 = unsorted
    long long nchunks;  // warp tasks of the long rows: chunk slots ccum[r] .. ccum[r+1]
    const int* ccum;
    double* cpart;      // [nchunks] chunk sums
    int* carr;          // [n_block_rows] chunk arrival counters
};

constexpr int kPrChunk = 2048;  // arcs per warp task of a long row

__device__ double block_sum(double x, double* sh) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(kAllLanes, x, o);
    if (lane == 0) sh[wid] = x;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x == 0)
        for (int w = 0; w < kPrThreads / 32; ++w) s += sh[w];
    __syncthreads();
    return s;
}

__global__ void __launch_bounds__(kPrThreads) k_pagerank(PrParams p) {
    __shared__ double sh[kPrThreads / 32];
    GridTeam team{p.ctl, p.ctl, (int)gridDim.x, p.budget};
    const long long nthr = (long long)gridDim.x * blockDim.x;
    const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const int lane = threadIdx.x & 31;
    const long long nwarps = nthr >> 5, wid = tid >> 5;
    const double base = (1.0 - p.delta) / (double)p.n;
    double* rank = p.rank;
    double* nxt = p.nxt;
    for (long long v = tid; v < p.n; v += nthr) rank[v] = 1.0 / (double)p.n;
    if (!team.sync()) return;
    for (int it = 0;; ++it) {
        for (long long u = tid; u < p.n; u += nthr) {
            const int d = p.off[u + 1] - p.off[u];
            p.contrib[u] = d > 0 ? rank[u] / (double)d : 0.0;
        }
        if (!team.sync()) return;
        double mine = 0.0;  // |change| of the rows this lane finished
        if (p.n_warp_rows >= 0) {
            // long rows: 2048-arc warp tasks; a chunk's sum (lane-strided,
            // then a fixed xor tree) goes to its slot, and the warp that
            // finishes a row's last chunk adds the slots in chunk order
            for (long long t = wid; t < p.nchunks; t += nwarps) {
                int lo = 0, hi = p.n_block_rows;  // ccum[lo] <= t < ccum[hi]
                while (hi - lo > 1) {
                    const int mid = (lo + hi) >> 1;
                    if (p.ccum[mid] <= t) lo = mid;
                    else hi = mid;
                }
                const int r = lo, c0 = p.ccum[r], nch = p.ccum[r + 1] - c0;
                const int b = p.roff[r] + (int)(t - c0) * kPrChunk, e = min(p.roff[r + 1], b + kPrChunk);
                double s = 0.0;
                for (int j = b + lane; j < e; j += 32) s += p.contrib[p.radj[j]];
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(kAllLanes, s, o);
                int last = 0;
                if (lane == 0) {
                    p.cpart[t] = s;
                    __threadfence();
                    last = atomicAdd(&p.carr[r], 1) == nch - 1;
                }
                last = __shfl_sync(kAllLanes, last, 0);
                if (last && lane == 0) {
                    __threadfence();
                    double tot = __ldcg(&p.cpart[c0]);
                    for (int k = 1; k < nch; ++k) tot += __ldcg(&p.cpart[c0 + k]);
                    nxt[r] = base + p.delta * tot;
                    p.carr[r] = 0;  // ready for the next sweep (after its barriers)
                }
            }
            for (long long r = p.n_block_rows + wid; r < p.n_warp_rows; r += nwarps) {
                const int b = p.roff[r], l = p.roff[r + 1] - b;
                double s = 0.0;
                for (int e = b + lane; e < b + l; e += 32) s += p.contrib[p.radj[e]];
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(kAllLanes, s, o);
                if (lane == 0) {
                    const double val = base + p.delta * s;
                    mine += fabs(val - rank[r]);
                    nxt[r] = val;
                }
            }
            for (long long v = p.n_warp_rows + tid; v < p.n; v += nthr) {
                const int b = p.roff[v], l = p.roff[v + 1] - b;
                double s = 0.0;
                // four arcs' loads in flight, added in CSR order
                int e = b;
                for (; e + 4 <= b + l; e += 4) {
                    const int u0 = p.radj[e], u1 = p.radj[e + 1], u2 = p.radj[e + 2], u3 = p.radj[e + 3];
                    const double c0 = p.contrib[u0], c1 = p.contrib[u1], c2 = p.contrib[u2], c3 = p.contrib[u3];
                    s += c0;
                    s += c1;
                    s += c2;
                    s += c3;
                }
                for (; e < b + l; ++e) s += p.contrib[p.radj[e]];
                const double val = base + p.delta * s;
                mine += fabs(val - rank[v]);
                nxt[v] = val;
            }
        }
        for (long long g0 = wid * 32; p.n_warp_rows < 0 && g0 < p.n; g0 += nwarps * 32) {
            const long long v = g0 + lane;
            int beg = 0, len = 0;
            if (v < p.n) {
                beg = p.roff[v];
                len = p.roff[v + 1] - beg;
            }
            if (v < p.n && len < 32) {
                double s = 0.0;
                for (int e = beg; e < beg + len; ++e) s += p.contrib[p.radj[e]];
                const double val = base + p.delta * s;
                mine += fabs(val - rank[v]);
                nxt[v] = val;
            }
            unsigned int longs = __ballot_sync(kAllLanes, v < p.n && len >= 32);
            while (longs) {
                const int j = __ffs(longs) - 1;
                longs &= longs - 1;
                const int b = __shfl_sync(kAllLanes, beg, j), l = __shfl_sync(kAllLanes, len, j);
                double s = 0.0;
                for (int e = b + lane; e < b + l; e += 32) s += p.contrib[p.radj[e]];
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(kAllLanes, s, o);
                if (lane == 0) {
                    const long long w = g0 + j;
                    const double val = base + p.delta * s;
                    mine += fabs(val - rank[w]);
                    nxt[w] = val;
                }
            }
        }
        if (p.n_block_rows > 0) {
            // the long rows' changes, once their sums are in, by a fixed thread each
            if (!team.sync()) return;
            for (long long r = tid; r < p.n_block_rows; r += nthr) mine += fabs(nxt[r] - rank[r]);
        }
        const double bs = block_sum(mine, sh);
        if (threadIdx.x == 0) p.partial[blockIdx.x] = bs;
        if (!team.sync()) return;
        if (blockIdx.x == 0 && threadIdx.x == 0) {
            double diff = 0.0;
            for (int b = 0; b < (int)gridDim.x; ++b) diff += *(volatile double*)&p.partial[b];
            *p.diff_out = diff;
            *p.iters = it + 1;
            *(volatile int*)p.go = (diff > p.beta && it + 1 < p.max_iter) ? 1 : 0;
        }
        if (!team.sync()) return;
        double* t = rank;
        rank = nxt;
        nxt = t;
        if (*(volatile int*)p.go == 0) break;
    }
    // the last sweep's ranks end in p.rank
    if (rank != p.rank)
        for (long long v = tid; v < p.n; v += nthr) p.rank[v] = rank[v];
}

}  // namespace

int pagerank_blocks() {
    int dev = 0, sms = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_pagerank, kPrThreads, 0);
    if (per > 8) per = 8;
    return sms * per;
}

cudaError_t launch_pagerank(int n, const int* off, const int* roff, const int* radj, const int* row_class,
                            long long nchunks, const int* ccum, double* cpart, int* carr,
                            double delta, double beta, int max_iter, double* rank, double* scratch, Ctl* ctl, int* iters,
                            double* diff_out, int* go, long long budget, int blocks, cudaStream_t st) {
    PrParams p;
    p.nchunks = row_class ? nchunks : 0;
    p.ccum = ccum;
    p.cpart = cpart;
    p.carr = carr;
    p.n_block_rows = row_class ? row_class[0] : -1;
    p.n_warp_rows = row_class ? row_class[1] : -1;
    p.n = n;
    p.off = off;
    p.roff = roff;
    p.radj = radj;
    p.delta = delta;
    p.beta = beta;
    p.max_iter = max_iter;
    p.rank = rank;
    p.nxt = scratch;
    p.contrib = scratch + n;
    p.partial = scratch + 2 * (size_t)n;
    p.ctl = ctl;
    p.iters = iters;
    p.diff_out = diff_out;
    p.go = go;
    p.budget = budget;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(blocks);
    cfg.blockDim = dim3(kPrThreads);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k_pagerank, p);
}

}  // namespace bcx
