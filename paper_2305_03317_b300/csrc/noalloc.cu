// bc_compute_noalloc: the batched BC computation for callers that cannot
// allocate device memory.
//
// Who needs it: code that runs inside a host framework which owns all device
// memory through its own pool and forbids any other allocation (to keep a hard
// memory cap or to avoid the allocator's implicit synchronisation), and code
// on latency-critical paths that must not enter the CUDA allocator at all.
// Such a caller passes its CSR, sources and output already on the device; all
// working state of the computation lives in one statically sized device array
// defined in this file, so the call itself allocates nothing.
//
// Limits (checked before any device work): n <= kNaMaxN vertices, the CSR in
// int32 with m < 2^31; batches of 32 sources.  The graph is used as given (no
// relabelling); offsets and index range are checked on the device, symmetry,
// self-loops and duplicates are not.  The array is shared by every call in
// the process and keeps the previous call's contents: each call clears what
// must start at zero, and two calls that overlap on the GPU race on it.
#include <cuda_runtime.h>

#include <cstring>

#include "../../include/bc.h"
#include "bc_internal.cuh"

using namespace bcx;

namespace {

constexpr int kNaK = 32;                      // sources per traversal
constexpr long long kNaMaxN = 32768;          // vertices
constexpr long long kNaMaxBatches = 2048;     // batches per launch (65536 sources)
constexpr size_t kAlign = 256;

constexpr size_t up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

// Region sizes for n = kNaMaxN at width 32 (one mask word per vertex).
constexpr size_t kV = up(sizeof(uint32_t) * kNaMaxN);
constexpr size_t kSig = up(sizeof(unsigned long long) * kNaMaxN * kNaK);
constexpr size_t kSigE = up(sizeof(int) * kNaMaxN * kNaK);
constexpr size_t kEnt = up(sizeof(int) * kNaMaxN * kNaK);       // level-list capacity n * K
constexpr size_t kSmallK = up(sizeof(unsigned long long) * kNaK);
constexpr size_t kLvlI = up(sizeof(int) * kLevelSlots);
constexpr size_t kLvlL = up(sizeof(long long) * kLevelSlots);
constexpr size_t kCtl = up(sizeof(Ctl));
constexpr size_t kBst = up(sizeof(int) * kNaMaxBatches);
constexpr size_t kSrc = up(sizeof(int) * kNaMaxBatches * kNaK);
constexpr size_t kMisc = up(64);

// offsets of each region
constexpr size_t oV = 0;
constexpr size_t oF0 = oV + kV;
constexpr size_t oF1 = oF0 + kV;
constexpr size_t oF2 = oF1 + kV;
constexpr size_t oSig = oF2 + kV;
constexpr size_t oRho = oSig + kSig;
constexpr size_t oSigE = oRho + kSig;
constexpr size_t oRhoE = oSigE + kSigE;
constexpr size_t oEnt = oRhoE + kSigE;
constexpr size_t oEmask = oEnt + kEnt;
constexpr size_t oStamp = oEmask + kEnt;
constexpr size_t oHent = oStamp + kV;
constexpr size_t oHmask = oHent + kSmallK;
constexpr size_t oHpre = oHmask + kSmallK;
constexpr size_t oScrV = oHpre + kSmallK;
constexpr size_t oScrE = oScrV + kSmallK;
constexpr size_t oScrOr = oScrE + kSmallK;
constexpr size_t oArr = oScrOr + kSmallK;
constexpr size_t oHcum = oArr + kMisc;
constexpr size_t oCnt = oHcum + kMisc;
constexpr size_t oHcnt = oCnt + kLvlI;
constexpr size_t oStart = oHcnt + kLvlI;
constexpr size_t oHstart = oStart + kLvlI;
constexpr size_t oHchunks = oHstart + kLvlI;
constexpr size_t oDsum = oHchunks + kLvlI;
constexpr size_t oFull = oDsum + kLvlL;
constexpr size_t oCtl = oFull + kLvlL;
constexpr size_t oBst = oCtl + kCtl;
constexpr size_t oSrc = oBst + kBst;
constexpr size_t oJob = oSrc + kSrc;
constexpr size_t oFlags = oJob + kMisc;
constexpr size_t kScratchBytes = oFlags + kMisc;  // about 37 MB

enum : int { NA_BAD_OFFSETS = 1, NA_BAD_INDEX = 2, NA_BAD_SOURCE = 4 };

}  // namespace

// The working state of every bc_compute_noalloc call (see the file comment).
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

namespace {

// flags[0]: NA_* bits; flags[1]: the longest row (arcs), which bounds every
// path-count sum (rows are summed whole here, and a row may repeat an arc).
__global__ void k_na_check_csr(const int* off, const int* adj, int n, long long m, int* flags) {
    const long long nthr = (long long)gridDim.x * blockDim.x;
    const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (tid == 0 && (off[0] != 0 || (long long)off[n] != m)) atomicOr(flags, NA_BAD_OFFSETS);
    int longest = 0;
    for (long long v = tid; v < n; v += nthr) {
        const int d = off[v + 1] - off[v];
        if (d < 0) atomicOr(flags, NA_BAD_OFFSETS);
        else longest = d > longest ? d : longest;
    }
    if (longest > 0) atomicMax(flags + 1, longest);
    for (long long e = tid; e < m; e += nthr) {
        const int w = adj[e];
        if (w < 0 || w >= n) atomicOr(flags, NA_BAD_INDEX);
    }
}

// Sources of one launch into the [batch][32] column table (-1 pads the last batch).
__global__ void k_na_sources(const int* src, int count, int total, int n, int* dst, int* flags) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= total) return;
    int s = -1;
    if (i < count) {
        s = src[i];
        if (s < 0 || s >= n) {
            atomicOr(flags, NA_BAD_SOURCE);
            s = -1;
        }
    }
    dst[i] = s;
}

__global__ void k_na_job(double** slot, double* out) { *slot = out; }

// Device address of the scratch array on the current device.  Host code
// cannot use the symbol's name as a device pointer, so every call asks the
// runtime (with the caller's device current) instead of caching the address:
// after cudaDeviceReset the module is loaded again and the array may move.
cudaError_t scratch_address(unsigned char** out) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    *out = (unsigned char*)p;
    return cudaSuccess;
}

// Bits of x (0 for 0): a sum of x terms below 2^(64 - na_bits(x)) fits 64 bits.
int na_bits(unsigned long long x) {
    int b = 0;
    while (x) {
        ++b;
        x >>= 1;
    }
    return b;
}

bc_status na_fail(bc_status st, const char* msg) {
    set_last_error(msg);  // reported by bc_last_error() on this thread
    return st;
}

}  // namespace

extern "C" bc_status bc_compute_noalloc(const int32_t* offsets, const int32_t* indices, int32_t n, int64_t m,
                                        const int32_t* sources, int32_t nsrc, double* out_bc, bc_stream_t stream) {
    if (n < 0 || m < 0 || nsrc < 0) return na_fail(BC_E_INVALID_ARG, "negative size");
    if (n > kNaMaxN) return na_fail(BC_E_LIMIT, "bc_compute_noalloc: more vertices than its static scratch holds (32768)");
    if (m >= (1ll << 31) - 1) return na_fail(BC_E_LIMIT, "bc_compute_noalloc: m beyond int32 CSR");
    if (!offsets || (m > 0 && !indices) || (n > 0 && !out_bc) || (nsrc > 0 && !sources))
        return na_fail(BC_E_INVALID_ARG, "NULL pointer");
    cudaStream_t st = (cudaStream_t)stream;
    unsigned char* base = nullptr;
    cudaError_t e = scratch_address(&base);
    if (e != cudaSuccess) return na_fail(BC_E_CUDA, cudaGetErrorString(e));
    int* flags = (int*)(base + oFlags);
    if (n == 0) return BC_OK;

    // the caller's CSR must be safe to index
    if ((e = cudaMemsetAsync(flags, 0, 2 * sizeof(int), st)) != cudaSuccess)
        return na_fail(BC_E_CUDA, cudaGetErrorString(e));
    k_na_check_csr<<<592, 256, 0, st>>>(offsets, indices, n, m, flags);
    int hcheck[2] = {0, 0};
    if ((e = cudaGetLastError()) != cudaSuccess ||
        (e = cudaMemcpyAsync(hcheck, flags, 2 * sizeof(int), cudaMemcpyDeviceToHost, st)) != cudaSuccess ||
        (e = cudaStreamSynchronize(st)) != cudaSuccess)
        return na_fail(BC_E_CUDA, cudaGetErrorString(e));
    if (hcheck[0]) return na_fail(BC_E_INVALID_GRAPH, "offsets not monotone or an index outside [0, n)");
    int hflags = 0;

    KParams p;
    memset(&p, 0, sizeof p);
    p.n = n;
    p.n_nz = n;       // no relabelling: isolated vertices stay where they are
    p.n_heavy = 0;    // every row runs on the grouped path
    p.first_leaf = n; // no relabelling: degree-1 rows are not a suffix, none is left out
    p.m_nz = m;
    p.off = offsets;
    p.adj = indices;
    p.src = (const int*)(base + oSrc);
    p.V = (uint32_t*)(base + oV);
    p.F[0] = (uint32_t*)(base + oF0);
    p.F[1] = (uint32_t*)(base + oF1);
    p.F[2] = (uint32_t*)(base + oF2);
    p.sig = (unsigned long long*)(base + oSig);
    p.rho = (double*)(base + oRho);
    p.sig_e = (int*)(base + oSigE);
    p.rho_e = (int*)(base + oRhoE);
    p.ent = (int*)(base + oEnt);
    p.emask = (uint32_t*)(base + oEmask);
    p.hent = (int*)(base + oHent);
    p.hmask = (uint32_t*)(base + oHmask);
    p.hpre = (int*)(base + oHpre);
    p.cap = (long long)n * kNaK;
    p.hcap = kNaK;
    p.hcum = (const int*)(base + oHcum);
    p.scr_v = (unsigned long long*)(base + oScrV);
    p.scr_e = (int*)(base + oScrE);
    p.scr_or = (uint32_t*)(base + oScrOr);
    p.arr = (int*)(base + oArr);
    p.stamp = (int*)(base + oStamp);
    p.la.cnt = (int*)(base + oCnt);
    p.la.hcnt = (int*)(base + oHcnt);
    p.la.start = (int*)(base + oStart);
    p.la.hstart = (int*)(base + oHstart);
    p.la.hchunks = (int*)(base + oHchunks);
    p.la.dsum = (long long*)(base + oDsum);
    p.la.fulldeg = (long long*)(base + oFull);
    p.ctl = (Ctl*)(base + oCtl);
    p.gctl = p.ctl;  // one team: its control block is the launch-wide one
    p.nteams = 1;
    p.team_bytes = 0;
    p.level_slots = kLevelSlots;
    p.batch_status = (int*)(base + oBst);
    p.job_bc = (double* const*)(base + oJob);
    p.col_job = nullptr;
    p.direction = 0;
    p.alpha = 14.0f;
    p.beta = 24.0f;
    p.budget = 40000000000ll;
    p.group = 32;
    // rows are summed whole (never chunked here), and nothing stops a row from
    // repeating an arc, so the bound comes from the longest row: a sum of
    // `longest` terms below 2^sum_bits cannot wrap 64 bits
    p.sum_bits = 64 - na_bits((unsigned long long)(hcheck[1] > 1 ? hcheck[1] : 1));
    p.dense_min = 32;  // batch width 32: only arcs matching every column go column-mapped

    // the output accumulates every batch in source order; the job table points at it
    k_na_job<<<1, 1, 0, st>>>((double**)(base + oJob), out_bc);
    if ((e = cudaMemsetAsync(base + oHcum, 0, kMisc, st)) != cudaSuccess) return na_fail(BC_E_CUDA, cudaGetErrorString(e));

    bool inexact = false;
    for (int ext = 0; ext < 2; ++ext) {
        p.ext = ext;
        if ((e = cudaMemsetAsync(out_bc, 0, sizeof(double) * (size_t)n, st)) != cudaSuccess)
            return na_fail(BC_E_CUDA, cudaGetErrorString(e));
        int per_sm = 0;
        const int blocks = max_coop_blocks(kNaK, ext != 0, &per_sm);
        if (blocks < 1) return na_fail(BC_E_CUDA, "persistent kernel cannot be resident");
        p.team_blocks = blocks;
        bool need_ext = false;
        inexact = false;
        for (long long s0 = 0; s0 < nsrc; s0 += kNaMaxBatches * kNaK) {
            const int count = (int)((nsrc - s0) < kNaMaxBatches * kNaK ? (nsrc - s0) : kNaMaxBatches * kNaK);
            const int nbatch = (count + kNaK - 1) / kNaK;
            const int total = nbatch * kNaK;
            p.nbatch = nbatch;
            if ((e = cudaMemsetAsync(flags, 0, sizeof(int), st)) != cudaSuccess ||
                (e = cudaMemsetAsync(base + oCtl, 0, kCtl, st)) != cudaSuccess ||
                (e = cudaMemsetAsync(base + oBst, 0, sizeof(int) * nbatch, st)) != cudaSuccess ||
                (e = cudaMemsetAsync(base + oArr, 0, kMisc, st)) != cudaSuccess)
                return na_fail(BC_E_CUDA, cudaGetErrorString(e));
            k_na_sources<<<(total + 255) / 256, 256, 0, st>>>(sources + s0, count, total, n, (int*)(base + oSrc), flags);
            if ((e = cudaGetLastError()) != cudaSuccess) return na_fail(BC_E_CUDA, cudaGetErrorString(e));
            if ((e = launch_batches(kNaK, p, blocks, st)) != cudaSuccess) return na_fail(BC_E_CUDA, cudaGetErrorString(e));
            Ctl ctl;
            int bst[kNaMaxBatches];
            if ((e = cudaMemcpyAsync(&hflags, flags, sizeof(int), cudaMemcpyDeviceToHost, st)) != cudaSuccess ||
                (e = cudaMemcpyAsync(&ctl, base + oCtl, sizeof(Ctl), cudaMemcpyDeviceToHost, st)) != cudaSuccess ||
                (e = cudaMemcpyAsync(bst, base + oBst, sizeof(int) * nbatch, cudaMemcpyDeviceToHost, st)) !=
                    cudaSuccess ||
                (e = cudaStreamSynchronize(st)) != cudaSuccess)
                return na_fail(BC_E_CUDA, cudaGetErrorString(e));
            if (hflags & NA_BAD_SOURCE) return na_fail(BC_E_SOURCE, "a source id is outside [0, n)");
            if (ctl.err & ERR_TIMEOUT) return na_fail(BC_E_TIMEOUT, "a grid-barrier wait exceeded its cycle budget");
            if (ctl.err & ERR_LIMIT) return na_fail(BC_E_LIMIT, "BFS deeper than 65534 levels");
            if (ctl.err) return na_fail(BC_E_CUDA, "internal device error");
            for (int b = 0; b < nbatch; ++b) {
                if (bst[b] & BST_NEED_EXT) need_ext = true;
                else if (!(bst[b] & BST_DONE)) return na_fail(BC_E_CUDA, "internal: batch not completed");
                if (bst[b] & BST_INEXACT) inexact = true;
            }
            if (need_ext) break;
        }
        if (!need_ext) return inexact ? BC_W_SIGMA_INEXACT : BC_OK;
        // a path count passed 2^64: redo every batch in the extended form
    }
    return na_fail(BC_E_SIGMA_RANGE, "path count beyond the extended range");
}
