// Internal types shared by the libbc CUDA sources (not part of the C ABI).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace bcx {

constexpr int kChunk = 1024;        // arcs per ordered partial sum (fixed: results depend on it);
                                    // rows longer than this are "heavy" and split into chunk tasks
constexpr int kMaxLevel = 65534;    // levels are uint16; 0xFFFF marks "not reached"
constexpr int kThreads = 256;       // threads per block of the persistent kernels
constexpr int kWarps = kThreads / 32;
constexpr int kLevelSlots = kMaxLevel + 3;
constexpr uint16_t kNoLevel = 0xFFFF;

// Ctl::err bits (fatal for the launch)
enum : int { ERR_TIMEOUT = 1, ERR_SIGMA_RANGE = 2, ERR_LIMIT = 4, ERR_CAPACITY = 8, ERR_INTERNAL = 16 };
// per-batch status bits
enum : int { BST_DONE = 1, BST_INEXACT = 2, BST_NEED_EXT = 4 };
// trace tags: kind << 24 | level (kinds below)
enum : int { TR_INIT = 1, TR_PULL = 2, TR_PUSH = 3, TR_SIGMA = 4, TR_BACK = 5, TR_BC = 6, TR_PREFIX = 7 };

struct Ctl {
    unsigned int bar_count;
    unsigned int bar_gen;
    int err;
    int flags;                 // BST_* bits raised inside the current batch
    unsigned int wq[8];        // dynamic work counters, two per phase slot
    int max_levels;            // deepest BFS over the launch
    int pull_levels;
    int push_levels;
    int last_levels;           // levels of the last batch (debug runs)
    int trace_n;               // pairs written to the trace
    unsigned int bc_next;      // global control: the next batch allowed to add into BC
    int pad[2];
    unsigned long long dag_pairs;      // (arc, column) terms of the forward path-count sums: sum of E_dag(s)
    unsigned long long reached_pairs;  // (vertex, column) pairs reached, sources included: sum of n_s
};

// Level bookkeeping, indexed by BFS level.
struct LevelArrays {
    int* cnt;            // light entries of the level
    int* hcnt;           // heavy entries of the level
    int* start;          // first light entry index
    int* hstart;         // first heavy entry index
    long long* dsum;     // sum of degrees of the level's entries
    long long* fulldeg;  // sum of degrees of vertices whose every column was reached at that level
    int* hchunks;        // number of 1024-arc chunk tasks of the level's heavy entries
};

struct KParams {
    // graph (relabelled: ids sorted by degree descending, heavy rows first, isolated last)
    int n, n_nz, n_heavy;
    // undirected graphs: ids [first_leaf, n_nz) have degree 1 (their one neighbour
    // is their parent, so no successor at any level >= 1); n when not used
    int first_leaf;
    long long m_nz;
    const int* off;
    const int* adj;
    const int* ioff;           // directed graphs: in-CSR (transpose) for the pull steps; null = undirected
    const int* iadj;
    // sources, relabelled, [nbatch][K]; -1 = unused column
    const int* src;
    int nbatch;
    // per-slot state
    uint32_t* V;               // [n][W] reached-column masks
    uint32_t* F[3];            // [n][W] frontier masks of three consecutive levels
    unsigned long long* sig;   // [n][K] path counts (mantissa in the extended form); delta bits after the sweep
    int* sig_e;                // [n][K] extended-form exponent (may be null when ext == 0)
    double* rho;               // [n][K] (1 + delta) / sigma (mantissa in the extended form)
    int* rho_e;                // [n][K]
    int* ent;                  // light level lists (vertex ids), level by level
    uint32_t* emask;           // [cap][W] columns of each light entry at its level
    int* hent;                 // heavy level lists
    uint32_t* hmask;           // [hcap][W]
    int* hpre;                 // [hcap] exclusive chunk prefix within the entry's level
    long long cap, hcap;
    // heavy rows (degree > kChunk): ids [0, n_heavy); chunk slots hcum[r] .. hcum[r+1)
    const int* hcum;           // [n_heavy + 1]
    unsigned long long* scr_v; // [hcum[n_heavy]][K] chunk partial sums
    int* scr_e;                // [hcum[n_heavy]][K] partial exponents (extended form)
    uint32_t* scr_or;          // [hcum[n_heavy]][W] chunk OR of matched masks
    int* arr;                  // [n_heavy] chunk arrival counters (zero between phases)
    int* stamp;                // [n] push-claim stamps
    LevelArrays la;
    Ctl* ctl;                  // this team's control block (barrier, work counters, batch flags)
    Ctl* gctl;                 // launch-wide control block (errors, statistics, BC order, trace)
    int* batch_status;         // [nbatch]
    double* const* job_bc;     // [njobs] accumulated BC per job (relabelled ids, device pointers)
    const int* col_job;        // [nbatch][K] job of each column; null = every column is job 0
    // options
    int direction;             // 0 auto, 1 push, 2 pull
    float alpha, beta;
    long long budget;          // barrier spin budget (cycles)
    int ext;                   // run the extended path-count form
    int forward_only;          // debug: stop after the forward sweep (no delta, no BC)
    long long* trace;          // optional phase trace: (tag, globaltimer ns) pairs; null = off
    int trace_cap;             // pairs the trace buffer holds
    int group;                 // light rows per warp task (1..32)
    int sum_bits;              // forward terms below 2^sum_bits cannot make a sum wrap 64 bits
    int dense_min;             // matched columns from which an arc is summed column-mapped (K >= 32)
    // teams: gridDim.x = nteams * team_blocks; team t owns blocks [t*team_blocks, (t+1)*team_blocks)
    // and the workspace slice at +t*team_bytes of every per-team array; batches go round-robin
    int team_blocks;
    int nteams;
    int team;                  // set in the kernel's team view
    int rank;                  // block index inside the team (team view)
    long long team_bytes;
    int level_slots;           // entries of each level array (>= levels + 3)
};

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

// x * 2^n, the value of scalbn(x, n): for a normal x whose scaled value is
// normal too, the exponent field moves by n (integer arithmetic, exact);
// zeros, subnormals, infinities and results outside the normal range take
// scalbn itself.
__device__ __forceinline__ double scale2(double x, int n) {
    const long long b = __double_as_longlong(x);
    const int e = (int)((b >> 52) & 0x7FF);
    if (e != 0 && e != 0x7FF && n > -0x7FF && n < 0x7FF) {
        const int ne = e + n;
        if (ne > 0 && ne < 0x7FF) return __longlong_as_double(b + (long long)n * (1LL << 52));
    }
    return scalbn(x, n);
}

// Real value r * 2^e (r a double) summed with alignment to the larger exponent.
__device__ __forceinline__ void xd_add(double& ar, int& ae, double xr, int xe) {
    if (xr == 0.0) return;
    if (ar == 0.0) { ar = xr; ae = xe; return; }
    if (xe > ae) {
        ar = scale2(ar, ae - xe);
        ae = xe;
        ar += xr;
    } else {
        ar += scale2(xr, xe - ae);
    }
}

// ------------------------------------------------------------------ barrier
// Barrier over the blocks of one team (a plain block barrier for one-block
// teams); errors are read from the launch-wide control block.
struct GridTeam {
    Ctl* ctl;
    Ctl* gctl;
    int nblocks;
    long long budget;

    // Returns false when the launch has failed (timeout or a fatal error).
    __device__ bool sync() {
        __shared__ int s_bad;
        __syncthreads();
        if (nblocks == 1) {
            if (threadIdx.x == 0) s_bad = *(volatile int*)&gctl->err != 0;
            __syncthreads();
            return !s_bad;
        }
        if (threadIdx.x == 0) {
            int bad = 0;
            volatile unsigned int* genp = &ctl->bar_gen;
            volatile int* errp = &gctl->err;
            unsigned int g = *genp;
            __threadfence();
            unsigned int arrived = atomicAdd(&ctl->bar_count, 1u);
            if (arrived == (unsigned int)nblocks - 1) {
                atomicExch(&ctl->bar_count, 0u);
                __threadfence();
                atomicAdd(&ctl->bar_gen, 1u);
            } else {
                long long t0 = clock64();
                while (*genp == g) {
                    if (*errp) { bad = 1; break; }
                    if (clock64() - t0 > budget) { atomicOr(&gctl->err, ERR_TIMEOUT); bad = 1; break; }
                    __nanosleep(32);
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

// Host-side launchers (bc_kernels.cu)
cudaError_t launch_batches(int K, const KParams& p, int blocks, cudaStream_t st);
int max_coop_blocks(int K, bool ext, int* per_sm);
cudaError_t launch_unpermute(const double* bc_rel, const int* inv, double* out, int n, cudaStream_t st);
cudaError_t launch_collect_status(const Ctl* ctl, const int* bstat, int nbatch, int* out, cudaStream_t st);
cudaError_t launch_team_reset(Ctl* ctl0, int* arr0, long long team_bytes, int nteams, int arr_ints, cudaStream_t st);
cudaError_t launch_map_sources(const int* src_orig, int nsrc, const int* inv, int n, int K, int* dst,
                               int nbatch, int* bad, cudaStream_t st);
cudaError_t launch_bfs_extract(const KParams& p, int K, int levels, int ncols, const int* inv, long long n,
                               unsigned short* lvl, int* level_out, double* sig_out, int* exp_out, cudaStream_t st);
// Weighted BC (weighted.cu): one cooperative launch per batch of 32 sources;
// weights of the relabelled arcs looked up from the original sorted CSR
// (err bits: 1 rows not sorted, 2 a weight <= 0, 4 asymmetric weights).
// One direction of a weighted graph for weighted BC: rows with their arc
// weights, split into heavy rows (more than kChunk arcs, the relabelled
// prefix [0, n_heavy), run as kChunk-arc chunk tasks) and light ones.
struct WCsr {
    const int* off;
    const int* adj;
    const int* w;       // nullptr where only rows and indices are read
    int n_heavy;        // heavy rows
    long long hchunks;  // their chunk tasks
    const int* hcum;    // [n_heavy + 1] chunk prefix
};
int wbc_blocks();
// ord: [n] ints; hist: kWbcHistWords words (bucket counts and the largest key);
// dag: [m] words; visited: [4] counters.
constexpr int kWbcHistWords = 4096 + 2;
cudaError_t launch_wbc(int n, const WCsr& out, const WCsr& in, int* arr, void* scratch, const int* src,
                       long long* dist, unsigned long long* sig, double* inv, double* del, double* rho, int* mark,
                       int* ord, unsigned int* hist, unsigned int* dag, double* bc, Ctl* ctl, int* changed,
                       int* passes, unsigned long long* visited, long long budget, int blocks, cudaStream_t st);
// Weights of the relabelled arcs; err bits: 1 rows not sorted, 2 a weight
// <= 0, 4 asymmetric weights.
cudaError_t launch_weight_ingest(const int* ooff, const int* oadj, const int* ow, const int* perm, const int* noff,
                                 const int* nadj, int n, int* nw, int* err, bool check_symmetry, cudaStream_t st);
// Level table [n][K] (0xFFFF = unreached) of a forward-only batch; and the
// levels of columns [0, L) of such a table at each of nsrc sources (original
// ids): keys[nsrc][L].
cudaError_t launch_level_table(const KParams& p, int K, int levels, unsigned short* lvl, long long n,
                               cudaStream_t st);
cudaError_t launch_source_keys(const unsigned short* lvl, int K, int L, long long n, const int* src, int nsrc,
                               const int* inv, unsigned short* keys, cudaStream_t st);
cudaError_t launch_debug_extract(const KParams& p, int K, int levels, int* level_rel, unsigned long long* sig_rel,
                                 int* sige_rel, cudaStream_t st);

// PageRank (pagerank.cu): scratch holds 2n + blocks doubles
int pagerank_blocks();
// row_class (rows sorted by length; null = not sorted): first rows shorter than
// 8192 and than 32 arcs
cudaError_t launch_pagerank(int n, const int* off, const int* roff, const int* radj, const int* row_class,
                            long long nchunks, const int* ccum, double* cpart, int* carr,
                            double delta, double beta, int max_iter, double* rank, double* scratch, Ctl* ctl, int* iters,
                            double* diff_out, int* go, long long budget, int blocks, cudaStream_t st);

// Graphs of large diameter (deep.cu): one source per block, block barriers
// only.  Per-block slices of `stride` entries: rec (one 32-byte record per
// vertex: the extended-form path count sm x 2^se, rho x 2^re and the level
// tag, so that one sector holds what a neighbour test reads), order (the
// vertices in BFS order) and orow (their out-row bounds); lvl: level_slots
// level starts per block.  A tag is
// epoch << 16 | level; tags of older epochs read as unseen, so a slice needs
// no reset between sources: source j (0-based) of block b in a launch uses
// epoch epoch0 + j, and the host keeps every epoch of a launch below 2^16,
// clearing the records (tag 0) when the count wraps.  delta: [nsrc][n]
// dependencies, cleared by the host (only reached vertices other than the
// source are written).  status[i]: BST_DONE | BST_INEXACT, or ERR_LIMIT << 8;
// depth[i]: levels of source i.  The counters add sum E_dag and sum n_s over
// the launch.
struct __align__(32) DeepRec {
    unsigned long long sm;  // path count mantissa
    double rho;             // rho mantissa
    unsigned int tag;       // epoch << 16 | level
    int se;                 // path count exponent
    int re;                 // rho exponent
    int pad;
};
struct DeepParams {
    int n;
    const int* off;
    const int* adj;
    const int* ioff;   // directed: in-CSR for the path-count sums; null = undirected
    const int* iadj;
    int n_heavy;       // rows above kChunk arcs: ids [0, n_heavy), summed per chunk
    const int* src;    // [nsrc] relabelled ids
    int nsrc;
    long long stride;
    DeepRec* rec;
    int* order;
    int2* orow;        // [k]: out-row bounds (off[v], off[v + 1]) of order[k], stored by its claimer
    int* lvl;
    int level_slots;   // lvl entries per block (>= deepest level + 3)
    unsigned int epoch0;
    double* delta;
    int* status;
    int* depth;
    unsigned long long* dag_pairs;
    unsigned long long* reached_pairs;
    // forward sweep only (multi-source BFS): when level_out is set, no reverse
    // sweep runs and source i writes row i of level_out (distance or -1) and,
    // when given, sig_out / exp_out (path counts as bc_bfs defines them), in
    // original ids through inv; delta is unused
    const int* inv;
    int* level_out;
    double* sig_out;
    int* exp_out;
};
cudaError_t launch_deep(const DeepParams& p, int blocks, int threads, cudaStream_t st);
int deep_blocks_per_sm(int threads);  // resident blocks of k_deep per SM (0 on error)
// bc[v] += delta[0][v] + ... + delta[nsrc-1][v], in that order
cudaError_t launch_deep_accumulate(const double* delta, int nsrc, long long n, double* bc, cudaStream_t st);

// Thread-local detail returned by bc_last_error() (bc_api.cu)
void set_last_error(const char* msg);

// Ingest (ingest.cu)
struct IngestOut {
    int* off;       // [n+1] device
    int* adj;       // [m] device
    int* perm;      // [n] new -> original
    int* inv;       // [n] original -> new
    int* ioff;      // directed: [n+1] in-CSR (transpose of the relabelled CSR), else null
    int* iadj;      // directed: [m]
    int max_deg;
    int max_in_deg; // directed: longest in-row, else 0
    int n_nz;
    int reason;     // 0 ok, else 1 offsets, 2 index range, 3 self-loop, 4 duplicate, 5 asymmetric
};
typedef void* (*AllocFn)(size_t, cudaStream_t);
typedef void (*FreeFn)(void*, cudaStream_t);
cudaError_t ingest(const int* d_off_in, const int* d_adj_in, int n, long long m, bool validate, bool directed,
                   cudaStream_t st, AllocFn alloc, FreeFn dfree, IngestOut* out, bool* oom);

}  // namespace bcx
