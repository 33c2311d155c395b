// libbc host runtime: the C ABI declared in include/bc.h.
//
// Owns graph lifetime (device-resident relabelled CSR), per-graph workspaces
// sized for a batch width, the batching of a source list into traversals of
// K columns, and the launch of the persistent kernel.  No computation of the
// method happens on the host: it only marshals sizes, pointers and statuses.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "../../include/bc.h"
#include "bc_internal.cuh"

using namespace bcx;

// ------------------------------------------------------------------ errors
static thread_local std::string t_err;

static bc_status fail(bc_status st, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    t_err = buf;
    return st;
}

void bcx::set_last_error(const char* msg) { t_err = msg; }

static bc_status cuda_fail(cudaError_t e, const char* what) {
    return fail(BC_E_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

// ------------------------------------------------------------------ allocator hook
struct AllocHook {
    bc_alloc_fn alloc = nullptr;
    bc_free_fn free_fn = nullptr;
    void* ctx = nullptr;
};
static std::mutex g_alloc_mu;
static AllocHook g_hook;

struct DevBuf {
    void* p = nullptr;
    size_t bytes = 0;
    AllocHook hook;  // the hook that allocated it
};

static void* dev_alloc_raw(size_t bytes, cudaStream_t st, AllocHook* used) {
    AllocHook h;
    {
        std::lock_guard<std::mutex> lk(g_alloc_mu);
        h = g_hook;
    }
    if (used) *used = h;
    if (bytes == 0) bytes = 16;
    if (h.alloc) return h.alloc(bytes, (bc_stream_t)st, h.ctx);
    {
        // the device's default pool keeps up to 256 MB of freed memory between
        // synchronisations (default 0: every sync returns it, and the next
        // call's small buffers are mapped anew); a process-local setting
        static std::once_flag once[64];
        int dev = 0;
        cudaGetDevice(&dev);
        if (dev >= 0 && dev < 64)
            std::call_once(once[dev], [dev]() {
                cudaMemPool_t pool;
                if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
                    unsigned long long keep = 256ull << 20;
                    cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
                }
                cudaGetLastError();
            });
    }
    void* p = nullptr;
    if (cudaMallocAsync(&p, bytes, st) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return p;
}

static void dev_free_raw(void* p, cudaStream_t st, const AllocHook& h) {
    if (!p) return;
    if (h.alloc) {
        if (h.free_fn) h.free_fn(p, (bc_stream_t)st, h.ctx);
    } else {
        cudaFreeAsync(p, st);
    }
}

// for ingest (plain function pointers; the hook in force at the call is used)
static void* ingest_alloc(size_t b, cudaStream_t st) { return dev_alloc_raw(b, st, nullptr); }
static void ingest_free(void* p, cudaStream_t st) {
    AllocHook h;
    {
        std::lock_guard<std::mutex> lk(g_alloc_mu);
        h = g_hook;
    }
    dev_free_raw(p, st, h);
}

static bool buf_ensure(DevBuf& b, size_t bytes, cudaStream_t st) {
    if (b.p && b.bytes >= bytes) return true;
    if (b.p) dev_free_raw(b.p, st, b.hook);
    b.p = dev_alloc_raw(bytes, st, &b.hook);
    b.bytes = b.p ? bytes : 0;
    return b.p != nullptr;
}

static void buf_release(DevBuf& b, cudaStream_t st) {
    if (b.p) dev_free_raw(b.p, st, b.hook);
    b.p = nullptr;
    b.bytes = 0;
}

// ------------------------------------------------------------------ graph
// Per-team arrays live in one arena: team t's slice starts at t * team_bytes and
// every slice has the same layout (offsets below).  Launch-wide arrays are
// separate buffers.
struct TeamLayout {
    size_t V = 0, F0 = 0, F1 = 0, F2 = 0, sig = 0, rho = 0, sig_e = 0, rho_e = 0, ent = 0, emask = 0;
    size_t hent = 0, hmask = 0, hpre = 0, stamp = 0, scr_v = 0, scr_e = 0, scr_or = 0, arr = 0;
    size_t cnt = 0, hcnt = 0, start = 0, hstart = 0, hchunks = 0, dsum = 0, fulldeg = 0, ctl = 0;
    size_t bytes = 0;
    long long cap = 0, hcap = 0;
    int arr_ints = 0, level_slots = 0;
};

static TeamLayout team_layout(int n_vert, int n_heavy, long long hchunks, int K, bool ext, int capf) {
    TeamLayout L;
    const size_t n = (size_t)(n_vert > 0 ? n_vert : 1);
    const size_t W = K >= 32 ? (size_t)K / 32 : 1;
    const size_t nh = (size_t)(n_heavy > 0 ? n_heavy : 1);
    const size_t hc = (size_t)(hchunks > 0 ? hchunks : 1);
    L.cap = (long long)n * capf;
    L.hcap = (long long)nh * K;
    L.arr_ints = (int)nh;
    L.level_slots = (int)std::min<long long>(kLevelSlots, (long long)n + 3);
    size_t o = 0;
    auto take = [&](size_t bytes) {
        const size_t at = o;
        o += (bytes + 255) / 256 * 256;
        return at;
    };
    L.V = take(4 * n * W);
    L.F0 = take(4 * n * W);
    L.F1 = take(4 * n * W);
    L.F2 = take(4 * n * W);
    L.sig = take(8 * n * K);
    L.rho = take(8 * n * K);
    if (ext) {
        L.sig_e = take(4 * n * K);
        L.rho_e = take(4 * n * K);
    }
    L.ent = take(4 * (size_t)L.cap);
    L.emask = take(4 * W * (size_t)L.cap);
    L.hent = take(4 * (size_t)L.hcap);
    L.hmask = take(4 * W * (size_t)L.hcap);
    L.hpre = take(4 * (size_t)L.hcap);
    L.stamp = take(4 * n);
    L.scr_v = take(8 * hc * K);
    if (ext) L.scr_e = take(4 * hc * K);
    L.scr_or = take(4 * hc * W);
    L.arr = take(4 * nh);
    const size_t ls = (size_t)L.level_slots;
    L.cnt = take(4 * ls);
    L.hcnt = take(4 * ls);
    L.start = take(4 * ls);
    L.hstart = take(4 * ls);
    L.hchunks = take(4 * ls);
    L.dsum = take(8 * ls);
    L.fulldeg = take(8 * ls);
    L.ctl = take(sizeof(Ctl));
    L.bytes = o;
    return L;
}

struct Workspace {
    int K = 0;
    bool ext = false;
    int nteams = 0;
    TeamLayout lay;
    DevBuf arena;  // nteams * lay.bytes
    DevBuf gctl, bstat, bc, src, bad, jobptr, coljob, trace;
    void release(cudaStream_t st) {
        DevBuf* all[] = {&arena, &gctl, &bstat, &bc, &src, &bad, &jobptr, &coljob, &trace};
        for (DevBuf* b : all) buf_release(*b, st);
    }
    size_t bytes() const {
        const DevBuf* all[] = {&arena, &gctl, &bstat, &bc, &src, &bad, &jobptr, &coljob, &trace};
        size_t t = 0;
        for (const DevBuf* b : all) t += b->bytes;
        return t;
    }
    char* at(size_t off) const { return (char*)arena.p + off; }
};

// Entry-list capacity per vertex: a vertex enters a level list at most once per
// distinct level across the batch's columns, so K bounds it; the first try
// uses a smaller factor and the call reruns with K on overflow.
static int cap_factor(int K, int sticky) { return sticky > 0 ? sticky : (K < 24 ? K : 24); }

// Bytes a single-team workspace needs (admission estimate for serving).
static size_t ws_need(int n, int K, int n_heavy, long long hc, bool ext, int nbatch, int njobs, int capf) {
    const TeamLayout L = team_layout(n, n_heavy, hc, K, ext, capf);
    return L.bytes + sizeof(Ctl) + sizeof(int) * (size_t)(nbatch > 0 ? nbatch : 1) * (1 + 2 * K) +
           sizeof(double) * (size_t)(n > 0 ? n : 1) + sizeof(double*) * (size_t)(njobs > 0 ? njobs : 1);
}

struct bc_graph {
    int n = 0;
    long long m = 0;
    int max_deg = 0;
    int n_nz = 0;
    int n_heavy = -1;      // rows with degree > kChunk (a prefix of the new ids); -1 = not yet counted
    int first_leaf = 1 << 30;  // first new id of degree 1 (degrees are non-increasing); set with n_heavy
    long long hchunk_total = 0;
    bool directed = false;
    int max_in_deg = 0;  // directed: longest in-row (forward sums run over whole in-rows)
    DevBuf off, adj, perm, inv, hcum;
    DevBuf ioff, iadj;  // directed: in-CSR for the pull steps
    DevBuf w;           // weighted graphs: arc weights in relabelled arc order (empty otherwise)
    DevBuf wdist, wsig, winv, wdel, wrho, wmark, wbc, wctl, wsrc, wscr, warr;  // weighted BC state, kept between calls
    DevBuf word, whist;  // weighted BC: row order by mean distance, its bucket counts
    DevBuf wdag;         // weighted BC: per out-arc DAG masks of the current batch
    AllocHook hook;
    std::mutex mu;                                 // bc_compute / plans: the per-width workspaces below
    std::map<int, std::unique_ptr<Workspace>> ws;  // by batch width
    std::mutex state_mu;                           // the lazily set facts below (concurrent serving runs)
    bool sticky_ext = false;
    std::map<int, int> sticky_cap;                 // entry capacity factor that sufficed, by width
    bc_run_stats last{};
    std::vector<long long> last_trace;             // (tag, t_ns) pairs of the last traced call
    cudaStream_t last_stream = nullptr;
    std::atomic<int> users{0};  // plans and queued serving jobs that refer to the graph
    std::mutex lm_mu;           // the landmark table below, built once on first use
    DevBuf landmark;            // [n][32] uint16 levels of the BFS from each of the 32 first relabelled vertices
    int lm_levels = -1;         // levels of that BFS; -1 = not built
    // PageRank facts and buffers (under mu, built on first use): row classes,
    // the chunk prefix of the long rows, rank / scratch / chunk sums / counters
    int depth_seen = -1;  // deepest BFS (levels) of any completed traversal on the graph; -1 = none yet
    // per-source form: per-block records, per-block BFS order and level starts, dependency rows, status;
    // the records of blocks [0, deep_blocks) at stride deep_stride hold tags of epochs below deep_epoch
    DevBuf deep_state, deep_order, deep_delta, deep_aux;
    unsigned int deep_epoch = 1;
    long long deep_stride = -1;
    long long deep_blocks = 0;
    int pr_cls[2] = {-1, -1};
    long long pr_nchunks = 0;
    DevBuf pr_ccum, pr_rank, pr_scratch, pr_cpart, pr_carr, pr_ctl, pr_small;
};

// The per-source form's depth rule (see want_deep): at least kDeepMinDepth
// levels of at most kDeepMaxWidth vertices on average.
constexpr int kDeepMinDepth = 48;
constexpr int kDeepMaxWidth = 8192;
static bool deep_by_depth(const bc_graph* g, int depth) {
    return depth >= kDeepMinDepth && (double)g->n_nz <= (double)kDeepMaxWidth * depth;
}

// ------------------------------------------------------------------ helpers
static bool is_device_ptr(const void* p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// Heavy rows and their chunk prefix, once per graph: degrees are non-increasing
// in new ids, so the heavy rows are a prefix found by binary search; the
// prefix of chunk counts is built on the host from their offsets.
static bc_status ensure_heavy(bc_graph* g, cudaStream_t st) {
    std::lock_guard<std::mutex> lk(g->state_mu);
    if (g->n_heavy >= 0) return BC_OK;
    int lo = 0, hi = g->n_nz;  // first r with deg(r) <= kChunk
    const int* off = (const int*)g->off.p;
    while (lo < hi) {
        int mid = (lo + hi) / 2;
        int two[2];
        cudaError_t e = cudaMemcpyAsync(two, off + mid, sizeof two, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) return cuda_fail(e, "heavy-row count");
        if (two[1] - two[0] > kChunk) lo = mid + 1;
        else hi = mid;
    }
    const int nh = lo;
    // rows of degree 1 follow every longer row: the first of them
    int llo = nh, lhi = g->n_nz;
    while (llo < lhi) {
        int mid = (llo + lhi) / 2;
        int two[2];
        cudaError_t e = cudaMemcpyAsync(two, off + mid, sizeof two, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) return cuda_fail(e, "degree-1 row count");
        if (two[1] - two[0] > 1) llo = mid + 1;
        else lhi = mid;
    }
    std::vector<int> ho((size_t)nh + 1), cum((size_t)nh + 1);
    cudaError_t e = cudaMemcpyAsync(ho.data(), off, sizeof(int) * ((size_t)nh + 1), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "heavy-row offsets");
    cum[0] = 0;
    for (int r = 0; r < nh; ++r) cum[r + 1] = cum[r] + (ho[r + 1] - ho[r] + kChunk - 1) / kChunk;
    if (!buf_ensure(g->hcum, sizeof(int) * ((size_t)nh + 1), st)) return fail(BC_E_NOMEM, "heavy-row table");
    e = cudaMemcpyAsync(g->hcum.p, cum.data(), sizeof(int) * ((size_t)nh + 1), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "heavy-row table");
    g->first_leaf = llo;
    g->n_heavy = nh;
    g->hchunk_total = cum[nh];
    return BC_OK;
}

// Workspace for `nteams` teams, each sized for graphs of at most n_vert
// vertices, n_heavy heavy rows and hchunks heavy chunks.
static bool ws_ensure_dims(Workspace* w, int n_vert, int n_heavy, long long hchunks, int K, bool ext, int nbatch,
                           int njobs, int capf, int nteams, cudaStream_t st) {
    const TeamLayout L = team_layout(n_vert, n_heavy, hchunks, K, ext, capf);
    const size_t n = (size_t)(n_vert > 0 ? n_vert : 1);
    const size_t nb = (size_t)(nbatch > 0 ? nbatch : 1);
    // keep a larger arena when it already fits the new layout's total
    const size_t need = L.bytes * (size_t)(nteams > 0 ? nteams : 1);
    bool ok = buf_ensure(w->arena, need, st);
    ok &= buf_ensure(w->gctl, sizeof(Ctl), st);
    ok &= buf_ensure(w->bstat, sizeof(int) * nb, st);
    ok &= buf_ensure(w->bc, sizeof(double) * n, st);
    ok &= buf_ensure(w->src, sizeof(int) * nb * K, st);
    ok &= buf_ensure(w->coljob, sizeof(int) * nb * K, st);
    ok &= buf_ensure(w->bad, sizeof(int), st);
    ok &= buf_ensure(w->jobptr, sizeof(double*) * (size_t)(njobs > 0 ? njobs : 1), st);
    if (!ok) {
        fail(BC_E_NOMEM, "device allocation failed for a batch-width-%d workspace (n=%d, %d teams)", K, n_vert, nteams);
        return false;
    }
    w->K = K;
    w->ext = ext;
    w->nteams = nteams;
    w->lay = L;
    return true;
}

static bool ws_ensure(Workspace* w, bc_graph* g, int K, bool ext, int nbatch, int njobs, int capf, int nteams,
                      cudaStream_t st) {
    return ws_ensure_dims(w, g->n, g->n_heavy, g->hchunk_total, K, ext, nbatch, njobs, capf, nteams, st);
}

// Bits of x (0 for 0): a sum of x terms below 2^(64 - bits_needed(x)) fits 64 bits.
static int bits_needed(unsigned long long x) {
    int b = 0;
    while (x) {
        ++b;
        x >>= 1;
    }
    return b;
}

// Matched columns from which an arc is cheaper summed column-mapped (one warp
// step per arc) than as compacted pairs; measured on R-MAT scale 22 (4096
// sources): 32 of 128 once the column-mapped sums stay in registers between
// arcs of one owner (48 before), and 32 of 64; at 32 columns the two forms tie.
static int default_dense_min(int K) { return 32; }

static KParams make_params(bc_graph* g, Workspace* w, int nbatch, const bc_options& o, bool ext, int team_blocks) {
    KParams p;
    memset(&p, 0, sizeof p);
    const TeamLayout& L = w->lay;
    p.n = g->n;
    p.n_nz = g->n_nz;
    p.n_heavy = g->n_heavy;
    p.first_leaf = g->directed ? g->n : g->first_leaf;  // undirected only: a directed out-degree 1 may lead on
    p.m_nz = g->m;
    p.off = (const int*)g->off.p;
    p.adj = (const int*)g->adj.p;
    p.ioff = g->directed ? (const int*)g->ioff.p : nullptr;
    p.iadj = g->directed ? (const int*)g->iadj.p : nullptr;
    p.src = (const int*)w->src.p;
    p.nbatch = nbatch;
    p.V = (uint32_t*)w->at(L.V);
    p.F[0] = (uint32_t*)w->at(L.F0);
    p.F[1] = (uint32_t*)w->at(L.F1);
    p.F[2] = (uint32_t*)w->at(L.F2);
    p.sig = (unsigned long long*)w->at(L.sig);
    p.rho = (double*)w->at(L.rho);
    p.sig_e = ext ? (int*)w->at(L.sig_e) : nullptr;
    p.rho_e = ext ? (int*)w->at(L.rho_e) : nullptr;
    p.ent = (int*)w->at(L.ent);
    p.emask = (uint32_t*)w->at(L.emask);
    p.hent = (int*)w->at(L.hent);
    p.hmask = (uint32_t*)w->at(L.hmask);
    p.hpre = (int*)w->at(L.hpre);
    p.cap = L.cap;
    p.hcap = L.hcap;
    p.hcum = (const int*)g->hcum.p;
    p.scr_v = (unsigned long long*)w->at(L.scr_v);
    p.scr_e = ext ? (int*)w->at(L.scr_e) : nullptr;
    p.scr_or = (uint32_t*)w->at(L.scr_or);
    p.arr = (int*)w->at(L.arr);
    p.stamp = (int*)w->at(L.stamp);
    p.la.cnt = (int*)w->at(L.cnt);
    p.la.hcnt = (int*)w->at(L.hcnt);
    p.la.start = (int*)w->at(L.start);
    p.la.hstart = (int*)w->at(L.hstart);
    p.la.dsum = (long long*)w->at(L.dsum);
    p.la.fulldeg = (long long*)w->at(L.fulldeg);
    p.la.hchunks = (int*)w->at(L.hchunks);
    p.ctl = (Ctl*)w->at(L.ctl);
    p.gctl = (Ctl*)w->gctl.p;
    p.batch_status = (int*)w->bstat.p;
    p.job_bc = (double* const*)w->jobptr.p;
    p.col_job = nullptr;
    p.direction = o.direction;
    p.alpha = o.alpha > 0 ? o.alpha : 14.0f;
    p.beta = o.beta > 0 ? o.beta : 24.0f;
    p.budget = o.barrier_budget > 0 ? o.barrier_budget : 40000000000ll;
    p.ext = ext ? 1 : 0;
    p.forward_only = 0;
    p.group = o.group_vertices > 0 ? o.group_vertices : 32;
    p.dense_min = o.dense_min > 0 ? o.dense_min : default_dense_min(w->K);
    // forward sums have at most 1024 terms (chunked rows); directed graphs sum whole in-rows
    p.sum_bits = g->directed ? 64 - bits_needed((unsigned long long)g->max_in_deg) : 64 - 10;
    p.trace = nullptr;
    p.trace_cap = 0;
    p.team_blocks = team_blocks;
    p.nteams = w->nteams;
    p.team_bytes = (long long)L.bytes;
    p.level_slots = L.level_slots;
    return p;
}

// Reset the launch-wide and per-team control blocks before a launch.
static cudaError_t reset_controls(Workspace* w, int nbatch, cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(w->gctl.p, 0, sizeof(Ctl), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(w->bstat.p, 0, sizeof(int) * (size_t)(nbatch > 0 ? nbatch : 1), st);
    if (e == cudaSuccess)
        e = launch_team_reset((Ctl*)w->at(w->lay.ctl), (int*)w->at(w->lay.arr), (long long)w->lay.bytes, w->nteams,
                              w->lay.arr_ints, st);
    return e;
}

static int choose_width(int n, int nsrc, int requested) {
    if (requested > 0) return requested;
    // automatic: wide batches amortise row reads over more sources; keep the
    // per-batch state within a few GB and do not pad tiny requests.
    if (nsrc <= 1) return 1;
    if (nsrc <= 32) return 32;
    const double bytes128 = (double)n * 128 * 20;
    if (nsrc >= 256 && bytes128 < 24e9) return 128;
    return 64;
}

static bc_status check_opts(const bc_options& o) {
    if (o.batch_width != 0 && o.batch_width != 1 && o.batch_width != 32 && o.batch_width != 64 &&
        o.batch_width != 128)
        return fail(BC_E_INVALID_ARG, "batch_width must be 0, 1, 32, 64 or 128 (got %d)", o.batch_width);
    if (o.direction < 0 || o.direction > 2) return fail(BC_E_INVALID_ARG, "direction must be 0, 1 or 2");
    if (o.group_vertices < 0 || o.group_vertices > 32) return fail(BC_E_INVALID_ARG, "group_vertices must be in [0, 32]");
    if (o.blocks_per_sm < 0 || o.barrier_budget < 0 || o.alpha < 0 || o.beta < 0 || o.teams < 0 || o.dense_min < 0)
        return fail(BC_E_INVALID_ARG, "negative option value");
    if (o.source_order < 0 || o.source_order > 2) return fail(BC_E_INVALID_ARG, "source_order must be 0, 1 or 2");
    if (o.deep_form < 0 || o.deep_form > 2) return fail(BC_E_INVALID_ARG, "deep_form must be 0, 1 or 2");
    return BC_OK;
}

static int grid_blocks(int K, bool ext, int blocks_per_sm, int share) {
    int per_sm = 0;
    const int maxb = max_coop_blocks(K, ext, &per_sm);
    int sms = 0, dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    int bps = blocks_per_sm > 0 ? blocks_per_sm : per_sm;
    if (bps > per_sm) bps = per_sm;
    int blocks = bps * sms;
    if (blocks > maxb) blocks = maxb;
    if (share > 1) blocks = blocks / share;
    return blocks;
}

// Teams for a launch, host arithmetic only (exported as bc_team_rule): blocks
// per team grow with the graph's arcs m; no more teams than the nbatch batches
// or the grid's blocks; the teams' arena slices (team_bytes each) within 30%
// of free_bytes and 24 GB; forced > 0 asks for that many teams.
static void team_rule(long long m, int K, int nbatch, int blocks, size_t team_bytes, size_t free_bytes, int forced,
                      int* nteams, int* team_blocks) {
    int T;
    if (forced > 0) {
        T = forced;
    } else {
        // blocks per team: about one per 2^19 arcs on large graphs, and on
        // smaller ones about 0.7 * m^0.24 at width 128, in proportion to the
        // width (measured optimum with many 128-wide batches: 7 blocks at R-MAT
        // 10, 11 at 12, 15 at 14, 18 at 16, 27 at 18; one team per batch on a
        // whole grid ran R-MAT 16 with 316 batches in 457 ms against 175-191 ms
        // with 16-32 teams; one-source batches of R-MAT 12 run best one block
        // each: 45.7 ms against 67.3 ms on 9-block teams); at least two teams
        // when there are two batches (a second batch in flight hides the
        // first's level-barrier waits: R-MAT 22, 1261 -> 1245 ms)
        long long per = std::max<long long>((m >> 19) + 1,
                                            (long long)(0.7 * std::pow((double)m, 0.24) * K / 128.0));
        // a one-source batch gains little from a team past 32 blocks: R-MAT 22
        // with 256 sources ran 1493 ms on 2 teams of 222 blocks and 969 ms on 13
        // of 34 (9-20 teams within 0.3%); R-MAT 20 with 512 sources 583 ms on 6
        // teams, 492 on 13, 481 on 27 (R-MAT 18 and below keep their teams)
        if (K == 1) per = std::min<long long>(per, 32);
        if (per < 1) per = 1;
        T = (int)std::max<long long>(1, blocks / std::min<long long>(per, blocks));
        if (nbatch >= 2) T = std::max(T, 2);
    }
    T = std::min(T, std::max(1, nbatch));
    T = std::min(T, blocks);
    const double budget = std::min(0.3 * (double)free_bytes, 24e9);
    while (T > 1 && (double)T * (double)team_bytes > budget) --T;
    if (forced <= 0 && T > 1) {
        // the fewest teams that take the batches in the same number of rounds,
        // so the last round is not a few batches on a mostly idle grid
        // (R-MAT 18, 32 batches: 29 teams 139 ms, 16 teams 109 ms)
        const int rounds = (nbatch + T - 1) / T;
        T = (nbatch + rounds - 1) / rounds;
    }
    *nteams = T;
    *team_blocks = blocks / T;
}

static void choose_teams(long long m, int K, int nbatch, int blocks, size_t team_bytes, int forced, int* nteams,
                         int* team_blocks) {
    size_t fr = 0, tot = 0;
    if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) {
        cudaGetLastError();
        fr = (size_t)16 << 30;
    }
    team_rule(m, K, nbatch, blocks, team_bytes, fr, forced, nteams, team_blocks);
}

// One traversal run of a source list (original ids, device) on workspace w:
// map sources, launch the persistent kernel over all batches, read the status.
// job_bc buffers (relabelled, one per job) are accumulated, not cleared.
struct RunOut {
    bool need_ext = false;
    bool inexact = false;
    bool capacity = false;
    float kernel_ms = 0.f;
    Ctl ctl{};
};

static bc_status run_core(bc_graph* g, Workspace* w, const int* d_src_orig, int nsrc, int K, int team_blocks,
                          const bc_options& o, bool ext, const std::vector<double*>& job_bc,
                          const std::vector<int>* col_job, bool forward_only, cudaStream_t st, RunOut* ro) {
    const int nbatch = (nsrc + K - 1) / K;
    cudaError_t e;
    if ((e = cudaMemsetAsync(w->bad.p, 0, sizeof(int), st)) != cudaSuccess) return cuda_fail(e, "memset");
    if ((e = launch_map_sources(d_src_orig, nsrc, (const int*)g->inv.p, g->n, K, (int*)w->src.p, nbatch,
                                (int*)w->bad.p, st)) != cudaSuccess)
        return cuda_fail(e, "map sources");
    if ((e = cudaMemcpyAsync(w->jobptr.p, job_bc.data(), sizeof(double*) * job_bc.size(), cudaMemcpyHostToDevice,
                             st)) != cudaSuccess)
        return cuda_fail(e, "job table");
    if (col_job && (e = cudaMemcpyAsync(w->coljob.p, col_job->data(), sizeof(int) * col_job->size(),
                                        cudaMemcpyHostToDevice, st)) != cudaSuccess)
        return cuda_fail(e, "column table");
    int bad = 0;
    if ((e = cudaMemcpyAsync(&bad, w->bad.p, sizeof(int), cudaMemcpyDeviceToHost, st)) != cudaSuccess)
        return cuda_fail(e, "source check");
    if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return cuda_fail(e, "source check");
    if (bad) return fail(BC_E_SOURCE, "a source id is outside [0, %d)", g->n);
    if ((e = reset_controls(w, nbatch, st)) != cudaSuccess) return cuda_fail(e, "reset");
    KParams p = make_params(g, w, nbatch, o, ext, team_blocks);
    p.forward_only = forward_only ? 1 : 0;
    if (col_job) p.col_job = (const int*)w->coljob.p;
    const int kTraceCap = 1 << 16;
    if (o.trace) {
        if (!buf_ensure(w->trace, sizeof(long long) * 2 * kTraceCap, st)) return fail(BC_E_NOMEM, "trace buffer");
        p.trace = (long long*)w->trace.p;
        p.trace_cap = kTraceCap;
    }
    cudaEvent_t ev[2];
    cudaEventCreate(&ev[0]);
    cudaEventCreate(&ev[1]);
    cudaEventRecord(ev[0], st);
    e = launch_batches(K, p, team_blocks * w->nteams, st);
    cudaEventRecord(ev[1], st);
    if (e != cudaSuccess) {
        cudaEventDestroy(ev[0]);
        cudaEventDestroy(ev[1]);
        return cuda_fail(e, "persistent kernel launch");
    }
    std::vector<int> bst(nbatch);
    if ((e = cudaMemcpyAsync(&ro->ctl, w->gctl.p, sizeof(Ctl), cudaMemcpyDeviceToHost, st)) != cudaSuccess)
        return cuda_fail(e, "status read");
    if ((e = cudaMemcpyAsync(bst.data(), w->bstat.p, sizeof(int) * nbatch, cudaMemcpyDeviceToHost, st)) !=
        cudaSuccess)
        return cuda_fail(e, "status read");
    e = cudaStreamSynchronize(st);
    if (e == cudaSuccess) cudaEventElapsedTime(&ro->kernel_ms, ev[0], ev[1]);
    cudaEventDestroy(ev[0]);
    cudaEventDestroy(ev[1]);
    if (e != cudaSuccess) return cuda_fail(e, "persistent kernel");
    const Ctl& ctl = ro->ctl;
    if (o.trace) {
        const int nrec = ctl.trace_n < kTraceCap ? ctl.trace_n : kTraceCap;
        g->last_trace.assign((size_t)2 * nrec, 0);
        if (nrec > 0 && (e = cudaMemcpy(g->last_trace.data(), w->trace.p, sizeof(long long) * 2 * nrec,
                                        cudaMemcpyDeviceToHost)) != cudaSuccess)
            return cuda_fail(e, "trace read");
    }
    if (ctl.err & ERR_TIMEOUT) return fail(BC_E_TIMEOUT, "a grid-barrier wait exceeded its cycle budget");
    if (ctl.err & ERR_LIMIT) return fail(BC_E_LIMIT, "BFS deeper than %d levels", kMaxLevel);
    if (ctl.err == ERR_CAPACITY) {
        ro->capacity = true;
        return BC_OK;
    }
    if (ctl.err) return fail(BC_E_CUDA, "internal device error 0x%x", ctl.err);
    ro->need_ext = false;
    ro->inexact = false;
    for (int b = 0; b < nbatch; ++b) {
        if (bst[b] & BST_NEED_EXT) ro->need_ext = true;
        else if (!(bst[b] & BST_DONE)) return fail(BC_E_CUDA, "internal: batch %d not completed", b);
        if (bst[b] & BST_INEXACT) ro->inexact = true;
    }
    return BC_OK;
}

// A full call: batches of K, reruns when a count overflows 64 bits (extended
// form) or the level lists overflow (full capacity), accumulation into job
// buffers (cleared first).
static bc_status run_jobs(bc_graph* g, Workspace* w, const int* d_src, int nsrc, const bc_options& o, int blocks_share,
                          const std::vector<double*>& job_bc, const std::vector<int>* col_job, bool forward_only,
                          cudaStream_t st, bc_run_stats* stats, int* K_out, bool* ext_out, int* levels_out) {
    const int K = choose_width(g->n, nsrc, o.batch_width);
    const int nbatch = (nsrc + K - 1) / K;
    bc_status err = ensure_heavy(g, st);
    if (err != BC_OK) return err;
    bool ext;
    int capf;
    {
        std::lock_guard<std::mutex> lk(g->state_mu);
        ext = g->sticky_ext;
        capf = cap_factor(K, g->sticky_cap.count(K) ? g->sticky_cap[K] : 0);
    }
    bc_run_stats s{};
    s.batch_width = K;
    s.batches = nbatch;
    for (int attempt = 0; attempt < 4; ++attempt) {
        const int blocks = grid_blocks(K, ext, o.blocks_per_sm, blocks_share);
        if (blocks < 1) return fail(BC_E_CUDA, "persistent kernel cannot be resident (occupancy 0)");
        int nteams = 1, team_blocks = blocks;
        const TeamLayout L = team_layout(g->n, g->n_heavy, g->hchunk_total, K, ext, capf);
        choose_teams(g->m, K, nbatch, blocks, L.bytes, o.teams, &nteams, &team_blocks);
        s.grid_blocks = nteams * team_blocks;
        s.teams = nteams;
        if (!ws_ensure(w, g, K, ext, nbatch, (int)job_bc.size(), capf, nteams, st)) return BC_E_NOMEM;
        for (double* jb : job_bc) {
            cudaError_t e = cudaMemsetAsync(jb, 0, sizeof(double) * (size_t)(g->n > 0 ? g->n : 1), st);
            if (e != cudaSuccess) return cuda_fail(e, "memset");
        }
        RunOut ro;
        bc_status r = run_core(g, w, d_src, nsrc, K, team_blocks, o, ext, job_bc, col_job, forward_only, st, &ro);
        if (r != BC_OK) return r;
        s.kernel_launches += 3;  // source mapping, control reset, traversal
        s.kernel_ms += ro.kernel_ms;
        s.max_levels = ro.ctl.max_levels;
        s.pull_levels += ro.ctl.pull_levels;
        s.push_levels += ro.ctl.push_levels;
        s.dag_arcs = (int64_t)ro.ctl.dag_pairs;  // the launch that settles the call counts
        s.reached = (int64_t)ro.ctl.reached_pairs;
        if (ro.capacity) {
            if (capf >= K) return fail(BC_E_CUDA, "internal: level-list capacity exceeded at the bound");
            capf = K;
            {
                std::lock_guard<std::mutex> lk(g->state_mu);
                g->sticky_cap[K] = K;
            }
            continue;
        }
        if (ro.need_ext && !ext) {
            // rerun the whole call in the extended form, so that every source is
            // accumulated in list order exactly as in a single pass
            ext = true;
            {
                std::lock_guard<std::mutex> lk(g->state_mu);
                g->sticky_ext = true;
            }
            continue;
        }
        if (ro.need_ext) return fail(BC_E_SIGMA_RANGE, "path count beyond the extended range");
        if (ext) s.ext_batches = nbatch;
        {
            std::lock_guard<std::mutex> lk(g->state_mu);
            g->depth_seen = std::max(g->depth_seen, ro.ctl.max_levels);
        }
        if (stats) *stats = s;
        if (K_out) *K_out = K;
        if (ext_out) *ext_out = ext;
        if (levels_out) *levels_out = ro.ctl.last_levels;
        return ro.inexact ? BC_W_SIGMA_INEXACT : BC_OK;
    }
    return fail(BC_E_CUDA, "internal: reruns did not settle");
}

// ------------------------------------------------------------------ autotuning
// Tuned knobs per graph-size bucket: (log2 n, log2 average degree, log2 of
// max/average degree).  None of the knobs changes results (every sum has a
// fixed order), so a tuned setting only changes speed.
struct TuneKey {
    int ln, lavg, lskew;
    bool operator<(const TuneKey& o) const {
        if (ln != o.ln) return ln < o.ln;
        if (lavg != o.lavg) return lavg < o.lavg;
        return lskew < o.lskew;
    }
};
struct TuneVal {
    int K = 0, group = 0;
    float alpha = 0.f;
    double rate = 0.0;  // source-arcs per second measured on the sample
};
static std::mutex g_tune_mu;
static std::map<TuneKey, TuneVal> g_tune;

static int ilog2(double x) {
    int l = 0;
    while (x >= 2.0 && l < 62) {
        x *= 0.5;
        ++l;
    }
    return l;
}

static TuneKey tune_key(const bc_graph* g) {
    const double nz = g->n_nz > 0 ? (double)g->n_nz : 1.0;
    const double avg = (double)g->m / nz > 1.0 ? (double)g->m / nz : 1.0;
    return TuneKey{ilog2((double)(g->n > 0 ? g->n : 1)), ilog2(avg), ilog2((double)(g->max_deg > 0 ? g->max_deg : 1) / avg)};
}

// Fill unset knobs of o from the graph's bucket, when it has been tuned.
static void apply_tuning(const bc_graph* g, int nsrc, bc_options& o) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tune.find(tune_key(g));
    if (it == g_tune.end()) return;
    const TuneVal& v = it->second;
    if (o.batch_width == 0 && v.K > 0 && (v.K == 1 || nsrc > v.K / 2)) o.batch_width = v.K;
    if (o.alpha == 0.f && v.alpha > 0.f) o.alpha = v.alpha;
    if (o.group_vertices == 0 && v.group > 0) o.group_vertices = v.group;
}

// ------------------------------------------------------------------ serving
// Continuous batching: worker threads (one CUDA stream and one workspace each)
// take queued jobs in arrival order as soon as a worker is free and the
// device-memory budget admits its workspace; small jobs queued on the same
// graph are packed into the same traversal (their columns side by side).
// source grouping (defined with the C entry points below, used by the serving workers)
extern "C" {
static bool want_grouping(const bc_graph* g, int nsrc, const bc_options& o);
static bc_status group_sources(bc_graph* g, const int* d_src, int nsrc, cudaStream_t st, DevBuf& out,
                               bc_run_stats* acc, std::vector<int>* host_out);
}

namespace {

struct Job {
    bc_job id = 0;
    bc_graph* g = nullptr;
    std::vector<int> src;
    double* out = nullptr;
    bc_status result = BC_PENDING;
    bool done = false;
    bool grouped = false;  // src already in the grouped order (source_order)
    std::chrono::steady_clock::time_point t_submit, t_done;
};

struct Server {
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<std::shared_ptr<Job>> queue;
    std::map<bc_job, std::shared_ptr<Job>> jobs;
    std::vector<std::thread> workers;
    int slots = 1;        // one full-GPU traversal at a time measured best (packing still mixes jobs)
    bool paused = false;  // set while the slot count changes
    long long budget = 0;  // bytes; 0 = decided at start
    long long reserved = 0;
    int running = 0, peak = 0;
    long long completed = 0;
    bc_job next_id = 1;
    bool started = false;
    int pack_limit = 1024;  // sources per packed traversal (saturated R-MAT 14-22 pool, source-arcs/s:
                            // 256 -> 3.06e11, 1024 -> 3.2e11, 4096 -> 3.17e11)
};

Server& server() {
    static Server* s = new Server();  // never destroyed: workers may outlive static teardown
    return *s;
}

void worker_main(int slot) {
    Server& S = server();
    cudaStream_t st;
    cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    Workspace ws;
    DevBuf dsrc, jobbufs;
    long long my_reserved = 0;
    for (;;) {
        std::vector<std::shared_ptr<Job>> batch;
        long long grow = 0;
        int share = 1;  // this run takes 1/share of the GPU's persistent blocks
        {
            std::unique_lock<std::mutex> lk(S.mu);
            for (;;) {
                if (S.paused || slot >= S.slots) {
                    S.cv_work.wait(lk);
                    continue;
                }
                // first admissible job in arrival order
                size_t lead = S.queue.size();
                for (size_t i = 0; i < S.queue.size(); ++i) {
                    const auto& j = S.queue[i];
                    const int K = choose_width(j->g->n, (int)j->src.size(), 0);
                    int nh;
                    long long hc;
                    bool sext;
                    {
                        std::lock_guard<std::mutex> glk(j->g->state_mu);
                        nh = j->g->n_heavy > 0 ? j->g->n_heavy : 0;
                        hc = j->g->hchunk_total;
                        sext = j->g->sticky_ext;
                    }
                    const long long need = (long long)ws_need(j->g->n, K, nh, hc, sext, 64, 64, cap_factor(K, 0)) +
                                           (long long)sizeof(double) * j->g->n * 64;
                    grow = need > my_reserved ? need - my_reserved : 0;
                    if (S.reserved + grow <= S.budget || S.running == 0) { lead = i; break; }
                }
                if (lead < S.queue.size()) {
                    auto L = S.queue[lead];
                    batch.push_back(L);
                    S.queue.erase(S.queue.begin() + (long)lead);
                    int total = (int)L->src.size();
                    for (size_t i = 0; i < S.queue.size() && total < S.pack_limit && batch.size() < 64;) {
                        auto& j = S.queue[i];
                        if (j->g == L->g && total + (int)j->src.size() <= S.pack_limit) {
                            total += (int)j->src.size();
                            batch.push_back(j);
                            S.queue.erase(S.queue.begin() + (long)i);
                        } else {
                            ++i;
                        }
                    }
                    S.reserved += grow;
                    my_reserved += grow;
                    share = S.slots;
                    S.running++;
                    if (S.running > S.peak) S.peak = S.running;
                    break;
                }
                S.cv_work.wait(lk);
            }
        }
        // run the packed jobs
        bc_graph* g = batch[0]->g;
        int nsrc = 0;
        for (auto& j : batch) nsrc += (int)j->src.size();
        bc_options o;
        memset(&o, 0, sizeof o);
        apply_tuning(g, nsrc, o);
        const int K = choose_width(g->n, nsrc, o.batch_width);
        bc_status r = BC_OK;
        // a graph known to be deep: every job through the direct call, which picks
        // the per-source form by the same rule, so each result is the direct call's
        int seen;
        {
            std::lock_guard<std::mutex> lk(g->state_mu);
            seen = g->depth_seen;
        }
        const bool deep = deep_by_depth(g, seen);
        std::vector<bc_status> jr(batch.size(), BC_OK);
        if (deep) {
            for (size_t k = 0; k < batch.size(); ++k)
                jr[k] = bc_compute_ex(g, batch[k]->src.data(), (int)batch[k]->src.size(), batch[k]->out, st, nullptr);
        }
        // each job's sources in the order bc_compute would take them, so that a
        // job's result is the same alone, packed or computed directly
        for (auto& j : batch) {
            if (deep) break;
            if (r != BC_OK || j->grouped || !want_grouping(g, (int)j->src.size(), o)) continue;
            const int n1 = (int)j->src.size();
            DevBuf tmp;
            if (!buf_ensure(dsrc, sizeof(int) * (size_t)n1, st)) {
                r = fail(BC_E_NOMEM, "serving buffers");
                break;
            }
            cudaError_t e = cudaMemcpyAsync(dsrc.p, j->src.data(), sizeof(int) * (size_t)n1, cudaMemcpyHostToDevice, st);
            bc_run_stats gs{};
            std::vector<int> grouped;
            r = e == cudaSuccess ? group_sources(g, (const int*)dsrc.p, n1, st, tmp, &gs, &grouped)
                                 : cuda_fail(e, "source copy");
            buf_release(tmp, st);
            if (r == BC_OK) {
                j->src.swap(grouped);
                j->grouped = true;
            }
        }
        if (!deep) {
            std::vector<int> all;
            std::vector<int> owner;  // job index per source
            for (size_t j = 0; j < batch.size(); ++j) {
                all.insert(all.end(), batch[j]->src.begin(), batch[j]->src.end());
                owner.insert(owner.end(), batch[j]->src.size(), (int)j);
            }
            const int nbatch = (nsrc + K - 1) / K;
            std::vector<int> col_job((size_t)nbatch * K, 0);
            for (int i = 0; i < nbatch * K; ++i) col_job[i] = i < nsrc ? owner[i] : (int)batch.size() - 1;
            const size_t nn = (size_t)(g->n > 0 ? g->n : 1);
            if (r == BC_OK && (!buf_ensure(dsrc, sizeof(int) * (size_t)nsrc, st) ||
                               !buf_ensure(jobbufs, sizeof(double) * nn * batch.size(), st))) {
                r = fail(BC_E_NOMEM, "serving buffers");
            }
            if (r == BC_OK) {
                cudaError_t e = cudaMemcpyAsync(dsrc.p, all.data(), sizeof(int) * (size_t)nsrc, cudaMemcpyHostToDevice, st);
                if (e != cudaSuccess) r = cuda_fail(e, "source copy");
            }
            std::vector<double*> jb;
            for (size_t j = 0; j < batch.size(); ++j) jb.push_back((double*)jobbufs.p + nn * j);
            if (r == BC_OK) {  // runs on the same graph proceed concurrently (own workspace and stream)
                r = run_jobs(g, &ws, (const int*)dsrc.p, nsrc, o, share, jb, &col_job, false, st, nullptr, nullptr,
                             nullptr, nullptr);
            }
            if (r >= 0) {
                for (size_t j = 0; j < batch.size(); ++j) {
                    cudaError_t e = launch_unpermute(jb[j], (const int*)g->inv.p, batch[j]->out, g->n, st);
                    if (e != cudaSuccess) { r = cuda_fail(e, "unpermute"); break; }
                }
                cudaError_t e = cudaStreamSynchronize(st);
                if (e != cudaSuccess && r >= 0) r = cuda_fail(e, "serving run");
            }
        }
        const long long have = (long long)(ws.bytes() + dsrc.bytes + jobbufs.bytes);
        {
            std::lock_guard<std::mutex> lk(S.mu);
            const auto now = std::chrono::steady_clock::now();
            for (size_t k = 0; k < batch.size(); ++k) {
                auto& j = batch[k];
                j->result = deep ? jr[k] : r;
                j->done = true;
                j->t_done = now;
                j->g->users--;
            }
            S.running--;
            S.completed += (long long)batch.size();
            S.reserved += have - my_reserved;
            my_reserved = have;
        }
        S.cv_done.notify_all();
        S.cv_work.notify_all();
    }
}

void server_start_locked(Server& S) {
    if (S.started) return;
    if (S.budget <= 0) {
        size_t fr = 0, tot = 0;
        cudaMemGetInfo(&fr, &tot);
        S.budget = (long long)(0.8 * (double)fr);
    }
    for (int i = 0; i < S.slots; ++i) {
        S.workers.emplace_back(worker_main, i);
        S.workers.back().detach();
    }
    S.started = true;
}

}  // namespace

// ------------------------------------------------------------------ many graphs, one captured sequence
// Every item (graph, sources, output) gets: source mapping, one persistent
// cooperative launch over all its batches, a status word, the unpermute into
// its output.  Items are grouped by batch width; one workspace per width,
// sized for the largest graph of the group, serves its items in stream order.
// The whole sequence is recorded once into a CUDA graph and replayed by
// bc_many_run; items whose status asks for the extended path-count form or
// larger level lists are redone afterwards through bc_compute_ex.
struct ManyItem {
    bc_graph* g = nullptr;
    std::vector<int> src;      // original ids (host copy)
    long long src_off = 0;     // into the plan's device source buffer
    double* out = nullptr;
    int K = 0, nbatch = 0;
    bool deep = false;         // the per-source form: run at each replay by bc_compute_ex, not recorded
};

struct bc_many_plan {
    std::vector<ManyItem> items;
    std::map<int, std::unique_ptr<Workspace>> ws;  // by width
    DevBuf dsrc, dstatus;
    bc_options opt{};
    cudaStream_t cap_stream = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    int launches = 0;
};

static void many_release(bc_many_plan* pl) {
    if (pl->exec) cudaGraphExecDestroy(pl->exec);
    if (pl->graph) cudaGraphDestroy(pl->graph);
    cudaStream_t st = pl->cap_stream;
    if (st) cudaStreamSynchronize(st);
    for (auto& kv : pl->ws) kv.second->release(st);
    buf_release(pl->dsrc, st);
    buf_release(pl->dstatus, st);
    if (st) {
        cudaStreamSynchronize(st);
        cudaStreamDestroy(st);
    }
}

// Record the per-item sequence on the plan's capture stream.
static bc_status many_record(bc_many_plan* pl) {
    cudaStream_t st = pl->cap_stream;
    cudaError_t e = cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return cuda_fail(e, "begin capture");
    bc_status r = BC_OK;
    int launches = 0;
    for (size_t i = 0; i < pl->items.size() && r == BC_OK; ++i) {
        ManyItem& it = pl->items[i];
        if (it.deep) continue;  // run at replay time, outside the recorded graph
        bc_graph* g = it.g;
        Workspace* w = pl->ws[it.K].get();
        const int blocks = grid_blocks(it.K, false, pl->opt.blocks_per_sm, 1);
        // this item's teams: as many as its batches and the workspace's slices allow
        int nteams = 1, team_blocks = blocks;
        choose_teams(g->m, it.K, it.nbatch, blocks, w->lay.bytes, pl->opt.teams, &nteams, &team_blocks);
        nteams = std::min(nteams, w->nteams);
        team_blocks = blocks / nteams;
        const int saved = w->nteams;
        w->nteams = nteams;
        KParams p = make_params(g, w, it.nbatch, pl->opt, false, team_blocks);
        int* status = (int*)pl->dstatus.p + i;
        e = reset_controls(w, it.nbatch, st);
        w->nteams = saved;
        if (e != cudaSuccess ||
            (e = cudaMemsetAsync(w->bc.p, 0, sizeof(double) * (size_t)(g->n > 0 ? g->n : 1), st)) != cudaSuccess ||
            (e = launch_map_sources((const int*)pl->dsrc.p + it.src_off, (int)it.src.size(), (const int*)g->inv.p,
                                    g->n, it.K, (int*)w->src.p, it.nbatch, (int*)w->bad.p, st)) != cudaSuccess ||
            (e = launch_batches(it.K, p, team_blocks * nteams, st)) != cudaSuccess ||
            (e = launch_collect_status((const Ctl*)w->gctl.p, (const int*)w->bstat.p, it.nbatch, status, st)) !=
                cudaSuccess ||
            (e = launch_unpermute((const double*)w->bc.p, (const int*)g->inv.p, it.out, g->n, st)) != cudaSuccess) {
            r = cuda_fail(e, "recording the many-graph sequence");
        }
        launches += 5;  // control reset, source mapping, traversal, status, unpermute
    }
    cudaGraph_t graph = nullptr;
    e = cudaStreamEndCapture(st, &graph);
    if (r != BC_OK) {
        if (graph) cudaGraphDestroy(graph);
        return r;
    }
    if (e != cudaSuccess) return cuda_fail(e, "end capture");
    pl->graph = graph;
    e = cudaGraphInstantiate(&pl->exec, graph, 0);
    if (e != cudaSuccess) return cuda_fail(e, "graph instantiate");
    pl->launches = launches;
    return BC_OK;
}

// ------------------------------------------------------------------ C ABI
extern "C" {

bc_status bc_set_allocator(bc_alloc_fn alloc, bc_free_fn free_fn, void* ctx) {
    if ((alloc == nullptr) != (free_fn == nullptr))
        return fail(BC_E_INVALID_ARG, "alloc and free must be both set or both NULL");
    std::lock_guard<std::mutex> lk(g_alloc_mu);
    g_hook.alloc = alloc;
    g_hook.free_fn = free_fn;
    g_hook.ctx = ctx;
    return BC_OK;
}

bc_status bc_graph_create(const int32_t* offsets, const int32_t* indices, int32_t n, int64_t m, uint32_t flags,
                          bc_stream_t stream, bc_graph** out) {
    if (!out) return fail(BC_E_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (n < 0 || m < 0) return fail(BC_E_INVALID_ARG, "negative size (n=%d, m=%lld)", n, (long long)m);
    if (!offsets || (m > 0 && !indices)) return fail(BC_E_INVALID_ARG, "offsets/indices NULL");
    if (flags & ~(BC_UNDIRECTED | BC_INPUT_ON_DEVICE | BC_SKIP_VALIDATION))
        return fail(BC_E_INVALID_ARG, "unknown flag bits 0x%x", flags);
    const bool directed = !(flags & BC_UNDIRECTED);
    if (m >= (1ll << 31) - 1 || n >= (1 << 30)) return fail(BC_E_LIMIT, "graph beyond int32 CSR limits");
    cudaStream_t st = (cudaStream_t)stream;
    std::unique_ptr<bc_graph> g(new bc_graph());
    g->n = n;
    g->m = m;
    g->directed = directed;
    const int* d_off = offsets;
    const int* d_adj = indices;
    DevBuf in_off, in_adj;
    if (!(flags & BC_INPUT_ON_DEVICE)) {
        if (!buf_ensure(in_off, sizeof(int) * ((size_t)n + 1), st) ||
            !buf_ensure(in_adj, sizeof(int) * (size_t)(m > 0 ? m : 1), st)) {
            buf_release(in_off, st);
            buf_release(in_adj, st);
            return fail(BC_E_NOMEM, "device allocation failed for the input copy");
        }
        cudaError_t e = cudaMemcpyAsync(in_off.p, offsets, sizeof(int) * ((size_t)n + 1), cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess && m > 0)
            e = cudaMemcpyAsync(in_adj.p, indices, sizeof(int) * (size_t)m, cudaMemcpyHostToDevice, st);
        if (e != cudaSuccess) {
            buf_release(in_off, st);
            buf_release(in_adj, st);
            return cuda_fail(e, "input copy");
        }
        d_off = (const int*)in_off.p;
        d_adj = (const int*)in_adj.p;
    }
    IngestOut io;
    bool oom = false;
    {
        std::lock_guard<std::mutex> lk(g_alloc_mu);
        g->hook = g_hook;
    }
    cudaError_t e = ingest(d_off, d_adj, n, m, !(flags & BC_SKIP_VALIDATION), directed, st, ingest_alloc, ingest_free,
                           &io, &oom);
    buf_release(in_off, st);
    buf_release(in_adj, st);
    auto adopt = [&](DevBuf& b, void* p, size_t bytes) { b.p = p; b.bytes = bytes; b.hook = g->hook; };
    adopt(g->off, io.off, sizeof(int) * ((size_t)n + 1));
    adopt(g->adj, io.adj, sizeof(int) * (size_t)(m > 0 ? m : 1));
    adopt(g->perm, io.perm, sizeof(int) * (size_t)(n > 0 ? n : 1));
    adopt(g->inv, io.inv, sizeof(int) * (size_t)(n > 0 ? n : 1));
    if (io.ioff) adopt(g->ioff, io.ioff, sizeof(int) * ((size_t)n + 1));
    if (io.iadj) adopt(g->iadj, io.iadj, sizeof(int) * (size_t)(m > 0 ? m : 1));
    auto drop = [&]() {
        buf_release(g->off, st); buf_release(g->adj, st); buf_release(g->perm, st); buf_release(g->inv, st);
        buf_release(g->ioff, st); buf_release(g->iadj, st);
    };
    if (oom) { drop(); return fail(BC_E_NOMEM, "device allocation failed during ingest"); }
    if (e != cudaSuccess) { drop(); return cuda_fail(e, "ingest"); }
    if (io.reason) {
        static const char* why[] = {"", "offsets not monotone, offsets[0] != 0 or offsets[n] != m",
                                    "an index outside [0, n)", "a self-loop", "a duplicate arc",
                                    "an arc without its reverse (graph not symmetric)"};
        drop();
        return fail(BC_E_INVALID_GRAPH, "invalid CSR: %s", why[io.reason]);
    }
    g->max_deg = io.max_deg;
    g->max_in_deg = io.max_in_deg;
    // rows are sorted by out-degree; in a directed graph a vertex without out-arcs
    // can still be reached, so every vertex takes part in the pull steps
    g->n_nz = directed ? n : io.n_nz;
    *out = g.release();
    return BC_OK;
}

bc_status bc_graph_destroy(bc_graph* g) {
    if (!g) return fail(BC_E_INVALID_ARG, "graph is NULL");
    if (g->users.load() > 0)
        return fail(BC_E_BUSY, "graph still used by %d plan items or unfinished serving jobs", g->users.load());
    cudaStream_t st = g->last_stream;
    cudaStreamSynchronize(st);
    for (auto& kv : g->ws) kv.second->release(st);
    buf_release(g->off, st);
    buf_release(g->adj, st);
    buf_release(g->perm, st);
    buf_release(g->ioff, st);
    buf_release(g->iadj, st);
    buf_release(g->landmark, st);
    for (DevBuf* b : {&g->deep_state, &g->deep_order, &g->deep_delta, &g->deep_aux}) buf_release(*b, st);
    for (DevBuf* b : {&g->pr_ccum, &g->pr_rank, &g->pr_scratch, &g->pr_cpart, &g->pr_carr, &g->pr_ctl, &g->pr_small})
        buf_release(*b, st);
    for (DevBuf* b : {&g->w, &g->wdist, &g->wsig, &g->winv, &g->wdel,
                      &g->wrho, &g->wmark, &g->wbc, &g->wctl, &g->wsrc, &g->wscr, &g->warr, &g->word, &g->whist, &g->wdag})
        buf_release(*b, st);
    buf_release(g->inv, st);
    cudaStreamSynchronize(st);
    delete g;
    return BC_OK;
}

bc_status bc_graph_create_weighted(const int32_t* offsets, const int32_t* indices, const int32_t* weights, int32_t n,
                                   int64_t m, uint32_t flags, bc_stream_t stream, bc_graph** out) {
    if (!out) return fail(BC_E_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (m > 0 && !weights) return fail(BC_E_INVALID_ARG, "weights NULL");
    bc_graph* g = nullptr;
    bc_status r = bc_graph_create(offsets, indices, n, m, flags, stream, &g);
    if (r != BC_OK) return r;
    cudaStream_t st = (cudaStream_t)stream;
    const bool on_dev = (flags & BC_INPUT_ON_DEVICE) != 0;
    DevBuf doff, dadj, dw, derr;
    auto bail = [&](bc_status rr) {
        buf_release(doff, st);
        buf_release(dadj, st);
        buf_release(dw, st);
        buf_release(derr, st);
        if (rr != BC_OK) bc_graph_destroy(g);
        return rr;
    };
    if (!buf_ensure(g->w, sizeof(int) * (size_t)(m > 0 ? m : 1), st) || !buf_ensure(derr, sizeof(int), st))
        return bail(fail(BC_E_NOMEM, "weight buffers"));
    const int *ooff = offsets, *oadj = indices, *ow = weights;
    cudaError_t e = cudaMemsetAsync(derr.p, 0, sizeof(int), st);
    if (!on_dev && e == cudaSuccess) {
        if (!buf_ensure(doff, sizeof(int) * ((size_t)n + 1), st) || !buf_ensure(dadj, sizeof(int) * (size_t)(m > 0 ? m : 1), st) ||
            !buf_ensure(dw, sizeof(int) * (size_t)(m > 0 ? m : 1), st))
            return bail(fail(BC_E_NOMEM, "weight ingest buffers"));
        e = cudaMemcpyAsync(doff.p, offsets, sizeof(int) * ((size_t)n + 1), cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess && m > 0) e = cudaMemcpyAsync(dadj.p, indices, sizeof(int) * (size_t)m, cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess && m > 0) e = cudaMemcpyAsync(dw.p, weights, sizeof(int) * (size_t)m, cudaMemcpyHostToDevice, st);
        ooff = (const int*)doff.p;
        oadj = (const int*)dadj.p;
        ow = (const int*)dw.p;
    }
    if (e == cudaSuccess)
        e = launch_weight_ingest(ooff, oadj, ow, (const int*)g->perm.p, (const int*)g->off.p, (const int*)g->adj.p, n,
                                 (int*)g->w.p, (int*)derr.p, !g->directed && !(flags & BC_SKIP_VALIDATION), st);
    int herr = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&herr, derr.p, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return bail(cuda_fail(e, "weight ingest"));
    if (!(flags & BC_SKIP_VALIDATION) && herr)
        return bail(fail(BC_E_INVALID_GRAPH, "weights: %s%s%s", (herr & 1) ? "rows not sorted ascending; " : "",
                         (herr & 2) ? "a weight <= 0; " : "", (herr & 4) ? "the two arcs of an edge differ" : ""));
    *out = g;
    return bail(BC_OK);
}

bc_status bc_compute_weighted(bc_graph* g, const int32_t* sources, int32_t nsrc, double* out_bc, bc_stream_t stream) {
    if (!g) return fail(BC_E_INVALID_ARG, "graph is NULL");
    if (!g->w.p) return fail(BC_E_INVALID_ARG, "the graph has no weights (bc_graph_create_weighted)");
    if (nsrc < 0 || (nsrc > 0 && !sources)) return fail(BC_E_INVALID_ARG, "bad source list");
    if (!out_bc && g->n > 0) return fail(BC_E_INVALID_ARG, "out_bc is NULL");
    cudaStream_t st = (cudaStream_t)stream;
    std::lock_guard<std::mutex> lk(g->mu);
    g->last_stream = st;
    if (g->n == 0) return BC_OK;
    const size_t n = (size_t)g->n;
    bc_status r = ensure_heavy(g, st);
    if (r != BC_OK) return r;
    constexpr int KW = 32;
    const int nbatch = (nsrc + KW - 1) / KW;
    const size_t cells = n * KW;
    DevBuf hsrc;
    const int* d_src = sources;
    if (nsrc > 0 && !is_device_ptr(sources)) {
        for (int i = 0; i < nsrc; ++i)
            if (sources[i] < 0 || sources[i] >= g->n)
                return fail(BC_E_SOURCE, "source %d (entry %d) is outside [0, %d)", sources[i], i, g->n);
        if (!buf_ensure(hsrc, sizeof(int) * (size_t)nsrc, st)) return fail(BC_E_NOMEM, "source buffer");
        cudaError_t e = cudaMemcpyAsync(hsrc.p, sources, sizeof(int) * (size_t)nsrc, cudaMemcpyHostToDevice, st);
        if (e != cudaSuccess) {
            buf_release(hsrc, st);
            return cuda_fail(e, "source copy");
        }
        d_src = (const int*)hsrc.p;
    }
    DevBuf grouped;
    auto done = [&](bc_status rr) {
        buf_release(hsrc, st);
        buf_release(grouped, st);
        return rr;
    };
    // batches of sources with similar hub distances (the rule and order of
    // bc_compute): their 32 columns then agree on the row order below
    bc_run_stats pre{};
    {
        bc_options o;
        memset(&o, 0, sizeof o);
        if (nbatch > 1 && want_grouping(g, nsrc, o)) {
            bc_status gr = group_sources(g, d_src, nsrc, st, grouped, &pre, nullptr);
            if (gr < 0) return done(gr);
            d_src = (const int*)grouped.p;
        }
    }
    if (!buf_ensure(g->wdist, 8 * cells, st) || !buf_ensure(g->wsig, 8 * cells, st) || !buf_ensure(g->winv, 8 * cells, st) ||
        !buf_ensure(g->wdel, 8 * cells, st) || !buf_ensure(g->wrho, 8 * cells, st) || !buf_ensure(g->wmark, 8 * n, st) ||
        !buf_ensure(g->wbc, 8 * n, st) || !buf_ensure(g->wctl, sizeof(Ctl) + 8 * sizeof(int) + 32, st) ||
        !buf_ensure(g->wsrc, sizeof(int) * (size_t)(nbatch > 0 ? nbatch : 1) * KW + sizeof(int), st) ||
        !buf_ensure(g->wscr, 24 * KW * (size_t)std::max(1ll, g->hchunk_total), st) ||
        !buf_ensure(g->warr, sizeof(int) * (size_t)std::max(1, g->n_heavy), st) ||
        !buf_ensure(g->word, sizeof(int) * n, st) || !buf_ensure(g->whist, sizeof(unsigned int) * kWbcHistWords, st) ||
        !buf_ensure(g->wdag, sizeof(unsigned int) * (size_t)(g->m > 0 ? g->m : 1), st))
        return done(fail(BC_E_NOMEM, "weighted BC buffers"));
    const WCsr wout{(const int*)g->off.p, (const int*)g->adj.p, (const int*)g->w.p, g->n_heavy, g->hchunk_total,
                    (const int*)g->hcum.p};
    // in-arcs serve only the dependency loop's stamps (rows and indices)
    const WCsr win = !g->directed ? wout
                                  : WCsr{(const int*)g->ioff.p, (const int*)g->iadj.p, nullptr, 0, 0, nullptr};
    const size_t narr = (size_t)std::max(1, g->n_heavy);
    Ctl* ctl = (Ctl*)g->wctl.p;
    int* changed = (int*)((char*)g->wctl.p + sizeof(Ctl));
    int* passes = changed + 4;
    static_assert((sizeof(Ctl) + 8 * sizeof(int)) % 8 == 0, "visited counters need 8-byte alignment");
    unsigned long long* visited = (unsigned long long*)(changed + 8);  // arcs, rows, mask arcs, mask lanes
    int* bad = (int*)g->wsrc.p + (size_t)(nbatch > 0 ? nbatch : 1) * KW;
    cudaError_t e = cudaMemsetAsync(g->wbc.p, 0, 8 * n, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(g->wctl.p, 0, sizeof(Ctl) + 8 * sizeof(int) + 32, st);
    if (e == cudaSuccess && nbatch > 0) {
        e = cudaMemsetAsync(bad, 0, sizeof(int), st);
        if (e == cudaSuccess)
            e = launch_map_sources(d_src, nsrc, (const int*)g->inv.p, g->n, KW, (int*)g->wsrc.p, nbatch, bad, st);
    }
    int hbad = 0;
    if (e == cudaSuccess && nbatch > 0) e = cudaMemcpyAsync(&hbad, bad, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return done(cuda_fail(e, "weighted set-up"));
    if (hbad) return done(fail(BC_E_SOURCE, "a source id is outside [0, %d)", g->n));
    const int blocks = wbc_blocks();
    if (blocks < 1) return done(fail(BC_E_CUDA, "weighted BC kernel cannot be resident"));
    cudaEvent_t ev[2];
    cudaEventCreate(&ev[0]);
    cudaEventCreate(&ev[1]);
    cudaEventRecord(ev[0], st);
    for (int b = 0; b < nbatch && e == cudaSuccess; ++b) {
        // fresh barrier and pass flags per launch (pass counts accumulate)
        e = cudaMemsetAsync(ctl, 0, sizeof(Ctl), st);
        if (e == cudaSuccess) e = cudaMemsetAsync(changed, 0, 4 * sizeof(int), st);
        if (e == cudaSuccess) e = cudaMemsetAsync(g->warr.p, 0, sizeof(int) * narr, st);
        if (e == cudaSuccess) e = cudaMemsetAsync(g->wmark.p, 0, 8 * n, st);
        if (e == cudaSuccess)
            e = launch_wbc(g->n, wout, win, (int*)g->warr.p, g->wscr.p, (const int*)g->wsrc.p + (size_t)b * KW,
                           (long long*)g->wdist.p,
                           (unsigned long long*)g->wsig.p, (double*)g->winv.p, (double*)g->wdel.p,
                           (double*)g->wrho.p, (int*)g->wmark.p, (int*)g->word.p, (unsigned int*)g->whist.p,
                           (unsigned int*)g->wdag.p, (double*)g->wbc.p, ctl, changed, passes, visited,
                           40000000000ll, blocks, st);
        int herr = 0;
        if (e == cudaSuccess) e = cudaMemcpyAsync(&herr, &ctl->err, sizeof(int), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e == cudaSuccess && herr) {
            cudaEventDestroy(ev[0]);
            cudaEventDestroy(ev[1]);
            if (herr & ERR_SIGMA_RANGE) return done(fail(BC_E_SIGMA_RANGE, "a weighted path count reached 2^64"));
            if (herr & ERR_TIMEOUT) return done(fail(BC_E_TIMEOUT, "a grid-barrier wait exceeded its cycle budget"));
            return done(fail(BC_E_CUDA, "weighted BC kernel error 0x%x", herr));
        }
    }
    cudaEventRecord(ev[1], st);
    int hp[3] = {0, 0, 0}, hflags = 0;
    unsigned long long hv[4] = {0, 0, 0, 0};
    if (e == cudaSuccess) e = launch_unpermute((const double*)g->wbc.p, (const int*)g->inv.p, out_bc, g->n, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(hp, passes, sizeof hp, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(hv, visited, sizeof hv, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&hflags, &ctl->flags, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    float ms = 0.f;
    if (e == cudaSuccess) cudaEventElapsedTime(&ms, ev[0], ev[1]);
    cudaEventDestroy(ev[0]);
    cudaEventDestroy(ev[1]);
    if (e != cudaSuccess) return done(cuda_fail(e, "weighted BC"));
    bc_run_stats s{};
    s.batch_width = KW;
    s.batches = nbatch;
    s.max_levels = hp[0];    // passes of the distance loop, summed over batches
    s.pull_levels = hp[1];   // passes of the path-count loop
    s.push_levels = hp[2];   // passes of the dependency loop
    s.grid_blocks = blocks;
    s.kernel_launches = 2 + nbatch + pre.kernel_launches;  // source mapping, one per batch, unpermute, grouping
    s.kernel_ms = ms;
    s.order_ms = pre.kernel_ms;
    s.teams = 1;
    s.arcs_visited = (int64_t)hv[0];
    s.rows_visited = (int64_t)hv[1];
    s.mask_arcs = (int64_t)hv[2];
    s.mask_lanes = (int64_t)hv[3];
    g->last = s;
    return done((hflags & BST_INEXACT) ? BC_W_SIGMA_INEXACT : BC_OK);
}

bc_status bc_graph_info(const bc_graph* g, int32_t* n, int64_t* m, int32_t* max_degree, int32_t* n_nonisolated) {
    if (!g) return fail(BC_E_INVALID_ARG, "graph is NULL");
    if (n) *n = g->n;
    if (m) *m = g->m;
    if (max_degree) *max_degree = g->max_deg;
    if (n_nonisolated) *n_nonisolated = g->n_nz;
    return BC_OK;
}

bc_status bc_graph_export(const bc_graph* g, int32_t* perm, int32_t* offsets, int32_t* indices) {
    if (!g) return fail(BC_E_INVALID_ARG, "graph is NULL");
    cudaError_t e = cudaSuccess;
    if (perm && g->n > 0) e = cudaMemcpy(perm, g->perm.p, sizeof(int) * (size_t)g->n, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && offsets)
        e = cudaMemcpy(offsets, g->off.p, sizeof(int) * ((size_t)g->n + 1), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && indices && g->m > 0)
        e = cudaMemcpy(indices, g->adj.p, sizeof(int) * (size_t)g->m, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e, "export");
    return BC_OK;
}

// Source grouping (bc_options.source_order).  Two sources at the same
// distances from the graph's hubs reach most vertices at the same levels, so
// in one batch their columns match the same arcs: more arcs reach the
// column-mapped threshold and fewer single (arc, column) pairs remain.  The
// key of a source is its distance vector to the 32 highest-degree vertices
// (relabelled ids 0..31), read from the graph's landmark table (one
// forward-only traversal of those 32 vertices, built on first use and kept;
// undirected: d(h, s) = d(s, h)); sources are stably sorted by it,
// nearest-hub distance first.  Levels are exact integers, so the order does
// not depend on anything but the graph and the list.
static bool want_grouping(const bc_graph* g, int nsrc, const bc_options& o) {
    if (o.source_order == 1 || g->directed || g->n_nz < 32) return false;
    if (o.source_order == 2) return true;
    return nsrc >= 256 && g->n_nz >= 2048 && (double)g->max_deg * g->n_nz >= 16.0 * (double)g->m;
}

// The landmark table is a fact of the graph: built once, on first use, by a
// forward-only traversal of the 32 first relabelled vertices in a 32-wide
// workspace of its own (freed right after), then kept ([n][32] uint16).
static bc_status ensure_landmarks(bc_graph* g, cudaStream_t st, bc_run_stats* acc) {
    constexpr int L = 32;
    std::lock_guard<std::mutex> lk(g->lm_mu);
    if (g->lm_levels >= 0) return BC_OK;
    Workspace tmp;
    auto done = [&](bc_status r) {
        cudaStreamSynchronize(st);
        tmp.release(st);
        return r;
    };
    if (!buf_ensure(tmp.bc, sizeof(double) * (size_t)g->n, st) ||
        !buf_ensure(g->landmark, sizeof(unsigned short) * (size_t)g->n * L, st))
        return done(fail(BC_E_NOMEM, "landmark table"));
    bc_options o;
    memset(&o, 0, sizeof o);
    o.batch_width = L;
    std::vector<double*> jb{(double*)tmp.bc.p};
    bc_run_stats rs{};
    int kused = 0, levels = 0;
    bool ext = false;
    bc_status r = run_jobs(g, &tmp, (const int*)g->perm.p, L, o, 1, jb, nullptr, true, st, &rs, &kused, &ext, &levels);
    if (r < 0) return done(r);
    KParams p = make_params(g, &tmp, 1, o, ext, 1);
    cudaError_t e = launch_level_table(p, L, levels, (unsigned short*)g->landmark.p, g->n, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return done(cuda_fail(e, "landmark table"));
    g->lm_levels = levels;
    acc->kernel_launches += rs.kernel_launches + (levels > 0 ? 1 : 0);
    acc->kernel_ms += rs.kernel_ms;
    return done(BC_OK);
}

static bc_status group_sources(bc_graph* g, const int* d_src, int nsrc, cudaStream_t st, DevBuf& out,
                               bc_run_stats* acc, std::vector<int>* host_out) {
    constexpr int L = 32;
    bc_status r = ensure_landmarks(g, st, acc);
    if (r != BC_OK) return r;
    const int levels = g->lm_levels;
    DevBuf keys;
    std::vector<unsigned short> hk((size_t)nsrc * L);
    std::vector<int> hs(nsrc);
    if (!buf_ensure(keys, sizeof(unsigned short) * hk.size(), st)) return fail(BC_E_NOMEM, "grouping buffers");
    cudaEvent_t ev[2];
    cudaEventCreate(&ev[0]);
    cudaEventCreate(&ev[1]);
    cudaEventRecord(ev[0], st);
    cudaError_t e = launch_source_keys((const unsigned short*)g->landmark.p, L, L, g->n, d_src, nsrc,
                                       (const int*)g->inv.p, (unsigned short*)keys.p, st);
    cudaEventRecord(ev[1], st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(hk.data(), keys.p, sizeof(unsigned short) * hk.size(), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(hs.data(), d_src, sizeof(int) * (size_t)nsrc, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    float kms = 0.f;
    if (e == cudaSuccess) cudaEventElapsedTime(&kms, ev[0], ev[1]);
    cudaEventDestroy(ev[0]);
    cudaEventDestroy(ev[1]);
    buf_release(keys, st);
    if (e != cudaSuccess) return cuda_fail(e, "source grouping");
    acc->kernel_launches += 1;
    acc->kernel_ms += kms;
    // levels are below `levels`; 0xFFFF (unreached) ranks after them
    std::vector<int> idx(nsrc), nxt(nsrc), cnt((size_t)levels + 2);
    for (int i = 0; i < nsrc; ++i) idx[i] = i;
    auto digit = [&](int i, int j) {
        const unsigned short v = hk[(size_t)i * L + j];
        return v == 0xFFFFu || v > levels ? levels + 1 : (int)v;
    };
    if (levels + 1 < 16) {
        // shallow graphs: 4 bits per landmark, the 32 digits packed most
        // significant first into two words; ties keep the given order
        struct Packed {
            unsigned long long hi, lo;
            int i;
        };
        std::vector<Packed> pk(nsrc);
        for (int i = 0; i < nsrc; ++i) {
            unsigned long long hi = 0, lo = 0;
            for (int j = 0; j < 16; ++j) hi = hi << 4 | (unsigned long long)digit(i, j);
            for (int j = 16; j < L; ++j) lo = lo << 4 | (unsigned long long)digit(i, j);
            pk[i] = Packed{hi, lo, i};
        }
        std::sort(pk.begin(), pk.end(), [](const Packed& a, const Packed& b) {
            if (a.hi != b.hi) return a.hi < b.hi;
            if (a.lo != b.lo) return a.lo < b.lo;
            return a.i < b.i;
        });
        for (int i = 0; i < nsrc; ++i) idx[i] = pk[i].i;
    }
    // deeper graphs: stable LSD counting sort, least significant landmark first
    for (int j = L - 1; levels + 1 >= 16 && j >= 0; --j) {
        std::fill(cnt.begin(), cnt.end(), 0);
        for (int i = 0; i < nsrc; ++i) cnt[digit(idx[i], j)]++;
        for (int d = 0, run = 0; d < (int)cnt.size(); ++d) {
            const int c = cnt[d];
            cnt[d] = run;
            run += c;
        }
        for (int i = 0; i < nsrc; ++i) nxt[cnt[digit(idx[i], j)]++] = idx[i];
        idx.swap(nxt);
    }
    std::vector<int> grouped(nsrc);
    for (int i = 0; i < nsrc; ++i) grouped[i] = hs[idx[i]];
    if (host_out) *host_out = grouped;
    if (!buf_ensure(out, sizeof(int) * (size_t)nsrc, st)) return fail(BC_E_NOMEM, "source buffer");
    e = cudaMemcpyAsync(out.p, grouped.data(), sizeof(int) * (size_t)nsrc, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "source copy");
    return BC_OK;
}

// ------------------------------------------------------------------ per-source form (deep graphs)

// The per-source form (deep.cu) over a source list (original ids, device):
// rounds of R sources, each one launch of `blocks` blocks (one source at a
// time per block) writing R dependency rows, then the rows added to bc_rel
// (relabelled, cleared first) in list order.  Memory: per block 44 bytes per
// vertex plus its level starts; per source of a round 8 bytes per vertex;
// together within min(30% of free memory, 24 GB).
struct DeepPlan {
    int threads = 0, sms = 0;
    long long blocks = 0, R = 0, stride = 0;
    int slots = 0;
};

// Launch shape of the per-source form: the widest block (1024, 512 or 256
// threads) whose resident grid still covers the sources, as many blocks as
// are resident (or wanted), and rounds of R sources within the memory budget.
static bc_status deep_plan(const bc_graph* g, int nsrc, const bc_options& o, bool forward_only, DeepPlan* pl) {
    const int n = g->n;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (sms < 1) sms = 1;
    int threads = 256, per_sm = deep_blocks_per_sm(256);
    for (int t : {1024, 512}) {
        const int b = deep_blocks_per_sm(t);
        if (b > 0 && (long long)b * sms >= nsrc) {
            threads = t;
            per_sm = b;
            break;
        }
    }
    if (per_sm < 1) return fail(BC_E_CUDA, "per-source kernel cannot be resident (occupancy 0)");
    if (o.blocks_per_sm > 0 && o.blocks_per_sm < per_sm) per_sm = o.blocks_per_sm;
    const long long stride = ((long long)n + 31) & ~31LL;
    const int slots = (int)std::min<long long>(kLevelSlots, (long long)n + 3);
    // a round's dependency rows: 8 bytes per vertex and source (none when forward only)
    const double per_block = 44.0 * (double)stride + 4.0 * (double)slots, per_src = forward_only ? 0.0 : 8.0 * n;
    size_t fr = 0, tot = 0;
    if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) {
        cudaGetLastError();
        fr = 0;
    }
    const double held = (double)(g->deep_state.bytes + g->deep_order.bytes + g->deep_delta.bytes);
    const double budget = std::min(0.3 * ((double)fr + held), 24e9);
    long long blocks = std::min<long long>((long long)per_sm * sms, nsrc);
    blocks = std::min<long long>(blocks, (long long)(budget / (per_block + per_src)));
    if (blocks < 1) return fail(BC_E_NOMEM, "per-source form: no room for one block's state");
    long long R = forward_only ? (long long)nsrc : (long long)((budget - (double)blocks * per_block) / per_src);
    R = std::max<long long>(blocks, std::min<long long>(R, nsrc));
    R = std::min<long long>(R, blocks * 0x8000LL);  // epochs of one launch stay below 2^16
    pl->threads = threads;
    pl->sms = sms;
    pl->blocks = blocks;
    pl->R = R;
    pl->stride = stride;
    pl->slots = slots;
    return BC_OK;
}

// Outputs of a forward-only run (bc_bfs): [nsrc][n] rows in original ids.
struct BfsOut {
    int* level;
    double* sigma;
    int* sigma_exp;
};

static bc_status run_deep(bc_graph* g, const int* d_src, int nsrc, const bc_options& o, cudaStream_t st,
                          double* bc_rel, bc_run_stats* out, const BfsOut* bfs = nullptr) {
    const int n = g->n;
    bc_status hr = ensure_heavy(g, st);
    if (hr != BC_OK) return hr;
    DeepPlan pl;
    if ((hr = deep_plan(g, nsrc, o, bfs != nullptr, &pl)) != BC_OK) return hr;
    const int threads = pl.threads, slots = pl.slots;
    const long long blocks = pl.blocks, R = pl.R, stride = pl.stride;
    const size_t rec_bytes = sizeof(DeepRec) * (size_t)blocks * (size_t)stride;
    const size_t ord_bytes = (sizeof(int) + sizeof(int2)) * (size_t)blocks * (size_t)stride;
    const size_t lvl_bytes = sizeof(int) * (size_t)blocks * (size_t)slots;
    const size_t aux_bytes = 2 * sizeof(unsigned long long) + sizeof(int) * ((size_t)nsrc + 2 * (size_t)R + 1);
    void* old_state = g->deep_state.p;
    if (!buf_ensure(g->deep_state, rec_bytes, st) || !buf_ensure(g->deep_order, ord_bytes + lvl_bytes, st) ||
        (!bfs && !buf_ensure(g->deep_delta, sizeof(double) * (size_t)R * n, st)) ||
        !buf_ensure(g->deep_aux, aux_bytes, st))
        return fail(BC_E_NOMEM, "per-source form buffers");
    if (g->deep_state.p != old_state) g->deep_stride = -1;  // fresh memory: clear before use
    char* ap = (char*)g->deep_aux.p;
    unsigned long long* ctr = (unsigned long long*)ap;
    int* src_rel = (int*)(ap + 2 * sizeof(unsigned long long));
    int* status = src_rel + nsrc;
    int* depth = status + R;
    int* bad = depth + R;
    cudaError_t e = cudaMemsetAsync(ap, 0, aux_bytes, st);
    if (e == cudaSuccess) e = launch_map_sources(d_src, nsrc, (const int*)g->inv.p, n, 1, src_rel, nsrc, bad, st);
    int hbad = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&hbad, bad, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "per-source form setup");
    if (hbad) return fail(BC_E_SOURCE, "a source id is outside [0, %d)", n);
    if (!bfs && (e = cudaMemsetAsync(bc_rel, 0, sizeof(double) * (size_t)n, st)) != cudaSuccess)
        return cuda_fail(e, "memset");
    DeepParams p{};
    p.n = n;
    p.off = (const int*)g->off.p;
    p.adj = (const int*)g->adj.p;
    p.ioff = g->directed ? (const int*)g->ioff.p : nullptr;
    p.iadj = g->directed ? (const int*)g->iadj.p : nullptr;
    p.n_heavy = g->n_heavy;
    p.stride = stride;
    p.rec = (DeepRec*)g->deep_state.p;
    p.order = (int*)g->deep_order.p;
    p.orow = (int2*)((char*)g->deep_order.p + sizeof(int) * (size_t)blocks * (size_t)stride);
    p.lvl = (int*)((char*)g->deep_order.p + ord_bytes);
    p.level_slots = slots;
    p.delta = bfs ? nullptr : (double*)g->deep_delta.p;
    p.inv = (const int*)g->inv.p;
    p.status = status;
    p.depth = depth;
    p.dag_pairs = ctr;
    p.reached_pairs = ctr + 1;
    bc_run_stats s{};
    s.batch_width = 1;
    s.batches = nsrc;
    s.grid_blocks = (int)blocks;
    s.teams = (int)blocks;
    s.deep_sources = nsrc;
    s.kernel_launches = 1;  // source mapping
    bool inexact = false;
    std::vector<int> hst((size_t)R), hdp((size_t)R);
    for (long long r0 = 0; r0 < nsrc; r0 += R) {
        const int cnt = (int)std::min<long long>(R, nsrc - r0);
        const int nb = (int)std::min<long long>(blocks, cnt);
        const unsigned iters = (unsigned)((cnt + nb - 1) / nb);  // sources (epochs) per block
        if (g->deep_stride != stride || g->deep_blocks < nb || g->deep_epoch + iters - 1 > 0xFFFFu) {
            // records of another layout, fresh memory or every epoch used: tag 0 everywhere
            if ((e = cudaMemsetAsync(p.rec, 0, rec_bytes, st)) != cudaSuccess) return cuda_fail(e, "memset");
            g->deep_stride = stride;
            g->deep_blocks = blocks;
            g->deep_epoch = 1;
            s.kernel_launches += 1;
        }
        p.epoch0 = g->deep_epoch;
        g->deep_epoch += iters;
        p.src = src_rel + r0;
        p.nsrc = cnt;
        if (bfs) {
            const size_t row0 = (size_t)r0 * (size_t)n;
            p.level_out = bfs->level + row0;
            p.sig_out = bfs->sigma ? bfs->sigma + row0 : nullptr;
            p.exp_out = bfs->sigma_exp ? bfs->sigma_exp + row0 : nullptr;
        } else if ((e = cudaMemsetAsync(p.delta, 0, sizeof(double) * (size_t)cnt * (size_t)n, st)) != cudaSuccess) {
            return cuda_fail(e, "memset");
        }
        cudaEvent_t ev[2];
        cudaEventCreate(&ev[0]);
        cudaEventCreate(&ev[1]);
        cudaEventRecord(ev[0], st);
        e = launch_deep(p, nb, threads, st);
        cudaEventRecord(ev[1], st);
        if (e == cudaSuccess && !bfs) e = launch_deep_accumulate(p.delta, cnt, n, bc_rel, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(hst.data(), status, sizeof(int) * cnt, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(hdp.data(), depth, sizeof(int) * cnt, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        float ms = 0.f;
        if (e == cudaSuccess) cudaEventElapsedTime(&ms, ev[0], ev[1]);
        cudaEventDestroy(ev[0]);
        cudaEventDestroy(ev[1]);
        if (e != cudaSuccess) return cuda_fail(e, "per-source kernel");
        s.kernel_ms += ms;
        s.kernel_launches += bfs ? 1 : 2;
        for (int i = 0; i < cnt; ++i) {
            if (hst[i] == (ERR_LIMIT << 8)) return fail(BC_E_LIMIT, "BFS deeper than %d levels", kMaxLevel);
            if (!(hst[i] & BST_DONE)) return fail(BC_E_CUDA, "internal: source %lld not completed", r0 + i);
            inexact |= (hst[i] & BST_INEXACT) != 0;
            s.max_levels = std::max(s.max_levels, hdp[i]);
        }
    }
    unsigned long long hc[2] = {0, 0};
    if ((e = cudaMemcpyAsync(hc, ctr, sizeof hc, cudaMemcpyDeviceToHost, st)) == cudaSuccess)
        e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "per-source counters");
    s.dag_arcs = (int64_t)hc[0];
    s.reached = (int64_t)hc[1];
    {
        std::lock_guard<std::mutex> lk(g->state_mu);
        g->depth_seen = std::max(g->depth_seen, s.max_levels);
    }
    *out = s;
    return inexact ? BC_W_SIGMA_INEXACT : BC_OK;
}

// Automatic choice of the per-source form (bc_options.deep_form = 0), for a
// width left to the library: the graph's depth as seen by earlier
// traversals (on a sparse graph with none yet, one source, relabelled vertex
// 0, is first run in the per-source form into `scratch`, n doubles, to learn
// it).  The per-source form runs when the BFS is deep (kDeepMinDepth levels
// or more), its levels are narrow (on average at most kDeepMaxWidth
// vertices), and the memory budget leaves a block for every source or SM.
static bool want_deep(bc_graph* g, int nsrc, const bc_options& o, cudaStream_t st, double* scratch,
                      bc_run_stats* pre, bool forward_only = false) {
    if (o.deep_form == 1) return false;
    if (o.deep_form == 2) return true;
    if (o.batch_width != 0) return false;
    auto deep_enough = [&](int d) { return deep_by_depth(g, d); };
    int seen;
    {
        std::lock_guard<std::mutex> lk(g->state_mu);
        seen = g->depth_seen;
    }
    const bool probe = seen < 0 && nsrc >= 64 && g->n_nz >= 256 && g->m <= 8LL * g->n_nz;
    if (seen < 0 ? !probe : !deep_enough(seen)) return false;
    // room next: a graph whose per-block state leaves too few blocks runs
    // batched whatever its depth, and needs no probe
    DeepPlan pl;
    if (deep_plan(g, nsrc, o, forward_only, &pl) != BC_OK) {
        cudaGetLastError();
        return false;
    }
    if (pl.blocks < std::min<long long>(nsrc, pl.sms)) return false;
    if (probe) {
        bc_run_stats ps{};
        bc_options po;
        memset(&po, 0, sizeof po);
        if (run_deep(g, (const int*)g->perm.p, 1, po, st, scratch, &ps) >= 0) {
            seen = ps.max_levels;
            pre->kernel_launches += ps.kernel_launches;
        } else {
            cudaGetLastError();
        }
    }
    return deep_enough(seen);
}

bc_status bc_compute_ex(bc_graph* g, const int32_t* sources, int32_t nsrc, double* out_bc, bc_stream_t stream,
                        const bc_options* opt) {
    if (!g) return fail(BC_E_INVALID_ARG, "graph is NULL");
    if (nsrc < 0) return fail(BC_E_INVALID_ARG, "nsrc < 0");
    if (nsrc > 0 && !sources) return fail(BC_E_INVALID_ARG, "sources is NULL");
    if (!out_bc && g->n > 0) return fail(BC_E_INVALID_ARG, "out_bc is NULL");
    bc_options o;
    memset(&o, 0, sizeof o);
    if (opt) o = *opt;
    bc_status cs = check_opts(o);
    if (cs != BC_OK) return cs;
    cudaStream_t st = (cudaStream_t)stream;
    const bc_options given = o;  // the form choice follows the caller's knobs, not tuned ones
    apply_tuning(g, nsrc, o);
    std::lock_guard<std::mutex> lk(g->mu);
    g->last_stream = st;
    if (g->n == 0) return BC_OK;
    if (nsrc == 0) {
        cudaError_t e = cudaMemsetAsync(out_bc, 0, sizeof(double) * (size_t)g->n, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) return cuda_fail(e, "zero output");
        g->last = bc_run_stats{};
        return BC_OK;
    }
    const int* d_src = sources;
    DevBuf tmp;
    if (!is_device_ptr(sources)) {
        for (int i = 0; i < nsrc; ++i)
            if (sources[i] < 0 || sources[i] >= g->n)
                return fail(BC_E_SOURCE, "source %d (entry %d) is outside [0, %d)", sources[i], i, g->n);
        if (!buf_ensure(tmp, sizeof(int) * (size_t)nsrc, st)) return fail(BC_E_NOMEM, "source buffer");
        cudaError_t e = cudaMemcpyAsync(tmp.p, sources, sizeof(int) * (size_t)nsrc, cudaMemcpyHostToDevice, st);
        if (e != cudaSuccess) {
            buf_release(tmp, st);
            return cuda_fail(e, "source copy");
        }
        d_src = (const int*)tmp.p;
    }
    const int K = choose_width(g->n, nsrc, o.batch_width);
    auto& slot = g->ws[K];
    if (!slot) slot.reset(new Workspace());
    Workspace* w = slot.get();
    if (!buf_ensure(w->bc, sizeof(double) * (size_t)g->n, st)) {
        buf_release(tmp, st);
        return fail(BC_E_NOMEM, "output buffer");
    }
    bc_run_stats pre{};
    DevBuf grouped;
    if (want_grouping(g, nsrc, o)) {
        bc_status gr = group_sources(g, d_src, nsrc, st, grouped, &pre, nullptr);
        if (gr < 0) {
            buf_release(tmp, st);
            buf_release(grouped, st);
            return gr;
        }
        d_src = (const int*)grouped.p;
    }
    std::vector<double*> jb{(double*)w->bc.p};
    bc_run_stats stats{};
    bc_status r;
    if (want_deep(g, nsrc, given, st, (double*)w->bc.p, &pre))
        r = run_deep(g, d_src, nsrc, o, st, (double*)w->bc.p, &stats);
    else
        r = run_jobs(g, w, d_src, nsrc, o, 1, jb, nullptr, false, st, &stats, nullptr, nullptr, nullptr);
    stats.kernel_launches += pre.kernel_launches;
    stats.order_ms = pre.kernel_ms;
    if (r >= 0) {
        cudaError_t e = launch_unpermute((const double*)w->bc.p, (const int*)g->inv.p, out_bc, g->n, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) r = cuda_fail(e, "unpermute");
        stats.kernel_launches += 1;
        g->last = stats;
    }
    buf_release(tmp, st);
    buf_release(grouped, st);
    return r;
}

bc_status bc_source_batches(bc_graph* g, const int32_t* sources, int32_t nsrc, const bc_options* opt,
                            int32_t* order, int32_t* batch_width, bc_stream_t stream) {
    if (!g) return fail(BC_E_INVALID_ARG, "graph is NULL");
    if (nsrc < 0) return fail(BC_E_INVALID_ARG, "nsrc < 0");
    if (nsrc > 0 && (!sources || !order)) return fail(BC_E_INVALID_ARG, "sources or order is NULL");
    bc_options o;
    memset(&o, 0, sizeof o);
    if (opt) o = *opt;
    bc_status cs = check_opts(o);
    if (cs != BC_OK) return cs;
    cudaStream_t st = (cudaStream_t)stream;
    apply_tuning(g, nsrc, o);
    if (batch_width) *batch_width = choose_width(g->n, nsrc, o.batch_width);
    if (nsrc == 0) return BC_OK;
    std::lock_guard<std::mutex> lk(g->mu);
    g->last_stream = st;
    std::vector<int> hs(nsrc);
    DevBuf dsrc;
    cudaError_t e = cudaSuccess;
    if (is_device_ptr(sources))
        e = cudaMemcpyAsync(hs.data(), sources, sizeof(int) * (size_t)nsrc, cudaMemcpyDeviceToHost, st);
    else
        memcpy(hs.data(), sources, sizeof(int) * (size_t)nsrc);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "source copy");
    for (int i = 0; i < nsrc; ++i)
        if (hs[i] < 0 || hs[i] >= g->n) return fail(BC_E_SOURCE, "source %d (entry %d) is outside [0, %d)", hs[i], i, g->n);
    if (want_grouping(g, nsrc, o)) {
        if (!buf_ensure(dsrc, sizeof(int) * (size_t)nsrc, st)) return fail(BC_E_NOMEM, "source buffer");
        e = cudaMemcpyAsync(dsrc.p, hs.data(), sizeof(int) * (size_t)nsrc, cudaMemcpyHostToDevice, st);
        if (e != cudaSuccess) {
            buf_release(dsrc, st);
            return cuda_fail(e, "source copy");
        }
        DevBuf grouped;
        bc_run_stats pre{};
        std::vector<int> go;
        bc_status r = group_sources(g, (const int*)dsrc.p, nsrc, st, grouped, &pre, &go);
        buf_release(grouped, st);
        buf_release(dsrc, st);
        if (r < 0) return r;
        hs.swap(go);
    }
    memcpy(order, hs.data(), sizeof(int) * (size_t)nsrc);
    return BC_OK;
}

}  // extern "C"

// out[v] = parts[0][v] + parts[1][v] + ... + parts[nranks-1][v], added left to
// right in rank order, so the result does not depend on how the parts arrived.
__global__ void k_reduce_ranks(const double* __restrict__ parts, int nranks, long long n, double* __restrict__ out) {
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride) {
        double acc = parts[v];
        for (int r = 1; r < nranks; ++r) acc += parts[(size_t)r * (size_t)n + (size_t)v];
        out[v] = acc;
    }
}

extern "C" {

bc_status bc_reduce_ranks(const double* parts, int32_t nranks, int64_t n, double* out, bc_stream_t stream) {
    if (nranks < 1 || n < 0) return fail(BC_E_INVALID_ARG, "nranks < 1 or n < 0");
    if (n == 0) return BC_OK;
    if (!parts || !out) return fail(BC_E_INVALID_ARG, "parts or out is NULL");
    cudaStream_t st = (cudaStream_t)stream;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const long long want = (n + 255) / 256, cap = 8LL * (sms > 0 ? sms : 1);
    k_reduce_ranks<<<(unsigned)(want < cap ? want : cap), 256, 0, st>>>(parts, nranks, (long long)n, out);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "rank reduction");
    return BC_OK;
}

bc_status bc_bfs(bc_graph* g, const int32_t* sources, int32_t nsrc, int32_t* level, double* sigma, int32_t* sigma_exp,
                 bc_stream_t stream) {
    if (!g) return fail(BC_E_INVALID_ARG, "graph is NULL");
    if (nsrc < 0) return fail(BC_E_INVALID_ARG, "nsrc < 0");
    if (nsrc > 0 && !sources) return fail(BC_E_INVALID_ARG, "sources is NULL");
    if (nsrc > 0 && g->n > 0 && !level) return fail(BC_E_INVALID_ARG, "level is NULL");
    if (sigma_exp && !sigma) return fail(BC_E_INVALID_ARG, "sigma_exp needs sigma");
    cudaStream_t st = (cudaStream_t)stream;
    std::lock_guard<std::mutex> lk(g->mu);
    g->last_stream = st;
    if (g->n == 0 || nsrc == 0) return BC_OK;
    const size_t n = (size_t)g->n;
    cudaError_t e = cudaSuccess;  // every output cell is written by the extraction
    const int* d_src = sources;
    DevBuf tmp;
    if (!is_device_ptr(sources)) {
        for (int i = 0; i < nsrc; ++i)
            if (sources[i] < 0 || sources[i] >= g->n)
                return fail(BC_E_SOURCE, "source %d (entry %d) is outside [0, %d)", sources[i], i, g->n);
        if (!buf_ensure(tmp, sizeof(int) * (size_t)nsrc, st)) return fail(BC_E_NOMEM, "source buffer");
        e = cudaMemcpyAsync(tmp.p, sources, sizeof(int) * (size_t)nsrc, cudaMemcpyHostToDevice, st);
        if (e != cudaSuccess) {
            buf_release(tmp, st);
            return cuda_fail(e, "source copy");
        }
        d_src = (const int*)tmp.p;
    }
    bc_options o;
    memset(&o, 0, sizeof o);
    apply_tuning(g, nsrc, o);
    const int K = choose_width(g->n, nsrc, o.batch_width);
    o.batch_width = K;
    auto& slot = g->ws[K];
    if (!slot) slot.reset(new Workspace());
    Workspace* w = slot.get();
    if (!buf_ensure(w->bc, sizeof(double) * n, st)) {
        buf_release(tmp, st);
        return fail(BC_E_NOMEM, "buffers");
    }
    {
        // deep graphs: the per-source form, forward only, writes the rows itself
        bc_options given;
        memset(&given, 0, sizeof given);
        bc_run_stats pre{};
        if (want_deep(g, nsrc, given, st, (double*)w->bc.p, &pre, true)) {
            const BfsOut bo{level, sigma, sigma_exp};
            bc_run_stats stats{};
            bc_status rd = run_deep(g, d_src, nsrc, given, st, nullptr, &stats, &bo);
            if (rd >= 0) {
                stats.kernel_launches += pre.kernel_launches;
                g->last = stats;
            }
            buf_release(tmp, st);
            return rd;
        }
    }
    DevBuf lvl;  // [n][K] uint16 level table of one batch
    bc_status r = buf_ensure(lvl, sizeof(unsigned short) * n * (size_t)K, st) ? BC_OK : fail(BC_E_NOMEM, "buffers");
    bool inexact = false;
    bc_run_stats total{};
    for (int b0 = 0; r >= 0 && b0 < nsrc; b0 += K) {
        // one forward-only traversal per batch, then its rows of the output
        const int cnt = nsrc - b0 < K ? nsrc - b0 : K;
        std::vector<double*> jb{(double*)w->bc.p};
        bc_run_stats stats{};
        int kused = 0, levels = 0;
        bool ext = false;
        r = run_jobs(g, w, d_src + b0, cnt, o, 1, jb, nullptr, true, st, &stats, &kused, &ext, &levels);
        if (r < 0) break;
        inexact |= r == BC_W_SIGMA_INEXACT;
        total.batch_width = kused;
        total.batches += 1;
        total.kernel_launches += stats.kernel_launches + (levels > 0 ? 2 : 1);  // level table, rows
        total.kernel_ms += stats.kernel_ms;
        total.max_levels = std::max(total.max_levels, levels);
        total.pull_levels += stats.pull_levels;
        total.push_levels += stats.push_levels;
        total.ext_batches += ext ? 1 : 0;
        total.grid_blocks = stats.grid_blocks;
        total.teams = stats.teams;
        KParams p = make_params(g, w, 1, o, ext, 1);
        const size_t row0 = (size_t)b0 * n;
        e = launch_bfs_extract(p, kused, levels, cnt, (const int*)g->inv.p, (long long)n, (unsigned short*)lvl.p,
                               level + row0, sigma ? sigma + row0 : nullptr, sigma_exp ? sigma_exp + row0 : nullptr, st);
        if (e != cudaSuccess) r = cuda_fail(e, "bfs extract");
    }
    if (r >= 0) {
        e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) r = cuda_fail(e, "bfs");
        g->last = total;
    }
    buf_release(tmp, st);
    buf_release(lvl, st);
    if (r >= 0 && inexact) r = BC_W_SIGMA_INEXACT;
    return r;
}

// First relabelled row shorter than len arcs (rows are sorted by length, longest first).
static int first_row_shorter(bc_graph* g, int len, cudaStream_t st, cudaError_t* err) {
    int lo = 0, hi = g->n;
    const int* off = (const int*)g->off.p;
    while (lo < hi) {
        const int mid = (lo + hi) / 2;
        int two[2];
        cudaError_t e = cudaMemcpyAsync(two, off + mid, sizeof two, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) {
            *err = e;
            return 0;
        }
        if (two[1] - two[0] >= len) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

bc_status bc_pagerank(bc_graph* g, double delta, double beta, int32_t max_iter, double* out_rank, int32_t* iterations,
                      double* last_diff, bc_stream_t stream) {
    if (!g) return fail(BC_E_INVALID_ARG, "graph is NULL");
    if (!(delta >= 0.0 && delta <= 1.0) || !(beta >= 0.0) || max_iter < 1)
        return fail(BC_E_INVALID_ARG, "need 0 <= delta <= 1, beta >= 0 and max_iter >= 1");
    if (g->n > 0 && !out_rank) return fail(BC_E_INVALID_ARG, "out_rank is NULL");
    cudaStream_t st = (cudaStream_t)stream;
    std::lock_guard<std::mutex> lk(g->mu);
    g->last_stream = st;
    if (iterations) *iterations = 0;
    if (last_diff) *last_diff = 0.0;
    if (g->n == 0) return BC_OK;
    const size_t n = (size_t)g->n;
    const int blocks = pagerank_blocks();
    if (blocks < 1) return fail(BC_E_CUDA, "PageRank kernel cannot be resident");
    cudaError_t e = cudaSuccess;
    if (g->pr_cls[0] < 0) {
        // facts of the graph, once: undirected rows are sorted by length, so the
        // row classes are the first rows shorter than 8192 and 32 arcs; the long
        // rows' 2048-arc chunk prefix
        int cls[2] = {0, 0};
        const int bounds[2] = {8192, 32};
        if (!g->directed)
            for (int i = 0; i < 2 && e == cudaSuccess; ++i) cls[i] = first_row_shorter(g, bounds[i], st, &e);
        std::vector<int> hoff((size_t)cls[0] + 1), hc((size_t)cls[0] + 1, 0);
        if (e == cudaSuccess && cls[0] > 0) {
            e = cudaMemcpyAsync(hoff.data(), g->off.p, sizeof(int) * ((size_t)cls[0] + 1), cudaMemcpyDeviceToHost, st);
            if (e == cudaSuccess) e = cudaStreamSynchronize(st);
            for (int r = 0; r < cls[0]; ++r) hc[r + 1] = hc[r] + (hoff[r + 1] - hoff[r] + 2047) / 2048;
        }
        if (e != cudaSuccess) return cuda_fail(e, "PageRank set-up");
        if (!buf_ensure(g->pr_ccum, sizeof(int) * hc.size(), st)) return fail(BC_E_NOMEM, "PageRank buffers");
        e = cudaMemcpyAsync(g->pr_ccum.p, hc.data(), sizeof(int) * hc.size(), cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) return cuda_fail(e, "PageRank set-up");
        g->pr_cls[0] = cls[0];
        g->pr_cls[1] = cls[1];
        g->pr_nchunks = hc[cls[0]];
    }
    const int cls0 = g->pr_cls[0];
    if (!buf_ensure(g->pr_rank, sizeof(double) * n, st) ||
        !buf_ensure(g->pr_scratch, sizeof(double) * (2 * n + blocks), st) ||
        !buf_ensure(g->pr_ctl, sizeof(Ctl), st) || !buf_ensure(g->pr_small, 64, st) ||
        !buf_ensure(g->pr_cpart, sizeof(double) * (size_t)(g->pr_nchunks + 1), st) ||
        !buf_ensure(g->pr_carr, sizeof(int) * (size_t)(cls0 + 1), st))
        return fail(BC_E_NOMEM, "PageRank buffers");
    DevBuf& rank = g->pr_rank;
    DevBuf& scratch = g->pr_scratch;
    DevBuf& ctl = g->pr_ctl;
    DevBuf& small = g->pr_small;
    auto release = [&]() {};  // the buffers stay with the graph
    e = cudaMemsetAsync(ctl.p, 0, sizeof(Ctl), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(small.p, 0, 64, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(g->pr_carr.p, 0, sizeof(int) * (size_t)(cls0 + 1), st);
    int* d_iters = (int*)small.p;
    int* d_go = (int*)small.p + 1;
    double* d_diff = (double*)small.p + 1;
    const int* roff = g->directed ? (const int*)g->ioff.p : (const int*)g->off.p;
    const int* radj = g->directed ? (const int*)g->iadj.p : (const int*)g->adj.p;
    if (e == cudaSuccess)
        e = launch_pagerank(g->n, (const int*)g->off.p, roff, radj, g->directed ? nullptr : g->pr_cls, g->pr_nchunks,
                            (const int*)g->pr_ccum.p, (double*)g->pr_cpart.p, (int*)g->pr_carr.p, delta, beta,
                            max_iter, (double*)rank.p, (double*)scratch.p, (Ctl*)ctl.p, d_iters, d_diff, d_go,
                            40000000000ll, blocks, st);
    if (e == cudaSuccess) e = launch_unpermute((const double*)rank.p, (const int*)g->inv.p, out_rank, g->n, st);
    int h_it = 0, h_err = 0;
    double h_diff = 0.0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h_it, d_iters, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h_diff, d_diff, sizeof(double), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h_err, &((Ctl*)ctl.p)->err, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    release();
    if (e != cudaSuccess) return cuda_fail(e, "PageRank");
    if (h_err & ERR_TIMEOUT) return fail(BC_E_TIMEOUT, "a grid-barrier wait exceeded its cycle budget");
    if (h_err) return fail(BC_E_CUDA, "PageRank kernel error 0x%x", h_err);
    if (iterations) *iterations = h_it;
    if (last_diff) *last_diff = h_diff;
    bc_run_stats s{};
    s.kernel_launches = 2;
    s.grid_blocks = blocks;
    s.max_levels = h_it;
    g->last = s;
    return BC_OK;
}

bc_status bc_compute(bc_graph* g, const int32_t* sources, int32_t nsrc, double* out_bc, bc_stream_t stream) {
    return bc_compute_ex(g, sources, nsrc, out_bc, stream, nullptr);
}

bc_status bc_last_trace(const bc_graph* g, int64_t* out, int32_t cap, int32_t* count) {
    if (!g || !count || (cap > 0 && !out) || cap < 0) return fail(BC_E_INVALID_ARG, "bad argument");
    const int nrec = (int)(g->last_trace.size() / 2);
    const int k = nrec < cap ? nrec : cap;
    for (int i = 0; i < 2 * k; ++i) out[i] = g->last_trace[i];
    *count = k;
    return BC_OK;
}

bc_status bc_last_run_stats(const bc_graph* g, bc_run_stats* st) {
    if (!g || !st) return fail(BC_E_INVALID_ARG, "NULL argument");
    *st = g->last;
    return BC_OK;
}

bc_status bc_debug_source(bc_graph* g, int32_t s, int32_t* level, double* sigma_mant, int32_t* sigma_exp) {
    if (!g) return fail(BC_E_INVALID_ARG, "graph is NULL");
    if (s < 0 || s >= g->n) return fail(BC_E_SOURCE, "source %d outside [0, %d)", s, g->n);
    std::lock_guard<std::mutex> lk(g->mu);
    cudaStream_t st = nullptr;
    g->last_stream = st;
    DevBuf dsrc, dlev, dsig, dsige;
    const size_t n = (size_t)g->n;
    if (!buf_ensure(dsrc, sizeof(int), st) || !buf_ensure(dlev, sizeof(int) * n, st) ||
        !buf_ensure(dsig, sizeof(unsigned long long) * n, st) || !buf_ensure(dsige, sizeof(int) * n, st)) {
        buf_release(dsrc, st); buf_release(dlev, st); buf_release(dsig, st); buf_release(dsige, st);
        return fail(BC_E_NOMEM, "debug buffers");
    }
    cudaMemcpyAsync(dsrc.p, &s, sizeof(int), cudaMemcpyHostToDevice, st);
    bc_options o;
    memset(&o, 0, sizeof o);
    o.batch_width = 32;
    auto& slot = g->ws[32];
    if (!slot) slot.reset(new Workspace());
    Workspace* w = slot.get();
    int K = 0, levels = 0;
    bool ext = false;
    bc_status r = buf_ensure(w->bc, sizeof(double) * n, st) ? BC_OK : fail(BC_E_NOMEM, "debug buffers");
    if (r == BC_OK) {
        std::vector<double*> jb{(double*)w->bc.p};
        r = run_jobs(g, w, (const int*)dsrc.p, 1, o, 1, jb, nullptr, true, st, nullptr, &K, &ext, &levels);
    }
    KParams p = make_params(g, w, 1, o, ext, 1);
    if (r < 0) {
        buf_release(dsrc, st); buf_release(dlev, st); buf_release(dsig, st); buf_release(dsige, st);
        return r;
    }
    cudaError_t e = launch_debug_extract(p, 32, levels, (int*)dlev.p, (unsigned long long*)dsig.p, (int*)dsige.p, st);
    std::vector<int> lev(n), sige(n), perm(n);
    std::vector<unsigned long long> sig(n);
    if (e == cudaSuccess) e = cudaMemcpyAsync(lev.data(), dlev.p, sizeof(int) * n, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(sig.data(), dsig.p, sizeof(unsigned long long) * n, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(sige.data(), dsige.p, sizeof(int) * n, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(perm.data(), g->perm.p, sizeof(int) * n, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    buf_release(dsrc, st); buf_release(dlev, st); buf_release(dsig, st); buf_release(dsige, st);
    if (e != cudaSuccess) return cuda_fail(e, "debug extract");
    for (size_t r2 = 0; r2 < n; ++r2) {
        const int v = perm[r2];
        if (level) level[v] = lev[r2];
        int ex = 0;
        double mant = std::frexp((double)sig[r2], &ex);  // representation only: m * 2^e -> [0.5,1) * 2^x
        if (sigma_mant) sigma_mant[v] = mant;
        if (sigma_exp) sigma_exp[v] = sig[r2] ? ex + sige[r2] : 0;
    }
    return r;
}

bc_status bc_many_create(const bc_item* items, int32_t nitems, const bc_options* opt, bc_stream_t stream,
                         bc_many_plan** out) {
    if (!out || nitems < 0 || (nitems > 0 && !items)) return fail(BC_E_INVALID_ARG, "bad argument");
    *out = nullptr;
    bc_options o;
    memset(&o, 0, sizeof o);
    if (opt) o = *opt;
    bc_status cs = check_opts(o);
    if (cs != BC_OK) return cs;
    cudaStream_t ust = (cudaStream_t)stream;
    std::unique_ptr<bc_many_plan> pl(new bc_many_plan());
    pl->opt = o;
    long long total_src = 0;
    // items, validated on the host; per-width dimensions
    struct Dims { int n = 0, nh = 0, nb = 0, teams = 1; long long hc = 0; };
    std::map<int, Dims> dims;
    for (int i = 0; i < nitems; ++i) {
        const bc_item& x = items[i];
        if (!x.graph || x.nsrc < 0 || (x.nsrc > 0 && !x.sources) || (!x.out_bc && x.graph->n > 0))
            return fail(BC_E_INVALID_ARG, "item %d: bad graph, sources or output", i);
        bc_graph* g = x.graph;
        for (int k = 0; k < x.nsrc; ++k)
            if (x.sources[k] < 0 || x.sources[k] >= g->n)
                return fail(BC_E_SOURCE, "item %d: source %d outside [0, %d)", i, x.sources[k], g->n);
        bc_status r = ensure_heavy(g, ust);
        if (r != BC_OK) return r;
        ManyItem it;
        it.g = g;
        it.src.assign(x.sources, x.sources + x.nsrc);
        if (want_grouping(g, x.nsrc, o)) {
            // the order bc_compute would use, fixed once here
            DevBuf dsrc, grouped;
            bc_run_stats gs{};
            r = buf_ensure(dsrc, sizeof(int) * (size_t)x.nsrc, ust) ? BC_OK : fail(BC_E_NOMEM, "source buffer");
            cudaError_t e = cudaSuccess;
            if (r == BC_OK &&
                (e = cudaMemcpyAsync(dsrc.p, x.sources, sizeof(int) * (size_t)x.nsrc, cudaMemcpyHostToDevice, ust)) !=
                    cudaSuccess)
                r = cuda_fail(e, "source copy");
            if (r == BC_OK) r = group_sources(g, (const int*)dsrc.p, x.nsrc, ust, grouped, &gs, &it.src);
            cudaStreamSynchronize(ust);
            buf_release(dsrc, ust);
            buf_release(grouped, ust);
            if (r != BC_OK) return r;
        }
        it.out = x.out_bc;
        it.K = choose_width(g->n, x.nsrc, o.batch_width);
        it.nbatch = (x.nsrc + it.K - 1) / it.K;
        it.src_off = total_src;
        total_src += x.nsrc;
        if (g->n > 0 && x.nsrc > 0) {
            // deep graphs take the per-source form, by bc_compute's rule (a depth probe included)
            std::lock_guard<std::mutex> lk(g->mu);
            DevBuf scratch;
            bc_run_stats pre{};
            if (!buf_ensure(scratch, sizeof(double) * (size_t)g->n, ust)) return fail(BC_E_NOMEM, "probe buffer");
            it.deep = want_deep(g, x.nsrc, o, ust, (double*)scratch.p, &pre);
            cudaStreamSynchronize(ust);
            buf_release(scratch, ust);
        }
        if (it.deep) {
            pl->items.push_back(std::move(it));
            continue;
        }
        Dims& d = dims[it.K];
        d.n = std::max(d.n, g->n);
        d.nh = std::max(d.nh, g->n_heavy);
        d.hc = std::max(d.hc, g->hchunk_total);
        d.nb = std::max(d.nb, it.nbatch);
        {
            const int blocks = grid_blocks(it.K, false, o.blocks_per_sm, 1);
            int T = 1, B = blocks;
            const TeamLayout L = team_layout(g->n, g->n_heavy, g->hchunk_total, it.K, false, cap_factor(it.K, 0));
            choose_teams(g->m, it.K, it.nbatch, blocks, L.bytes, o.teams, &T, &B);
            d.teams = std::max(d.teams, T);
        }
        pl->items.push_back(std::move(it));
    }
    cudaError_t e = cudaStreamCreateWithFlags(&pl->cap_stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) return cuda_fail(e, "stream");
    cudaStream_t st = pl->cap_stream;
    auto bail = [&](bc_status r) {
        many_release(pl.get());
        return r;
    };
    for (auto& kv : dims) {
        std::unique_ptr<Workspace> w(new Workspace());
        // slices for the most teams any item of this width uses, each sized for the
        // largest graph of the width (capped by the same memory budget)
        const TeamLayout L = team_layout(kv.second.n, kv.second.nh, kv.second.hc, kv.first, false, cap_factor(kv.first, 0));
        size_t fr = 0, tot = 0;
        cudaMemGetInfo(&fr, &tot);
        int T = kv.second.teams;
        while (T > 1 && (double)T * (double)L.bytes > std::min(0.3 * (double)fr, 24e9)) --T;
        if (!ws_ensure_dims(w.get(), kv.second.n, kv.second.nh, kv.second.hc, kv.first, false, kv.second.nb, 1,
                            cap_factor(kv.first, 0), T, st))
            return bail(BC_E_NOMEM);
        double* jb = (double*)w->bc.p;
        if ((e = cudaMemcpyAsync(w->jobptr.p, &jb, sizeof(double*), cudaMemcpyHostToDevice, st)) != cudaSuccess ||
            (e = cudaStreamSynchronize(st)) != cudaSuccess)
            return bail(cuda_fail(e, "job table"));
        pl->ws[kv.first] = std::move(w);
    }
    if (!buf_ensure(pl->dsrc, sizeof(int) * (size_t)(total_src > 0 ? total_src : 1), st) ||
        !buf_ensure(pl->dstatus, sizeof(int) * (size_t)(nitems > 0 ? nitems : 1), st))
        return bail(fail(BC_E_NOMEM, "plan buffers"));
    std::vector<int> all;
    all.reserve((size_t)total_src);
    for (auto& it : pl->items) all.insert(all.end(), it.src.begin(), it.src.end());
    if (total_src > 0 &&
        (e = cudaMemcpyAsync(pl->dsrc.p, all.data(), sizeof(int) * all.size(), cudaMemcpyHostToDevice, st)) !=
            cudaSuccess)
        return bail(cuda_fail(e, "source copy"));
    if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return bail(cuda_fail(e, "plan set-up"));
    bc_status r = many_record(pl.get());
    if (r != BC_OK) return bail(r);
    for (auto& it : pl->items) it.g->users++;
    *out = pl.release();
    return BC_OK;
}

bc_status bc_many_run(bc_many_plan* pl, bc_stream_t stream, bc_status* item_status) {
    if (!pl) return fail(BC_E_INVALID_ARG, "plan is NULL");
    cudaStream_t st = (cudaStream_t)stream;
    const size_t ni = pl->items.size();
    if (ni == 0) return BC_OK;
    cudaError_t e = cudaGraphLaunch(pl->exec, st);
    std::vector<int> status(ni);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(status.data(), pl->dstatus.p, sizeof(int) * ni, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "many-graph run");
    bc_status overall = BC_OK;
    for (size_t i = 0; i < ni; ++i) {
        const int w = status[i];
        bc_status r;
        if (pl->items[i].deep) {
            // the per-source form, in the item's fixed source order
            ManyItem& it = pl->items[i];
            bc_options od = pl->opt;
            od.deep_form = 2;
            od.source_order = 1;
            r = bc_compute_ex(it.g, it.src.data(), (int)it.src.size(), it.out, stream, &od);
        } else if ((w >> 8) & ERR_TIMEOUT) {
            r = fail(BC_E_TIMEOUT, "item %zu: a grid-barrier wait exceeded its cycle budget", i);
        } else if ((w >> 8) & ERR_LIMIT) {
            r = fail(BC_E_LIMIT, "item %zu: BFS deeper than %d levels", i, kMaxLevel);
        } else if ((w >> 8) || (w & (BST_NEED_EXT | 0x80))) {
            // extended path-count form or larger level lists: redo this item alone
            ManyItem& it = pl->items[i];
            r = bc_compute_ex(it.g, it.src.data(), (int)it.src.size(), it.out, stream, &pl->opt);
        } else {
            r = (w & BST_INEXACT) ? BC_W_SIGMA_INEXACT : BC_OK;
        }
        if (item_status) item_status[i] = r;
        if (r < 0 && overall >= 0) overall = r;
        else if (r == BC_W_SIGMA_INEXACT && overall == BC_OK) overall = r;
    }
    return overall;
}

bc_status bc_many_destroy(bc_many_plan* pl) {
    if (!pl) return fail(BC_E_INVALID_ARG, "plan is NULL");
    many_release(pl);
    for (auto& it : pl->items) it.g->users--;
    delete pl;
    return BC_OK;
}

bc_status bc_many_info(const bc_many_plan* pl, int32_t* items, int32_t* kernel_launches) {
    if (!pl) return fail(BC_E_INVALID_ARG, "plan is NULL");
    if (items) *items = (int32_t)pl->items.size();
    if (kernel_launches) *kernel_launches = pl->launches;
    return BC_OK;
}

bc_status bc_autotune(bc_graph* g, const int32_t* sources, int32_t nsrc, bc_stream_t stream, bc_options* best,
                      double* best_rate) {
    if (!g || nsrc <= 0 || !sources) return fail(BC_E_INVALID_ARG, "autotune needs a graph and host sources");
    if (is_device_ptr(sources)) return fail(BC_E_INVALID_ARG, "autotune takes host sources");
    for (int i = 0; i < nsrc; ++i)
        if (sources[i] < 0 || sources[i] >= g->n) return fail(BC_E_SOURCE, "source %d outside [0, %d)", sources[i], g->n);
    cudaStream_t st = (cudaStream_t)stream;
    // sample: the whole list on small graphs (so that team parallelism is what
    // the real call sees), a few wide batches on large ones
    const int cap_s = g->m <= (1ll << 24) ? 8192 : 512;
    const int S = nsrc < cap_s ? nsrc : cap_s;
    DevBuf out;
    if (!buf_ensure(out, sizeof(double) * (size_t)(g->n > 0 ? g->n : 1), st)) return fail(BC_E_NOMEM, "autotune buffer");
    auto measure = [&](const bc_options& o, double* rate) -> bc_status {
        bc_options q = o;  // every knob explicit, so an older tuned entry cannot leak in
        if (q.alpha == 0.f) q.alpha = 14.f;
        if (q.group_vertices == 0) q.group_vertices = 32;
        bc_status r = bc_compute_ex(g, sources, S, (double*)out.p, stream, &q);  // warm (allocations)
        if (r < 0) return r;
        r = bc_compute_ex(g, sources, S, (double*)out.p, stream, &q);
        if (r < 0) return r;
        const double ms = g->last.kernel_ms > 0 ? g->last.kernel_ms : 1e-3;
        *rate = (double)S * (double)g->m / (ms * 1e-3);
        return BC_OK;
    };
    bc_options cur;
    memset(&cur, 0, sizeof cur);
    double cur_rate = -1.0;
    // coordinate descent: width, then the pull threshold, then the grouping
    std::vector<int> widths;
    if (S <= 64) widths.push_back(1);
    for (int K : {32, 64, 128})
        if (K <= 2 * S) widths.push_back(K);
    for (int K : widths) {
        bc_options o = cur;
        o.batch_width = K;
        double rate = 0;
        bc_status r = measure(o, &rate);
        if (r < 0) {
            buf_release(out, st);
            return r;
        }
        if (rate > cur_rate) { cur_rate = rate; cur = o; }
    }
    const bc_options base = cur;
    for (float alpha : {5.f, 40.f}) {
        bc_options o = base;
        o.alpha = alpha;
        double rate = 0;
        if (measure(o, &rate) == BC_OK && rate > cur_rate) { cur_rate = rate; cur = o; }
    }
    const bc_options base2 = cur;
    for (int grp : {8, 16}) {
        bc_options o = base2;
        o.group_vertices = grp;
        double rate = 0;
        if (measure(o, &rate) == BC_OK && rate > cur_rate) { cur_rate = rate; cur = o; }
    }
    buf_release(out, st);
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        TuneVal v;
        v.K = cur.batch_width;
        v.alpha = cur.alpha;
        v.group = cur.group_vertices;
        v.rate = cur_rate;
        g_tune[tune_key(g)] = v;
    }
    if (best) *best = cur;
    if (best_rate) *best_rate = cur_rate;
    return BC_OK;
}

bc_status bc_tuning_cache(const char* path, int32_t save) {
    if (!path) return fail(BC_E_INVALID_ARG, "path is NULL");
    std::lock_guard<std::mutex> lk(g_tune_mu);
    if (save) {
        FILE* f = fopen(path, "w");
        if (!f) return fail(BC_E_INVALID_ARG, "cannot write %s", path);
        fprintf(f, "{\"bc_tuning\": [\n");
        size_t i = 0;
        for (const auto& kv : g_tune) {
            fprintf(f, "  {\"log2_n\": %d, \"log2_avg_degree\": %d, \"log2_skew\": %d, \"batch_width\": %d, "
                       "\"alpha\": %.3f, \"group_vertices\": %d, \"rate\": %.6e}%s\n",
                    kv.first.ln, kv.first.lavg, kv.first.lskew, kv.second.K, kv.second.alpha, kv.second.group,
                    kv.second.rate, ++i < g_tune.size() ? "," : "");
        }
        fprintf(f, "]}\n");
        fclose(f);
        return BC_OK;
    }
    FILE* f = fopen(path, "r");
    if (!f) return fail(BC_E_INVALID_ARG, "cannot read %s", path);
    char line[512];
    int loaded = 0;
    while (fgets(line, sizeof line, f)) {
        TuneKey k;
        TuneVal v;
        if (sscanf(line, " {\"log2_n\": %d, \"log2_avg_degree\": %d, \"log2_skew\": %d, \"batch_width\": %d, "
                         "\"alpha\": %f, \"group_vertices\": %d, \"rate\": %lf",
                   &k.ln, &k.lavg, &k.lskew, &v.K, &v.alpha, &v.group, &v.rate) == 7) {
            g_tune[k] = v;
            ++loaded;
        }
    }
    fclose(f);
    return BC_OK;
}

bc_status bc_team_rule(int64_t m, int32_t batch_width, int32_t nbatch, int32_t blocks, uint64_t team_bytes,
                       uint64_t free_bytes, int32_t teams, int32_t* nteams, int32_t* team_blocks) {
    if (m < 0 || batch_width < 1 || nbatch < 0 || blocks < 1 || teams < 0 || !nteams || !team_blocks)
        return fail(BC_E_INVALID_ARG, "bc_team_rule: m >= 0, batch_width >= 1, nbatch >= 0, blocks >= 1, teams >= 0 "
                                      "and non-NULL outputs");
    int T = 1, B = blocks;
    team_rule(m, batch_width, nbatch, blocks, (size_t)team_bytes, (size_t)free_bytes, teams, &T, &B);
    *nteams = T;
    *team_blocks = B;
    return BC_OK;
}

bc_status bc_server_config(int32_t slots, int64_t memory_budget) {
    if (slots < 1 || slots > 64 || memory_budget < 0)
        return fail(BC_E_INVALID_ARG, "slots must be in [1, 64] and the budget >= 0");
    Server& S = server();
    std::unique_lock<std::mutex> lk(S.mu);
    if (!S.started) {
        S.slots = slots;
        S.budget = memory_budget;
        return BC_OK;
    }
    // running: the slot count may grow.  New jobs wait until every traversal
    // in flight has finished, so runs sized for different shares of the GPU
    // never have to be co-resident.
    if (slots < S.slots) return fail(BC_E_INVALID_ARG, "the slot count can only grow while the server runs");
    if (memory_budget > 0) S.budget = memory_budget;
    if (slots == S.slots) return BC_OK;
    S.paused = true;
    S.cv_done.wait(lk, [&] { return S.running == 0; });
    for (int i = S.slots; i < slots; ++i) {
        S.workers.emplace_back(worker_main, i);
        S.workers.back().detach();
    }
    S.slots = slots;
    S.paused = false;
    S.cv_work.notify_all();
    return BC_OK;
}

bc_status bc_batch_submit(bc_graph* g, const int32_t* sources, int32_t nsrc, double* out_bc, bc_job* job) {
    if (!g || !job) return fail(BC_E_INVALID_ARG, "NULL argument");
    if (nsrc < 0 || (nsrc > 0 && !sources)) return fail(BC_E_INVALID_ARG, "bad source list");
    if (!out_bc && g->n > 0) return fail(BC_E_INVALID_ARG, "out_bc is NULL");
    if (nsrc > 0 && is_device_ptr(sources)) return fail(BC_E_INVALID_ARG, "bc_batch_submit takes host sources");
    for (int i = 0; i < nsrc; ++i)
        if (sources[i] < 0 || sources[i] >= g->n)
            return fail(BC_E_SOURCE, "source %d (entry %d) is outside [0, %d)", sources[i], i, g->n);
    auto j = std::make_shared<Job>();
    j->g = g;
    j->src.assign(sources, sources + nsrc);
    j->out = out_bc;
    j->t_submit = std::chrono::steady_clock::now();
    Server& S = server();
    {
        std::lock_guard<std::mutex> lk(S.mu);
        server_start_locked(S);
        j->id = S.next_id++;
        S.jobs[j->id] = j;
        if (nsrc == 0 || g->n == 0) {
            cudaError_t e = g->n ? cudaMemset(out_bc, 0, sizeof(double) * (size_t)g->n) : cudaSuccess;
            j->result = e == cudaSuccess ? BC_OK : cuda_fail(e, "zero output");
            j->done = true;
            j->t_done = std::chrono::steady_clock::now();
            S.completed++;
        } else {
            g->users++;
            S.queue.push_back(j);
        }
    }
    S.cv_work.notify_all();
    *job = j->id;
    return BC_OK;
}

static bc_status poll_impl(bc_job job, double* latency_s, int64_t timeout_ms, bool wait) {
    Server& S = server();
    std::unique_lock<std::mutex> lk(S.mu);
    auto it = S.jobs.find(job);
    if (it == S.jobs.end()) return fail(BC_E_INVALID_ARG, "unknown or already released job %llu", (unsigned long long)job);
    std::shared_ptr<Job> j = it->second;
    if (wait && !j->done) {
        auto pred = [&] { return j->done; };
        if (timeout_ms < 0) S.cv_done.wait(lk, pred);
        else S.cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), pred);
    }
    if (!j->done) return BC_PENDING;
    if (latency_s) *latency_s = std::chrono::duration<double>(j->t_done - j->t_submit).count();
    S.jobs.erase(it);
    return j->result;
}

bc_status bc_poll(bc_job job) { return poll_impl(job, nullptr, 0, false); }
bc_status bc_poll_ex(bc_job job, double* latency_s) { return poll_impl(job, latency_s, 0, false); }
bc_status bc_wait(bc_job job, int64_t timeout_ms) { return poll_impl(job, nullptr, timeout_ms, true); }
bc_status bc_wait_ex(bc_job job, int64_t timeout_ms, double* latency_s) {
    return poll_impl(job, latency_s, timeout_ms, true);
}

bc_status bc_server_stats(int32_t* peak_concurrency, int64_t* completed) {
    Server& S = server();
    std::lock_guard<std::mutex> lk(S.mu);
    if (peak_concurrency) *peak_concurrency = S.peak;
    if (completed) *completed = S.completed;
    return BC_OK;
}

bc_status bc_server_reset_stats(void) {
    Server& S = server();
    std::lock_guard<std::mutex> lk(S.mu);
    S.peak = S.running;
    S.completed = 0;
    return BC_OK;
}

bc_status bc_cancel(bc_job job) {
    Server& S = server();
    {
        std::lock_guard<std::mutex> lk(S.mu);
        auto it = S.jobs.find(job);
        if (it == S.jobs.end())
            return fail(BC_E_INVALID_ARG, "unknown or already released job %llu", (unsigned long long)job);
        std::shared_ptr<Job> j = it->second;
        if (j->done) return fail(BC_E_BUSY, "job %llu has already finished", (unsigned long long)job);
        auto q = std::find(S.queue.begin(), S.queue.end(), j);
        if (q == S.queue.end()) return fail(BC_E_BUSY, "job %llu is running; it will finish", (unsigned long long)job);
        S.queue.erase(q);
        j->result = BC_E_CANCELLED;  // out_bc is not written
        j->done = true;
        j->t_done = std::chrono::steady_clock::now();
        j->g->users--;
    }
    S.cv_done.notify_all();
    return BC_OK;
}

const char* bc_status_string(bc_status st) {
    switch (st) {
        case BC_OK: return "BC_OK";
        case BC_PENDING: return "BC_PENDING";
        case BC_W_SIGMA_INEXACT: return "BC_W_SIGMA_INEXACT";
        case BC_E_INVALID_ARG: return "BC_E_INVALID_ARG";
        case BC_E_INVALID_GRAPH: return "BC_E_INVALID_GRAPH";
        case BC_E_SOURCE: return "BC_E_SOURCE";
        case BC_E_NOMEM: return "BC_E_NOMEM";
        case BC_E_TIMEOUT: return "BC_E_TIMEOUT";
        case BC_E_CUDA: return "BC_E_CUDA";
        case BC_E_SIGMA_RANGE: return "BC_E_SIGMA_RANGE";
        case BC_E_LIMIT: return "BC_E_LIMIT";
        case BC_E_BUSY: return "BC_E_BUSY";
        case BC_E_CANCELLED: return "BC_E_CANCELLED";
    }
    return "BC_UNKNOWN";
}

const char* bc_last_error(void) { return t_err.c_str(); }

}  // extern "C"
