/*
 * libbc -- exact betweenness centrality (Brandes) on one NVIDIA B300 (sm_103a).
 *
 * The operation is the paper's computeBC (Appendix A, BC listing): for each
 * source s in a list, a level-synchronous BFS from s counts shortest paths
 * (sigma, the iterateInBFS body), then a reverse level-by-level sweep over the
 * BFS DAG accumulates the dependency
 *     delta_s(v) = sum over DAG successors w of (sigma_v / sigma_w)(1 + delta_s(w))
 * (the iterateInReverse body), and BC(v) += delta_s(v) for every v != s.
 * The graph is unweighted, undirected (symmetric) or directed, given as int32
 * CSR (Section 3.1: the backend keeps graphs in CSR); bc_compute_weighted
 * covers graphs (undirected or directed) with positive integer arc weights.  The result is the raw
 * sum over the listed sources: no halving for undirected graphs, no
 * normalisation, no extrapolation from sampled sources.  A source listed twice
 * counts twice.
 *
 * Numerics: path counts are exact unsigned 64-bit integers; a batch whose
 * counts could pass 2^64 is rerun in an extended-range form (64-bit mantissa,
 * 32-bit exponent), which equals the plain form bit for bit while counts stay
 * below 2^64.  delta and BC are IEEE double.  BC_W_SIGMA_INEXACT
 * reports that some count reached 2^53 (the double conversion in the backward
 * sweep then rounds).  Results are deterministic: every sum runs in a fixed
 * order (CSR row order, in fixed 1024-arc chunks; sources in list order, or in
 * the grouped order of bc_options.source_order, which depends only on the
 * graph and the list, so a direct call, a plan and a served job agree).
 *
 * Threading: a bc_graph may be used by one host thread at a time for
 * bc_compute / bc_bfs / bc_pagerank / bc_compute_weighted / bc_debug_source
 * (calls on one graph serialise); bc_batch_submit / bc_poll are thread-safe.  Every traversal is
 * a cooperative launch sized to its share of the GPU: a full-GPU call issued
 * while serving slots run waits for their blocks, its bounded waits then
 * limiting how long (BC_E_TIMEOUT past the barrier budget).
 * Error detail: bc_last_error() returns a thread-local message for the last
 * failing call on the calling thread.
 */
#ifndef LIBBC_BC_H
#define LIBBC_BC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Same type as cudaStream_t / CUstream (0 = the legacy default stream). */
typedef struct CUstream_st* bc_stream_t;

typedef struct bc_graph bc_graph;
typedef uint64_t bc_job;

typedef enum {
    BC_OK = 0,
    BC_PENDING = 1,            /* bc_poll: job not finished yet */
    BC_W_SIGMA_INEXACT = 2,    /* finished; some path count >= 2^53, so delta used a rounded count */
    BC_E_INVALID_ARG = -1,     /* null pointer, negative size, unknown flag or option value */
    BC_E_INVALID_GRAPH = -2,   /* offsets not monotone / offsets[0] != 0 / offsets[n] != m, index out of
                                  range, self-loop, duplicate arc, or (BC_UNDIRECTED) an arc without its
                                  reverse */
    BC_E_SOURCE = -3,          /* a source id outside [0, n) */
    BC_E_NOMEM = -4,           /* device allocation failed (allocator hook returned NULL) */
    BC_E_TIMEOUT = -5,         /* a bounded device wait (grid barrier) ran out; results not written */
    BC_E_CUDA = -6,            /* a CUDA runtime call failed; bc_last_error() has the CUDA message */
    BC_E_SIGMA_RANGE = -7,     /* a path count exceeded even the extended range (2^(2^31)) */
    BC_E_LIMIT = -8,           /* a size limit: BFS depth > 65534 levels, or n/m beyond int32 */
    BC_E_BUSY = -9,            /* bc_graph_destroy: a plan or an unfinished serving job still uses the graph;
                                  bc_cancel: the job is already running or finished */
    BC_E_CANCELLED = -10       /* bc_poll / bc_wait: the job was withdrawn by bc_cancel before it ran */
} bc_status;

/* bc_graph_create flags */
#define BC_UNDIRECTED 1u        /* the CSR is symmetric (checked); without it the CSR is the
                                   out-adjacency of a directed graph (arc v -> w listed in row v) */
#define BC_INPUT_ON_DEVICE 2u   /* offsets/indices are device pointers (else host pointers) */
#define BC_SKIP_VALIDATION 4u   /* trust the input (self-loops/duplicates/asymmetry unchecked) */

/*
 * Device memory hook.  alloc(bytes, stream, ctx) returns device memory or NULL;
 * free(ptr, stream, ctx) releases it.  Passing alloc = free = NULL restores the
 * default (cudaMallocAsync / cudaFreeAsync on the given stream).  Applies to
 * allocations made after the call; memory is released with the hook that
 * allocated it.
 */
typedef void* (*bc_alloc_fn)(size_t bytes, bc_stream_t stream, void* ctx);
typedef void (*bc_free_fn)(void* ptr, bc_stream_t stream, void* ctx);
bc_status bc_set_allocator(bc_alloc_fn alloc, bc_free_fn free_fn, void* ctx);

/*
 * Ingest (paper Section 3.1: CSR graph copied to the device once).
 * offsets[n+1], indices[m] (int32, host or device per flags) are copied; the
 * caller keeps ownership.  On the device the graph is validated, relabelled
 * by degree (descending, ties by original id) and stored with every row
 * sorted ascending.  Blocks until the graph is ready.  n may be 0.
 * Directed graphs (no BC_UNDIRECTED): shortest paths follow arcs; the device
 * also keeps the in-adjacency (the transpose), which the forward pull steps
 * read; BC is the raw sum over the listed sources, as for undirected graphs.
 */
bc_status bc_graph_create(const int32_t* offsets, const int32_t* indices, int32_t n, int64_t m,
                          uint32_t flags, bc_stream_t stream, bc_graph** out);
/* Frees the graph and its workspaces.  Returns BC_E_BUSY (and frees nothing)
 * while a bc_many_plan built over it exists or a serving job on it has not
 * finished; destroy the plan / wait for the jobs first.  Not to be called
 * concurrently with a bc_compute on the same graph. */
bc_status bc_graph_destroy(bc_graph* g);

/* Size facts of an ingested graph (any pointer may be NULL). */
bc_status bc_graph_info(const bc_graph* g, int32_t* n, int64_t* m, int32_t* max_degree,
                        int32_t* n_nonisolated);

/*
 * The relabelled graph, copied to HOST buffers: perm[n] (perm[r] = original id
 * of new id r), offsets[n+1], indices[m] (new ids, rows sorted).  Any pointer
 * may be NULL.  For inspection and tests.
 */
bc_status bc_graph_export(const bc_graph* g, int32_t* perm, int32_t* offsets, int32_t* indices);

/* Tuning knobs; zero-initialise and set what you need (0 = automatic). */
typedef struct {
    int32_t batch_width;     /* sources per traversal: 1 (plain per-source), 32, 64 or 128; 0 = auto */
    int32_t direction;       /* 0 = auto push/pull switching, 1 = push only, 2 = pull only */
    float alpha;             /* switch to pull when frontier arcs * alpha > unvisited arcs (0 = 14) */
    float beta;              /* back to push when frontier vertices * beta < non-isolated vertices (0 = 24) */
    int32_t group_vertices;  /* rows of degree <= 1024 handled per warp task, 1..32 (0 = 32); results do not
                                depend on it (sums follow fixed 1024-arc chunks of each row) */
    int32_t blocks_per_sm;   /* persistent-grid residency, also of the per-source form (0 = occupancy maximum) */
    int64_t barrier_budget;  /* device cycles a grid-barrier wait may spin before BC_E_TIMEOUT
                                (0 = about 20 s; tests may set 1 to force a timeout) */
    int32_t trace;           /* 1 = record a device timestamp at the end of every grid-wide phase */
    int32_t teams;           /* independent groups of blocks, each running its own batches (0 = auto:
                                one block per ~2^19 arcs per team, at most one team per batch) */
    int32_t dense_min;       /* batch widths >= 32: an arc matching at least this many columns of its row's
                                batch is summed by the whole warp, one lane per column group, instead of one
                                (arc, column) pair per lane (0 = auto); results do not depend on it */
    int32_t source_order;    /* bc_compute, bc_many_create (fixed once at creation) and, with the automatic
                                rule, each serving job: 1 = batches take the sources in the order given; 2 =
                                sources are first grouped by their distances to the graph's 32 highest-degree
                                vertices (a 32-source forward traversal, once per graph), so that a batch holds
                                sources that
                                reach most vertices at the same levels and more arcs are summed column-mapped;
                                0 = auto: 2 on undirected graphs with at least 256 sources, 2048 non-isolated
                                vertices and a maximum degree of at least 16 times the mean, else 1.  Only the
                                order in which per-source dependencies are added to BC changes (rounding); the
                                grouping depends on the graph and the source list alone, so results stay the
                                same for every batch width and direction setting.  The landmark levels are
                                kept with the graph ([n][32] uint16), built on the first grouped call */
    int32_t deep_form;       /* bc_compute / bc_compute_ex: 1 = always the batched traversal; 2 = the per-source
                                form for graphs of large diameter: every block of one launch runs whole sources
                                alone, level by level with block barriers only, so that thousands of levels of a
                                few thousand vertices do not each cost grid-wide barriers; 0 = auto: 2 when
                                batch_width is 0, the graph's BFS depth is known to be at least 48 levels of
                                at most 8192 vertices on average (from an earlier call, or from a one-source
                                probe that the first call with at least 64 sources on a graph of mean degree at
                                most 8 runs) and the memory budget leaves a block per source or SM, else 1.
                                Same arithmetic, same sums in the same order: the two forms give the same bits.
                                The per-source form takes blocks_per_sm and ignores the batched traversal's
                                knobs (width, direction, alpha, beta, grouping of rows, teams, dense_min) and
                                trace (it records no phase trace) */
} bc_options;

/*
 * BC over a source list (paper Appendix A, computeBC; sources in ORIGINAL ids,
 * host or device pointer).  out_bc: device array of n doubles, overwritten,
 * in original ids.  Work is ordered on `stream`; the call returns after the
 * results are final (it reads a device status word).  nsrc == 0 writes zeros.
 * Returns BC_OK or BC_W_SIGMA_INEXACT on success.
 */
bc_status bc_compute(bc_graph* g, const int32_t* sources, int32_t nsrc, double* out_bc,
                     bc_stream_t stream);
bc_status bc_compute_ex(bc_graph* g, const int32_t* sources, int32_t nsrc, double* out_bc,
                        bc_stream_t stream, const bc_options* opt);

/*
 * Splitting one job over several GPUs (sources are independent: the paper's
 * computeBC loops over its source set, Appendix A, and BC is a sum over it).
 * Every rank holds the same graph, takes a share of the job's batches, runs
 * bc_compute_ex on its share, and the ranks' partial BC vectors are summed.
 *
 * bc_source_batches: the order in which bc_compute_ex(g, sources, nsrc, ..., opt)
 * would batch the list (grouped by hub distances under the automatic rule of
 * bc_options.source_order, else as given; it depends on the graph and the list
 * alone) and the batch width it would use.  sources: host or device, original
 * ids; order: HOST int32[nsrc], written; batch_width: host, may be NULL.
 * Batch b is order[b*K, (b+1)*K).  A rank that runs a sub-list of whole
 * batches with batch_width = K and source_order = 1 gets, per column, the
 * bits the full call computes.  BC_E_SOURCE for an id outside [0, n).
 */
bc_status bc_source_batches(bc_graph* g, const int32_t* sources, int32_t nsrc, const bc_options* opt,
                            int32_t* order, int32_t* batch_width, bc_stream_t stream);

/*
 * Sum of per-rank partial results in a fixed order: out[v] = parts[0][v] +
 * parts[1][v] + ... + parts[nranks-1][v], added left to right (device arrays;
 * parts is [nranks][n] row-major, out[n]; out may not overlap parts).  The
 * order is that of the ranks, whatever order the parts arrived in, so the
 * result repeats bit for bit.  Returns when out is final.
 */
bc_status bc_reduce_ranks(const double* parts, int32_t nranks, int64_t n, double* out, bc_stream_t stream);

/*
 * Multi-source BFS: the forward sweep of bc_compute alone (Section 2.3.2,
 * iterateInBFS: levels and shortest-path counts) for each listed source, the
 * same kernels and batching (on deep graphs, by bc_compute's automatic rule of
 * bc_options.deep_form, the per-source form; the same values either way).  sources: nsrc original ids (host or device).
 * level: device int32[nsrc][n], row i = distance from sources[i] (-1 when
 * unreachable), original vertex ids; required when n > 0 and nsrc > 0.
 * sigma: device double[nsrc][n] or NULL = number of shortest paths (exact below
 * 2^53, rounded above and the call returns BC_W_SIGMA_INEXACT; +inf beyond the
 * double range unless sigma_exp is given).  sigma_exp: device int32[nsrc][n] or
 * NULL; when given, sigma holds a mantissa in [0.5, 1) and the count is
 * sigma * 2^sigma_exp (0 and 0 when unreachable).  Overwrites the outputs; the
 * call returns after they are final.  Counterpart of the paper's BFS
 * construct as a standalone operation (no backward sweep, no BC).
 */
bc_status bc_bfs(bc_graph* g, const int32_t* sources, int32_t nsrc, int32_t* level, double* sigma,
                 int32_t* sigma_exp, bc_stream_t stream);

/*
 * PageRank as the paper's computePR (Appendix A, PR listing): ranks start at
 * 1/n; each sweep sets rank(v) = (1 - delta)/n + delta * sum over arcs u -> v
 * of rank(u) / outdeg(u) (all vertices at once), and sweeps repeat while the
 * L1 change of the sweep exceeds beta and fewer than max_iter have run.  No
 * redistribution of the rank of vertices without out-arcs (as in the
 * listing).  out_rank: device double[n], original ids.  iterations /
 * last_diff (host, may be NULL): sweeps run and the last L1 change.  Every
 * sum has a fixed order: repeated calls give the same bits.  Requires
 * 0 <= delta <= 1, beta >= 0, max_iter >= 1.
 */
bc_status bc_pagerank(bc_graph* g, double delta, double beta, int32_t max_iter, double* out_rank,
                      int32_t* iterations, double* last_diff, bc_stream_t stream);

/*
 * Weighted graphs (positive int32 arc weights), undirected (BC_UNDIRECTED) or
 * directed.  weights[m] is parallel to indices[m] of the input CSR (host or
 * device, as the flags say), whose rows must be sorted ascending.  Undirected:
 * both arcs of an edge carry the same weight.  Directed: each arc has its own
 * weight.  Checks (unless
 * BC_SKIP_VALIDATION): the CSR rules of bc_graph_create, sorted rows,
 * weights > 0, symmetric weights when undirected, else BC_E_INVALID_GRAPH.
 * The result is a regular graph (every unweighted call works on it, ignoring
 * the weights) that bc_compute_weighted also accepts.
 */
bc_status bc_graph_create_weighted(const int32_t* offsets, const int32_t* indices, const int32_t* weights,
                                   int32_t n, int64_t m, uint32_t flags, bc_stream_t stream, bc_graph** out);

/*
 * Weighted BC over a source list (original ids, host or device): the paper's
 * BC accumulation (Appendix A, BC listing) over the shortest-path DAG of
 * weighted distances, the distances found by the fixed-point Min relaxation
 * of the paper's SSSP program (Section 2.3).  Path counts are exact below
 * 2^64 (BC_W_SIGMA_INEXACT once one reaches 2^53, BC_E_SIGMA_RANGE at
 * 2^64); BC is the raw sum over the listed sources, as for bc_compute.
 * On a directed graph paths follow the arcs: distances and path counts are
 * pushed along out-arcs, dependencies pulled over them.  Sources are batched in the
 * grouped order of bc_compute's automatic rule (undirected skewed graphs,
 * 256 sources or more); the order changes rounding only.
 * Batches of 32 sources, one launch each; results repeat bit for bit.
 * BC_E_INVALID_ARG if the graph has no weights.  bc_last_run_stats reports
 * max_levels / pull_levels / push_levels = passes of the distance, path-count
 * and dependency loops, summed over batches.
 */
bc_status bc_compute_weighted(bc_graph* g, const int32_t* sources, int32_t nsrc, double* out_bc, bc_stream_t stream);

/* Per-call facts of the last bc_compute / bc_compute_ex / bc_bfs on this graph. */
typedef struct {
    int32_t batch_width;     /* width used */
    int32_t batches;         /* traversals run */
    int32_t max_levels;      /* deepest BFS (levels, source = level 0) */
    int32_t pull_levels;     /* forward levels run in pull (bottom-up) form, summed over batches */
    int32_t push_levels;     /* forward levels run in push (top-down) form */
    int32_t ext_batches;     /* batches rerun in the extended-range path-count form */
    int32_t grid_blocks;     /* persistent grid size */
    int32_t kernel_launches; /* kernels launched by the call */
    float kernel_ms;         /* device time of the persistent traversal launches (CUDA events on the call's stream) */
    int32_t teams;           /* teams of the last launch */
    float order_ms;          /* device time of the source grouping: the key gather, plus the graph's landmark
                                traversal on the first grouped call (0 when the sources were not grouped; not
                                part of kernel_ms) */
    int64_t arcs_visited;    /* bc_compute_weighted: arcs read by all passes of all batches (0 otherwise) */
    int64_t rows_visited;    /* bc_compute_weighted: rows recomputed by all passes of all batches */
    int64_t mask_arcs;       /* bc_compute_weighted: of arcs_visited, the arcs the path-count and dependency
                                loops read through the batch's DAG masks (an index and a mask word, no
                                neighbour distance row) */
    int64_t mask_lanes;      /* bc_compute_weighted: (arc, column) pairs those reads used (one count add or one
                                rho read each) */
    int64_t dag_arcs;        /* unweighted calls: terms of the forward path-count sums, i.e. the sum over the
                                call's sources of E_dag(s) = #{arcs (v, w): d_s(w) = d_s(v) + 1} (last launch) */
    int64_t reached;         /* unweighted calls: sum over the call's sources of the vertices reached, source
                                included (last launch) */
    int32_t deep_sources;    /* sources run in the per-source form of bc_options.deep_form (0: batched form) */
} bc_run_stats;
bc_status bc_last_run_stats(const bc_graph* g, bc_run_stats* st);

/*
 * Phase trace of the last call made with bc_options.trace = 1: up to `cap`
 * records of (tag, t_ns) as int64 pairs in `out` (host), *count = records.
 * tag = kind << 24 | level, kind 1 init, 2 pull level, 3 push discovery,
 * 4 path-count sum after push, 5 reverse level, 6 BC accumulation, 7 chunk
 * prefix; t_ns = device global timer at the end of the phase.
 */
bc_status bc_last_trace(const bc_graph* g, int64_t* out, int32_t cap, int32_t* count);

/*
 * Autotuner: measures the traversal on a sample of the given sources (host,
 * original ids; the whole list, up to 8192, on graphs of at most 2^24 arcs,
 * else the first 512) for batch widths 32/64/128 (and 1 for samples of at
 * most 64 sources), the pull threshold
 * (alpha) and the light-row grouping, by coordinate descent, and records the
 * fastest setting for the graph's size bucket (log2 n, log2 average degree,
 * log2 max/average degree).  Later bc_compute / bc_compute_ex calls on graphs
 * of that bucket use it for every knob left at 0.  No knob changes results.
 * best / best_rate (source-arcs per second on the sample) may be NULL.
 */
bc_status bc_autotune(bc_graph* g, const int32_t* sources, int32_t nsrc, bc_stream_t stream, bc_options* best,
                      double* best_rate);
/* Load (save = 0) or write (save = 1) the tuned settings as a JSON file. */
bc_status bc_tuning_cache(const char* path, int32_t save);

/*
 * Many graphs in one recorded sequence: for each item, BC over its sources
 * (host array, original ids, copied at create) on its graph into its output
 * (device, n doubles).  bc_many_create groups the items by batch width,
 * allocates one workspace per width, and records every item's work (source
 * mapping, one persistent launch over all of its batches, a status word, the
 * unpermute) into a CUDA graph; bc_many_run replays it on `stream`, then
 * redoes alone any item that needed the extended path-count form or larger
 * level lists, and returns the worst status (per item in item_status[nitems],
 * may be NULL).  Items on graphs that bc_compute's automatic rule sends to the
 * per-source form (bc_options.deep_form; decided at create, a depth probe
 * included) are not recorded: bc_many_run runs them after the replay through
 * bc_compute_ex in that form.  Outputs must stay alive while the plan is run.
 * Results are bitwise those of bc_compute on each item.
 */
typedef struct bc_many_plan bc_many_plan;
typedef struct {
    bc_graph* graph;
    const int32_t* sources;
    int32_t nsrc;
    double* out_bc;
} bc_item;
bc_status bc_many_create(const bc_item* items, int32_t nitems, const bc_options* opt, bc_stream_t stream,
                         bc_many_plan** out);
bc_status bc_many_run(bc_many_plan* plan, bc_stream_t stream, bc_status* item_status);
bc_status bc_many_destroy(bc_many_plan* plan);
/* Items in the plan and kernel launches recorded in its graph. */
bc_status bc_many_info(const bc_many_plan* plan, int32_t* items, int32_t* kernel_launches);

/*
 * Serving: continuous batching over resident graphs.  bc_batch_submit queues a
 * job (sources copied from host memory at submit time; out_bc is a device
 * array of n doubles that must stay alive until bc_poll returns a final
 * status).  Jobs are admitted as execution slots and device memory free up;
 * admitted jobs run concurrently on their own streams.  bc_poll returns
 * BC_PENDING until done, then the job's final status once, releasing the id.
 * A job's result is bitwise the same whether it runs alone or among others.
 * Jobs on a graph that an earlier traversal showed deep (bc_options.deep_form's
 * depth rule) run one by one through bc_compute_ex, which picks the per-source
 * form; its per-source state is the graph's and is not part of the admission
 * budget.
 */
bc_status bc_batch_submit(bc_graph* g, const int32_t* sources, int32_t nsrc, double* out_bc,
                          bc_job* job);
bc_status bc_poll(bc_job job);
/* As bc_poll; on a final status also writes the job's submit-to-completion time in seconds. */
bc_status bc_poll_ex(bc_job job, double* latency_s);
/* Blocks until the job is final (timeout_ms < 0: no limit; when it passes: BC_PENDING), then
 * returns and releases like bc_poll. */
bc_status bc_wait(bc_job job, int64_t timeout_ms);
bc_status bc_wait_ex(bc_job job, int64_t timeout_ms, double* latency_s);
/* Serving facts: jobs admitted concurrently at peak, total completed (since start or the last reset). */
bc_status bc_server_stats(int32_t* peak_concurrency, int64_t* completed);
/* Starts a new measurement window: peak = the traversals running now, completed = 0. */
bc_status bc_server_reset_stats(void);
/*
 * Withdraws a job that is still queued (not yet admitted): it will not run,
 * out_bc is not written, and its bc_poll / bc_wait then returns BC_E_CANCELLED
 * (releasing the id).  BC_E_BUSY when the job is already running or finished
 * (it completes normally); BC_E_INVALID_ARG for an unknown or released id.
 */
bc_status bc_cancel(bc_job job);
/* Slots (traversals run concurrently, each on 1/slots of the GPU; default 1, which measured
 * best: jobs queued on the same graph are still packed into one traversal) and the device-memory
 * budget for admission (bytes; 0 = 80% of free).  While the server runs the slot count may only
 * grow; the call then waits until the traversals in flight have finished. */
bc_status bc_server_config(int32_t slots, int64_t memory_budget);

/*
 * Inspection: the team split that bc_compute and plans use for a traversal
 * (host arithmetic only, no device work; the calls pass their graph's arc
 * count m, the batch width, the batch count, the cooperative grid's blocks,
 * the arena bytes of one team and the device's free bytes at the call).
 * A team has about one block per 2^19 arcs on large graphs, at least about
 * 0.7 * m^0.24 * batch_width / 128 blocks on smaller ones, at most 32 when
 * batch_width is 1; at least two teams when there are two batches; no more
 * teams than batches or blocks; the teams' slices within 30% of free_bytes
 * (and 24 GB); then the fewest teams that need the same number of rounds.
 * teams > 0 asks for that many (still capped by batches, blocks and memory).
 * Writes nteams and team_blocks (blocks / nteams).  BC_E_INVALID_ARG for
 * m < 0, batch_width < 1, nbatch < 0, blocks < 1, teams < 0 or NULL outputs.
 */
bc_status bc_team_rule(int64_t m, int32_t batch_width, int32_t nbatch, int32_t blocks, uint64_t team_bytes,
                       uint64_t free_bytes, int32_t teams, int32_t* nteams, int32_t* team_blocks);

/*
 * Test/inspection: levels and path counts of ONE source (original id) in
 * original ids.  level[v] = BFS depth or -1; sigma(v) = sigma_mant[v] *
 * 2^sigma_exp[v] exactly when the count is below 2^53 (mantissa in [0.5,1)).
 * Host output buffers of n entries; any may be NULL.
 */
bc_status bc_debug_source(bc_graph* g, int32_t s, int32_t* level, double* sigma_mant, int32_t* sigma_exp);

/*
 * BC for callers that cannot allocate device memory (the paper has no
 * counterpart; this is an addition of this library).  Some host code may not
 * call cudaMalloc: a framework that owns the whole device through its own pool
 * and forbids other allocations (to hold a hard memory cap), or a
 * latency-critical path that must never enter the CUDA allocator.  Such a
 * caller passes everything on the device: offsets[n+1] and indices[m] (int32
 * undirected CSR, used as given: offsets and index range are checked
 * (BC_E_INVALID_GRAPH), symmetry, self-loops and duplicates are not; rows are
 * summed whole, so the longest row sets the count at which a batch moves to
 * the extended-range form), sources[nsrc] (original ids, BC_E_SOURCE outside
 * [0, n)), and out_bc[n] (overwritten with the same raw BC as bc_compute,
 * within 1e-9 relative).  All working state lives in one static device array
 * of about 37 MB that every GPU loading the library holds until exit; hence
 * n <= 32768 vertices (BC_E_LIMIT beyond), batches of 32 sources.  The call
 * allocates nothing.  It is synchronous: it waits on `stream` (and reads
 * status words back into host memory) before it returns, with the result
 * final.  Each call looks up the array's address on the calling thread's
 * current device (cudaGetSymbolAddress), so that device must be the one that
 * holds the caller's buffers.  Every call shares the array and it keeps the
 * last call's contents (each call clears what must start at zero): calls that
 * overlap on the GPU, from several streams or threads, race and must not be
 * issued.
 */
bc_status bc_compute_noalloc(const int32_t* offsets, const int32_t* indices, int32_t n, int64_t m,
                             const int32_t* sources, int32_t nsrc, double* out_bc, bc_stream_t stream);

const char* bc_status_string(bc_status st);
const char* bc_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* LIBBC_BC_H */
