/*
 * peers.h -- C ABI of the B300 library for exact effective resistance by the implicit-inverse
 * query sweep (PEERS, arXiv 2606.31535).
 *
 * Problem (PEERS §II-A, eq. 1-4; §IV-A, eq. 15-18).  For an undirected graph G = (V, E, w)
 * with positive conductances, L_G = D - W is its Laplacian (eq. 1).  Grounding a node g and
 * deleting its row and column gives the SPD reduced Laplacian L_r.  The effective resistance
 * of a pair (s, t) is R_st = (e_s - e_t)^T L_r^{-1} (e_s - e_t) (eq. 2, eq. 15), with the unit
 * vector of g dropped when an endpoint is g (eq. 4).  The library factors L_r = L D L^T (unit
 * lower L; the paper's eq. 3 writes the equivalent L L^T) and returns
 *     R_st = sum_k y_k^2 / d_k,   L y = e_s - e_t          (eq. 16-18),
 * walking for each query only the elimination-tree path(s) on which y is non-zero (Lemma 1),
 * never forming L^{-1}.
 *
 * Call sequence: peers_create -> peers_analyze (host) -> peers_factor (device) ->
 * peers_query (device sweep) -> peers_free_* / peers_destroy.
 *
 * Conventions shared by all calls:
 *   - Every function returns PEERS_OK (0) or a negative PEERS_E* status; peers_strerror()
 *     names it.  On error no output handle is created and *out is set to NULL.
 *   - Callers own every array they pass in; the library copies what it keeps.  Handles are
 *     owned by the library until freed with their peers_free_* / peers_destroy call.
 *   - Device work is issued on the context's CUDA stream; calls return after that work has
 *     finished unless stated otherwise.
 *   - One context per host thread; handles may be shared read-only between contexts on the
 *     same device.
 */
#ifndef PEERS_H
#define PEERS_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---------------------------------------------------------------------- */
#define PEERS_OK 0
#define PEERS_EINVAL (-1)        /* malformed input: asymmetric CSR, self-loop, duplicate edge,
                                    w <= 0 or not finite, index out of range, bad argument */
#define PEERS_ENOTCONNECTED (-2) /* the graph is not connected (L_r would be singular) */
#define PEERS_ENOTSPD (-3)       /* a pivot d_k <= 0 or not finite during the factorization */
#define PEERS_ENOMEM (-4)        /* host or device allocation failed */
#define PEERS_ECUDA (-5)         /* a CUDA runtime call failed (device lost, bad stream, ...) */
#define PEERS_ETIMEOUT (-6)      /* a bounded device-side wait ran out */
#define PEERS_ENOTREADY (-7)     /* result not available yet (non-blocking calls) */

/* ---- flags ----------------------------------------------------------------------------- */
#define PEERS_OUT_DEVICE 1  /* peers_query: R is a device pointer (else a host pointer) */

typedef struct peers_ctx peers_ctx;           /* device + CUDA stream + scratch */
typedef struct peers_symbolic peers_symbolic; /* host plan: ordering, etree, supernodes,
                                                 query grouping (no device memory) */
typedef struct peers_numeric peers_numeric;   /* device-resident L panels, D, plan copy */

/* Options of peers_analyze.  Zero-initialise and set what you need; NULL means defaults. */
typedef struct peers_options {
  int32_t ordering;     /* 0 = auto (coordinate nested dissection when coords are given,
                           else BFS level-structure nested dissection); 1 = coordinate ND;
                           2 = BFS ND; 3 = natural order (tests only) */
  int32_t nd_leaf;      /* nested-dissection leaf size (0 = default 32) */
  int32_t relax_small;  /* amalgamate supernodes up to this many columns (0 = default 8) */
  int32_t relax_max;    /* amalgamate up to this many columns when extra zeros <= relax_frac
                           (0 = default 32) */
  double relax_frac;    /* tolerated fraction of explicit zeros in an amalgamated supernode
                           (0 = default 0.15) */
  int64_t carry_budget; /* device bytes of query fronts carried between levels per wave
                           (0 = default 48 GiB); a smaller budget splits the queries into more
                           waves walked one after another */
  int32_t qcap[4];      /* sweep tile caps: at most qcap[c] queries per CTA for supernodes
                           whose front has N rows in class c = [0,128), [128,512), [512,2048),
                           [2048,inf); 0 = the largest tile that fits (up to 32) */
  int64_t front_smem;   /* shared-memory bytes a sweep CTA may give its query fronts (0 = the
                           default: tiles sized for 200 KiB, fronts up to the 227 KiB per-CTA
                           limit).  A supernode whose front does not fit even with one query
                           keeps its fronts in global memory instead (results are unchanged
                           bit for bit); a small value forces that path, e.g. for tests */
  int64_t one_stream;   /* nonzero: the factorization, the selected inversion and the block
                           inverse run on the context's stream alone, without the lanes
                           (independent subtrees on concurrent streams), the factorization's
                           split column blocks (three streams) or the block inverse's
                           concurrent narrow launches.  Every result is the same bit for bit;
                           the default schedule is faster.  For tests and comparison. */
  int64_t reserved[4];
} peers_options;

/* Statistics of an analysis (all counts exact). */
typedef struct peers_info {
  int64_t n;              /* graph nodes */
  int64_t n_reduced;      /* n - 1 (ground removed) */
  int64_t nnz_a;          /* strictly-lower entries of L_r */
  int64_t nnz_l;          /* stored entries of the supernodal L incl. diagonal and
                             explicit zeros: sum over supernodes of (n_c+n_b)*n_c */
  int64_t nsuper;         /* supernodes */
  int64_t levels;         /* supernodal etree height + 1 (one sweep launch per level) */
  int64_t max_nc, max_nb; /* largest supernode width and below-diagonal row count */
  int64_t nq;             /* queries */
  int64_t nq_trivial;     /* queries with u == v (R = 0, no work) */
  int64_t nq_two_branch;  /* listed pairs whose two etree paths merge above the start */
  int64_t walk_entries;   /* W = sum_q sum_{s on path(q)} (n'(n'-1)/2 + n_b n' + n'), the
                             per-query walk's factor entries (n' = columns of s at or after
                             the query's first non-zero); bytes streamed = 8 W */
  int64_t walk_fma;       /* FMAs the sweep kernels execute (block-aligned; >= useful work) */
  int64_t factor_fma;     /* FMAs of the numeric factorization (dense blocks) */
  int64_t device_bytes;   /* device memory of peers_factor + peers_query (footprint) */
  double t_order, t_symbolic, t_queries; /* host seconds of the analysis phases */
  int64_t nsuper_spilled; /* supernodes whose sweep fronts live in global memory (fronts
                             larger than a CTA's shared memory; see peers_options) */
  int64_t front_bytes;    /* bytes of query fronts one sweep reads from and writes to the
                             carry buffer between levels (single-path queries) */
  int64_t lanes;          /* concurrent streams of independent subtrees (0: one stream) */
  int64_t split_blocks;   /* factorization column blocks whose update runs split over three
                             streams (0 under peers_options.one_stream) */
} peers_info;

/* ---- context --------------------------------------------------------------------------- */

/* Creates a context on CUDA device `device`.  `cuda_stream` is a cudaStream_t to issue all
 * work on (the caller keeps ownership), or NULL for a library-owned non-blocking stream.
 * Errors: PEERS_EINVAL (no such device), PEERS_ECUDA. */
int peers_create(peers_ctx **out, int device, void *cuda_stream);
void peers_destroy(peers_ctx *ctx);

/* ---- analysis (host only; PEERS Alg. 8 step 1: ground, fill-reducing order, structure) -- */

/* Builds the plan for graph (n nodes; symmetric CSR indptr[n+1] int64, indices[nnz] int32,
 * w[nnz] conductance of each stored entry, both directions equal) grounded at node `ground`,
 * for the queries (qu[i], qv[i]), i < nq.  nq < 0 or qu == NULL selects all edges, in the
 * order "u ascending, then each CSR neighbour v > u in CSR order".  `coords` (n x dim, row
 * major, may be NULL) only guides the ordering.  `ctx` may be NULL: no device is touched.
 * Queries with u == v give R = 0; a query touching the ground follows eq. 4.
 * Large graphs and query sets are analysed on up to 8 host threads (at most the hardware's
 * count, and at most the environment variable PEERS_ANALYSIS_THREADS when it is set to a
 * positive number); the plan does not depend on the thread count.  The caller's buffers are
 * only read, and only during the call.
 * Errors: PEERS_EINVAL, PEERS_ENOTCONNECTED, PEERS_ENOMEM. */
int peers_analyze(peers_ctx *ctx, int64_t n, const int64_t *indptr, const int32_t *indices,
                  const double *w, int32_t ground, int64_t nq, const int32_t *qu,
                  const int32_t *qv, const double *coords, int dim, const peers_options *opt,
                  peers_symbolic **out);
int peers_symbolic_info(const peers_symbolic *sym, peers_info *info);
/* Number of queries of the plan (the length of R in peers_query). */
int64_t peers_num_queries(const peers_symbolic *sym);
/* Device bytes that peers_factor + peers_query will hold for this plan. */
int64_t peers_footprint_bytes(const peers_symbolic *sym);
void peers_free_symbolic(peers_symbolic *sym);

/* Structure export for tests (host arrays sized by peers_info):
 *   perm[n_reduced]      graph node (ground excluded) eliminated k-th
 *   sn_first[nsuper+1]   first column of each supernode (columns are contiguous)
 *   sn_parent[nsuper]    parent supernode (-1 for a root)
 *   sn_nb[nsuper]        below-diagonal row count n_b
 *   sn_level[nsuper]     height above the leaves
 * Any pointer may be NULL. */
int peers_symbolic_export(const peers_symbolic *sym, int32_t *perm, int32_t *sn_first,
                          int32_t *sn_parent, int32_t *sn_nb, int32_t *sn_level);

/* ---- numeric factorization (device) ------------------------------------------------------ */

/* Numeric supernodal L D L^T of the grounded Laplacian on the context's device (multifrontal,
 * one level of the supernodal etree at a time).  `w` (same layout as in peers_analyze, may be
 * NULL) replaces the conductances for a refactorization on the same pattern; NULL reuses the
 * ones given to peers_analyze.  The result stays resident in device memory.
 * Errors: PEERS_ENOTSPD, PEERS_ENOMEM, PEERS_ECUDA, PEERS_EINVAL. */
int peers_factor(peers_ctx *ctx, const peers_symbolic *sym, const double *w, peers_numeric **out);
/* Copies the diagonal D (n_reduced entries, elimination order) to host memory. */
int peers_numeric_diag(peers_ctx *ctx, const peers_numeric *num, double *d_host);
void peers_free_numeric(peers_numeric *num);

/* ---- implicit inverse by etree blocks (the paper's order of work) ------------------------- */

/* The same results as peers_query by another route: the entries of Z = L^{-1} that the paper's
 * row-wise implicit inversion visits (§III-A/C, eq. 11, Lemma 1) are computed block by block,
 * Z[P_t, C_t] for every supernode t over its ancestor path P_t, top-down (one launch per tree
 * depth, each block a staircase GEMM from its ancestors' blocks), and each query then reads
 * its two columns: R_st = sum_i (Z[i,s] - Z[i,t])^2 / d_i (eq. 12, eq. 18).  Work is about the
 * paper's O(n^alpha nnz(L)) (Thm 4), far below the per-query walk, but device memory holds all
 * of nnz(Z) at once (peers_blockinv_bytes); the call fails with PEERS_ENOMEM when it does not
 * fit.  The device memory is allocated and freed inside the call.  The host-side plan (block
 * offsets, tiles, the per-query column list; about 24 bytes per query plus 12 per entry of
 * the factor's row structure) is built by the first call on `sym` (or by peers_blockinv_bytes
 * / _fma) and kept with the handle for later calls, until peers_retile or peers_autotune
 * rebuild the sweep plan or the handle is freed.  Calls on one `sym` from several threads
 * are safe.  Errors: PEERS_EINVAL, PEERS_ENOMEM, PEERS_ECUDA. */
int peers_query_blockinv(peers_ctx *ctx, const peers_symbolic *sym, const peers_numeric *num,
                         double *R, int flags);
/* Device bytes peers_query_blockinv needs for this plan. */
int64_t peers_blockinv_bytes(const peers_symbolic *sym);
/* FMAs of its block GEMMs (the dominant kernel), counting the staircase's skipped zeros out. */
int64_t peers_blockinv_fma(const peers_symbolic *sym);

/* ---- selected inversion (all-edge resistances from the inverse on the pattern of L) ------- */

/* The same results for every query that lies inside the pattern of L (every graph edge and
 * every pair touching the ground): Sigma = L_r^{-1} is computed only on the pattern of L by
 * Takahashi's recurrences in supernodal form, top-down, and R_uv = Sigma_uu + Sigma_vv -
 * 2 Sigma_uv (eq. 2).  The work is about one factorization, far below both the walk and the
 * block inverse; the memory is two depths of dense inverse fronts.  The paper does not use it
 * (§II-C); it is an independent second route to the same numbers.  A plan with listed pairs
 * outside the pattern is rejected with PEERS_EINVAL (use peers_query).  The host-side plan is
 * kept with `sym` after the first call, as for peers_query_blockinv (rebuilt for a device with
 * another SM count).  The first call on a factor also copies that plan to the device and
 * allocates its working buffers (T^{-1}, M and two depths of inverse fronts per stream of
 * independent subtrees: about 2.7 GB for a 1M-node mesh), which stay with `num` for later calls
 * until it is freed or the plan is rebuilt; calls on one `num` are serialised.  Errors:
 * PEERS_EINVAL, PEERS_ENOMEM, PEERS_ECUDA. */
int peers_query_selinv(peers_ctx *ctx, const peers_symbolic *sym, const peers_numeric *num,
                       double *R, int flags);
/* Useful multiply-adds of the selected inversion for this plan: Sigma[B,C], the lower
 * triangle of Sigma[C,C], and the phase that forms T^{-1} and M = P T^{-1}. */
int64_t peers_selinv_fma(const peers_symbolic *sym);

/* ---- spectral sparsification (PEERS §II-B, Alg. 1) ---------------------------------------- */

/* Draws q edges with probability p_e proportional to w_e R_e and weights each drawn edge by
 * w_e / (q p_e), summed over its draws (Alg. 1).  All pointers are device pointers: w and R
 * (m entries each, e.g. the conductances and the resistances of an all-edge peers_query),
 * u (q uniform numbers in [0, 1) supplied by the caller: the call draws no random numbers of
 * its own), count (m int64, the number of draws of each edge) and weight (m, the sparsifier's
 * conductance of each edge; 0 for edges never drawn).
 * Reproducibility: scores are quantised once in FP64 to k_e = floor(w_e R_e S) with
 * S = floor(2^62 / m) / max_e(w_e R_e), so p_e = k_e / sum(k) and draw i picks the first edge
 * whose cumulative weight exceeds floor(u_i sum(k)) -- exact integer work, the same on any
 * machine.  Errors: PEERS_EINVAL, PEERS_ENOMEM, PEERS_ECUDA. */
int peers_sparsify(peers_ctx *ctx, int64_t m, const double *w, const double *R, int64_t q,
                   const double *u, int64_t *count, double *weight);

/* ---- tile shapes --------------------------------------------------------------------------- */

/* Re-tiles a factored plan's sweep with new per-size-class caps (see peers_options.qcap) and
 * re-uploads its work lists.  Results are unchanged bit for bit: column blocks stay aligned,
 * so a query's arithmetic never depends on its tile.  Only the speed changes. */
int peers_retile(peers_ctx *ctx, peers_symbolic *sym, peers_numeric *num, const int32_t qcap[4]);

/* Autotuner for the sweep's tile shapes: for each front-size class it times every candidate
 * cap (1, 2, 4, 8, 16, 32 queries per CTA) on the heaviest supernodes of that class of this
 * plan, keeps the fastest and re-tiles the plan (as peers_retile).  `cache_path` (may be NULL)
 * names a text file of "<GPU name>|class<c>|<cap>" lines: classes found there are not measured
 * again, and the measured ones are added.  qcap_out receives the caps, gain_out the speed-up of
 * each class's chosen cap over the largest tile on the timed supernodes (1 when not measured).
 * The timing runs overwrite the plan's carried fronts; results of later peers_query calls are
 * unaffected.  This is the batching tuner of the sweep; the paper has no counterpart. */
int peers_autotune(peers_ctx *ctx, peers_symbolic *sym, peers_numeric *num,
                   const char *cache_path, int32_t qcap_out[4], double gain_out[4]);

/* ---- the sweep (device) ------------------------------------------------------------------ */

/* Effective resistance of every query of the plan into R[0 .. peers_num_queries(sym)), in the
 * plan's query order.  R is a device pointer when flags has PEERS_OUT_DEVICE, else a host
 * pointer.  One launch per level of the supernodal etree walks every query from its starting
 * supernode to the root (eq. 16-18 over the etree path of Lemma 1).  A pair whose endpoints'
 * etree paths only meet above the lower endpoint's supernode (a listed non-edge pair) is
 * walked as two branches that merge at their lowest common supernode, with one more small
 * launch per wave to combine the branches' sums.
 * Errors: PEERS_EINVAL, PEERS_ENOMEM, PEERS_ECUDA. */
int peers_query(peers_ctx *ctx, const peers_symbolic *sym, const peers_numeric *num, double *R,
                int flags);

/* The sweep of peers_query for callers that cannot let the library allocate device memory:
 * a framework that owns all device memory through its own pool, or a latency-bound loop that
 * cannot afford the device-wide synchronisation a cudaMalloc or cudaFree may cause.  The
 * paper has no counterpart; this is a deployment variant of the same kernels.
 *   - Inputs are the plan and its resident factor (peers_factor allocated those earlier);
 *     the output R_device is a device array of peers_num_queries(sym) doubles, written in
 *     the plan's query order.  The call allocates and frees nothing.
 *   - Scratch: the fronts carried between levels and the running sums live in one static
 *     device array of 2 Mi doubles (16 MiB) compiled into the library; every GPU that loads
 *     the library holds it until the process exits.  A plan fits when its largest wave's
 *     query slots x (max n_b + 1) <= 2 Mi doubles.  peers_analyze counts exactly
 *     8 (max n_b + 1) bytes per slot against peers_options.carry_budget, so any plan analysed
 *     with carry_budget <= 16 MiB fits (its queries are split into more waves).  A plan that
 *     does not fit is rejected with PEERS_EINVAL and a message naming both sizes.
 *   - The call returns after the sweep has finished: it synchronises the context's stream.
 *   - The first call on a device looks up the array's device address (cudaGetSymbolAddress)
 *     and caches it; make that first call before any stream capture.
 *   - All calls share the one array, which keeps the last call's contents.  Nothing in it
 *     needs to start at zero (each carry is written before it is read); R is cleared by the
 *     call.  Calls that overlap on the GPU (other streams, other contexts, other threads)
 *     race on the array: serialise them.
 * Errors: PEERS_EINVAL, PEERS_ECUDA. */
int peers_query_noalloc(peers_ctx *ctx, const peers_symbolic *sym, const peers_numeric *num,
                        double *R_device);

/* ---- batched sweep of many graphs -------------------------------------------------------- */

/* Many independent graphs, each with its own plan and factor, swept together: the graphs'
 * level sequences are aligned at the top (every graph's root level in the last launch) and
 * the t-th level from the top of every graph becomes one persistent kernel launch (CTAs pull
 * work items of all graphs until the level is done), so G graphs of heights H_g take
 * max_g H_g launches.  With PEERS_BATCH_CUDA_GRAPH the launch sequence is
 * captured into a CUDA graph on the first peers_batch_query and replayed afterwards.  Each
 * graph's results are bit-identical to its own peers_query (an item's arithmetic depends
 * only on its supernode and queries).  The handles must outlive the batch.  This is the
 * batching pattern of the sweep; the paper's own parallel driver is Alg. 8. */
typedef struct peers_batch peers_batch;
#define PEERS_BATCH_CUDA_GRAPH 1
int peers_batch_create(peers_ctx *ctx, int32_t count, const peers_symbolic *const *syms,
                       const peers_numeric *const *nums, int flags, peers_batch **out);
/* R[i] receives graph i's peers_num_queries(syms[i]) results (host pointers, or device
 * pointers with PEERS_OUT_DEVICE); R may be NULL to leave them in the batch. */
int peers_batch_query(peers_ctx *ctx, peers_batch *b, double *const *R, int flags);
/* out[0] steps (aligned levels), out[1] work items, out[2] launches per query,
 * out[3] device bytes held by the batch. */
int peers_batch_info(const peers_batch *b, int64_t out[4]);
void peers_batch_free(peers_batch *b);
/* One-shot: create, query once (no graph capture), free. */
int peers_query_batch(peers_ctx *ctx, int32_t count, const peers_symbolic *const *syms,
                      const peers_numeric *const *nums, double *const *R, int flags);

/* ---- serving: continuous batching of requests ------------------------------------------- */

/* A request loop on one device.  Each submitted request (a graph and its queries, copied at
 * submit) is analysed and factored by one of `workers` host threads on its own CUDA stream,
 * admitted when its device footprint (peers_footprint_bytes) fits in `mem_budget_bytes`
 * next to the admitted requests and at most `max_active` are admitted, and then swept by
 * continuous batching: one persistent launch per step carries work of every active request;
 * requests join at the next step after their factor is ready and leave after their last
 * level.  Each step gives every active request a share of a fixed amount of work (a few
 * milliseconds of the device) from its current etree level -- the whole level when it is
 * smaller -- so a step's length does not depend on the largest request in the mix.  Device
 * memory of the requests comes from a memory pool of the server with stream-ordered
 * allocation and release, so requests joining and leaving never synchronise the device.
 * Results equal peers_query's bit for bit, alone or in the mix.
 * mem_budget_bytes <= 0 selects 64 GiB; max_active <= 0 selects 64; workers <= 0 selects 4. */
typedef struct peers_server peers_server;
typedef struct peers_server_stats {
  int64_t submitted, completed, failed, queries;
  int64_t steps, launches;      /* sweep steps run, kernel launches */
  int64_t peak_bytes;           /* largest admitted footprint sum */
  double wall_s;                /* first submit to last completion */
  double qps;                   /* completed queries / wall_s */
  double p50_s, p99_s, mean_s;  /* request latency, submit to results ready */
  int64_t max_step_requests;    /* most requests with work in one step */
  int64_t request_steps;        /* sum over completed requests of the steps that carried their
                                   work; above `steps` exactly when requests shared steps */
  int64_t ready;                /* factored requests waiting to join the sweep */
} peers_server_stats;
/* `opt` (may be NULL) is applied to the analysis of every request (ordering, tile caps,
 * carry budget). */
int peers_server_create(int device, int64_t mem_budget_bytes, int32_t max_active,
                        int32_t workers, const peers_options *opt, peers_server **out);
/* Same graph/query arguments as peers_analyze; returns a ticket. */
int peers_server_submit(peers_server *sv, int64_t n, const int64_t *indptr,
                        const int32_t *indices, const double *w, int32_t ground, int64_t nq,
                        const int32_t *qu, const int32_t *qv, const double *coords, int dim,
                        int64_t *ticket);
/* 1 = results ready, 0 = not yet, < 0 = the request failed with that status. */
int peers_server_poll(peers_server *sv, int64_t ticket);
/* Blocks until the request is done, copies up to `cap` results into host R (may be NULL),
 * stores the request's latency, and releases the ticket. */
int peers_server_wait(peers_server *sv, int64_t ticket, double *R, int64_t cap,
                      double *latency_s);
int peers_server_get_stats(peers_server *sv, peers_server_stats *out);
/* hold != 0: factored requests wait (stats.ready counts them) instead of joining the sweep;
 * hold == 0: they join at the next step.  Lets a caller start a known set of requests in the
 * same step.  Destroying the server releases a hold. */
int peers_server_hold(peers_server *sv, int hold);
/* Finishes the admitted and queued requests, then stops the threads and frees everything. */
void peers_server_destroy(peers_server *sv);

/* Counters of the last peers_factor / peers_query on a context.  Device times are filled only
 * while timing is enabled (peers_set_timing(ctx, 1)); counts and bytes always. */
typedef struct peers_stats {
  double sweep_s;          /* device seconds of the sweep launches of the last peers_query */
  double max_launch_s;     /* longest single sweep launch */
  double factor_s;         /* device seconds of the last peers_factor */
  int64_t sweep_launches;  /* kernels launched by the last peers_query */
  int64_t factor_launches; /* kernels launched by the last peers_factor */
  int64_t h2d_bytes;       /* host-to-device bytes of the last peers_factor + peers_query */
  int64_t d2h_bytes;       /* device-to-host bytes of the last peers_query (+ factor status) */
} peers_stats;
int peers_set_timing(peers_ctx *ctx, int enable);
int peers_last_stats(const peers_ctx *ctx, peers_stats *out);

/* Device milliseconds per step of the last timed call on the context, into
 * ms[0 .. min(count, cap)), where the steps are: for peers_query, each sweep launch (one per
 * etree level, leaves first, summed over waves); for peers_query_selinv, each tree depth of
 * the part above the concurrent subtrees (root first; a step includes the wait for that
 * depth's T^{-1} and M, which are formed beside the depths above it), then the concurrent
 * subtrees, which run on several CUDA streams at once, as one step; for
 * peers_query_blockinv, the diagonal inverses, M, each tree depth of Z blocks
 * (root first) and the query pass.  Returns the step count or a negative status (PEERS_EINVAL for a null context, or a
 * null ms with cap > 0). */
int64_t peers_last_level_times(const peers_ctx *ctx, double *ms, int64_t cap);

/* Measures the FP64 throughput of the context's device with short register-only kernels
 * (about 0.2 s), in TFLOP/s with 2 flops per multiply-add, into the caller's array of 3:
 *   tflops[0]  DFMA on the CUDA cores;
 *   tflops[1]  mma.sync m8n8k4 f64 (the FP64 tensor path);
 *   tflops[2]  both at once, alternate warps of one kernel: near tflops[0] + tflops[1] if the
 *              two use separate hardware, near max(tflops[0], tflops[1]) if they share it.
 * tflops[0] is the sweep's roofline denominator: the sweep is bound by FP64 FMA throughput.
 * Returns PEERS_EINVAL for a null argument, PEERS_ECUDA if a launch fails. */
int peers_fp64_peak(peers_ctx *ctx, double tflops[3]);

/* Measures every shape of the FP64 tensor instruction mma.sync .f64 (register-only kernels,
 * about 0.2 s), in TFLOP/s with 2 flops per multiply-add, into the caller's array of 4:
 *   tflops[0] m8n8k4, tflops[1] m16n8k4, tflops[2] m16n8k8, tflops[3] m16n8k16.
 * The sweep's dense multi-query solve would move from DFMA (peers_fp64_peak's tflops[0]) to
 * the FP64 tensor path only if one of these shapes were faster.
 * Returns PEERS_EINVAL for a null argument, PEERS_ECUDA if a launch fails. */
int peers_fp64_mma_shapes(peers_ctx *ctx, double tflops[4]);

/* ---- misc ------------------------------------------------------------------------------- */
const char *peers_strerror(int status);
/* Message of the last failed call on this host thread ("" if none). */
const char *peers_last_error(void);
/* Library version string. */
const char *peers_version(void);

#ifdef __cplusplus
}
#endif
#endif /* PEERS_H */
