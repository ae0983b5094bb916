/*
 * di.h - C ABI of the GB300 D-iteration library (libdi.so).
 *
 * The library solves X = P X + B (Eq. 1) for a sparse contractive P of the
 * PageRank form P = d Q (Eq. 2), q_kj = 1/#out_j for every edge j -> k and a
 * zero column for a dangling j, or optionally its 1/N completion (Sec. 2.2),
 * by fluid diffusion (D-iteration,
 * Eqs. defF/defH): diffusing node i moves its fluid F_i into its history H_i
 * and adds p_ki F_i to the fluid of every child k.  Nodes are chosen by the
 * cyclic threshold rule of Sec. 2.4: every node with |F_i| >= T diffuses,
 * then T <- T / alpha.  H converges to X with |X - H|_1 <= |F|_1 / (1 - d)
 * (Sec. 2, error bound).
 *
 * Conventions
 *   - Every call returns a di_status; nothing aborts the process.  On an
 *     error, di_last_error() returns a message for the calling thread.
 *   - Node ids are int32 (N <= 2^31 - 1); the graph must have fewer than
 *     2^31 edges.
 *   - "device pointer" arguments are CUDA global-memory addresses on the
 *     current device; the caller owns and keeps them alive for the call.
 *     "host pointer" arguments are ordinary (pageable or pinned) memory.
 *   - The library owns di_graph objects and everything it allocates for
 *     them; di_graph_destroy frees it all.
 *   - All calls are made on the stream in di_opts.stream (or the one passed
 *     explicitly); NULL means the legacy default stream.  Calls that return
 *     results in host memory synchronise that stream before returning.
 *   - A di_graph is not thread-safe: concurrent solves on one graph object
 *     must be serialised by the caller (its scratch memory is shared).
 */
#ifndef DI_H
#define DI_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#if defined(__GNUC__)
#define DI_API __attribute__((visibility("default")))
#else
#define DI_API
#endif

typedef enum {
    DI_OK = 0,
    DI_EINVAL = 1,    /* invalid argument (validated before any GPU work) */
    DI_ENOMEM = 2,    /* device or host allocation failed */
    DI_ECUDA = 3,     /* a CUDA call failed; di_last_error() names it */
    DI_ENOCONV = 4,   /* the level cap was reached before |F|_1 <= tol */
    DI_ETIMEOUT = 5,  /* a bounded device wait gave up (no GPU fault) */
    DI_ENONFINITE = 6 /* the residual became NaN or Inf (bad B or H0) */
} di_status;

typedef struct di_graph di_graph;

/* Shape of the push kernels (see di_autotune): a frontier node whose out-row
 * has at most thread_max_deg edges is pushed by one thread, one of at most
 * warp_max_deg edges by a warp, a longer one by the whole CTA (the
 * warp-tile push, propagation 4, sends every row above thread_max_deg to a
 * warp); the push runs push_ctas_per_sm CTAs per SM (0 = the occupancy
 * maximum; it also caps the persistent loop's grid, propagation 7).
 * push_window = 1 gives the frontier push of propagations 3 and 7 a
 * shared-memory copy of the fluid around each tile of 256 frontier nodes
 * (targets within the graph's locality radius of the tile are added there and
 * flushed with coalesced reductions).  Defaults: 16, 512, 0, 0. */
typedef struct {
    int32_t thread_max_deg;    /* 1 .. 1024 */
    int32_t warp_max_deg;      /* thread_max_deg .. 2^30 */
    int32_t push_ctas_per_sm;  /* 0 .. 64 */
    int32_t push_window;       /* 0 or 1 */
} di_tune;

/* Solver options.  Fill with di_opts_default() and change what you need. */
typedef struct {
    double alpha;          /* threshold decay T <- T/alpha, > 1; default 1.5 (Sec. 2.4) */
    int fluid_fp64;        /* 1: fluid F in FP64; 0: FP32 fluid, FP64 history (default) */
    int recompute_every;   /* FP32 fluid: exact FP64 residual F = B + P H - H every this
                              many levels; 0 (default) = no level rule */
    int max_levels;        /* level cap -> DI_ENOCONV; default 100000 */
    int warm_start;        /* 1: H holds H0 on entry and F0 = B + P H0 - H0; the first
                              threshold is then |F0|_1 / N (a cold start uses max |F0|) */
    int warm_fallback;     /* with warm_start: fall back to H0 = 0 when |F0|_1 > |B|_1 */
    int l2_window;         /* 1: keep the fluid vector L2-resident (access-policy window) */
    int timing;            /* 1: run the levels host-driven with a CUDA event around every
                              kernel and fill the per-kernel times of di_stats (slower) */
    int propagation;       /* how a level diffuses its frontier.  Levels of modes 0-2 drain
                              the whole frontier first, then send its fluid: 0 gather over
                              in-edges (binned rows) on dense levels, scatter on sparse
                              ones; 1 the same with a flat edge-parallel gather; 2 always
                              scatter.  3 (default): asynchronous push - each frontier node
                              is drained with an atomic exchange when its row is pushed, so
                              fluid arriving earlier in the level goes with it; 4: the same
                              asynchronous push with warp-level tiles (each warp drains 32
                              frontier nodes at a time; no block-wide barrier); 5: the
                              level in one launch - each CTA selects nodes in its chunks
                              of F and pushes them at once, with no frontier list;
                              6: the level in one launch over contiguous node chunks in node
                              order (the cyclic sweep of Sec. 2.4 at GPU width): targets
                              within a window around the chunk and targets of very high
                              in-degree are added in shared memory and flushed with
                              coalesced reductions, fluid sent to a later chunk is diffused
                              in the same level; rows are pushed edge-parallel per warp;
                              7: the levels of mode 3 in one persistent cooperative launch
                              per segment between exact residuals - selection and push
                              phases separated by bounded grid barriers (see spin_limit),
                              whose last CTA runs the control; the phases are timed on the
                              device (di_stats.level_seconds / select_seconds) */
    int push_ratio;        /* auto: a level is dense (gather) when its active edges times
                              push_ratio reach the edge count; default 8 */
    int exact_residual;    /* form of the exact FP64 residual B + P H - H: 1 gather over the
                              in-rows binned by length (no atomics, fixed summation order);
                              2 in-edges in source-blocked order (blocks of 2^22 sources,
                              so the gathered H stays in L2), runs of equal destination
                              summed over the warp and added with FP64 reds;
                              0 (default) = 2 */
    int selection;         /* frontier rule: 0 (default) |F_i| >= T; 1 the weighted score
                              |F_i| / ((#in_i + 1)(#out_i + 1)) >= T that Sec. 2.4 names as
                              the ideal diffusion order (T_0 and the empty-level rule then
                              use the largest score; the stop rule keeps |F|_1).
                              Needs propagation 3, 4 or 7 */
    int dangling;          /* columns of nodes without out-edges: 0 (default) zero, so
                              sum X < 1; 1 the uniform 1/N completion of Sec. 2.2
                              (p_kj = d/N for every k), which makes the columns of Q
                              stochastic.  The fluid a dangling node drains is spread
                              over all nodes as one uniform add in the next frontier
                              selection; the exact residual adds d/N sum_dangling H_j.
                              Needs propagation 3 to 7 and exact_residual 0 or 2
                              (di_solve_batched supports it as well) */
    double recompute_drop; /* FP32 fluid: exact FP64 residual whenever the running |F|_1
                              has fallen by this factor since the last exact value, so
                              that the FP32 rounding of the pushes stays a fraction of
                              about 2^-24 * recompute_drop of the residual; 0 = no drop
                              rule, else > 1; default 1024.  Either rule, and every stop
                              request, triggers an exact recomputation */
    long long spin_limit;  /* bound of a device wait, in microseconds: the grid barriers of
                              the persistent level loop (propagation 7) give up after it and
                              the solve returns DI_ETIMEOUT (no GPU fault; the context stays
                              usable); the push's wait for the frontier's tiles before its
                              slice sweeps (slice_sweeps) gives up after it and sweeps what
                              has landed (the result is unaffected).  No other kernel waits
                              on another CTA.  0 .. 2^40; default 2^20 (about 1 s) */
    void *stream;          /* cudaStream_t for all work; NULL = legacy default stream */
    int resweeps;          /* propagations 3-7: after a level's pass, select again at the
                              same T up to this many times (nodes whose fluid crossed T
                              while the level pushed - what the paper's sequential sweep
                              meets later in the same sweep) before T <- T / alpha; a pass
                              that selects nothing ends the level.  0 .. 8; default 0 */
    int slice_sweeps;      /* propagations 3 and 7: once the frontier's tiles are all
                              claimed, each CTA of the push sweeps its own slice of about
                              n / (push CTAs) consecutive nodes at the level's threshold
                              and diffuses every node with |F_i| >= T, up to this many
                              times - the nodes whose fluid crossed T while the level
                              pushed, which the sequential sweep of Sec. 2.4 diffuses in
                              the same sweep.  Unlike resweeps, no grid-wide pass: a node
                              that crosses T after its slice was swept keeps its fluid for
                              the next selection.  0 = off, 1 .. 4, or -1 (default): one
                              where it applies - propagation 3 or 7, selection 0, no
                              re-selection and no fluid window - and none elsewhere.  An
                              explicit count > 0 needs propagation 3 or 7 and selection 0,
                              and turns the fluid window of di_tune off for the solve */
} di_opts;

/* Statistics of one solve. */
typedef struct {
    int32_t levels;            /* threshold levels with a non-empty frontier */
    int32_t recomputes;        /* exact FP64 residual recomputations */
    int64_t node_diffusions;   /* nodes diffused (F_i moved into H_i) */
    int64_t edge_diffusions;   /* elementary node-to-node diffusions (Sec. 2.4 cost) */
    double resid_l1;           /* final |B + P H - H|_1, recomputed exactly in FP64 */
    double err_bound;          /* resid_l1 / (1 - d): bound on |X - H|_1 */
    double b_l1;               /* |B|_1 */
    double f0_l1;              /* |F0|_1 of the start actually used */
    double seconds;            /* device time of the solve (CUDA events) */
    int32_t warm_used;         /* 1 if the warm start was kept, 0 if plain/fallback */
    int32_t status;            /* the di_status the call returned */
    int64_t gpu_launches;      /* kernels this call launched */
    /* CUDA-event times, filled only when opts.timing = 1 */
    double level_seconds;      /* level kernels (frontier selection fused with the push);
                                  propagation 7: its selection and push phases, timed on the
                                  device in either loop mode */
    double recompute_seconds;  /* exact-residual kernels (timing mode launches them each level) */
    int32_t level_launches;    /* level kernels that did work (propagation 7: selection passes) */
    int32_t recompute_launches;/* exact residual recomputations */
    int32_t body_iterations;   /* iterations of the device-side level loop */
    int32_t slice_sweeps;      /* slice sweeps per level the push made (opts.slice_sweeps resolved) */
    double select_seconds;     /* timing mode, propagation 3/4 (propagation 7: always): the
                                  frontier-selection part of level_seconds */
    int64_t red_ops;           /* propagations 3, 6, 7: global L2 reduction sectors the push
                                  issued (a scattered red counts one, a coalesced flush of the
                                  shared-memory fluid window one per sector it touches); 0 for
                                  the other propagations */
    int64_t slice_nodes;       /* nodes diffused by the push's slice sweeps (opts.slice_sweeps) */
} di_stats;

/* Library version string. */
DI_API const char *di_version(void);

/* Message of the last failed call on this thread ("" if none). */
DI_API const char *di_last_error(void);

/* Defaults: alpha 1.5, FP32 fluid, recompute_every 0, recompute_drop 1024,
 * max_levels 100000, cold start (fallback on when warm), L2 window on,
 * timing off, propagation 3, push_ratio 8, exact_residual 0, selection 0,
 * dangling 0, spin_limit 2^20, stream NULL, resweeps 0, slice_sweeps -1 (auto).  Returns DI_EINVAL if
 * o is NULL. */
DI_API di_status di_opts_default(di_opts *o);

/*
 * Builds the device form of P's sparsity from a CSR of out-edges (Sec. 2.2):
 * row j of (row_ptr, col) lists the targets k of the edges j -> k, i.e. the
 * support of column j of P.  Duplicates count with their multiplicity and a
 * self-loop j -> j is the entry p_jj; a row with no entry is a dangling node
 * (zero column).  n >= 1 nodes, nnz >= 0 edges; row_ptr has n+1 entries
 * (row_ptr[0] = 0, non-decreasing, row_ptr[n] = nnz), col has nnz entries in
 * [0, n).  on_device = 0: row_ptr/col are host pointers; 1: device pointers.
 * The arrays are copied; the caller keeps ownership.  Validation failures
 * return DI_EINVAL (nothing allocated).  The library also derives the
 * transpose (in-edges) used by the exact residual and the node features.
 * stream: cudaStream_t or NULL.  *out receives the new graph.
 */
DI_API di_status di_graph_create(int64_t n, int64_t nnz, const int64_t *row_ptr,
                                 const int32_t *col, int on_device, void *stream,
                                 di_graph **out);

/* Frees a graph and all its device memory (NULL is a no-op). */
DI_API void di_graph_destroy(di_graph *g);

/* Shape of a graph; any output pointer may be NULL. */
DI_API di_status di_graph_info(const di_graph *g, int64_t *n, int64_t *nnz,
                               int64_t *n_dangling, int64_t *max_outdeg, int64_t *max_indeg,
                               int64_t *n_hot);

/*
 * Solves X = P X + B by D-iteration on one GPU until the exactly recomputed
 * residual satisfies |B + P H - H|_1 <= tol (the paper's stop rule
 * r/(1-d) <= Target_Error of Sec. 2.1 is tol = (1-d) Target_Error).
 *   B  device pointer, n doubles, finite (non-finite -> DI_ENONFINITE).
 *   d  damping factor in (0, 1) (P = d Q, Eq. 2).
 *   tol > 0, absolute L1 tolerance.
 *   H  device pointer, n doubles: in = H0 when opts->warm_start, out = H ~ X.
 *   F  device pointer, n doubles, or NULL: out = B + P H - H in FP64.
 *   opts NULL = defaults.  stats may be NULL.
 * Synchronous: returns after the solve completed on opts->stream.
 * Returns DI_OK, DI_ENOCONV (level cap; H and stats still valid),
 * DI_ENONFINITE, DI_EINVAL, DI_ENOMEM or DI_ECUDA.
 */
DI_API di_status di_solve(di_graph *g, const double *B, double d, double tol, double *H,
                          double *F, const di_opts *opts, di_stats *stats);

/*
 * di_solve with HOST buffers: copies B (and H0 when warm) to the device,
 * solves, and copies H (and F when non-NULL) back.  B, H, F are host
 * pointers of n doubles.  Uses library-owned device buffers.
 */
DI_API di_status di_solve_host(di_graph *g, const double *B, double d, double tol, double *H,
                               double *F, const di_opts *opts, di_stats *stats);

/*
 * Exact residual (the invariant F_n = B + P H_n - H_n that Eqs. defF/defH
 * imply): F = B + P H - H in FP64 for device vectors B, H (n doubles) into
 * the device vector F (n doubles); *r_l1 (host, may be NULL) receives
 * |F|_1.  Gathers over the in-edges in source-blocked order (form 2 of
 * di_opts.exact_residual); runs of equal destination are summed in
 * registers and over the warp, then added with FP64 reds, so the summation
 * order (not the set of terms) varies between runs.  Synchronous when
 * r_l1 != NULL.
 */
DI_API di_status di_residual(di_graph *g, const double *B, double d, const double *H,
                             double *F, double *r_l1, void *stream);

/*
 * Frontier selection of one threshold level (Sec. 2.4): writes to the
 * device array list (capacity n) the ids of all nodes with |F_i| >= T, in
 * no guaranteed order, and returns through host pointers the count, the
 * L1 norm sum |F_i| and max |F_i|.  F is a device vector of n floats
 * (fluid_fp64 = 0) or doubles (fluid_fp64 = 1).  The comparison is made in
 * the fluid's precision.  Synchronous.
 */
DI_API di_status di_frontier(di_graph *g, const void *F, int fluid_fp64, double T,
                             int32_t *list, int64_t *count, double *r_l1, double *max_abs,
                             void *stream);

/*
 * di_residual without any allocation (the paper has no counterpart: this is
 * a deployment facility).  For callers that must not call cudaMalloc on
 * their hot path - a serving loop whose device memory was reserved at
 * start-up, code running while another component owns the allocator, or a
 * process that cannot afford the implicit synchronisation of an allocation.
 * Same inputs and outputs as di_residual (B, H, F device pointers of n
 * doubles; r_l1 host pointer or NULL; synchronous when r_l1 != NULL); the
 * graph must have been created beforehand by di_graph_create.
 * Scratch memory is a fixed static device array inside libdi.so (8,430,080
 * bytes, held on every GPU that loads the library until exit), so the graph
 * may have at most 1,048,576 nodes and at most 4096 segments of 8192 in-edges
 * in its long in-rows; anything larger returns DI_EINVAL (use di_residual).
 * The first call on each device resolves the array's address for that
 * device: make it before any stream capture.  All calls share the one array:
 * calls that overlap on the GPU race and must be serialised by the caller.
 */
DI_API di_status di_residual_noalloc(const di_graph *g, const double *B, double d, const double *H,
                                     double *F, double *r_l1, void *stream);

/*
 * K-PID asynchronous D-iteration (Secs. 2.3-2.6) on one GPU: the nodes are
 * split into K contiguous ranges (kind 0: uniform, w_k = floor(k N / K);
 * kind 1: cost balanced, each range holding about L / K out-edges, Sec. 2.3).
 * The PID of range k keeps its own threshold T_k and diffuses its nodes to
 * their children inside the range only (Sec. 2.5, algorithm (*)); the fluid
 * owed to other ranges is P (H - H_old) restricted to external children and
 * is transmitted once its amount s_k exceeds r_k / K (Eq. send); a range that
 * receives fluid scales T_k by (r_k + received) / r_k, or sets T_k to the
 * received amount when it held no fluid (Sec. 2.6).  Every
 * round, all PIDs make one threshold level in the same launches; the stop is
 * decided on the exact FP64 residual, which includes the fluid still owed.
 * B, H (out), F (out, may be NULL) are device vectors of n doubles as in
 * di_solve.  Supports FP32 fluid, a cold start and the plain selection;
 * opts->alpha, max_levels, recompute_drop, dangling, timing and stream apply
 * (NULL opts = defaults).  dangling = 1 completes the columns of nodes
 * without out-edges by 1/N (Sec. 2.2): such a column has n_k rows in its own
 * range, diffused locally as a uniform add to the range's nodes at their next
 * selection, and N - n_k rows outside, owed and transmitted like external
 * edges (pid_ops counts both); the exact residual then uses the completed P.  timing = 1 runs the rounds
 * host-driven, one synchronisation per round, with CUDA events that fill
 * stats->select_seconds (k_pscan), level_seconds (selection, push and
 * transmission) and recompute_seconds (the IF body's kernels).  pid_ops / pid_sends (host, K entries, may be
 * NULL) receive each PID's elementary diffusions (local children plus
 * transmitted external edges) and its number of transmissions.  1 <= K <= 64.
 * Synchronous; the rounds run on the device in one CUDA graph (WHILE node),
 * which is kept on the graph object (with the ranges of the last K and kind,
 * the per-node range table and H_old) and reused by later calls; it is freed
 * with the graph.
 */
DI_API di_status di_solve_partitioned(di_graph *g, const double *B, double d, double tol, double *H,
                                      double *F, const di_opts *opts, int32_t K, int32_t kind,
                                      int64_t *pid_ops, int64_t *pid_sends, di_stats *stats);

/*
 * Batched solves (many right-hand sides of many graphs in one level loop).
 * Work item t is right-hand side r of graph g, numbered graph-major: the
 * items of graphs[0] first (r = 0 .. nrhs[0]-1), then those of graphs[1] ...
 * Every item is an independent D-iteration (Eqs. defF/defH) with its own
 * threshold schedule (Sec. 2.4) and its own stop rule.  di_batch_create lays
 * the items side by side in one device-resident union graph (one copy of
 * graph g per right-hand side, each starting on a multiple of 2048 nodes), so
 * all items advance together in the same kernel launches.  The graphs must
 * live on the current device; they are copied (the batch does not reference
 * them afterwards).  The union must stay below 2^31 nodes and 2^31 edges.
 * stream: cudaStream_t or NULL.  Synchronous.
 */
typedef struct di_batch di_batch;

DI_API di_status di_batch_create(const di_graph *const *graphs, int ng, const int *nrhs, void *stream,
                                 di_batch **out);

/* Frees a batch and all its device memory (NULL is a no-op). */
DI_API void di_batch_destroy(di_batch *b);

/* Items, union nodes (chunk-aligned) and union edges; outputs may be NULL. */
DI_API di_status di_batch_info(const di_batch *b, int *n_items, int64_t *n_union, int64_t *nnz_union);

/*
 * Solves every item of the batch: B[t], H[t] are device pointers of n_g
 * doubles (host array of n_items pointers); tol[t] > 0 is item t's absolute
 * L1 tolerance on |B + P H - H|_1 (host array).  d in (0, 1).  opts as for
 * di_solve (warm_start must be 0; timing = 1 runs the levels host-driven;
 * dangling = 1 completes the dangling columns of each item's graph by 1/n_g,
 * n_g the nodes of that graph; slice_sweeps: 0 .. 4 sweeps of each push
 * CTA's slice of the union at each item's selection threshold after the
 * frontier, as in di_solve, on the items whose frontier holds at least 1/32
 * of their nodes; -1 (default) none: with mostly sparse frontiers the
 * per-level wait costs more than it saves; spin_limit bounds the push's wait
 * for the frontier before a sweep).
 * item_stats (host array of n_items, may be NULL) receives each item's
 * statistics; total (may be NULL) the sums (levels = max over items,
 * gpu_launches and seconds of the whole call).  Returns DI_OK when every
 * item converged, DI_ENOCONV when at least one reached the level cap (its H
 * and statistics are still valid), DI_ENONFINITE, DI_EINVAL, DI_ENOMEM or
 * DI_ECUDA.  Synchronous on opts->stream.
 */
DI_API di_status di_solve_batched(di_batch *b, const double *const *B, double d, const double *tol,
                                  double *const *H, const di_opts *opts, di_stats *item_stats,
                                  di_stats *total);

/*
 * Learned warm start.  The paper starts from H_0 = 0 (F_0 = B); any H_0 is
 * as valid (F_0 = B + P H_0 - H_0 keeps the invariant of Eqs. defF/defH and
 * the bound |X - H|_1 <= |F|_1 / (1 - d)), so a good guess of X can shorten
 * the solve.  A small network predicts y_i = log(N x_i) from per-node
 * features and H0_i = exp(y_i) / N is handed to di_solve with
 * opts.warm_start = 1 (and warm_fallback = 1: H0 is dropped when
 * |F0|_1 > |B|_1).
 *
 * Features (DI_MODEL_NFEAT per node, float, row-major [n][9]): for node i
 * with in-degree m_i, out-degree o_i (edges with multiplicity), ld = log(1+m)
 * and s = 1/o (0 if dangling):
 *   x0 = ld_i, x1 = log(1 + o_i), x2/x3 = mean/max of ld_j over the in-edges
 *   j -> i, x4/x5 = mean of x2_j / max of x3_j over the in-edges,
 *   x6 = log(1 + sum s_j), x7 = log(1 + sum s_j a1_j) (a1_j = sum over j's
 *   in-edges of s), x8 = N B_i; empty means, maxima and sums are 0.
 *   Logarithms and 1/o are evaluated in FP32; sums over in-edges are
 *   accumulated in FP64 and rounded once to FP32.
 * Network: standardise (x - mu) / sd, then 9 -> 64 -> 64 -> 1 with ReLU
 * (BF16 tensor-core operands, FP32 accumulation), y = w3 . h2 + b3.
 * Parameters (DI_MODEL_NPARAM floats): W1 [64][16] (input columns 9..15 are
 * zero padding), b1 [64], W2 [64][64], b2 [64], w3 [64], b3 [1].  The model
 * "state" is mu [9], sd [9], then the parameters (DI_MODEL_STATE floats).
 */
#define DI_MODEL_NFEAT 9
#define DI_MODEL_NPARAM 5313
#define DI_MODEL_STATE (2 * DI_MODEL_NFEAT + DI_MODEL_NPARAM)

typedef struct di_model di_model;

typedef struct {
    int epochs;        /* passes over the training nodes (default 4) */
    int batch;         /* nodes per Adam step, drawn with replacement (default 65536) */
    double lr, beta1, beta2, eps;   /* Adam (defaults 1e-3, 0.9, 0.999, 1e-8) */
    uint64_t seed;     /* minibatch sampling (default 1) */
    void *stream;      /* cudaStream_t or NULL */
} di_train_opts;

DI_API di_status di_train_opts_default(di_train_opts *o);

/* New model on the current device: uniform He initialisation from seed
 * (SplitMix64), zero biases, identity standardisation (mu 0, sd 1). */
DI_API di_status di_model_create(uint64_t seed, di_model **out);

/* Frees a model (NULL is a no-op). */
DI_API void di_model_destroy(di_model *m);

/* Copies the model state (host array of DI_MODEL_STATE floats) out / in.
 * di_model_set rejects sd <= 0 or a non-finite mu with DI_EINVAL. */
DI_API di_status di_model_get(const di_model *m, float *state);
DI_API di_status di_model_set(di_model *m, const float *state);

/* Features of every node of g (device B of n doubles) into the device array
 * feat ([n][9] floats).  Asynchronous on stream. */
DI_API di_status di_features(di_model *m, di_graph *g, const double *B, float *feat, void *stream);

/* Network prediction y (device, n floats) for n feature rows (device
 * [n][9]).  Asynchronous on stream. */
DI_API di_status di_mlp_forward(const di_model *m, const float *feat, int64_t n, float *y, void *stream);

/* Mean squared error (1/n) sum (y_i - target_i)^2 over the n rows (device
 * feat [n][9], device target [n]) and its gradient with respect to the
 * parameters (host, DI_MODEL_NPARAM floats).  Synchronous. */
DI_API di_status di_mlp_grad(di_model *m, const float *feat, const float *target, int64_t n, float *grad,
                             double *loss, void *stream);

/* One Adam step with the gradient grad (host, DI_MODEL_NPARAM floats),
 * bias-corrected with the model's step count.  Synchronous. */
DI_API di_status di_model_adam(di_model *m, const float *grad, const di_train_opts *opts);

/* Trains m on ng graphs with right-hand sides B[g] and converged solutions
 * X[g] (device pointers of n_g doubles, e.g. H from di_solve): features,
 * target log(N x_i), standardisation statistics of the training features
 * (set into the model), then epochs of Adam steps on minibatches drawn over
 * all training nodes.  *final_loss (may be NULL) receives the mean squared
 * error over the last epoch.  Synchronous. */
DI_API di_status di_warmstart_train(di_model *m, di_graph *const *graphs, int ng, const double *const *B,
                                    const double *const *X, const di_train_opts *opts, double *final_loss);

/* H0 = exp(y) / N for every node of g (device H0, n doubles) from the
 * features of g and B (device); the exponential is taken in FP32 (any H0 is
 * a valid start, and F0 is formed from it exactly).  Asynchronous on stream. */
DI_API di_status di_warmstart_infer(di_model *m, di_graph *g, const double *B, double *H0, void *stream);

/* Model file: header, step, state, Adam moments (little-endian floats). */
DI_API di_status di_warmstart_save(const di_model *m, const char *path);
DI_API di_status di_warmstart_load(const char *path, di_model **out);

/*
 * Ceiling of the scattered memory operations of the push and the exact
 * residual.  A threshold level (Sec. 2.4) adds p_ki F_i into the fluid of
 * every child k (Eq. defF): one red.global.add per elementary diffusion at an
 * irregular target of the fluid vector, which the library keeps in L2; the
 * exact residual gathers one word per in-edge.  Their ceiling is the rate at
 * which the GPU processes such single-word operations, not the HBM copy
 * bandwidth.  This call measures it: ops operations by every thread of a
 * full-occupancy grid over a zeroed device array of `slots` words (a power of
 * two in [2^10, 2^30]; 2^24 floats is the fluid of a 2^24-node graph), after
 * one warm-up launch; *ops_per_s (host) receives the best rate of three
 * launches and *seconds (host, may be NULL) that launch's time.
 *   mode 0: red.global.add.f32 at pseudo-random slots with the L2 evict-last
 *           hint of the push;  1: the same in FP64;  2: 4-byte loads at
 *           pseudo-random slots (gathers);  3: red.global.add.f32 at
 *           consecutive slots per warp (coalesced, for contrast);
 *           4: atom.global.add.f32 at pseudo-random slots (fetch-and-add,
 *           the old value returned to the thread).
 * The array is allocated and freed by the call (this is a measurement, not a
 * solver step).  Synchronous on stream.  DI_EINVAL on a bad mode, size or
 * count; DI_ENOMEM / DI_ECUDA on CUDA failures.
 */
DI_API di_status di_probe_l2(int mode, int64_t slots, int64_t ops, double *ops_per_s, double *seconds,
                             void *stream);

/*
 * Autotuning of the push shape.  The paper's cost model counts elementary
 * diffusions only (Sec. 2.4); on a GPU the time per diffusion also depends
 * on how frontier rows are spread over threads, warps and CTAs, which
 * depends on the graph's degree mix.  di_autotune / di_batch_autotune time
 * complete solves of the caller's problem (plain D-iteration, the same
 * options) for candidate shapes - thread_max_deg in {4, 8, 16, 32}, with the
 * occupancy-maximum push grid and with half of it, and (di_autotune with
 * propagation 3 or 7) the default shape with the fluid window - keep the fastest, store
 * it in the graph or batch (used by every later solve) and return it.
 * cache_path (may be NULL) names a text file of JSON lines keyed by the
 * problem's size bucket (log2 of nodes and edges, items, fluid precision,
 * propagation): a hit is used without timing, a miss appends the result.
 * *best_seconds (may be NULL) receives the winner's time (0 on a cache hit).
 * The solves write the caller's H buffers (graph: a scratch buffer of the
 * library).  Synchronous.
 */
DI_API di_status di_tune_default(di_tune *t);
DI_API di_status di_graph_set_tune(di_graph *g, const di_tune *t);
DI_API di_status di_graph_get_tune(const di_graph *g, di_tune *t);
DI_API di_status di_batch_set_tune(di_batch *b, const di_tune *t);
DI_API di_status di_batch_get_tune(const di_batch *b, di_tune *t);
DI_API di_status di_autotune(di_graph *g, const double *B, double d, double tol, const di_opts *opts,
                             const char *cache_path, di_tune *best, double *best_seconds);
DI_API di_status di_batch_autotune(di_batch *b, const double *const *B, double d, const double *tol,
                                   double *const *H, const di_opts *opts, const char *cache_path,
                                   di_tune *best, double *best_seconds);

#ifdef __cplusplus
}
#endif

#endif /* DI_H */
