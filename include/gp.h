/*
 * gp.h -- C ABI of libgp, the push/pull graph-sweep library for NVIDIA GB300 (sm_103a).
 *
 * The library runs the per-iteration vertex-centric edge sweep studied in
 * "To Push or To Pull: On Reducing Communication and Synchronization in Graph
 * Computations" (Besta, Podstawski, Groner, Solomonik, Hoefler; HPDC 2017) in
 * its two forms (Section 3, "Push-Pull: Applicability"; Section 3.8):
 *   push -- the thread that owns vertex v writes state of other vertices: v
 *           scatters along its out-edges into shared state with atomics;
 *   pull -- only the owner of v writes v: v gathers along its in-edges into
 *           its own state, with no atomics;
 * applied to PageRank power iteration (Section 3.1; Algorithm 1) and to BFS
 * frontier expansion (Section 3.3; Algorithm 3): top-down = push, bottom-up =
 * pull, and a per-level switch between the two (Generic-Switch, Section 5).
 *
 * Conventions shared by every entry point
 *  - Status: every function returns GP_OK (0) or a negative gp_status.  No
 *    entry point aborts, prints or exits.  gp_status_string() names a status;
 *    gp_last_error() returns a message for the last failure on the calling
 *    host thread.
 *  - Memory kinds: "device" = CUDA device (or managed) memory of the current
 *    device; "host" = ordinary or pinned host memory; "any" = either (the
 *    library detects the kind and copies host data through its own device
 *    buffers, synchronising the stream before returning).
 *  - Streams: `stream` is a cudaStream_t passed as void* (NULL = the legacy
 *    default stream).  All device work of a call is enqueued on it.  A call
 *    returns once its work is enqueued, except that gp_pagerank reads its
 *    convergence flag back every few sweeps, gp_bfs reads its frontier
 *    counters back once per level, and any "any" output in host memory or a
 *    non-NULL stats pointer makes the call synchronise the stream.
 *  - Ownership: the caller owns every pointer it passes.  The library never
 *    frees caller memory.  Arrays handed to gp_graph_upload without
 *    GP_UPLOAD_COPY are read in place and must stay alive and unchanged until
 *    gp_graph_free.  Library-owned device memory (degree arrays, vertex bins,
 *    queues, bitmaps, partial sums) is obtained from the allocator registered
 *    with gp_set_allocator (default: stream-ordered allocation from a memory
 *    pool of the library's own per device, which keeps freed memory for reuse
 *    rather than returning it to the driver; cudaMallocAsync where the device
 *    has no pool support).
 *  - Graph layout (Section 2.2): neighbours of each vertex form one contiguous
 *    array; n+1 offsets (int64) mark where each vertex's list begins.  CSR
 *    lists out-neighbours (row u = heads of u->v; what push walks), CSC lists
 *    in-neighbours (column v = tails of u->v; what pull walks), Section 4.8
 *    ("Directed Graphs").  Indices are int32 (n < 2^31), offsets int64.
 *  - Threads: one graph handle may be used by one host thread at a time.
 */
#ifndef GP_H
#define GP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define GP_VERSION 1

/* Sweep form.  For PageRank: PUSH = scatter with FP32 atomics, PULL = gather
 * with no atomics, AUTO = the library picks one per graph (the result is the
 * same up to FP32 rounding).  For BFS: PUSH = top-down, PULL = bottom-up,
 * AUTO = switch per level. */
typedef enum gp_mode { GP_PUSH = 0, GP_PULL = 1, GP_AUTO = 2 } gp_mode;

typedef enum gp_status {
    GP_OK = 0,
    GP_ERR_INVALID = -1,       /* bad argument or malformed graph */
    GP_ERR_OOM = -2,           /* the allocator returned NULL */
    GP_ERR_CUDA = -3,          /* a CUDA runtime call failed (message in gp_last_error) */
    GP_ERR_NOT_CONVERGED = -4, /* sweep cap reached before tol; the last iterate is written */
    GP_ERR_TIMEOUT = -5,       /* a bounded device wait ran out */
    GP_ERR_UNSUPPORTED = -6    /* feature not available for this input */
} gp_status;

typedef struct gp_graph gp_graph; /* opaque handle */

/* ------------------------------------------------------------------ errors */

/* Static text for a status code (never NULL). */
const char *gp_status_string(int status);

/* Thread-local message describing the last failure on this host thread ("" if none). */
const char *gp_last_error(void);

/* GP_VERSION of the library actually loaded. */
int gp_version(void);

/* ------------------------------------------------------------------ memory */

/* Allocation callbacks for library-owned device memory.  alloc returns a device
 * pointer of at least `bytes` bytes aligned to 256 bytes, usable in stream
 * order on `stream`, or NULL on failure (the call then fails with GP_ERR_OOM).
 * free releases it in stream order.  Passing NULL for both restores the
 * default (the library's own pool, stream-ordered, freed memory kept for
 * reuse until gp_pool_trim).  Applies to later allocations
 * only; memory is always released with the callbacks that allocated it. */
typedef void *(*gp_alloc_fn)(size_t bytes, void *stream, void *ctx);
typedef void (*gp_free_fn)(void *ptr, size_t bytes, void *stream, void *ctx);
int gp_set_allocator(gp_alloc_fn alloc, gp_free_fn free_fn, void *ctx);

/* The library's default pool (one per device, created on first use) keeps the
 * memory that gp_graph_free and the entry points' temporary buffers give back,
 * so the next upload of a graph of the same size maps nothing new; that memory
 * stays held by the library, unusable by other allocators in the process
 * (PyTorch's included), until it is trimmed.  gp_pool_usage reports, for the
 * current device, the bytes the pool holds from the driver (reserved) and the
 * bytes handed out and not yet freed (used); both are 0 before first use.
 * gp_pool_trim synchronises the current device, then returns held memory to
 * the driver until at most keep_bytes stay reserved (memory in use is never
 * released).  Neither touches memory of a registered allocator (gp_set_allocator).
 * The small page-locked host blocks a graph uses for the kernels' status words
 * are kept in the same way when the graph is freed (page-locking is a driver
 * call that can take milliseconds) and reused by later graphs; gp_pool_trim
 * also frees the kept ones. */
int gp_pool_usage(int64_t *reserved_bytes, int64_t *used_bytes);
int gp_pool_trim(int64_t keep_bytes);

/* ------------------------------------------------------------------ graph */

#define GP_UPLOAD_VALIDATE 0x1u  /* check offsets (monotone, 0..m), indices (< n), and that
                                    CSR and CSC hold the same edge multiset; GP_ERR_INVALID
                                    with a message on failure (synchronises the stream) */
#define GP_UPLOAD_SYMMETRIC 0x2u /* the graph is symmetric: the CSC arguments may be NULL and
                                    the CSR arrays serve both directions */
#define GP_UPLOAD_COPY 0x4u      /* copy all arrays into library-owned device memory; the
                                    sources may be "any" memory and need not outlive the call */
#define GP_UPLOAD_NORMALIZE 0x8u /* weighted graphs: P_vu = w_uv / sum_v' w_uv' (else P_vu = w_uv) */

/*
 * Upload a graph and prepare its degree data (the paper's Section 2.2 layout;
 * Section 7.3 notes that pulling must also fetch the neighbours' degrees, so
 * 1/deg_out is precomputed here once).
 *   n, m          vertices and stored directed edges; 0 <= n < 2^31, m >= 0.
 *   csr_off       int64[n+1] "any"/device: out-edge offsets, csr_off[0] = 0, csr_off[n] = m.
 *   csr_idx       int32[m]: heads of the out-edges of each vertex.
 *   csr_w         float[m] or NULL: weight of each CSR edge (P_vu for u->v, see NORMALIZE).
 *   csc_off/idx/w the same edges grouped by head (in-edges); may be NULL with
 *                 GP_UPLOAD_SYMMETRIC.  csc_w must be given iff csr_w is.
 *   flags         GP_UPLOAD_* bits.
 * Without GP_UPLOAD_COPY all arrays must be device memory.  Unweighted:
 * P_vu = 1/deg_out(u).  Vertices with deg_out = 0 contribute nothing.
 * On success *out holds a new handle; on failure *out is NULL.
 */
int gp_graph_upload(gp_graph **out, int64_t n, int64_t m, const int64_t *csr_off, const int32_t *csr_idx,
                    const float *csr_w, const int64_t *csc_off, const int32_t *csc_idx, const float *csc_w,
                    unsigned flags, void *stream);

/* Release a handle and all library-owned memory (in order on the stream it was
 * uploaded with).  NULL is accepted. */
int gp_graph_free(gp_graph *g);

typedef struct gp_graph_info {
    int64_t n, m;
    int64_t max_out_degree, max_in_degree;
    int64_t pull_big_vertices; /* vertices with in-degree above pull_light_max (warp chunks) */
    int64_t pull_big_chunks;
    int64_t push_big_vertices; /* vertices with out-degree above push_light_max */
    int64_t push_big_chunks;
    int64_t isolated; /* vertices with no in- and no out-edges */
    int32_t symmetric, weighted;
    int64_t device_bytes; /* library-owned device memory held by the handle */
} gp_graph_info;

int gp_graph_info_get(const gp_graph *g, gp_graph_info *info);

/* ------------------------------------------------------------------ options */

/* Tunables (the autotuner writes these).  Correctness never depends on them. */
typedef struct gp_options {
    int32_t pull_light_max;   /* in-degree <= this: 32 vertices per warp, merged edge stream */
    int32_t push_light_max;   /* out-degree <= this: same for the push scatter and top-down BFS */
    int32_t chunk_edges;      /* edges per warp chunk for vertices above the light limits */
    int32_t blocks_per_sm;    /* resident blocks per SM for the grid-stride sweep kernels */
    int32_t poll_interval;    /* PageRank sweeps enqueued between convergence read-backs (at
                                 most two batches in flight; once two read-backs give the
                                 residual's rate of decrease, sweeps are enqueued only up to the
                                 predicted stopping sweep plus one, then a batch at a time if
                                 the iteration runs longer; the sweeps performed do not depend
                                 on it) */
    int32_t pr_auto_mode;     /* what GP_AUTO means for PageRank: GP_PUSH, GP_PULL, or -1 = rule */
    float bfs_alpha;          /* top-down -> bottom-up when m_f > m_u / alpha */
    float bfs_beta;           /* bottom-up -> top-down when n_f < n / beta (frontier shrinking) */
    int32_t push_fp64_accum;  /* push PageRank: 1 = accumulate the scattered updates with FP64
                                 atomics (ranks stay FP32), 0 = FP32 atomics, -1 = by size
                                 (default): FP64 unless its 8n-byte accumulator exceeds half
                                 the L2 cache and no vertex takes more than 4096 updates per
                                 sweep (then FP32, whose array stays in L2) */
    int32_t pull_hot_slots;   /* pull PageRank: contributions of this many highest out-degree
                                 vertices are served from shared memory (0 = off, <= 49152) */
    int32_t push_hot_slots;   /* push PageRank: updates to this many highest in-degree vertices are
                                 summed in shared memory per block, then flushed with one atomic
                                 per vertex and block (0 = off, <= 49152) */
    float sssp_alpha;         /* SSSP GP_AUTO: an iteration pulls when the active vertices'
                                 out-edges times sssp_alpha exceed the unsettled in-edges */
    float fe_alpha;           /* Frontier-Exploit PageRank GP_AUTO: an iteration pulls when the
                                 frontier's out-edges times fe_alpha exceed m */
    float bc_alpha;           /* betweenness centrality GP_AUTO: a step pulls when the push side's
                                 edges times bc_alpha exceed the pull side's */
    int32_t bfs_light_max;    /* BFS top-down levels (gp_bfs, gp_bfs_multi): frontier vertices with
                                 more out-edges than this are expanded as chunk_edges-sized chunks
                                 by whole warps, the others in 32-vertex tiles (default 32; its own
                                 setting, since the push sweep's best push_light_max can be far
                                 from the traversal's) */
    int32_t bfs_groups;       /* gp_bfs_multi called with groups 0: this many groups of blocks
                                 (0 = the library's choice, 16; at most 32).  Changing it frees
                                 the multi-search workspace, which the next call sizes anew */
} gp_options;

/* Fill *opt with the built-in defaults. */
int gp_options_default(gp_options *opt);

/* Replace the handle's options (rebuilds its vertex bins if the degree limits
 * or chunk size change; enqueued on `stream`). */
int gp_graph_set_options(gp_graph *g, const gp_options *opt, void *stream);

int gp_graph_get_options(const gp_graph *g, gp_options *opt);

/* ------------------------------------------------------------------ autotuning */

#define GP_TUNE_PULL 0x1u /* pull_light_max, chunk_edges, pull_hot_slots */
#define GP_TUNE_PUSH 0x2u /* push_light_max, blocks_per_sm, push_hot_slots */
#define GP_TUNE_AUTO 0x4u /* pr_auto_mode: the faster of pull and push for this graph */
#define GP_TUNE_BFS 0x8u  /* bfs_light_max, bfs_alpha, bfs_beta, then bfs_groups */
#define GP_TUNE_ALL 0xFu

typedef struct gp_tune_result {
    gp_options best;         /* the options left set on the graph */
    float pull_ms_per_sweep; /* best measured, 0 if not tuned */
    float push_ms_per_sweep;
    float bfs_ms;            /* all given sources, direction-switching */
    int32_t evaluated;       /* candidates timed */
} gp_tune_result;

/*
 * Pick options for this graph by timing candidates on the device (coordinate
 * descent over small sets, CUDA events on `stream`; a few PageRank sweeps or
 * the given BFS sources per candidate).  Results never depend on the options,
 * only speed does.  sources (host int32[nsources]) are needed for GP_TUNE_BFS.
 * Leaves the best options set on the graph.  Synchronises the stream.
 */
int gp_autotune(gp_graph *g, unsigned what, const int32_t *sources, int nsources, gp_tune_result *res, void *stream);

/* ------------------------------------------------------------------ PageRank */

typedef struct gp_pr_stats {
    int32_t iters_done; /* sweeps performed */
    int32_t mode_used;  /* GP_PUSH or GP_PULL */
    double residual;    /* L1 norm (FP64) of the change made by the last sweep */
    float ms;           /* device time of the call by CUDA events (0 when stats is NULL) */
    int32_t converged;  /* 1 if residual < tol (or tol == 0 and all sweeps ran) */
    /* Push sweeps' scattered updates, summed over the sweeps performed (all 0
     * for pull, which issues no atomics; Table 1's atomics row).  Every edge
     * update of a push sweep is exactly one of: an atomic sent to L2
     * (push_updates_l2), an atomic into a block's shared-memory accumulator of a
     * hot vertex (push_updates_shared), or folded into another lane's update for
     * the same vertex inside a warp (push_updates_merged); the three sum to
     * m * iters_done.  push_flush_l2 counts the L2 atomics that flush the
     * shared accumulators (one per touched hot vertex per block and sweep). */
    int64_t push_updates_l2, push_updates_shared, push_updates_merged, push_flush_l2;
} gp_pr_stats;

/*
 * PageRank power iteration (Section 3.1 formula; Algorithm 1, push- and
 * pull-based PageRank; damping d is the paper's f):
 *     y[v] = (1-d) s[v] + d * sum_{(u->v) in E} P_vu x[u]
 * Jacobi sweeps from x0; after each sweep the L1 norm of y - x is reduced in
 * FP64; iteration stops at the first sweep where it is below tol, or after
 * `iters` sweeps (then GP_ERR_NOT_CONVERGED, with the last iterate written).
 * tol = 0 runs exactly `iters` sweeps and returns GP_OK.
 *   mode            GP_PUSH (scatter with atomics: FP64 reductions in L2, or FP32
 *                   atomicAdd, as push_fp64_accum says), GP_PULL (gather, no
 *                   atomics) or GP_AUTO.
 *   damping         in (0, 1).
 *   iters           >= 1.
 *   personalization float[n] "any" or NULL (uniform 1/n): the teleport vector s.
 *   x0              float[n] "any" or NULL (1/n): starting vector.
 *   ranks_out       float[n] "any": the final iterate.
 *   stats           optional.
 * Ranks are FP32; sums are FP32 (tree order within a warp, so pull is
 * deterministic for fixed options; push is not, its atomics commute).
 */
int gp_pagerank(const gp_graph *g, int mode, float damping, int iters, double tol, const float *personalization,
                const float *x0, float *ranks_out, gp_pr_stats *stats, void *stream);

/*
 * Gradient of a loss on the PageRank fixed point (not in the paper: implicit
 * differentiation of x = (1-d) s + d P x, so no iterate is stored).  For
 * L with dL/dx = grad_ranks, the adjoint lambda solves
 *     (I - d P^T) lambda = grad_ranks
 * by the transposed sweep -- the pull sweep run over out-edges (CSR) for
 * GP_PULL, the push sweep run over in-edges (CSC) for GP_PUSH -- with the same
 * on-device convergence test as gp_pagerank (L1 change of lambda < tol, or
 * `iters` sweeps).  Then
 *     grad_personalization[v] = (1-d) lambda_v
 *     grad_weights[e]          = d lambda_v x_u            for CSR edge e = (u -> v)
 * i.e. dL/dP_vu for the stored transition entries (unweighted graphs: the
 * entries 1/deg_out(u); weighted: the weights as given).  For a graph uploaded
 * with GP_UPLOAD_NORMALIZE (P_vu = w_uv / S_u) grad_weights is the gradient
 * with respect to the raw weights: (x_u / S_u)(d lambda_v - lambda_u + g_u).
 *   ranks                 float[n] "any": the fixed point x the gradient is taken at.
 *   grad_ranks            float[n] "any": dL/dx.
 *   grad_weights          float[m] "any" or NULL, CSR edge order.
 *   grad_personalization  float[n] "any" or NULL.
 * Returns GP_ERR_NOT_CONVERGED (gradients still written) when tol > 0 is not met.
 */
int gp_pagerank_backward(const gp_graph *g, int mode, float damping, const float *ranks, const float *grad_ranks,
                         float *grad_weights, float *grad_personalization, int iters, double tol, gp_pr_stats *stats,
                         void *stream);

/* Replace the edge weights of a weighted graph (device arrays, caller-owned,
 * kept alive until the next call or gp_graph_free; csc_w may be NULL for a
 * symmetric graph whose CSC shares the CSR arrays).  The per-source normaliser
 * of a GP_UPLOAD_NORMALIZE graph is recomputed on `stream`.  Used by training
 * loops that update weights between forward passes. */
int gp_graph_set_weights(gp_graph *g, const float *csr_w, const float *csc_w, void *stream);

/* ------------------------------------------------------------------ BFS */

/* Per-level statistics are kept for the first GP_BFS_MAX_LEVELS levels; a
 * deeper search runs to the end all the same (levels, reached and the edge
 * counts cover every level). */
#define GP_BFS_MAX_LEVELS 512

typedef struct gp_bfs_stats {
    int32_t levels;         /* levels explored (depth + 1) */
    int32_t switches;       /* direction changes */
    int64_t reached;        /* vertices with level >= 0 */
    int64_t edges_examined; /* out-edges scanned top-down + in-edges scanned bottom-up */
    int64_t edges_reached;  /* sum of out-degrees of the reached vertices */
    float ms;               /* device time of the call by CUDA events */
    int8_t direction[GP_BFS_MAX_LEVELS]; /* GP_PUSH (top-down) / GP_PULL (bottom-up) per level */
    int64_t frontier[GP_BFS_MAX_LEVELS]; /* frontier size entering each level */
    int64_t examined[GP_BFS_MAX_LEVELS]; /* edges scanned by each level */
    int32_t init_ns;                     /* device time from kernel start to the first level (global timer) */
    int32_t level_ns[GP_BFS_MAX_LEVELS]; /* device time of each level, its frontier conversion and barrier included */
} gp_bfs_stats;

/*
 * Breadth-first search from `src` over out-edges (Section 3.3; Algorithm 3
 * with every ready counter = 1, so each vertex takes the level of the frontier
 * that first reaches it, plus one).
 *   mode        GP_PUSH: top-down every level -- frontier vertices scan their
 *               out-edges and claim unvisited heads with atomicCAS (Section 4.3,
 *               "Atomics/Locks": O(m) CAS);
 *               GP_PULL: bottom-up every level -- every unvisited vertex scans
 *               its in-edges for a frontier vertex and stops at the first one
 *               (owner-only writes, no atomics on vertex state);
 *               GP_AUTO: per-level switch (top-down -> bottom-up when the
 *               frontier's out-edges m_f exceed m_u/alpha, m_u = in-edges of
 *               unvisited vertices; back when the frontier shrinks below n/beta).
 *   level_out   int32[n] "any": BFS level, -1 if unreached.
 *   parent_out  int32[n] "any" or NULL: a BFS parent (parent[src] = src, -1 if
 *               unreached).  Levels are unique; parents are valid but may
 *               differ between runs (any frontier in-neighbour is correct).
 *   stats       NULL or filled on return (the call then waits for the search).
 * Synchronisation: with stats == NULL and both outputs in device memory the
 * call only enqueues the search on `stream` and returns; a grid-barrier
 * timeout of that search (GP_ERR_TIMEOUT, outputs incomplete) is then returned
 * by the next gp_bfs / gp_bfs_directed call on the same graph.  Otherwise the
 * call waits and reports the timeout itself.  Searches on one graph share its
 * workspace: issue them on one stream (or order the streams).
 */
int gp_bfs(const gp_graph *g, int32_t src, int mode, int32_t *level_out, int32_t *parent_out, gp_bfs_stats *stats,
           void *stream);

/* Per-search figures of gp_bfs_multi (the totals of gp_bfs_stats). */
typedef struct gp_bfs_summary {
    int32_t levels;         /* levels explored (depth + 1) */
    int32_t switches;       /* direction changes */
    int64_t reached;        /* vertices with level >= 0 */
    int64_t edges_examined; /* out-edges scanned top-down + in-edges scanned bottom-up */
    int64_t edges_reached;  /* sum of out-degrees of the reached vertices */
} gp_bfs_summary;

/*
 * Several independent searches (the same per-source search as gp_bfs: Section
 * 3.3, Algorithm 3, with gp_bfs's modes and direction rule) in one cooperative
 * launch.  The GPU's resident blocks are cut into `groups` equal groups, each
 * with its own frontier workspace and grid barrier; a group that finishes a
 * search takes the next one not yet started (the order in which searches run
 * is not fixed, their results are).  A search's levels cost a
 * fixed barrier and counter round trip each whatever the frontier's size, so
 * groups that never wait on one another overlap those costs.
 *   sources     host int32[nsources], each in [0, n) (repeats allowed).
 *   level_out   host array of nsources DEVICE pointers, each int32[n]: the
 *               levels of search i (as gp_bfs's level_out).
 *   parent_out  NULL, or a host array of nsources device pointers (int32[n]
 *               each): a BFS parent per vertex (as gp_bfs's parent_out).
 *   groups      0: the graph's bfs_groups option (gp_autotune's GP_TUNE_BFS
 *               sets it), or 16 when that is 0; the count is clamped to
 *               [1, min(nsources, resident blocks, 32)].
 *   summary     NULL, or host gp_bfs_summary[nsources] filled on return (the
 *               call then waits for the searches).
 * Returns GP_ERR_INVALID (nothing launched) for a source outside [0, n) or an
 * output pointer that is not device memory.  With summary == NULL the call only
 * enqueues the launch on `stream`; a grid-barrier timeout (GP_ERR_TIMEOUT,
 * outputs incomplete) is then returned by the next gp_bfs_multi on this graph.
 * Workspace: per group two n-entry queues and four n-bit bitmaps, kept with
 * the graph; calls on one graph share it, so issue them on one stream.
 */
int gp_bfs_multi(const gp_graph *g, const int32_t *sources, int nsources, int mode, int32_t *const *level_out,
                 int32_t *const *parent_out, int groups, gp_bfs_summary *summary, void *stream);

/* gp_bfs with the direction of every level chosen by the caller:
 * dirs[i] (GP_PUSH or GP_PULL) is used for level i, dirs[ndirs-1] for all
 * later levels; ndirs may exceed GP_BFS_MAX_LEVELS.  Levels do not depend on
 * the choice. */
int gp_bfs_directed(const gp_graph *g, int32_t src, const int8_t *dirs, int ndirs, int32_t *level_out,
                    int32_t *parent_out, gp_bfs_stats *stats, void *stream);

/* ------------------------------------------------------------------ Frontier-Exploit PageRank */

#define GP_FE_MAX_ITERS 1024

typedef struct gp_fe_stats {
    int32_t iterations;     /* iterations run */
    int32_t pushes, pulls;  /* iterations by direction */
    double residual_l1;     /* ||r||_1 of the residuals left (FP64 sum of the FP32 residuals) */
    double error_bound;     /* residual_l1 / (1 - damping): bound on ||x - x*||_1 for column-substochastic P */
    int64_t frontier_left;  /* vertices with |r| > eps when the run stopped (0: converged) */
    float ms;               /* device time of the call by CUDA events */
    int32_t init_ns;        /* device time before the first iteration */
    int8_t direction[GP_FE_MAX_ITERS];  /* per iteration: GP_PUSH / GP_PULL */
    int64_t frontier[GP_FE_MAX_ITERS];  /* frontier size entering each iteration */
    int64_t examined[GP_FE_MAX_ITERS];  /* edges scattered (push) or gathered (pull) */
    int32_t iter_ns[GP_FE_MAX_ITERS];   /* device time of each iteration */
} gp_fe_stats;

/*
 * PageRank with Frontier-Exploit (Section 5: only a frontier of vertices works
 * in an iteration) and Generic-Switch (push or pull per iteration), in residual
 * form: x starts at s (1/n uniform) and the residuals r at (1-d) s + d P x - x,
 * the change one PageRank sweep would make (one pull sweep at the start); each
 * iteration the
 * frontier F = {u : |r_u| > eps} moves its residuals into x and sends
 * d P_vu r_u to the out-neighbours:
 *     x_u += r_u (u in F);   r'_v = [v not in F] r_v + d sum_{u in F, u->v} P_vu r_u.
 * Since x + (I - dP)^-1 r equals the PageRank fixed point throughout, a run that
 * stops with F empty (converged) is within ||r||_1 / (1 - d) of it in L1
 * (stats->error_bound; P as in gp_pagerank: 1/deg_out, the weights as given, or
 * normalised weights).
 *   mode        GP_PUSH: F scatters over out-edges with FP64 atomic adds in L2;
 *               GP_PULL: every vertex gathers over its in-edges from F (owner
 *               writes, no atomics);
 *               GP_AUTO: per iteration, pull when F's out-edges times fe_alpha
 *               exceed m, else push.
 *   eps         frontier threshold on |r_u| (>= 0); eps < 0 keeps every vertex in
 *               the frontier: k iterations give the k-th PageRank sweep from s.
 *   iters       iteration cap.
 *   dirs, ndirs NULL, or the direction of each iteration (dirs[ndirs-1] after).
 *   personalization  float[n] "any" or NULL (uniform 1/n).
 *   ranks_out   float[n] "any": x.
 * Waits for completion.  GP_ERR_NOT_CONVERGED (ranks written) when the cap is
 * reached with a non-empty frontier; GP_ERR_INVALID for bad arguments.
 */
int gp_pagerank_fe(const gp_graph *g, int mode, float damping, double eps, int iters, const int8_t *dirs, int ndirs,
                   const float *personalization, float *ranks_out, gp_fe_stats *stats, void *stream);

/* ------------------------------------------------------------------ shortest paths */

#define GP_SSSP_MAX_ITERS 1024

typedef struct gp_sssp_stats {
    int32_t iterations;     /* relaxation iterations (all epochs) */
    int32_t epochs;         /* buckets processed */
    int64_t reached;        /* vertices with a finite distance */
    int64_t edges_examined; /* edges relaxed (push) or scanned (pull) */
    int32_t pushes, pulls;  /* iterations by direction */
    float ms;               /* device time of the call by CUDA events */
    int32_t init_ns;        /* device time before the first iteration */
    int8_t direction[GP_SSSP_MAX_ITERS]; /* per iteration (first GP_SSSP_MAX_ITERS): GP_PUSH / GP_PULL */
    int64_t bucket[GP_SSSP_MAX_ITERS];   /* bucket index (distance / delta) of the iteration's epoch */
    int64_t active[GP_SSSP_MAX_ITERS];   /* active vertices entering the iteration */
    int64_t examined[GP_SSSP_MAX_ITERS]; /* edges relaxed or scanned by the iteration */
    int32_t iter_ns[GP_SSSP_MAX_ITERS];  /* device time of the iteration (global timer) */
} gp_sssp_stats;

/*
 * Single-source shortest paths by Delta-Stepping (Section 3, the push- and
 * pull-based Delta-Stepping listing): epoch b settles the vertices whose
 * distance lies in [b*delta, (b+1)*delta); within an epoch, relaxation
 * iterations repeat until no vertex of the bucket improves.
 *   src         source vertex.
 *   delta       bucket width (> 0, finite): small widths approach Dijkstra's
 *               order, huge ones Bellman-Ford's; distances do not depend on it.
 *   mode        GP_PUSH: every iteration pushes (active vertices relax their
 *               out-edges with 64-bit atomicMin: O(m l) atomics);
 *               GP_PULL: every iteration pulls (unsettled vertices take the
 *               minimum over their in-edges from active vertices; owner-only
 *               writes, heavy in-lists combined by atomicMin over chunks);
 *               GP_AUTO: per iteration, pull when the active vertices'
 *               out-edges times sssp_alpha exceed the in-edges of the unsettled
 *               vertices, else push.
 *   dirs, ndirs NULL, or the direction of each iteration (GP_PUSH/GP_PULL,
 *               dirs[ndirs-1] for all later ones), overriding mode.
 *   dist_out    float[n] "any": shortest distance, +inf if unreachable.
 *   pred_out    int32[n] "any" or NULL: the smallest predecessor on a shortest
 *               path (pred[src] = src, -1 unreachable) -- unique, whatever the
 *               order of relaxations.  With zero-weight edges two vertices at
 *               the same distance can be each other's predecessor.
 *   stats       NULL or filled on return.
 * Weights: the graph's weights as uploaded (csr_w for out-edges, csc_w for
 * in-edges; weights must be >= 0, else GP_ERR_INVALID; checked once per graph),
 * 1 for every edge of an unweighted graph.  FP32 distances: sums along a path
 * are rounded as they are formed (exact while they are integers below 2^24).
 * Synchronisation as gp_bfs: with stats == NULL and device outputs the call
 * only enqueues the search; a grid-barrier timeout is then reported by the next
 * gp_sssp call on the graph.  GP_ERR_INVALID for a bad source, delta, mode or
 * direction; GP_ERR_TIMEOUT if a grid barrier wait ran out.
 */
int gp_sssp(const gp_graph *g, int32_t src, float delta, int mode, const int8_t *dirs, int ndirs, float *dist_out,
            int32_t *pred_out, gp_sssp_stats *stats, void *stream);

/* ------------------------------------------------------------------ triangle counting */

typedef struct gp_tc_stats {
    int64_t triangles; /* number of triangles (sum of the counts / 3) */
    int64_t probes;    /* list elements searched for (shorter list of every ordered edge) */
    float ms;          /* device time of the call by CUDA events */
    int32_t mode_used; /* GP_PUSH or GP_PULL */
} gp_tc_stats;

/*
 * Per-vertex triangle counts by the NodeIterator of Section 3 (push- and
 * pull-based Triangle Counting): for every v and every ordered pair (w1, w2) of
 * v's neighbours with w1 adjacent to w2, GP_PULL adds one to tc[v] (every count
 * written only by the warp that owns v) and GP_PUSH adds one to tc[w1] with a
 * fetch-and-add; both halve.  GP_AUTO runs the pull form (no atomics).  The
 * graph must have been uploaded as symmetric (GP_UPLOAD_SYMMETRIC) and be simple
 * (no duplicate edges; self-loops are skipped).
 *   tc_out      int64[n] "any" or NULL: triangles containing each vertex.
 *   total_out   host int64 or NULL: number of triangles.
 *   stats       NULL or filled on return.
 * Waits for completion.  GP_ERR_INVALID for a directed graph, a bad mode or no
 * output.
 */
int gp_triangles(const gp_graph *g, int mode, int64_t *tc_out, int64_t *total_out, gp_tc_stats *stats, void *stream);

/* ------------------------------------------------------------------ betweenness centrality */

#define GP_BC_MAX_STEPS 1024

typedef struct gp_bc_stats {
    int64_t sources;        /* sources processed */
    int64_t levels;         /* non-empty BFS levels, summed over the sources */
    int64_t reached;        /* vertices reached (source included), summed over the sources */
    int64_t edges_examined; /* adjacency entries read by all steps of all sources */
    int64_t pushes, pulls;  /* steps by direction, all sources, both phases */
    float ms;               /* device time of the call by CUDA events */
    int32_t steps;          /* steps of the first source recorded below */
    int8_t direction[GP_BC_MAX_STEPS]; /* GP_PUSH / GP_PULL */
    int8_t phase[GP_BC_MAX_STEPS];     /* 0: forward (path counting), 1: backward (dependencies) */
    int32_t level[GP_BC_MAX_STEPS];    /* forward: the frontier's level l; backward: the level l
                                          whose dependencies pass to level l-1 */
    int64_t frontier[GP_BC_MAX_STEPS]; /* vertices of level l */
    int64_t examined[GP_BC_MAX_STEPS]; /* adjacency entries read by the step */
    int32_t step_ns[GP_BC_MAX_STEPS];  /* device time of the step (global timer) */
} gp_bc_stats;

/*
 * Betweenness centrality by Brandes' scheme (Section 3, the push- and
 * pull-based BC listing), summed over a set of sources (all n vertices: the
 * exact centrality; a sample: the usual estimate up to the factor n / k):
 *   bc(v) = sum over sources s != v of delta_s(v),
 *   delta_s(v) = sum over t of sigma_st(v) / sigma_st,
 * sigma_st the number of shortest s-t paths (edges counted with multiplicity,
 * unit lengths, out-edges followed) and sigma_st(v) those through v.
 * Per source a forward phase counts shortest paths level by level (sigma of a
 * vertex = sum over its predecessors one level closer), then a backward phase
 * from the deepest level up accumulates the dependencies:
 *   delta(u) = sigma(u) * sum over successors w of (1 + delta(w)) / sigma(w).
 *   sources     int32[nsources] "any": source vertices (repeats count again).
 *   mode        GP_PUSH: every step pushes (forward: frontier vertices add
 *               their path counts to the next level with FP64 atomics, claiming
 *               new vertices by CAS; backward: each vertex adds its coefficient
 *               to its predecessors' sums with FP64 atomics);
 *               GP_PULL: every step pulls (forward: every unvisited vertex sums
 *               its predecessors' counts, no early exit; backward: each vertex
 *               sums its successors' coefficients; owner-only writes, heavy
 *               lists combined over chunks);
 *               GP_AUTO: per step, pull when the push side's edges times
 *               bc_alpha exceed the pull side's (forward: out-edges of the
 *               frontier against in-edges of the unvisited vertices; backward:
 *               in-edges of level l against out-edges of level l-1).
 *   dirs, ndirs NULL, or the direction of each step of every source (forward
 *               steps first, then backward ones; dirs[ndirs-1] for all later
 *               ones), overriding mode.
 *   bc_out      double[n] "any": the centralities (overwritten).  FP64
 *               throughout (path counts, coefficients, sums); results differ
 *               from a sequential FP64 evaluation only by summation order.
 *   stats       NULL or filled on return.
 * Synchronisation as gp_sssp: with stats == NULL and device memory for
 * sources and bc_out the call only enqueues the work; a grid-barrier timeout is
 * then reported by the next gp_bc call on the graph.  GP_ERR_INVALID for a
 * source outside [0, n), nsources < 0, a bad mode or direction;
 * GP_ERR_TIMEOUT if a grid barrier wait ran out.
 */
int gp_bc(const gp_graph *g, const int32_t *sources, int64_t nsources, int mode, const int8_t *dirs, int ndirs,
          double *bc_out, gp_bc_stats *stats, void *stream);

/* ------------------------------------------------------------------ batches of graphs */

typedef struct gp_batch gp_batch; /* opaque: a work plan over several uploaded graphs */

typedef struct gp_batch_stats {
    int32_t sweeps;  /* PageRank: sweeps run (the slowest vector's count) */
    int32_t levels;  /* BFS: levels explored by the deepest search */
    float ms;        /* device time of the persistent launch (CUDA events) */
    int32_t blocks;  /* resident blocks of the cooperative launch */
    int32_t jobs;    /* PageRank: (graph, column slice) jobs the vectors were split into */
    int32_t packed;  /* PageRank: columns their jobs left to packed jobs (see ppr_pack) */
} gp_batch_stats;

/* Tunables of a batch (gp_batch_autotune chooses them; results never depend on them). */
typedef struct gp_batch_options {
    int32_t big_in_degree; /* in-degree above which a vertex's in-edges are split into chunks
                              (PageRank) or scanned by a whole warp (bottom-up BFS) */
    int32_t chunk_edges;   /* in-edges per chunk */
    int32_t l2_budget_mb;  /* PageRank: the widest column slice (128, 64 or 32 columns, at most k_ppr) whose two iterates fit this many MiB is one job */
    float msbfs_alpha;     /* BFS: a graph's level goes bottom-up when its frontier's out-edges
                              times alpha exceed the in-edges of vertices some search misses */
    float msbfs_beta;      /* BFS: back to top-down when the frontier is below n / beta */
    int32_t ppr_start;     /* PageRank start vector: 1 = each vector's seed one-hot e_seed
                              (default), 0 = uniform 1/n */
    int32_t ppr_pack;      /* PageRank: a job (one graph, one column slice) stops once at most
                              this many of its columns still iterate; those continue, 32 to a
                              job, in packed jobs after all slices (0 = never; at most 128) */
    int32_t reserved[1];
} gp_batch_options;

int gp_batch_options_default(gp_batch_options *opt);
/* Replace the batch's options (rebuilds its work lists when the degree limit,
 * chunk size or budget change; synchronises the stream then). */
int gp_batch_set_options(gp_batch *b, const gp_batch_options *opt, void *stream);
int gp_batch_get_options(const gp_batch *b, gp_batch_options *opt);

typedef struct gp_batch_tune_result {
    gp_batch_options options; /* the chosen options (also installed in the batch) */
    float ppr_ms;             /* device time of ppr_sweeps fixed sweeps with them */
    float msbfs_ms;           /* device time of the multi-source search with them */
    int32_t trials;           /* timed candidates */
} gp_batch_tune_result;

/*
 * Autotuner of a batch (not in the paper): coordinate descent over the chunk
 * threshold {8..128}, chunk size {64, 128, 256} and L2 budget {48..192 MiB},
 * each candidate timed by CUDA events on `ppr_sweeps` fixed sweeps of
 * gp_ppr_batched with these seeds (host int32[ngraphs][k_ppr]; NULL skips the
 * PageRank axes), then over the BFS alpha {2..64} and beta {8, 24, 64} timed on
 * gp_msbfs_batched with these sources (host int32[ngraphs][nsrc]; NULL skips).
 * The best options stay installed.  Results never depend on the options.
 * Synchronises; the batch's previous outputs are overwritten.
 */
int gp_batch_autotune(gp_batch *b, const int32_t *seeds, const int32_t *sources, int nsrc, int ppr_sweeps,
                      gp_batch_tune_result *res, void *stream);

/*
 * Prepare batched runs over `ngraphs` uploaded graphs (the handles stay owned
 * by the caller and must outlive the batch).  k_ppr in {32, 64, 128, 256} is the
 * number of personalised PageRank vectors per graph.  Reads the in-degrees once
 * to lay out the work (vertex tiles per graph, warp chunks of in-edge lists
 * longer than 256) and allocates, per graph, two n x k_ppr iterates and the
 * n x 64 BFS level array.  Synchronises the stream.
 */
int gp_batch_create(gp_batch **out, gp_graph *const *graphs, int ngraphs, int k_ppr, void *stream);
int gp_batch_free(gp_batch *b);

/*
 * Personalised PageRank for every graph and every one-hot seed (Section 3.1
 * formula with s = e_seed), all graphs and vectors in one persistent
 * cooperative launch replayed from a CUDA graph (captured on first use and
 * whenever damping, iters or tol change).
 *   seeds       int32[ngraphs][k_ppr] host: the seed vertex of every vector.
 *   out         ngraphs pointers ("any", or NULL entries to skip) to float[n_i][k_ppr]
 *               (vertex-major: column j of graph i is out[i][v * k_ppr + j]).
 *   iters_done  int32[ngraphs][k_ppr] "any" or NULL: sweeps each vector ran.
 * Each vector starts from its seed's one-hot vector e_seed (options: ppr_start;
 * or from 1/n) and stops at its first sweep with L1 change < tol (or after
 * `iters`), exactly as gp_pagerank with that personalization and x0 would.  The
 * one-hot start lies in the seed's component, so none of the start's mass sits
 * in other components, where it would only decay as d^k: on R-MAT graphs it
 * meets tol 1e-6 in about a fifth of the sweeps the uniform start needs.
 * Returns GP_ERR_TIMEOUT if a grid barrier wait ran out.  Synchronises.
 */
int gp_ppr_batched(gp_batch *b, const int32_t *seeds, float damping, int iters, double tol, float *const *out,
                   int32_t *iters_done, gp_batch_stats *stats, void *stream);

/*
 * Multi-source BFS: nsrc <= 64 searches per graph (sources: host
 * int32[ngraphs][nsrc]) advanced together as 64-bit masks, pull levels with early
 * exit (Section 3.3, Algorithm 3 pulling), one persistent launch from a CUDA graph.
 *   levels_out  ngraphs pointers ("any", or NULL) to int32[n_i][64]: level of
 *               vertex v in search j at [v * 64 + j], -1 if unreached (columns
 *               >= nsrc stay -1).
 * Returns GP_ERR_TIMEOUT if a grid barrier wait ran out.  Synchronises.
 */
int gp_msbfs_batched(gp_batch *b, const int32_t *sources, int nsrc, int32_t *const *levels_out, gp_batch_stats *stats,
                     void *stream);

/* ------------------------------------------------------------------ sweep without allocation */

/* Largest graph (in vertices) gp_pull_sweep_noalloc accepts: the size of its static scratch. */
#define GP_NOALLOC_MAX_VERTICES (1 << 20)

/*
 * One pull PageRank sweep that allocates no device memory (the paper has no
 * counterpart: this entry point exists for callers that are not allowed to
 * allocate while they run -- code inside a framework hook that may only use
 * the buffers it is given, pipelines that reserve all device memory up front,
 * or processes whose memory is already claimed by another allocator).
 *     y[v] = (1-d) s[v] + d * sum_{u in in(v)} w_uv * x[u] * inv_deg[u]
 *     *residual_out = sum_v |y[v] - x[v]|   (FP64)
 * All arrays are device memory owned by the caller:
 *   csc_off int64[n+1], csc_idx int32[m]   in-edges (as for gp_graph_upload);
 *   csc_w   float[m] or NULL               edge factor w_uv (NULL: 1);
 *   inv_deg float[n]                       1/deg_out(u) (0 for dangling u), or the
 *                                          weight normaliser when csc_w is given;
 *   x       float[n]                       current iterate;
 *   personalization float[n] or NULL       teleport vector s (NULL: 1/n);
 *   y       float[n]                       new iterate (written);
 *   residual_out double[1]                 written on the device; NaN if an
 *                                          offset or index was out of range (the
 *                                          bad entries are skipped, never read).
 * Limits: 1 <= n <= GP_NOALLOC_MAX_VERTICES and m < 2^31, else GP_ERR_INVALID
 * with no device work.  Intermediate data (x*inv_deg and per-block residual
 * partials, 4 MiB + 8 KiB) lives in one array compiled into the library, which
 * every device that loads the library keeps until the process exits.  The
 * first call on a device looks up that array's device address (once per
 * device), so make the first call on each device before any stream capture.
 * All calls share the array: calls whose kernels overlap on the GPU (other
 * streams, other host threads) race and corrupt each other; serialise them.
 * Asynchronous on `stream`; no cudaMalloc/cudaFree or other allocating call.
 */
int gp_pull_sweep_noalloc(int64_t n, int64_t m, const int64_t *csc_off, const int32_t *csc_idx, const float *csc_w,
                          const float *inv_deg, const float *x, float damping, const float *personalization, float *y,
                          double *residual_out, void *stream);

/* ------------------------------------------------------------------ kernel timing */

/* When enabled, the library brackets each of its sweep-kernel launches with
 * CUDA events on the launching stream and accumulates their durations per
 * kernel name.  Off by default (no events recorded). */
int gp_profile_enable(int on);

typedef struct gp_kernel_time {
    char name[48];
    int64_t launches;
    double total_ms;
} gp_kernel_time;

/* Synchronise the recorded events, write up to `cap` entries (kernels sorted
 * by total time, descending) and return the number written in *count; reset
 * != 0 clears the accumulators afterwards. */
int gp_profile_read(gp_kernel_time *out, int cap, int *count, int reset);

/* ------------------------------------------------------------------ diagnostics */

/* Self-check of the binary64 -> binary32 rounding that the push epilogue uses
 * (integer operations on the IEEE 754 encodings, round to nearest, ties to
 * even; magnitudes below 2^-126 give signed zero).  For each of the n values of
 * the device array `in` (f64[n]) writes that rounding to `ours` and the
 * hardware conversion (__double2float_rn) to `hw` (device f32[n] each, caller-
 * owned).  Asynchronous on `stream`.  GP_ERR_INVALID for n < 0 or a NULL array
 * with n > 0. */
int gp_selftest_narrow(int64_t n, const double *in, float *ours, float *hw, void *stream);

/* Self-check of the bounded grid barrier that the persistent kernels (BFS,
 * batches) use between phases: one cooperative launch of one 128-thread block
 * per SM in which every block except `absent` enters a barrier whose waits give
 * up after a short limit (tens of milliseconds).  absent < 0: every block
 * arrives and the call returns GP_OK; otherwise the waiting blocks time out,
 * return, and the call returns GP_ERR_TIMEOUT with the device context intact.
 * Waits for completion.  GP_ERR_INVALID for absent >= the SM count. */
int gp_selftest_barrier(int absent, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* GP_H */
