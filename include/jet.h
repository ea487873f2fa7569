/*
 * jet.h — C ABI of the GB300 (sm_103a) Jet multilevel k-way graph partitioner.
 *
 * Method: Gilbert, Madduri, Boman, Rajamanickam, "Jet: Multilevel Graph
 * Partitioning on Graphics Processing Units".  Citations below name the
 * paper's sections, algorithms and equations.
 *
 * Graph format (Sec. 2.1 "Problem Definition"): an undirected graph without
 * self-loops or parallel edges in CSR form —
 *   xadj   int64[n+1], xadj[0] = 0, non-decreasing;
 *   adjncy int32[xadj[n]], every edge {u,v} stored as v in u's row and u in v's;
 *   vwgt   int32[n]  positive vertex weights, or NULL for unit weights;
 *   adjwgt int32[xadj[n]] positive edge weights, equal in both directions, or
 *          NULL for unit weights.
 * Limits: n < 2^31; sum of vwgt < 2^31; sum of adjwgt over all xadj[n] entries
 * < 2^31 (connectivities are exact 32-bit sums; cut and part weights are
 * 64-bit); 1 <= k <= JET_MAX_K.
 *
 * Memory: unless a function says otherwise, every array argument is a DEVICE
 * pointer on the context's device, allocated and owned by the caller; the
 * library never frees it.  Scalars returned through pointers (cut_out, ...)
 * are HOST pointers.  The library allocates its own device scratch (stream-
 * ordered, on the context's stream) and releases it before returning, except
 * for the hierarchy objects, which jet_hier_destroy releases.
 *
 * Streams and synchronisation: all work is enqueued on the context's stream;
 * every call returns only after its results are final (it synchronises that
 * stream), so callers may read outputs immediately.
 *
 * Determinism: results are a pure function of the inputs, k, eps, the options
 * and the seed — bit-identical across runs and equal to the CPU oracle's.
 * Ties are broken by the lowest part id, then the lowest vertex id.
 *
 * Errors: every call returns a status (JET_OK = 0, warnings > 0, errors < 0);
 * no exception or abort crosses the ABI.  After JET_ECUDA the context may be
 * unusable (the CUDA error is sticky); destroy it.
 */
#ifndef JET_H
#define JET_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define JET_MAX_K 1024
#define JET_MAX_LEVELS 64

/* status codes */
#define JET_OK 0
#define JET_WUNBALANCED 1   /* warning: the best partition found violates the balance limit */
#define JET_WITERLIMIT 2    /* warning: a level hit max_iters_per_level before the stop rule */
#define JET_EINVAL (-1)     /* bad argument: n < 0, k out of range, eps < 0, NULL required pointer */
#define JET_EGRAPH (-2)     /* invalid graph (only with JET_FLAG_VALIDATE): asymmetric, self-loop,
                               parallel edge, weight <= 0, id out of range */
#define JET_ENOMEM (-3)     /* device allocation failed */
#define JET_ECUDA (-4)      /* a CUDA call failed */
#define JET_ETIMEOUT (-5)   /* a bounded device wait ran out */
#define JET_EOVERFLOW (-6)  /* weight sums exceed the 2^31 limits above */

/* jet_options.flags */
#define JET_FLAG_VALIDATE 1u       /* check the input graph on the device first */
#define JET_FLAG_HOSTLOOP 2u       /* drive refinement iterations from the host (one launch
                                      sequence per iteration, mode read back each time)
                                      instead of the device-resident CUDA-graph loop */
#define JET_FLAG_PROFILE 4u        /* implies JET_FLAG_HOSTLOOP; records a CUDA event before every
                                      refinement kernel launch and after the last of each iteration
                                      (same kernels, same launch configuration) and fills
                                      jet_stats.kern_ms and sel_ms */
#define JET_FLAG_NO_LOCKS 16u      /* Jetlp ablations (Sec. 6.1.4, Table 2): ignore lock bits */
#define JET_FLAG_NO_AFTERBURN 32u  /*   M = X (skip the second filter) */
#define JET_FLAG_WEAK_AFTERBURN 64u/*   first filter keeps only F >= 0 */
#define JET_FLAG_BASELINE_LP 128u  /*   baseline LP: move iff F > 0, no afterburner, no locks */
#define JET_FLAG_STRICT_GAIN 512u  /* Jetlp ablation: first filter keeps only F > 0 (with
                                      JET_FLAG_NO_AFTERBURN: the baseline LP plus locks) */
#define JET_FLAG_TWO_HOP 256u      /* coarsening: add two-hop matches (Sec. 3.1) after heavy-edge matching;
                                      the plain method coarsens by heavy-edge matching alone */
#define JET_FLAG_NO_PDL 1024u      /* execution choice (results do not depend on it): launch every
                                      refinement kernel only after the previous one has finished,
                                      instead of letting it start early and wait on the device
                                      (programmatic dependent launch) */
#define JET_FLAG_GRID_LOOP 2048u   /* execution choice (results do not depend on it): levels above
                                      cluster_max_n run their whole refinement loop in one
                                      cooperative launch over the GPU (phases separated by grid
                                      barriers, each wait bounded: JET_ETIMEOUT if one runs out)
                                      instead of the CUDA-graph loop */

/* Hyper-parameters the paper names (defaults from jet_options_default):
 *   c_fine = 0.25, c_coarse = 0.75  first-filter ratio c (Sec. 4.1.2, Eq. gainconn_filter);
 *                                   held internally as round(c * 65536) / 65536
 *   phi = 0.999                     tolerance of Alg. 3 (held as round(phi * 1e6) / 1e6)
 *   max_no_improve = 12             iterations without a new best before stopping (Sec. 4)
 *   weak_limit = 2                  b_max Jetrw iterations before Jetrs (Sec. 4.2.2)
 *   coarsen_target = 0              stop coarsening at <= max(8k, 256) vertices (Sec. 3)
 *   max_levels = 64, max_iters_per_level = 10000 (safety caps), hem_rounds = 8
 * Execution choice (no counterpart in the paper; results do not depend on it):
 *   cluster_max_n = 4096            levels with at most this many vertices run their whole
 *                                   refinement loop in one thread-block-cluster launch; larger
 *                                   levels use the CUDA-graph loop; 0 = never
 *   cluster_blocks = 0              blocks (of 1024 threads) of that cluster: 0 = the largest the
 *                                   device runs (up to 16), else a power of two in [2, 16]
 *   barrier_polls = 0               polls a block of the persistent level loop (JET_FLAG_GRID_LOOP)
 *                                   makes at a grid barrier before it gives up and the call returns
 *                                   JET_ETIMEOUT; 0 = 2^22 (about a second or more, far above any
 *                                   phase); small values make the wait run out on purpose (tests)
 *   launch shapes of the refinement kernels (0 = the default in brackets; jet_autotune picks them):
 *   list_blocks_per_sm [4]          most blocks per SM of the list kernels (select, afterburner,
 *                                   rebalancing rows)
 *   list_items_per_block [64]       list entries per block below that cap
 *   apply_blocks_per_sm [list]      most blocks per SM of the apply kernel
 *   scan_blocks_per_sm [8]          most blocks per SM of the two scan kernels
 *   hub_degree [1024]               rows longer than this are taken by a whole block (shorter
 *                                   rows above 16 entries by one warp, up to 16 by one thread);
 *                                   0 or at least 32 */
typedef struct {
    double c_fine, c_coarse, phi;
    int32_t max_no_improve, weak_limit, coarsen_target, max_levels, max_iters_per_level, hem_rounds;
    uint32_t flags;
    int32_t cluster_max_n;
    int32_t cluster_blocks;
    int32_t barrier_polls;
    int32_t list_blocks_per_sm, list_items_per_block, apply_blocks_per_sm, scan_blocks_per_sm, hub_degree;
} jet_options;

/* Refinement kernels (one launch each per iteration of the CUDA-graph or host
 * loop), indices of jet_stats.kern_*; jet_kernel_name gives their names. */
#define JET_KERNELS 16
#define JET_K_LP_SCAN 0      /* Jetlp work list (Alg. 4: boundary, unlocked vertices) */
#define JET_K_LP_SELECT 1    /* Jetlp P_d, F and the first filter (Alg. 4, Eq. gainconn_filter) */
#define JET_K_AFTERBURN 2    /* Jetlp afterburner and second filter (Alg. 4, ord of Sec. 4.1.1) */
#define JET_K_APPLY 3        /* apply the moves (Alg. 3 updatePartsAndDS) + the Alg. 3 controller */
#define JET_K_RB_SCAN 4      /* rebalancing candidates (Alg. 5 first loop) */
#define JET_K_RB_CAND 5      /* rebalancing destinations and losses of listed candidates */
#define JET_K_RB_TILEHIST 6  /* rebalancing: weight of boundary-slot members per tile */
#define JET_K_RB_TILESCAN 7  /* rebalancing: scan of the tile sums */
#define JET_K_RB_TAKE 8      /* rebalancing: eviction in (slot, vertex id) order */
#define JET_K_RB_COOKIE 9    /* Jetrs destinations (cookie cutter, Sec. 4.2.2) */
#define JET_K_COUNT 10       /* kernels in use (indices below JET_KERNELS) */

/* Per-call statistics (jet_partition / jet_uncoarsen).  Times are CUDA-event
 * milliseconds on the context's stream. */
typedef struct {
    int32_t levels;
    int64_t n[JET_MAX_LEVELS], m[JET_MAX_LEVELS];          /* vertices / undirected edges per level */
    int32_t iters_lp[JET_MAX_LEVELS], iters_rw[JET_MAX_LEVELS], iters_rs[JET_MAX_LEVELS];
    int64_t cut_level[JET_MAX_LEVELS];                     /* cut after refining each level */
    int64_t edge_iters;        /* sum over levels of (iterations x m_level): refinement edge passes */
    int64_t fin_edge_iters;    /* the same, finest level only */
    float ms_coarsen, ms_init, ms_refine, ms_refine_finest, ms_total;
    int64_t cut, max_part_w;
    int64_t bytes_model;        /* algorithmic DRAM bytes of all refinement passes (byte model:
                                   compulsory streams, neighbour gathers taken as cache hits) */
    int64_t kernel_launches;    /* kernels executed by this call, device-loop iterations included */
    int64_t sel_launches[JET_MAX_LEVELS];  /* Jetlp select passes per level */
    int64_t sel_bytes[JET_MAX_LEVELS];     /* their algorithmic bytes, summed */
    float sel_ms[JET_MAX_LEVELS];          /* their CUDA-event time, summed (JET_FLAG_PROFILE only) */
    float ms_level[JET_MAX_LEVELS];        /* CUDA-event time of each level's projection + refinement */
    int32_t cluster_blocks[JET_MAX_LEVELS]; /* blocks of the thread-block cluster that ran the level's
                                               loop; 0 where the CUDA-graph or host loop ran it */
    /* per level and refinement kernel (JET_K_*): launches (0 where one cluster or cooperative launch
     * ran the whole loop), algorithmic DRAM bytes (the byte model of bytes_model, split by kernel)
     * and, with JET_FLAG_PROFILE, the CUDA-event time of the kernel's launches */
    int64_t kern_launches[JET_MAX_LEVELS][JET_KERNELS];
    int64_t kern_bytes[JET_MAX_LEVELS][JET_KERNELS];
    float kern_ms[JET_MAX_LEVELS][JET_KERNELS];
} jet_stats;

/* Name of refinement kernel i (JET_K_*), or NULL outside [0, JET_K_COUNT). */
const char *jet_kernel_name(int32_t i);

typedef struct jet_ctx jet_ctx;
typedef struct jet_hier jet_hier;

/* Fill *opt with the defaults listed above. */
void jet_options_default(jet_options *opt);

/* Create a context on CUDA device `device` that enqueues on `cuda_stream`
 * (a cudaStream_t; NULL = the legacy default stream).  opt may be NULL for
 * defaults.  The context owns no caller memory.  Returns JET_EINVAL for a bad
 * device or option, JET_ECUDA if the device cannot be used. */
int jet_ctx_create(int device, void *cuda_stream, const jet_options *opt, jet_ctx **out);
void jet_ctx_destroy(jet_ctx *ctx);

/* MLCoarsen of Alg. 1 (Sec. 3.1): repeated heavy-edge matching and edge
 * contraction (Alg. 2) until the graph has at most coarsen_target vertices,
 * coarsening stalls (a level keeps more than 95% of the vertices) or
 * max_levels is reached.  seed drives the matching's tie-break hash.  *out is
 * a device-resident hierarchy owned by the library (jet_hier_destroy); level 0
 * refers to the caller's arrays, which must stay valid while *out is used. */
int jet_coarsen(jet_ctx *ctx, int32_t n, const int64_t *xadj, const int32_t *adjncy,
                const int32_t *vwgt, const int32_t *adjwgt, int32_t k, uint64_t seed, jet_hier **out);
void jet_hier_destroy(jet_hier *h);

/* Level count and per-level sizes (host arrays of at least JET_MAX_LEVELS
 * entries; any may be NULL).  m is the number of undirected edges. */
int jet_hier_info(const jet_hier *h, int32_t *levels, int64_t *n_per_level, int64_t *m_per_level);

/* Device pointers of one level's CSR (rows sorted ascending, weights summed
 * over merged edges) and of its coarse map cmap (level -> level+1; NULL on the
 * coarsest level).  Valid until jet_hier_destroy. */
int jet_hier_level(const jet_hier *h, int32_t level, int32_t *n, const int64_t **xadj,
                   const int32_t **adjncy, const int32_t **vwgt, const int32_t **adjwgt,
                   const int32_t **cmap);

/* Alg. 1 after MLCoarsen: InitialPartition of the coarsest level (greedy
 * graph growing: vertices ordered by component, BFS level from the component's
 * lowest id, then id; cut into k consecutive pieces by weight), then
 * RefinePartition (Alg. 3) on it and, for each finer level, ProjectPartition
 * (P_i[v] = P_{i+1}[C_i[v]]) followed by RefinePartition.  part_out: device
 * int32[n of level 0].  stats may be NULL. */
int jet_uncoarsen(jet_ctx *ctx, const jet_hier *h, int32_t k, double eps, uint64_t seed,
                  int32_t *part_out, int64_t *cut_out, jet_stats *stats);

/* Jet refinement of one graph (Alg. 3 with Alg. 4 Jetlp, Alg. 5 Jetrw and the
 * Jetrs of Sec. 4.2.2) starting from part_inout (device int32[n], values in
 * [0,k)), which receives P_best.  is_finest selects c_fine (else c_coarse).
 * seed drives Jetrw's random destination.  *cut_out = cost of P_best.
 * Returns JET_WUNBALANCED if P_best still violates the limit
 * floor(ceil(W/k) * (10^6 + round(eps*10^6)) / 10^6). */
int jet_refine(jet_ctx *ctx, int32_t n, const int64_t *xadj, const int32_t *adjncy,
               const int32_t *vwgt, const int32_t *adjwgt, int32_t k, double eps,
               int32_t is_finest, uint64_t seed, int32_t *part_inout, int64_t *cut_out);

/* Host copy of the per-iteration record of the most recent jet_refine (or of
 * the finest level of the most recent jet_partition / jet_uncoarsen): kind
 * (0 Jetlp, 1 Jetrw, 2 Jetrs), |X| for Jetlp or the number of rebalancing
 * candidates, |M|, cut and max part weight after the iteration.  Host arrays
 * of `cap` entries (any may be NULL); *iters_out = iterations run. */
int jet_last_trace(jet_ctx *ctx, int32_t cap, int32_t *kind, int64_t *nx, int64_t *nm,
                   int64_t *cut, int64_t *maxw, int32_t *iters_out);

/* Alg. 1 end to end: jet_coarsen, then jet_uncoarsen.  part_out: device
 * int32[n].  stats may be NULL. */
int jet_partition(jet_ctx *ctx, int32_t n, const int64_t *xadj, const int32_t *adjncy,
                  const int32_t *vwgt, const int32_t *adjwgt, int32_t k, double eps,
                  uint64_t seed, int32_t *part_out, int64_t *cut_out, jet_stats *stats);

/* jet_partition on HOST arrays (same layout; vwgt/adjwgt may be NULL):
 * copies the graph to the device on the context's stream, partitions it and
 * copies part_out (host int32[n]) back. */
int jet_partition_host(jet_ctx *ctx, int32_t n, const int64_t *xadj, const int32_t *adjncy,
                       const int32_t *vwgt, const int32_t *adjwgt, int32_t k, double eps,
                       uint64_t seed, int32_t *part_out, int64_t *cut_out, jet_stats *stats);

/* Batched form: many independent graphs partitioned concurrently.  Each item
 * is one jet_partition (device arrays, its own k, eps and seed; results
 * bit-identical to a jet_partition call with the same arguments); `workers`
 * host threads (<= 0: 8) each drive their own stream and memory pool on the
 * context's device, so small graphs, whose refinement is latency-bound, fill
 * the GPU together.  The work starts after what is already enqueued on the
 * context's stream and is complete when the call returns.  Returns JET_OK
 * when every item succeeded or returned a warning, else the status of the
 * first failed item (each item's own status is in its `status`). */
typedef struct {
    int32_t n;                        /* vertices */
    const int64_t *xadj;              /* device int64[n+1] */
    const int32_t *adjncy;            /* device int32[xadj[n]] */
    const int32_t *vwgt, *adjwgt;     /* device, NULL = unit */
    int32_t k;
    double eps;
    uint64_t seed;
    int32_t *part_out;                /* device int32[n] */
    int64_t cut;                      /* out: cut of part_out */
    int32_t status;                   /* out: the item's jet_partition status */
    float ms;                         /* out: host wall time of the item on its worker */
} jet_batch_item;
int jet_partition_batch(jet_ctx *ctx, int32_t count, jet_batch_item *items, int32_t workers);

/* Autotuner of the execution choices (no counterpart in the paper; results
 * are bit-identical under every choice).  Times `items` (a batch, or one
 * graph with count = 1) with jet_partition_batch under each candidate, one
 * choice (stage) at a time, each stage keeping the best of the earlier ones:
 *   JET_TUNE_CLUSTER_BLOCKS  cluster_blocks in {16, 8, 4, 2} (at cluster_max_n 4096)
 *   JET_TUNE_CLUSTER_MAX_N   cluster_max_n in {0, 1024, 2048, 4096, 8192, 16384} (the largest
 *                            level that runs its whole refinement loop in one cluster launch)
 *   JET_TUNE_WORKERS         workers in {1, 2, 4, 8, 16} (count > 1 only)
 *   JET_TUNE_LIST_BLOCKS     list_blocks_per_sm in {2, 4, 8}
 *   JET_TUNE_APPLY_BLOCKS    apply_blocks_per_sm in {1, 2, 4}
 *   JET_TUNE_LIST_ITEMS      list_items_per_block in {32, 64, 128}
 *   JET_TUNE_SCAN_BLOCKS     scan_blocks_per_sm in {4, 8, 16}
 *   JET_TUNE_HUB_DEGREE      hub_degree in {256, 1024, 4096} (the degree threshold of the
 *                            block-per-row schedule)
 * — taking the median of `reps` timed runs (reps <= 0: 3) after one untimed
 * run, and writes every chosen option into the context's options.  The
 * items' outputs hold the last run's results.  report (may be NULL) lists
 * every candidate. */
#define JET_TUNE_MAX_CAND 48
#define JET_TUNE_CLUSTER_BLOCKS 0
#define JET_TUNE_CLUSTER_MAX_N 1
#define JET_TUNE_WORKERS 2
#define JET_TUNE_LIST_BLOCKS 3
#define JET_TUNE_APPLY_BLOCKS 4
#define JET_TUNE_LIST_ITEMS 5
#define JET_TUNE_SCAN_BLOCKS 6
#define JET_TUNE_HUB_DEGREE 7
typedef struct {
    /* chosen values (all but workers are now in the context's options) */
    int32_t cluster_max_n, cluster_blocks, workers;
    int32_t list_blocks_per_sm, apply_blocks_per_sm, list_items_per_block, scan_blocks_per_sm, hub_degree;
    int32_t ncand;                          /* candidates timed */
    int32_t cand_stage[JET_TUNE_MAX_CAND];  /* JET_TUNE_* of the stage */
    int32_t cand_value[JET_TUNE_MAX_CAND];  /* the value timed */
    float cand_ms[JET_TUNE_MAX_CAND];       /* median host wall time of the whole batch */
} jet_tune_report;
int jet_autotune(jet_ctx *ctx, int32_t count, jet_batch_item *items, int32_t reps, jet_tune_report *report);

/* --- single passes (for composition and per-pass checks) ---------------- */

/* Cost (Sec. 2.1) and part weights of `part`.  pw_out: device int64[k] or
 * NULL. */
int jet_cut(jet_ctx *ctx, int32_t n, const int64_t *xadj, const int32_t *adjncy,
            const int32_t *vwgt, const int32_t *adjwgt, int32_t k, const int32_t *part,
            int64_t *cut_out, int64_t *pw_out);

/* One Jetlp pass (Alg. 4) on `part` with lock set `locked` (device uint8[n],
 * nonzero = locked; NULL = none), first-filter ratio c.  Device outputs, each
 * int32/uint8 [n]: pd_out = P_d (P_s where undefined), gain_out = F
 * (INT32_MIN for negative infinity), inx_out = X membership, f2_out = the
 * afterburner gain F2 (0 outside X), inm_out = M membership.  Any output may
 * be NULL.  flags: the JET_FLAG_* ablation bits. */
int jet_lp_pass(jet_ctx *ctx, int32_t n, const int64_t *xadj, const int32_t *adjncy,
                const int32_t *vwgt, const int32_t *adjwgt, int32_t k, const int32_t *part,
                const uint8_t *locked, double c, uint32_t flags, int32_t *pd_out, int32_t *gain_out,
                uint8_t *inx_out, int32_t *f2_out, uint8_t *inm_out);

/* One rebalancing pass on `part`: strong = 0 runs Jetrw (Alg. 5; seed and
 * iter feed its random destination), strong = 1 runs Jetrs (Sec. 4.2.2).
 * dest_out: device int32[n], the new part of each moved vertex, -1 for the
 * others.  loss_out (device int32[n] or NULL): the eviction loss of each
 * candidate, INT32_MIN for non-candidates.  *nmoves_out / *ncand_out: host
 * counts (may be NULL). */
int jet_rebalance_pass(jet_ctx *ctx, int32_t n, const int64_t *xadj, const int32_t *adjncy,
                       const int32_t *vwgt, const int32_t *adjwgt, int32_t k, double eps,
                       int32_t strong, uint64_t seed, int32_t iter, const int32_t *part,
                       int32_t *dest_out, int32_t *loss_out, int64_t *nmoves_out, int64_t *ncand_out);

/* jet_lp_pass without any device allocation.  The paper has no counterpart:
 * this is for callers that cannot let a library allocate device memory — a
 * process whose memory is reserved up front by its own pool, a latency-bound
 * loop in which cudaMalloc/cudaFree would synchronise the device or grow the
 * memory pool, a host framework that only lends memory it owns.  Arguments,
 * outputs and results are those of jet_lp_pass (the JET_FLAG_VALIDATE graph
 * check is not run).
 * Scratch: a fixed device array of about 10 MiB inside the library, sized for
 * n <= JET_NOALLOC_MAX_N vertices; every GPU that loads the library holds it
 * until the process exits.  Larger n is rejected with JET_EINVAL (see
 * jet_last_error).  The first call on each device looks up the array's
 * device address (cudaGetSymbolAddress); make that first call before any
 * stream capture.  Like every call of this library it reads two counts back
 * to the host and synchronises the context's stream before it returns.  All
 * calls share the one array, which keeps the previous call's contents (the
 * pass clears what must start at zero): calls that can overlap on the GPU —
 * from several contexts, streams or host threads on the same device — race
 * and must be serialised by the caller.  No cudaMalloc, cudaFree or
 * allocating library routine is called (jet_alloc_count does not move). */
#define JET_NOALLOC_MAX_N 262144
int jet_lp_pass_noalloc(jet_ctx *ctx, int32_t n, const int64_t *xadj, const int32_t *adjncy,
                        const int32_t *vwgt, const int32_t *adjwgt, int32_t k, const int32_t *part,
                        const uint8_t *locked, double c, uint32_t flags, int32_t *pd_out, int32_t *gain_out,
                        uint8_t *inx_out, int32_t *f2_out, uint8_t *inm_out);

/* Heavy-edge matching of Sec. 3.1 (handshake rounds, see jet_coarsen) on one
 * graph: mate_out device int32[n] (partner or -1).  level salts the hash. */
int jet_hem(jet_ctx *ctx, int32_t n, const int64_t *xadj, const int32_t *adjncy,
            const int32_t *adjwgt, uint64_t seed, int32_t level, int32_t rounds, int32_t *mate_out);

/* Two-hop matching of Sec. 3.1, applied to a matching (mate_inout: device
 * int32[n], partner or -1, e.g. the output of jet_hem) the way jet_coarsen
 * does after heavy-edge matching when JET_FLAG_TWO_HOP is set: leaves (degree-1 vertices with the same
 * neighbour), then twins (same neighbourhood, identified by an order-free hash
 * of the neighbour ids; isolated vertices included), then relatives (same
 * matchmaker: the lowest-id neighbour that is matched when the stage starts
 * and has degree <= 1024); each stage only while more than 25% of the
 * vertices are unmatched; inside a group, pairs in ascending id.  added_out
 * (host int64[3], may be NULL) receives the vertices each stage matched.
 * Edge weights play no part.  JET_EINVAL for a bad argument. */
int jet_two_hop(jet_ctx *ctx, int32_t n, const int64_t *xadj, const int32_t *adjncy, int32_t *mate_inout,
                int64_t *added_out);

/* InitialPartition of Alg. 1 (the greedy graph growing described at
 * jet_uncoarsen) on one graph: part_out device int32[n]. */
int jet_initial_partition(jet_ctx *ctx, int32_t n, const int64_t *xadj, const int32_t *adjncy,
                          const int32_t *vwgt, int32_t k, int32_t *part_out);

/* Plain pipeline's partition of the coarsest level of `h`: the greedy initial
 * partition refined by Alg. 3 exactly as jet_uncoarsen refines that level
 * (same c, same level seed), without the finer levels.  part_out: device
 * int32[n of the coarsest level].  These are the training labels of the
 * learned initial partition. */
int jet_coarsest_refined(jet_ctx *ctx, const jet_hier *h, int32_t k, double eps, uint64_t seed, int32_t *part_out,
                         int64_t *cut_out);

/* --- learned initial partition (an extension: the paper uses Metis for the
 * initial partition of the coarsest graph, Sec. 3) ----------------------
 *
 * A message-passing network proposes the k-way partition of the coarsest
 * graph; the plain greedy initial partition stays its fallback and the result it must beat.
 *
 * Features (JET_LIP_FEATURES float32 per vertex, each ratio one IEEE float32
 * division of float32-converted integers, the divisor taken as 1 when 0):
 *   1, deg/max deg, vw/max vw, s = S/W, dist/max dist, wdeg/max wdeg,
 *   tri(2^j s) and tri(2^j s + 1/4) for j = 0..4, tri(y) = |2 (y - floor y) - 1|,
 * with S(v) the weight before v and dist(v) the BFS distance in the greedy
 * order of jet_initial_partition, wdeg the sum of v's edge weights.
 * Network (rows are vertices; H0 = features, d0 = 16, d1 = d2 = 64):
 *   A_l = mean of H_{l-1} over the neighbours (0 without neighbours),
 *   H_l = relu([H_{l-1}, A_l] W_l + b_l), l = 1..3, W_l: (2 d_{l-1}) x 64;
 *   logits = H_3 Wo + bo, Wo: 64 x k;  loss = mean cross-entropy of softmax.
 * The dense products run on the tensor cores with bf16 operands (rounded to
 * nearest even from the float32 values) and float32 accumulation; everything
 * else is float32.  Parameters are one float32 vector in the order W1, b1,
 * W2, b2, W3, b3, Wo, bo, matrices row-major (input index first):
 * jet_lip_num_params(k) entries.  Training uses Adam (beta1 0.9, beta2
 * 0.999, epsilon 1e-8) on float32 master parameters. */
#define JET_LIP_FEATURES 16
#define JET_LIP_HIDDEN 64
#define JET_LIP_MAX_K 256
#define JET_LIP_MAX_N (1 << 20)   /* largest coarsest graph the learned proposal is tried on */
typedef struct jet_lip jet_lip;

/* Parameter count for k parts, or -1 for k outside [2, JET_LIP_MAX_K]. */
int64_t jet_lip_num_params(int32_t k);

/* A model for k parts on the context's device, initialised from the HOST
 * array params (jet_lip_num_params(k) floats; the caller draws them).
 * Adam's moments start at zero.  Destroy with jet_lip_destroy. */
int jet_lip_create(jet_ctx *ctx, int32_t k, const float *params, jet_lip **out);
void jet_lip_destroy(jet_lip *m);
/* Copy the parameters to / from a HOST array; setting resets Adam. */
int jet_lip_get_params(jet_ctx *ctx, const jet_lip *m, float *params_out);
int jet_lip_set_params(jet_ctx *ctx, jet_lip *m, const float *params);

/* Input features of one graph: x_out device float32[n * JET_LIP_FEATURES]
 * (row-major).  Edge weights enter wdeg only; vwgt NULL = unit. */
int jet_lip_features(jet_ctx *ctx, int32_t n, const int64_t *xadj, const int32_t *adjncy, const int32_t *vwgt,
                     const int32_t *adjwgt, float *x_out);

/* Canonical labels of a partition: parts renumbered 0, 1, ... by the mean
 * position of their vertices in the greedy order (component, BFS distance,
 * id) — the order the features describe — compared exactly, equal means by
 * part id.  part: device int32[n] in [0, k); labels_out: device int32[n]. */
int jet_lip_labels(jet_ctx *ctx, int32_t n, const int64_t *xadj, const int32_t *adjncy, int32_t k,
                   const int32_t *part, int32_t *labels_out);

/* Forward pass on a graph (or a block-diagonal union of graphs, each row
 * aggregating its own neighbours): x device float32[n * 16], logits_out
 * device float32[n * k] (row-major). */
int jet_lip_forward(jet_ctx *ctx, const jet_lip *m, int32_t n, const int64_t *xadj, const int32_t *adjncy,
                    const float *x, float *logits_out);

/* Mean cross-entropy against labels (device int32[n] in [0, k); JET_EINVAL
 * otherwise) and its gradient: *loss_out host, grad_out device
 * float32[jet_lip_num_params(k)] in parameter order.  Weight gradients are
 * reduced over fixed row blocks in a fixed order: results are bit-identical
 * between runs. */
int jet_lip_loss_grad(jet_ctx *ctx, const jet_lip *m, int32_t n, const int64_t *xadj, const int32_t *adjncy,
                      const float *x, const int32_t *labels, float *loss_out, float *grad_out);

/* One Adam step with learning rate lr on that loss; *loss_out (host, may be
 * NULL) = the loss before the step. */
int jet_lip_train_step(jet_ctx *ctx, jet_lip *m, int32_t n, const int64_t *xadj, const int32_t *adjncy,
                       const float *x, const int32_t *labels, float lr, float *loss_out);

/* Balanced decode of logits (device float32[n * k]): a(v) = argmax (lowest
 * part on ties); margin = largest minus second largest logit (float32);
 * vertices visited by margin descending, then id ascending; a vertex takes
 * a(v) while that part's weight plus its own stays <= cap, else the lightest
 * part (lowest id on ties).  Logits must be finite.  part_out device int32[n]. */
int jet_lip_decode(jet_ctx *ctx, int32_t n, const float *logits, const int32_t *vwgt, int32_t k, int64_t cap,
                   int32_t *part_out);

/* The network's proposal for one graph: features, forward, decode with cap =
 * the balance limit of jet_refine for the model's k and eps. */
int jet_lip_initial_partition(jet_ctx *ctx, const jet_lip *m, int32_t n, const int64_t *xadj, const int32_t *adjncy,
                              const int32_t *vwgt, const int32_t *adjwgt, double eps, int32_t *part_out);

/* Learned form of Alg. 1 for the model's k: one jet_coarsen, the network's
 * proposal for the coarsest level, then jet_uncoarsen twice on that
 * hierarchy, concurrently (the second on a context and stream of its own):
 * from the greedy initial partition (the plain result, identical to
 * jet_partition's) and from the proposal.  The proposal's result is kept iff it is balanced while the plain
 * one is not, or both are alike in balance and its exactly computed cut is
 * <= the plain cut.  The proposal is skipped (plain kept) when the coarsest
 * level has more than JET_LIP_MAX_N vertices.  stats (may be NULL) describe
 * the kept run, with ms_total = the whole call; info (may be NULL) both. */
typedef struct {
    int64_t cut_plain, cut_learned;     /* cut_learned = -1 when the proposal was skipped */
    int32_t status_plain, status_learned;
    int32_t chosen;                     /* 1 learned kept, 0 plain kept */
    int32_t n_coarsest;
    float ms_coarsen, ms_plain, ms_proposal, ms_learned; /* CUDA-event times of the phases (the plain and
                                                          the learned uncoarsening overlap) */
} jet_learned_info;
int jet_partition_learned(jet_ctx *ctx, const jet_lip *m, int32_t n, const int64_t *xadj, const int32_t *adjncy,
                          const int32_t *vwgt, const int32_t *adjwgt, double eps, uint64_t seed, int32_t *part_out,
                          int64_t *cut_out, jet_stats *stats, jet_learned_info *info);

/* Fault injection on the host (a diagnostic for tests; the paper has no
 * counterpart): the nth device allocation the library attempts from now on
 * (nth >= 1) fails without reaching CUDA, as if the device were out of
 * memory, and the call that made it returns JET_ENOMEM after releasing what
 * it holds; one shot, process-wide.  nth = 0 disarms it.  No GPU state is
 * touched. */
void jet_debug_fail_alloc(int64_t nth);

/* Device allocations the library has made in this process so far (all
 * contexts and threads; every stream-ordered scratch allocation counts one).
 * A diagnostic: the paper has no counterpart. */
int64_t jet_alloc_count(void);

/* Human-readable name of a status code (static storage). */
const char *jet_status_string(int status);

/* Text describing the last failed CUDA call on the calling thread (for
 * diagnostics after JET_ECUDA / JET_ENOMEM; thread-local storage). */
const char *jet_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* JET_H */
