/*
 * hca_dbscan.h -- C ABI of the GB300 (sm_103a) HCA-DBSCAN library.
 *
 * HCA-DBSCAN (Mathur, Mehta, Singh; arXiv 1912.00323) clusters points with DBSCAN's
 * definitions (supplement, "The DBSCAN Algorithm", Definitions 1-5) by overlaying a grid of
 * hypercubes whose space diagonal is eps (Sec. 2, Algorithm 1), treating a hypercube that
 * holds at least MINPTS points as core as a whole, comparing representative points of
 * neighbouring hypercubes (Sec. 2, Algorithm 2), and merging hypercubes into clusters
 * (Algorithms 3-4).  Every step runs in this library's CUDA kernels.
 *
 * Result (identical for every entry point that computes labels):
 *   core(p)   iff |{q : dist(p,q) <= eps}| >= min_pts, p itself included (Definitions 1-2);
 *             dist(p,q) <= eps is decided as  fl64(sum_i (x_pi - x_qi)^2) <= fl64(eps*eps)
 *             with the sum taken in double precision in dimension order, which is exact
 *             for coordinates on a binary lattice.
 *   label(p)  core p: the smallest input index of a core point of its cluster (clusters are
 *             the connected components of core points, Definitions 3-5);
 *             non-core p within eps of a core point: the smallest label among those core
 *             points' clusters; otherwise -1 (noise).
 *
 * Conventions shared by all entry points:
 *   - points are row-major n x d (point i occupies elements [i*d, (i+1)*d)), of type float
 *     (HCA_F32) or double (HCA_F64), every coordinate finite;
 *   - labels are int32 in input order; the caller owns every buffer it passes;
 *   - the library owns only its workspace, taken from a library-private stream-ordered
 *     pool of device memory and returned to that pool before each call returns (except the
 *     graph a thread keeps for repeated calls, see hca_dbscan_device);
 *   - "device" entry points take device pointers and a CUDA stream passed as void*
 *     (a cudaStream_t; NULL = legacy default stream); they return once the result is
 *     complete on that stream;
 *   - every entry point returns HCA_OK (0) or a negative HCA_E* code; on a negative code the
 *     output buffers hold no result (they may have been partly written); n = 0 succeeds
 *     without touching any buffer.
 * Limits: 1 <= d <= 64, n < 2^31, 0 < eps finite, min_pts >= 1.  For d <= 4 the grid of
 * hypercubes (extent / (eps / sqrt(d)) cells per dimension) must fit 64-bit cell keys; for
 * d >= 5 the coarse grid (extent / eps cells in each of three dimensions) must fit them
 * (HCA_ERANGE otherwise).
 */
#ifndef HCA_DBSCAN_H
#define HCA_DBSCAN_H

#include <stdint.h>

#if defined(__GNUC__)
#define HCA_API __attribute__((visibility("default")))
#else
#define HCA_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

/* point coordinate types */
#define HCA_F32 0
#define HCA_F64 1

/* return codes */
#define HCA_OK 0
#define HCA_EINVAL (-1)    /* bad argument: n, d, eps, min_pts, dtype, NULL or non-finite input */
#define HCA_ENOMEM (-2)    /* device workspace could not be allocated */
#define HCA_ECUDA (-3)     /* a CUDA runtime call failed */
#define HCA_ERANGE (-4)    /* coordinate extent too large for the cell grid at this eps */
#define HCA_ENOTIMPL (-5)  /* supported by the interface, not by this build (a batched call whose
                              sets need more than 512 neighbour pencils in their union) */
#define HCA_EDEVICE (-6)   /* a kernel's own consistency check tripped (bounded loop limit,
                              full hash table); the outputs hold no result */
#define HCA_ETOOLARGE (-7) /* n above the fixed scratch of hca_radix_sort_pairs_noalloc */
#define HCA_ETIMEDOUT (-8) /* hca_wait: the job did not complete before the deadline */
#define HCA_ECANCELED (-9) /* the job was cancelled (hca_cancel, or the server shut down) */
#define HCA_EBUSY (-10)    /* hca_cancel: the job is already running */

/* largest n accepted by hca_radix_sort_pairs_noalloc */
#define HCA_SORT_NOALLOC_MAX_PAIRS (1 << 18)

/* flags for hca_dbscan_device_ex */
#define HCA_FLAG_TIMING 1     /* record CUDA events around each stage into stats->stage_ms */
#define HCA_FLAG_FP64_ONLY 2  /* decide every distance in FP64 (no FP32 filter); same result */
#define HCA_FLAG_NO_TENSOR_CORES 4  /* d >= 5, float input: compare pairs on the CUDA cores
                                       instead of the tensor-core distance tiles; same result */
#define HCA_FLAG_NO_GRAPH_CACHE 8   /* run the call's launches directly, without the graph
                                       kept for repeated calls (hca_dbscan_device) */

/* stages timed with HCA_FLAG_TIMING (index into hca_stats.stage_ms) */
#define HCA_STAGE_MINMAX 0    /* origin shift: per-dimension min / max (Sec. 2) */
#define HCA_STAGE_BIN 1       /* hypercube coordinates and cell keys (Algorithm 1) */
#define HCA_STAGE_SORT 2      /* radix sort of (key, index) (the pre-sort of Sec. 2) */
#define HCA_STAGE_CELLS 3     /* gather into cell order, run-length cell offsets */
#define HCA_STAGE_HASH 4      /* neighbour lookup table */
#define HCA_STAGE_CORE 5      /* dense cells and exact counts (Definition 2); d <= 4: with the
                                 chunk table of the representative pass */
#define HCA_STAGE_REPS 6      /* representative points (Algorithm 2): the selection kernel alone */
#define HCA_STAGE_MERGE 7     /* merging neighbouring cells, union-find (Algorithm 3) */
#define HCA_STAGE_LABELS 8    /* cluster ids, border and noise points (Algorithm 4) */
#define HCA_NUM_STAGES 9

typedef struct hca_stats {
    int64_t n_points;
    int64_t n_cells;          /* non-empty hypercubes */
    int64_t n_pencils;        /* non-empty lines of cells along the last dimension */
    int64_t n_dense_cells;    /* cells with >= min_pts points */
    int64_t n_core_points;
    int64_t n_clusters;
    int64_t n_noise;
    int32_t key_bits;         /* bits of the packed cell key */
    int32_t sort_passes;      /* 8-bit radix passes */
    int32_t kernel_launches;  /* kernels this call launched */
    int32_t reserved;
    float stage_ms[HCA_NUM_STAGES];
    /* work counters: 32-point chunks compared while counting neighbours (Definition 2),
       representative-point tests and hits (Algorithm 3), cell pairs that needed the
       exhaustive core x core test and its 32-point chunks, chunks compared for border points */
    int64_t n_count_chunks;
    int64_t n_rep_tests;
    int64_t n_rep_hits;
    int64_t n_exhaustive_pairs;
    int64_t n_exhaustive_chunks;
    int64_t n_border_chunks;
    /* d >= 5, float input: 128 x 128 tensor-core distance tiles computed (counts, unions and
       labels together) and the pairs of those tiles that fell in the guard band and were
       decided by the exact predicate */
    int64_t n_tc_tiles;
    int64_t n_tc_rechecks;
    /* d <= 4 (hypercube neighbour search): cells holding at least one core point (the cells
       with representative points, Algorithm 2); 0 on the coarse-grid path */
    int64_t n_core_cells;
    /* d >= 5, float input: point pairs (valid row x valid candidate) of the tensor-core tiles
       computed, and with HCA_FLAG_TIMING the CUDA-event time of the tensor-core kernel of the
       counts, unions and labels (one launch each) */
    int64_t n_tc_pairs;
    float tc_ms[3];
    int32_t reserved2;
    /* device workspace this call took from the library's pool (bytes; at most the bound of
       hca_workspace_bytes) */
    int64_t workspace_bytes;
} hca_stats;

/*
 * hca_dbscan -- cluster host-resident points; labels written to host memory.
 *   points  host, n*d values of `dtype`; read only.
 *   labels  host, n int32; written on success.
 * Copies the points to the device, runs hca_dbscan_device on an internal stream and copies
 * the labels back.  Synchronous.  (Algorithm 4, HYPERCUBE-BASED-ACCELERATED-DBSCAN.)
 */
HCA_API int hca_dbscan(const void *points, int32_t dtype, int64_t n, int32_t d, double eps,
               int32_t min_pts, int32_t *labels);

/*
 * hca_dbscan_device -- cluster device-resident points.
 *   d_points  device, n*d values of `dtype`, 4-byte (F32) or 8-byte (F64) aligned; read only.
 *   d_labels  device, n int32; written on success.
 *   stream    cudaStream_t as void*; all work is ordered on it.
 * Same result as hca_dbscan.  Returns after the labels are complete on `stream`.
 *
 * Repeated calls.  A call measures the points' extents first and builds its grid from them on
 * the host, so it waits for the GPU once before its main launch sequence, which it then
 * enqueues kernel by kernel.  When a host thread makes the same call twice in a row (same
 * device and CUDA context, same buffers, n, d, dtype, eps, min_pts, flags and tuning), the
 * second call also captures that sequence into a CUDA graph, with its measured extents as
 * declared extents (as hca_plan_create does), and later identical calls replay the graph:
 * one graph launch and one synchronisation per call.  The graph recomputes everything from
 * the points in the buffers at each launch, extents check included; points outside the
 * captured extents make that call run again without the graph (and the next repeat captures
 * anew).  The labels are the same either way: the grid origin does not change a label.  The
 * graph and its workspace stay with the thread until it makes a call with other arguments or
 * calls hca_graph_cache_release.  Calls with HCA_FLAG_TIMING or HCA_FLAG_NO_GRAPH_CACHE, and
 * the batched, plan, server and autotuner entry points, never use it.
 */
HCA_API int hca_dbscan_device(const void *d_points, int32_t dtype, int64_t n, int32_t d, double eps,
                      int32_t min_pts, int32_t *d_labels, void *stream);

/*
 * hca_dbscan_device_ex -- hca_dbscan_device with optional extra outputs.
 *   d_core  device, n uint8 (nullable): 1 for core points, 0 otherwise, input order.
 *   stats   host (nullable): counts of the run; stage times when flags has HCA_FLAG_TIMING
 *           (a call replayed from the graph of repeated calls reports the counts, not times).
 *   flags   bitwise OR of HCA_FLAG_*.
 */
HCA_API int hca_dbscan_device_ex(const void *d_points, int32_t dtype, int64_t n, int32_t d, double eps,
                         int32_t min_pts, int32_t *d_labels, uint8_t *d_core, void *stream,
                         hca_stats *stats, int32_t flags);

/*
 * hca_dbscan_batched -- cluster many independent point sets, each with its own dimension,
 * eps and MINPTS, in one call (the paper clusters one set per run; this batching has no
 * counterpart there).
 *   d_points   device, the sets' points concatenated: set s is a row-major n_s x d_per_set[s]
 *              block (n_s = offsets[s+1] - offsets[s]) that starts right after the block of
 *              set s - 1, i.e. at element sum_{t<s} n_t * d_per_set[t].
 *   offsets    host, n_sets + 1 non-decreasing int64 point offsets, offsets[0] = 0; empty sets
 *              are allowed.
 *   d_per_set  host, n_sets dimensions (1..64).
 *   eps, min_pts  host, n_sets values: each set's own parameters (Definitions 1-2).
 *   d_labels   device, offsets[n_sets] int32: set s's labels at [offsets[s], offsets[s+1]),
 *              with cluster ids that are indices WITHIN the set (the values a separate call on
 *              that set returns).
 *   d_core     device, optional core flags (laid out as d_labels); stats host, optional
 *              (totals over the sets; stage times summed over the d groups).
 * The sets of one d go through one pipeline: the set id sits above the cell key (the
 * hypercube key for d <= 4, the coarse-grid key for d >= 5), so one sort, one pencil hash and
 * one launch of each kernel serve every set of that d, and cells never mix sets.  The d groups
 * run one after another on `stream`, each with the tuning of its d; a group whose sets are
 * not consecutive is gathered into library workspace first and its labels scattered back.
 * Returns after the labels are complete on `stream`.
 */
HCA_API int hca_dbscan_batched(const void *d_points, int32_t dtype, int32_t n_sets, const int64_t *offsets,
                               const int32_t *d_per_set, const double *eps, const int32_t *min_pts,
                               int32_t *d_labels, uint8_t *d_core, void *stream, hca_stats *stats,
                               int32_t flags);

/*
 * Request server: asynchronous clustering jobs with continuous batching (the serving form of
 * the library; the paper has no counterpart).  Worker threads, each with its own CUDA stream,
 * repeatedly admit every queued job that fits the device-memory budget (in arrival order),
 * group the admitted jobs by (d, dtype) and cluster each group with one hca_dbscan_batched
 * call; jobs arriving while a batch runs join a later batch, and the workers keep several
 * batches in flight.  A job's result is the same as a separate hca_dbscan call on its points.
 */
typedef struct hca_request {
    const void *points;   /* n*d values of `dtype`, row-major; host or device memory */
    int32_t *labels;      /* n int32 in the same kind of memory; written when the job completes */
    int64_t n;
    int32_t d;
    int32_t dtype;
    double eps;
    int32_t min_pts;
    int32_t on_device;    /* 1: points and labels are device pointers, 0: host pointers */
} hca_request;

typedef struct hca_server hca_server;

/* Start a server on `device` with `workers` worker threads (1..16) and a device-memory budget
 * (bytes charged per job: its points and labels, the hca_workspace_bytes bound of its
 * workspace, and 16 bytes per point plus 1 KB of slack for sharing a call).  A job larger than
 * the whole budget runs alone.  Each worker keeps its staging buffers for the points and labels
 * on the device from batch to batch, and its clustering workspace comes from the library's
 * pool, which keeps freed blocks for the next call; every intermediate (sorted grid,
 * union-find state) stays on the device until the job's labels are copied out.  Within a batch
 * the (d, dtype) groups with the fewest coordinates run first.  The caller keeps every job's
 * buffers alive until the job completes. */
HCA_API int hca_server_create(hca_server **server, int32_t device, int64_t hbm_budget_bytes, int32_t workers);
/* Stop accepting jobs, cancel queued ones (HCA_ECANCELED), finish running ones, free. */
HCA_API int hca_server_destroy(hca_server *server);
/* Queue a job; *ticket identifies it.  Arguments are checked as in hca_dbscan. */
HCA_API int hca_submit(hca_server *server, const hca_request *request, int64_t *ticket);
/* 1: completed successfully; 0: queued or running; negative: the job's error code. */
HCA_API int hca_poll(hca_server *server, int64_t ticket);
/* Wait up to timeout_ms for the job; on completion return its code, store its submit-to-done
 * latency (ms, nullable) and forget the ticket; HCA_ETIMEDOUT if the deadline passed first. */
HCA_API int hca_wait(hca_server *server, int64_t ticket, int64_t timeout_ms, double *latency_ms);
/* Cancel a queued job (HCA_OK); HCA_EBUSY if it is already running. */
HCA_API int hca_cancel(hca_server *server, int64_t ticket);

/*
 * hca_radix_sort_pairs -- stable ascending sort of (key, value) pairs on the device, by key
 * bits [begin_bit, end_bit) (the pre-sort of Sec. 2 is done with this sort on cell keys).
 *   d_keys     device, n keys of key_bytes (4 or 8) bytes, 8-byte aligned; sorted in place.
 *   d_vals     device, n uint32 values; permuted with their keys in place.
 *   begin_bit, end_bit  0 <= begin_bit < end_bit <= 8*key_bytes.
 * Keys whose bits outside the range differ still sort only by the range (stable).
 * Returns after the sort is complete on `stream`.
 */
HCA_API int hca_radix_sort_pairs(void *d_keys, uint32_t *d_vals, int64_t n, int32_t key_bytes,
                         int32_t begin_bit, int32_t end_bit, void *stream);

/*
 * hca_radix_sort_pairs_noalloc -- hca_radix_sort_pairs without allocating device memory.
 * The paper has no counterpart: this entry point serves callers that cannot allocate device
 * memory while they run (a fixed memory budget set at start-up, a framework whose allocator
 * owns all device memory, code that must not risk the synchronisation cudaMalloc / cudaFree
 * can cause).  Same arguments and result as hca_radix_sort_pairs.
 *   n  at most HCA_SORT_NOALLOC_MAX_PAIRS (2^18); larger n returns HCA_ETOOLARGE.
 * Scratch: a fixed array of about 3.1 MiB inside the library (a __device__ variable: the
 * alternate keys and values of 2^18 pairs plus the sort's look-back words), held on every GPU
 * that loads the library until the process exits.  The first call in a CUDA context of a
 * device looks up that array's device address (cudaGetSymbolAddress) and caches it for that
 * context.  A cudaDeviceReset ends the
 * context, and the next call looks the address up again.  Calls no cudaMalloc, cudaFree or
 * other allocating routine.  Synchronous: the call reads the sort's status word back and
 * returns after the sort is complete on `stream`.
 * Every call uses the same array: calls whose work overlaps on the GPU (other streams, other
 * threads, without ordering between them) race and give wrong results; order them.  A call
 * leaves its scratch contents behind; none of them is read by the next call.
 */
HCA_API int hca_radix_sort_pairs_noalloc(void *d_keys, uint32_t *d_vals, int64_t n,
                                         int32_t key_bytes, int32_t begin_bit, int32_t end_bit,
                                         void *stream);

/*
 * Plans: one clustering call (1 <= d <= 64; the tuning of d at creation is fixed into it) whose
 * buffers and point extents are fixed up front, captured once into a CUDA graph and replayed.  The paper has no
 * counterpart; the result is the one hca_dbscan_device / hca_dbscan_batched give.  With the
 * extents declared, the grid, the stencil and the workspace are fixed before the first launch,
 * so a launch never waits for the host: the whole call is one graph launch.
 *   d_points, d_labels, d_core  device buffers bound to the plan (as in hca_dbscan_device_ex;
 *              d_core nullable); the caller may rewrite d_points between launches.
 *   box_min, box_max  host, d values (batched: d_per_set[s] values per set, set after set):
 *              every coordinate of every launch's points must lie in [box_min, box_max]; a
 *              launch whose points do not makes hca_plan_wait return HCA_ERANGE (its labels
 *              are then undefined).  A larger box gives the same labels (the grid origin does
 *              not change a label).
 * A batched plan takes the sets of hca_dbscan_batched (one d per set).  Its d groups are
 * captured one after another into the one graph (gathering and scattering included), so
 * hca_plan_launch is one graph launch for all of them.
 * hca_plan_create[_batched] synchronises (it sizes and allocates the workspace and captures
 * the graph; no kernel runs).  hca_plan_launch enqueues one clustering on `stream` and returns.
 * hca_plan_wait synchronises `stream` and returns the launch's code: HCA_OK, HCA_ERANGE (a
 * point outside its box), HCA_EINVAL (a NaN coordinate) or HCA_EDEVICE; `stats` (nullable)
 * receives its counts (every field but the stage and tensor-core times).
 * Launches of one plan share its workspace: order them (one stream, or wait in between).
 */
typedef struct hca_plan hca_plan;
HCA_API int hca_plan_create(hca_plan **out, const void *d_points, int32_t dtype, int64_t n, int32_t d,
                            double eps, int32_t min_pts, const double *box_min, const double *box_max,
                            int32_t *d_labels, uint8_t *d_core);
HCA_API int hca_plan_create_batched(hca_plan **out, const void *d_points, int32_t dtype, int32_t n_sets,
                                    const int64_t *offsets, const int32_t *d_per_set, const double *eps,
                                    const int32_t *min_pts, const double *box_min,
                                    const double *box_max, int32_t *d_labels, uint8_t *d_core);
HCA_API int hca_plan_launch(hca_plan *plan, void *stream);
HCA_API int hca_plan_wait(hca_plan *plan, void *stream, hca_stats *stats);
HCA_API int hca_plan_destroy(hca_plan *plan);

/*
 * hca_dbscan_literal_device -- the paper's Algorithms 2-4 as printed (an ablation, not DBSCAN),
 * for 1 <= d <= 4.  Hypercubes of side exactly eps / sqrt(d) from the per-dimension minimum
 * (Algorithm 1); per cube and each of the 3^d - 1 directions the representative point closest
 * to the cube's face, edge or corner in that direction, the smallest input index among equally
 * close points (Algorithm 2); neighbouring cubes are the offsets in [-R, R]^d, R =
 * ceil(sqrt(d)), without the cube itself and the corner cubes (Sec. 2, "Depth First Search");
 * two neighbouring cubes join when their representatives of complementary directions are
 * strictly closer than eps in double precision (Algorithm 3); every non-empty cube is in a
 * cluster (no MINPTS, no noise; Algorithm 4).  Labels: the smallest input index of the cluster.
 *   d_points, d_labels, stream  as hca_dbscan_device.
 * HCA_EINVAL for d > 4 or a NaN; HCA_ERANGE when the band indices need more than 64 key bits.
 * Synchronous.  Compare with hca_dbscan_device to see where the printed algorithm departs
 * from DBSCAN.
 */
HCA_API int hca_dbscan_literal_device(const void *d_points, int32_t dtype, int64_t n, int32_t d, double eps,
                                      int32_t *d_labels, void *stream);

/* Free the calling thread's graph of repeated calls and its workspace (hca_dbscan_device), if
 * it holds one; the thread's next calls start over.  HCA_OK.  The paper has no counterpart. */
HCA_API int hca_graph_cache_release(void);

/*
 * Tuning of the neighbour search and of the tensor-core tiles, per dimension d (process-wide,
 * all devices).  The paper has no counterpart: these choose how the same exact result is
 * computed (Sec. 2's hypercube neighbour enumeration, or the coarse grid of the d >= 5 path;
 * which cells use tensor-core tiles), never what is computed.
 *   path           0: by d (hypercube stencil for d <= 4, coarse grid for d >= 5);
 *                  1: hypercube stencil (d <= 4 only); 2: coarse grid (d >= 3 only).
 *   tc_min_count, tc_min_merge, tc_min_labels
 *                  coarse grid, float input: rows of a phase (all points / core points /
 *                  non-core points of a cell) from which that cell's counts / unions / labels
 *                  use tensor-core tiles; >= 1.
 *   tc_handoff     open rows at which a tensor-core count chunk hands them to the CUDA cores;
 *                  0..127.
 *   first_links    1: first-link pass in every coarse cell; 0: only in cells whose unions run
 *                  on the CUDA cores.
 *   cta_warps      coarse grid: warps per CTA of the CUDA-core chunk kernels (counts, first
 *                  links, unions, labels; one 32-point chunk per warp, its rows staged in the
 *                  CTA's shared memory): 2, 4 or 8.
 * Defaults: path 0, tc_handoff 32, first_links 1, cta_warps 4; thresholds 16 / 1 / 4 for
 * d <= 8 and 8 / 1 / 1 for d > 8.
 */
typedef struct hca_tuning {
    int32_t path;
    int32_t tc_min_count;
    int32_t tc_min_merge;
    int32_t tc_min_labels;
    int32_t tc_handoff;
    int32_t first_links;
    int32_t cta_warps;
} hca_tuning;

/* The tuning used for dimension d (1..64); HCA_EINVAL for a bad d or NULL out. */
HCA_API int hca_tuning_get(int32_t d, hca_tuning *out);
/* Set the tuning of dimension d; NULL restores the defaults.  HCA_EINVAL for a bad d or a
 * field out of range (nothing changes).  Takes effect for calls that start afterwards. */
HCA_API int hca_tuning_set(int32_t d, const hca_tuning *t);

/*
 * hca_autotune -- time candidate tunings for dimension d on the caller's device-resident points
 * (same arguments as hca_dbscan_device; the points are only read) and keep the fastest as the
 * tuning of d.  Each candidate runs once untimed and then `repeats` times (1..16) timed with CUDA
 * events on `stream`, keeping its minimum.  Candidates: both neighbour searches for d = 3, 4;
 * for the coarse grid with float input, first links on / off and several row thresholds; then,
 * on the coarse grid, 2 and 8 warps per CTA (cta_warps) with the rest of the fastest of those,
 * and with float input the tensor-core handoff at 8, 16, 32 and 64 open rows (tc_handoff).
 *   out       host, nullable: the tuning kept.   best_ms  host, nullable: its time.
 * Synchronous.  Returns HCA_OK, or the first error of a candidate run (nothing is changed).
 */
HCA_API int hca_autotune(const void *d_points, int32_t dtype, int64_t n, int32_t d, double eps,
                         int32_t min_pts, void *stream, int32_t repeats, hca_tuning *out,
                         double *best_ms);
/* hca_autotune for the sets of a batched call (arguments as hca_dbscan_batched): every d
 * present is tuned on its own sets and keeps its fastest candidate.
 *   out      host, nullable: 64 entries; entry d - 1 receives the tuning kept for each d
 *            present (the other entries are not written).
 *   best_ms  host, nullable: the sum over the d groups of their best times. */
HCA_API int hca_autotune_batched(const void *d_points, int32_t dtype, int32_t n_sets,
                                 const int64_t *offsets, const int32_t *d_per_set, const double *eps,
                                 const int32_t *min_pts, void *stream, int32_t repeats,
                                 hca_tuning *out, double *best_ms);

/*
 * hca_workspace_bytes -- the device memory one clustering call takes from the library's pool:
 * an upper bound for hca_dbscan_device / hca_dbscan_device_ex on n points of dimension d, for
 * any extents, eps and MINPTS, with the tuning of d in effect now and `flags`.  The host entry
 * point hca_dbscan adds its copies of the points and labels (n (d * element size + 4) bytes).
 * A batched call takes, per d group, at most this bound for the group's points plus a few
 * hundred bytes per set (more only through the power-of-two rounding of its hash table, below
 * 16 bytes per point), and a group whose sets are not consecutive also a compact copy of its
 * points, labels and core flags.  The paper has no counterpart: the request server admits jobs
 * by this bound.  Needs no device.
 *   bytes  host, written on success.
 */
HCA_API int hca_workspace_bytes(int64_t n, int32_t d, int32_t dtype, int32_t flags, int64_t *bytes);

/* Static description of a return code; never NULL. */
HCA_API const char *hca_strerror(int code);

/* Library version: major*10000 + minor*100 + patch. */
HCA_API int32_t hca_version(void);

#ifdef __cplusplus
}
#endif

#endif /* HCA_DBSCAN_H */
