// Internal declarations shared by the CUDA translation units of the HCA-DBSCAN library.
// Nothing here is part of the public ABI (include/hca_dbscan.h).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "../../include/hca_dbscan.h"

namespace hca {

constexpr int kMaxD = 4;            // dimensions handled by the hypercube-stencil path
constexpr int kMaxPencils = 512;    // neighbour pencil offsets per cell (d = 4 needs 179)
constexpr int kWarp = 32;
constexpr uint64_t kEmptyKey = ~0ull;
constexpr uint32_t kNoLabel = 0x7fffffffu;
constexpr uint32_t kLoopLimit = 1u << 22;  // cap of every loop that reads concurrently written data

// device-side status word bits (HCA_EDEVICE when non-zero)
constexpr uint32_t kErrHashFull = 1u;
constexpr uint32_t kErrLoop = 2u;
constexpr uint32_t kErrBox = 8u;   // a point lies outside the extents a plan declared

// Base tuning (include/hca_dbscan.h): dimension-chosen neighbour search; tensor-core tiles
// from 8 rows (counts, unions) and 2 non-core rows (labels); hand-off at 8 open count rows;
// first links everywhere.  The defaults per d (tune.cu) adjust the split from it.
constexpr hca_tuning kDefaultTuning = {0, 8, 8, 2, 32, 1, 4};

// Device counters and status, one struct per call in the workspace.
struct DevCounters {
    uint32_t n_cells;      // C: non-empty cells
    uint32_t n_pencils;    // P: non-empty pencils (cells sharing all but the last coordinate)
    uint32_t hash_mask;    // capacity - 1 of the pencil hash table
    uint32_t status;       // kErr* bits
    uint32_t n_dense;
    uint32_t n_core;
    uint32_t n_clusters;
    uint32_t n_noise;
    uint32_t n_core_cells;  // cells holding a core point (hypercube path)
    uint32_t n_list[3];     // hypercube path: cells to count, cells with core points, cells to label
    uint64_t minmax_enc[2 * kMaxD];  // order-preserving encodings of min (first kMaxD) / max per dim
    uint32_t nan_seen;
    uint32_t n_chunks;     // 32-point chunks of the coarse cells (high-dimensional path)
    uint32_t n_tc_chunks[4];  // work items of the tensor-core phases: counts, unions (the first window of
                              // every 128-row chunk), labels; [3]: the unions' other windows
    uint32_t tc_next[3];      // next unclaimed item of each tensor-core phase
    uint32_t n_tc_recount;    // chunks of the tensor-core recount of handed-over rows
    uint32_t tc_next_recount;
    uint32_t hd_next[4];      // next unclaimed 32-point chunk: counts, first links, unions, labels
    uint32_t lowd_next[5];    // next unclaimed batch (labels: [4])
    unsigned long long work[8];  // work counters (see hca_stats)
    unsigned long long tc_pairs;  // point pairs of the tensor-core tiles computed
    uint32_t digit_counts[8 * 256];  // radix digit counts per pass, filled while binning
};

// Grid of hypercubes (Algorithm 1) and everything a kernel needs to bin, pack and compare.
struct GridParams {
    int d;
    int64_t n;
    double origin[kMaxD];        // per-dimension minimum (origin shift, Sec. 2)
    float origin_f[kMaxD];
    double inv_side;             // 1 / cell side (cells per unit length)
    float inv_side_f;
    uint32_t ncell[kMaxD];       // cells per dimension
    uint32_t shift[kMaxD];       // bit offset of each coordinate in the packed key
    uint32_t bits[kMaxD];
    int key_bits;
    int prefix_shift;            // key >> prefix_shift = pencil key (all but the last coordinate)
    uint32_t min_pts;
    double eps2;                 // fl64(eps * eps): the exact predicate's threshold
    float lo32, hi32;            // FP32 filter: s < lo32 => within, s > hi32 => outside
    int bin_fp64;                // bin FP32 input in double precision
    int box_ok;                  // band coordinates exact enough in FP32 for cell-box tests
    float tau_box;               // widening of a cell box, band units
    float box_full, box_none;    // eps^2 in band units^2 times (1 -/+ 2^-12)
    int sel[3];                  // coarse-grid path: the three projected input dimensions
};

// Neighbour pencils: offsets of the first d-1 coordinates and the reach along the last one.
// Full list (every neighbour) and the upper half (pairs counted once) share the table:
// entries [0, n_half) are the offsets that are lexicographically >= 0.
struct Stencil {
    int n_all;
    int n_half;
    int8_t off[kMaxPencils][kMaxD - 1 > 0 ? kMaxD - 1 : 1];
    int8_t reach[kMaxPencils];   // max |delta_last| that can hold a point within eps
    uint16_t near[kMaxPencils];  // all pencils, nearest offsets first (counting order)
};

template <typename T, int D>
struct PadDim {
    static constexpr int value = (D == 3) ? 4 : D;
};

template <typename T, int D>
struct alignas(sizeof(T) * PadDim<T, D>::value) Pt {
    T x[PadDim<T, D>::value];
};

// Workspace carved out of one pool allocation per call.
struct Workspace {
    void *base;
    size_t bytes;
};

// ---------------------------------------------------------------------------------------
// Primitives implemented in sort.cu / scan.cu
// ---------------------------------------------------------------------------------------

// Exclusive scan of uint32 in[0, m) into out[0, m); total into *total (device, may be null).
// If m_dev is non-null the length is min(*m_dev, m_max); elements past it are left untouched.
// partials: device scratch of scan_partials_size(m_max) uint32.
size_t scan_partials_size(int64_t m_max);
void exclusive_scan_u32(const uint32_t *in, uint32_t *out, int64_t m_max, const uint32_t *m_dev,
                        uint32_t *total, uint32_t *partials, cudaStream_t s, int *launches);

// Elements per tile of the scan (the tile sums in `partials` are per this many elements).
constexpr int kScanTileElems = 2048;

// Run-length cells from first-of-cell flags (1 on the first point of every cell, points in
// cell order).  The kernel that wrote the flags also wrote the sum of every kScanTileElems-flag
// tile into partials[tile] (tiles = ceil(n / kScanTileElems)).  Scans those sums (the total,
// the cell count, into *n_cells), then per point replaces the flag by the point's cell id and
// writes the first point and the key of every cell, and cell_start[n_cells] = n.
// partials: scan_partials_size(n) uint32.  Two launches.
template <typename K>
void cells_from_flags(const K *keys, uint32_t *flags_cell_of, int64_t n, uint32_t *partials, uint32_t *n_cells,
                      uint32_t *cell_start, uint64_t *cell_key, cudaStream_t s, int *launches);

// Geometry of the onesweep radix sort (sort.cu): keys per tile, digits per pass, and the
// most passes a call can make.  The scratch of a sort of n pairs is sort_hist_elems(n)
// uint32: two words per tile and digit for the look-back, the digit counts of every pass,
// one ticket per pass and a status word.
constexpr int kSortTileKeys = 13312;
constexpr int kSortRadix = 256;
constexpr int kSortMaxPasses = 8;
constexpr int64_t sort_tiles_for(int64_t n) {
    return n <= kSortTileKeys ? 1 : (n + kSortTileKeys - 1) / kSortTileKeys;
}
constexpr size_t sort_hist_elems(int64_t n) {
    return (size_t)(2 * sort_tiles_for(n) * kSortRadix + kSortMaxPasses * kSortRadix + kSortMaxPasses + 2);
}

// LSD radix sort of (key, value) pairs by bits [begin_bit, end_bit), 8 bits per pass.
// Ping-pongs between (keys, vals) and (keys_alt, vals_alt); returns true when the sorted
// result ends up in the alternate buffers.  hist: sort_hist_size(n) uint32 of scratch
// (8-byte aligned; cleared by the sort itself).  A bounded look-back wait that ran out sets
// bit 2 of *err_out (device word; NULL: the status word inside hist, sort_status_word).
// `partials` is not used by the sort (callers may pass NULL).
inline size_t sort_hist_size(int64_t n) { return sort_hist_elems(n); }
uint32_t *sort_status_word(uint32_t *hist, int64_t n);
// digit_counts (optional, device): counts of every 8-bit digit of every pass, [pass][256],
// already computed by the caller.
template <typename K>
bool radix_sort_pairs(K *keys, uint32_t *vals, K *keys_alt, uint32_t *vals_alt, int64_t n,
                      int begin_bit, int end_bit, uint32_t *hist, uint32_t *partials,
                      cudaStream_t s, int *launches, uint32_t *err_out = nullptr,
                      const uint32_t *digit_counts = nullptr);

// Pool allocation (stream ordered) used by api.cu and the pipelines.
cudaError_t pool_alloc(void **p, size_t bytes, cudaStream_t s);
cudaError_t pool_free(void *p, cudaStream_t s);

int device_sm_count();

// Host orchestration of one clustering call, instantiated per (T, D) in lowd_*.cu.
struct RunArgs {
    const void *d_points = nullptr;
    int64_t n = 0;
    int d = 0;
    double eps = 0.0;
    int min_pts = 0;
    int32_t *d_labels = nullptr;
    uint8_t *d_core = nullptr;
    cudaStream_t stream = nullptr;
    hca_stats *stats = nullptr;
    int flags = 0;
    // batched calls (n_sets > 0): sets of consecutive points, each with its own eps and MINPTS
    int nsets = 0;
    const int64_t *h_off = nullptr;      // host, nsets + 1 point offsets
    const double *h_eps = nullptr;       // host, nsets
    const int32_t *h_minpts = nullptr;   // host, nsets
    hca_tuning tune = kDefaultTuning;    // neighbour search and tensor-core split of this call
    // Plans (d <= 4): declared extents box_mn / box_mx (host, D values per set, set-major) size
    // the grids instead of the measured ones, so nothing in the call waits for the host; a
    // device kernel flags a point outside its box (status kErrBox).
    const double *box_mn = nullptr, *box_mx = nullptr;
    size_t *ws_query = nullptr;          // set: store the workspace bytes needed, launch nothing
    void *ws_ext = nullptr;              // caller-owned workspace (nullptr: the call allocates)
    size_t ws_ext_bytes = 0;
    DevCounters *h_ext = nullptr;        // pinned host copy of the counters (nullptr: the thread's)
    void *h_stage = nullptr;             // pinned staging of the batched tables (deferred calls)
    bool deferred = false;               // no host synchronisation: the caller checks the status
    // optional outputs: the measured extents of a single-set call without declared extents
    // (host, 2 d values: d minima then d maxima), and the launch count and key bits of the call
    double *ext_out = nullptr;
    int *launches_out = nullptr;
    int *key_bits_out = nullptr;
};

// The tuning in effect for dimension d (tune.cu).
hca_tuning tuning_for(int d);

// The unique id of the calling thread's current CUDA context, 0 when there is none or the
// driver cannot say (sort_static.cu).
unsigned long long current_context_id();

// A plan of one set with the given flags (plan.cu; hca_plan_create is this with flags 0).
int plan_create_single(hca_plan **out, const void *d_points, int32_t dtype, int64_t n, int32_t d, double eps,
                       int32_t min_pts, const double *box_min, const double *box_max, int32_t *d_labels,
                       uint8_t *d_core, int32_t flags);

// api.cu: argument checks, dispatch to the pipelines, and the clustering calls with an
// explicit tuning.
int dispatch(const RunArgs &a, int32_t dtype);
int check_common(const void *pts, int32_t dtype, int64_t n, int32_t d, double eps, int32_t min_pts,
                 const void *labels);
int device_ex_tuned(const void *d_points, int32_t dtype, int64_t n, int32_t d, double eps, int32_t min_pts,
                    int32_t *d_labels, uint8_t *d_core, void *stream, hca_stats *stats, int32_t flags,
                    const hca_tuning &tune, double *ext_out = nullptr);
int batched_tuned(const void *d_points, int32_t dtype, int32_t n_sets, const int64_t *offsets, int32_t d,
                  const double *eps, const int32_t *min_pts, int32_t *d_labels, uint8_t *d_core, void *stream,
                  hca_stats *stats, int32_t flags, const hca_tuning &tune);
// multi.cu: batched calls with one d per set.  The sets are grouped by d (increasing d); a
// group whose sets are consecutive in the caller's buffers runs in place, any other group is
// gathered into a compact copy (points, labels, core flags, segment table) and scattered back.
struct SetGroup {
    int d = 0;
    std::vector<int32_t> sets;            // the call's set indices, increasing
    std::vector<int64_t> off;             // group-local point offsets (sets + 1)
    std::vector<double> eps;
    std::vector<int32_t> min_pts;
    std::vector<double> box_mn, box_mx;   // declared boxes of the sets, d values each (plans)
    std::vector<int64_t> far_pts;         // element offset of each set in the caller's points
    std::vector<int64_t> far_lab;         // point offset of each set in the caller's labels
    int64_t n = 0;                        // points of the group
    bool gather = false;                  // sets not consecutive: run on a compact copy
    int64_t first_point = 0;              // in place: first set's point offset
    size_t first_elem = 0;                // in place: first set's element offset
};
struct GroupBuffers {
    void *points;
    int32_t *labels;
    uint8_t *core;
    int64_t *table;
};
int group_sets(int32_t n_sets, const int64_t *offsets, const int32_t *d_per_set, const double *eps,
               const int32_t *min_pts, const double *box_mn, const double *box_mx, std::vector<SetGroup> &out);
size_t group_gather_bytes(const SetGroup &g, int32_t dtype, bool with_core);
void group_gather_layout(const SetGroup &g, int32_t dtype, bool with_core, void *buf, GroupBuffers &gb);
void group_table(const SetGroup &g, std::vector<int64_t> &t);
void group_gather(const SetGroup &g, int32_t dtype, const void *d_points, const GroupBuffers &gb, cudaStream_t s);
void group_scatter(const SetGroup &g, const GroupBuffers &gb, int32_t *d_labels, uint8_t *d_core, cudaStream_t s);
void add_stats(hca_stats &acc, const hca_stats &x);
int run_group(const SetGroup &g, const void *d_points, int32_t dtype, int32_t *d_labels, uint8_t *d_core,
              cudaStream_t s, hca_stats *stats, int32_t flags, const hca_tuning &tune);
// tune_by_d: nullable, 64 tunings indexed by d - 1 (NULL: the table of tune.cu)
int batched_mixed(const void *d_points, int32_t dtype, int32_t n_sets, const int64_t *offsets,
                  const int32_t *d_per_set, const double *eps, const int32_t *min_pts, int32_t *d_labels,
                  uint8_t *d_core, void *stream, hca_stats *stats, int32_t flags, const hca_tuning *tune_by_d);

template <typename T, int D>
int run_lowd(const RunArgs &a);
template <typename T, int DP>
int run_hd(const RunArgs &a);

}  // namespace hca

#define HCA_CUDA_TRY(expr)                                    \
    do {                                                      \
        cudaError_t _e = (expr);                              \
        if (_e != cudaSuccess) return HCA_ECUDA;              \
    } while (0)
