// Batched calls whose sets have different dimensions (include/hca_dbscan.h:
// hca_dbscan_batched with one d per set).  The sets are grouped by d; each group runs one
// segmented pipeline (the set id above the cell key, as for a single d).  A group whose sets
// are consecutive in the caller's buffers runs in place; the sets of any other group are
// gathered into a compact copy by one kernel, and their labels (and core flags) scattered back
// by another.
#include <map>
#include <string.h>

#include "hca_internal.cuh"

namespace hca {

namespace {

bool finite_pos(double x) { return x > 0.0 && x <= 1.7976931348623157e308; }

// dst[j] = src[far(j)] (gather, to_compact = 1) or dst[far(j)] = src[j] (scatter), for the
// compact index j in [0, total): j lies in segment k with compact_start[k] <= j <
// compact_start[k + 1], and far(j) = far_start[k] + (j - compact_start[k]).  Empty segments
// share their start with the next one; the search takes the last segment starting at or
// before j, which is the non-empty one holding j.
template <typename E>
__global__ void __launch_bounds__(256) k_copy_segments(const E *__restrict__ src, E *__restrict__ dst,
                                                       const int64_t *__restrict__ compact_start,
                                                       const int64_t *__restrict__ far_start, int nseg,
                                                       int64_t total, int to_compact) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < total; j += stride) {
        int lo = 0, hi = nseg - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (compact_start[mid] <= j) lo = mid;
            else hi = mid - 1;
        }
        const int64_t far = far_start[lo] + (j - compact_start[lo]);
        if (to_compact) dst[j] = src[far];
        else dst[far] = src[j];
    }
}

template <typename E>
void copy_segments(const void *src, void *dst, const int64_t *d_compact, const int64_t *d_far, int nseg,
                   int64_t total, bool to_compact, cudaStream_t s) {
    if (total <= 0 || nseg <= 0) return;
    const int sms = device_sm_count();
    int64_t blocks = (total + 255) / 256;
    const int64_t cap = (int64_t)(sms > 0 ? sms : 148) * 8;
    if (blocks > cap) blocks = cap;
    k_copy_segments<E><<<(unsigned)blocks, 256, 0, s>>>((const E *)src, (E *)dst, d_compact, d_far, nseg, total,
                                                        to_compact ? 1 : 0);
}

}  // namespace

int group_sets(int32_t n_sets, const int64_t *offsets, const int32_t *d_per_set, const double *eps,
               const int32_t *min_pts, const double *box_mn, const double *box_mx, std::vector<SetGroup> &out) {
    out.clear();
    if (n_sets < 1 || !offsets || !d_per_set || !eps || !min_pts) return HCA_EINVAL;
    if (offsets[0] != 0) return HCA_EINVAL;
    for (int32_t s = 0; s < n_sets; ++s) {
        if (offsets[s + 1] < offsets[s]) return HCA_EINVAL;
        if (d_per_set[s] < 1 || d_per_set[s] > 64) return HCA_EINVAL;
        if (!finite_pos(eps[s]) || min_pts[s] < 1) return HCA_EINVAL;
    }
    if (offsets[n_sets] >= ((int64_t)1 << 31)) return HCA_EINVAL;
    std::map<int, size_t> slot;
    for (int32_t s = 0; s < n_sets; ++s) {
        if (!slot.count(d_per_set[s])) slot[d_per_set[s]] = 0;
    }
    size_t k = 0;
    for (auto &kv : slot) kv.second = k++;
    out.resize(slot.size());
    for (auto &kv : slot) out[kv.second].d = kv.first;
    int64_t elem = 0, box = 0;
    for (int32_t s = 0; s < n_sets; ++s) {
        SetGroup &g = out[slot[d_per_set[s]]];
        const int64_t ns = offsets[s + 1] - offsets[s];
        if (g.sets.empty()) {
            g.first_point = offsets[s];
            g.first_elem = (size_t)elem;
            g.off.push_back(0);
        }
        g.sets.push_back(s);
        g.off.push_back(g.off.back() + ns);
        g.eps.push_back(eps[s]);
        g.min_pts.push_back(min_pts[s]);
        g.far_pts.push_back(elem);
        g.far_lab.push_back(offsets[s]);
        if (box_mn && box_mx) {
            g.box_mn.insert(g.box_mn.end(), box_mn + box, box_mn + box + g.d);
            g.box_mx.insert(g.box_mx.end(), box_mx + box, box_mx + box + g.d);
        }
        elem += ns * g.d;
        box += g.d;
    }
    for (SetGroup &g : out) {
        g.gather = (int64_t)(g.sets.back() - g.sets.front()) + 1 != (int64_t)g.sets.size();
        g.n = g.off.back();
    }
    return HCA_OK;
}

size_t group_gather_bytes(const SetGroup &g, int32_t dtype, bool with_core) {
    const size_t esz = dtype == HCA_F32 ? 4 : 8;
    const size_t k = g.sets.size();
    auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
    return al((size_t)g.n * g.d * esz) + al((size_t)g.n * 4) + (with_core ? al((size_t)g.n) : 0) +
           al(sizeof(int64_t) * (4 * k + 2));
}

void group_gather_layout(const SetGroup &g, int32_t dtype, bool with_core, void *buf, GroupBuffers &gb) {
    const size_t esz = dtype == HCA_F32 ? 4 : 8;
    auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
    char *b = (char *)buf;
    gb.points = b;
    b += al((size_t)g.n * g.d * esz);
    gb.labels = (int32_t *)b;
    b += al((size_t)g.n * 4);
    gb.core = nullptr;
    if (with_core) {
        gb.core = (uint8_t *)b;
        b += al((size_t)g.n);
    }
    gb.table = (int64_t *)b;
}

// The segment table of a gathered group: compact point-element starts (k + 1), far
// point-element starts (k), compact label starts (k + 1), far label starts (k).
void group_table(const SetGroup &g, std::vector<int64_t> &t) {
    const size_t k = g.sets.size();
    t.assign(4 * k + 2, 0);
    for (size_t i = 0; i <= k; ++i) t[i] = g.off[i] * g.d;
    for (size_t i = 0; i < k; ++i) t[k + 1 + i] = g.far_pts[i];
    for (size_t i = 0; i <= k; ++i) t[2 * k + 1 + i] = g.off[i];
    for (size_t i = 0; i < k; ++i) t[3 * k + 2 + i] = g.far_lab[i];
}

void group_gather(const SetGroup &g, int32_t dtype, const void *d_points, const GroupBuffers &gb, cudaStream_t s) {
    const int k = (int)g.sets.size();
    const int64_t *t = gb.table;
    if (dtype == HCA_F32)
        copy_segments<uint32_t>(d_points, gb.points, t, t + k + 1, k, g.n * g.d, true, s);
    else
        copy_segments<unsigned long long>(d_points, gb.points, t, t + k + 1, k, g.n * g.d, true, s);
}

void group_scatter(const SetGroup &g, const GroupBuffers &gb, int32_t *d_labels, uint8_t *d_core, cudaStream_t s) {
    const int k = (int)g.sets.size();
    const int64_t *t = gb.table + 2 * k + 1;
    copy_segments<uint32_t>(gb.labels, d_labels, t, t + k + 1, k, g.n, false, s);
    if (d_core && gb.core) copy_segments<uint8_t>(gb.core, d_core, t, t + k + 1, k, g.n, false, s);
}

void add_stats(hca_stats &acc, const hca_stats &x) {
    acc.n_points += x.n_points;
    acc.n_cells += x.n_cells;
    acc.n_pencils += x.n_pencils;
    acc.n_dense_cells += x.n_dense_cells;
    acc.n_core_points += x.n_core_points;
    acc.n_clusters += x.n_clusters;
    acc.n_noise += x.n_noise;
    acc.key_bits = acc.key_bits > x.key_bits ? acc.key_bits : x.key_bits;
    acc.sort_passes += x.sort_passes;
    acc.kernel_launches += x.kernel_launches;
    for (int i = 0; i < HCA_NUM_STAGES; ++i) acc.stage_ms[i] += x.stage_ms[i];
    acc.n_count_chunks += x.n_count_chunks;
    acc.n_rep_tests += x.n_rep_tests;
    acc.n_rep_hits += x.n_rep_hits;
    acc.n_exhaustive_pairs += x.n_exhaustive_pairs;
    acc.n_exhaustive_chunks += x.n_exhaustive_chunks;
    acc.n_border_chunks += x.n_border_chunks;
    acc.n_tc_tiles += x.n_tc_tiles;
    acc.n_tc_rechecks += x.n_tc_rechecks;
    acc.n_core_cells += x.n_core_cells;
    acc.n_tc_pairs += x.n_tc_pairs;
    acc.workspace_bytes += x.workspace_bytes;
    for (int i = 0; i < 3; ++i) acc.tc_ms[i] += x.tc_ms[i];
}

int run_group(const SetGroup &g, const void *d_points, int32_t dtype, int32_t *d_labels, uint8_t *d_core,
              cudaStream_t s, hca_stats *stats, int32_t flags, const hca_tuning &tune) {
    const size_t esz = dtype == HCA_F32 ? 4 : 8;
    if (!g.gather) {
        return batched_tuned((const char *)d_points + g.first_elem * esz, dtype, (int32_t)g.sets.size(),
                             g.off.data(), g.d, g.eps.data(), g.min_pts.data(), d_labels + g.first_point,
                             d_core ? d_core + g.first_point : nullptr, s, stats, flags, tune);
    }
    void *buf = nullptr;
    const bool with_core = d_core != nullptr;
    if (pool_alloc(&buf, group_gather_bytes(g, dtype, with_core), s) != cudaSuccess || !buf) return HCA_ENOMEM;
    GroupBuffers gb;
    group_gather_layout(g, dtype, with_core, buf, gb);
    std::vector<int64_t> t;
    group_table(g, t);
    int rc = HCA_OK;
    // pageable source: the copy has taken the table by the time it returns
    if (cudaMemcpyAsync(gb.table, t.data(), sizeof(int64_t) * t.size(), cudaMemcpyHostToDevice, s) != cudaSuccess)
        rc = HCA_ECUDA;
    if (rc == HCA_OK) {
        group_gather(g, dtype, d_points, gb, s);
        rc = batched_tuned(gb.points, dtype, (int32_t)g.sets.size(), g.off.data(), g.d, g.eps.data(),
                           g.min_pts.data(), gb.labels, gb.core, s, stats, flags, tune);
    }
    if (rc == HCA_OK) {
        group_scatter(g, gb, d_labels, d_core, s);
        if (stats) stats->kernel_launches += with_core ? 3 : 2;
        if (cudaGetLastError() != cudaSuccess) rc = HCA_ECUDA;
    }
    pool_free(buf, s);
    if (rc == HCA_OK && cudaStreamSynchronize(s) != cudaSuccess) rc = HCA_ECUDA;
    return rc;
}

int batched_mixed(const void *d_points, int32_t dtype, int32_t n_sets, const int64_t *offsets,
                  const int32_t *d_per_set, const double *eps, const int32_t *min_pts, int32_t *d_labels,
                  uint8_t *d_core, void *stream, hca_stats *stats, int32_t flags, const hca_tuning *tune_by_d) {
    std::vector<SetGroup> groups;
    int rc = group_sets(n_sets, offsets, d_per_set, eps, min_pts, nullptr, nullptr, groups);
    if (rc) return rc;
    if (dtype != HCA_F32 && dtype != HCA_F64) return HCA_EINVAL;
    if (stats) {
        hca_stats z = {};
        *stats = z;
    }
    const int64_t n = offsets[n_sets];
    if (n == 0) return HCA_OK;
    if (!d_points || !d_labels) return HCA_EINVAL;
    const size_t esz = dtype == HCA_F32 ? 4 : 8;
    if (((uintptr_t)d_points) % esz || ((uintptr_t)d_labels) % 4) return HCA_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    for (const SetGroup &g : groups) {
        if (g.n == 0) continue;
        hca_stats st = {};
        const hca_tuning t = tune_by_d ? tune_by_d[g.d - 1] : tuning_for(g.d);
        rc = run_group(g, d_points, dtype, d_labels, d_core, s, stats ? &st : nullptr, flags, t);
        if (rc) return rc;
        if (stats) add_stats(*stats, st);
    }
    return HCA_OK;
}

}  // namespace hca
