// Tuning table and autotuner (include/hca_dbscan.h: hca_tuning_get / _set, hca_autotune,
// hca_autotune_batched).  The table holds, per dimension d, the neighbour search and the
// tensor-core split used by every clustering call of that d; the autotuner times candidate
// tunings on the caller's data with CUDA events and keeps the fastest.  None of the choices
// changes a label.
#include <float.h>
#include <mutex>
#include <vector>

#include "hca_internal.cuh"

namespace hca {

namespace {

constexpr int kMaxDim = 64;
std::mutex g_tune_mu;
hca_tuning g_tune[kMaxDim + 1];
bool g_tune_init = false;

// Defaults per d: the coarse-grid split measured fastest across the workloads, with first
// links in every cell (leaving them out of tensor-core cells wins a few percent on many small
// sets but loses up to 8x on a set of a million points) — d <= 8: thresholds 16 / 1 / 4;
// d > 8 (the 16-D anisotropic clusters): 8 / 1 / 1.  Tensor-core count chunks hand over at 32
// open rows (the tensor-core recount takes them, in windows: against 8, 5% faster on the d = 8
// sets of the batched workload, 7-14% on the largest d = 9 and 16 serving jobs, equal on the
// 16-D workload).  From one core row on the unions of every
// cell with a core point run on the tensor cores: a cell of one to three core points next to
// a cluster streams the cluster's core points, 128 per tile there against 32 per warp step on
// the CUDA cores.
hca_tuning default_tuning(int d) {
    hca_tuning t = kDefaultTuning;
    if (d <= 8) {
        t.tc_min_count = 16;
        t.tc_min_merge = 1;
        t.tc_min_labels = 4;
        t.first_links = 1;
    } else {
        t.tc_min_count = 8;
        t.tc_min_merge = 1;
        t.tc_min_labels = 1;
        t.first_links = 1;
    }
    return t;
}

void ensure_init() {  // caller holds g_tune_mu
    if (g_tune_init) return;
    for (int d = 0; d <= kMaxDim; ++d) g_tune[d] = default_tuning(d);
    g_tune_init = true;
}

bool valid_tuning(int d, const hca_tuning &t) {
    if (t.path < 0 || t.path > 2) return false;
    if (t.path == 1 && d > 4) return false;
    if (t.path == 2 && d < 3) return false;
    if (t.tc_min_count < 1 || t.tc_min_merge < 1 || t.tc_min_labels < 1) return false;
    if (t.tc_handoff < 0 || t.tc_handoff > 127) return false;
    if (t.first_links != 0 && t.first_links != 1) return false;
    if (t.cta_warps != 2 && t.cta_warps != 4 && t.cta_warps != 8) return false;
    return true;
}

// Candidates for dimension d: the neighbour searches that exist for d, and for the coarse grid
// with float input the first-link choice and six row-threshold sets (counts, unions, labels).
std::vector<hca_tuning> candidates(int d, int32_t dtype) {
    std::vector<hca_tuning> out;
    std::vector<int> paths;
    if (d <= 2) paths = {1};
    else if (d <= 4) paths = {1, 2};
    else paths = {2};
    const int mins[6][3] = {{8, 8, 2}, {32, 8, 2}, {8, 4, 1}, {16, 16, 4}, {8, 1, 1}, {16, 1, 4}};
    for (int path : paths) {
        hca_tuning t = default_tuning(d);
        t.path = path;
        if (path == 1 || dtype != HCA_F32) {
            out.push_back(t);  // nothing else applies
            continue;
        }
        for (int links = 1; links >= 0; --links)
            for (const auto &m : mins) {
                t.first_links = links;
                t.tc_min_count = m[0];
                t.tc_min_merge = m[1];
                t.tc_min_labels = m[2];
                out.push_back(t);
            }
    }
    return out;
}

// Time `run` (one clustering on `s`) under every candidate: one untimed run, then `repeats`
// timed runs, minimum kept.  Then, on the coarse grid, the CTA size of the CUDA-core chunk
// kernels (2 and 8 warps besides the default 4) with the rest of the fastest candidate, and
// with float input the open rows at which a tensor-core count chunk hands over (8, 16, 32, 64).
// Stores the fastest for d.
template <typename Run>
int tune_with(int d, int32_t dtype, cudaStream_t s, int repeats, Run run, hca_tuning *out, double *best_ms) {
    if (repeats < 1 || repeats > 16) return HCA_EINVAL;
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess) return HCA_ECUDA;
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return HCA_ECUDA;
    }
    int rc = HCA_OK;
    double best = DBL_MAX;
    hca_tuning pick = default_tuning(d);
    auto trial = [&](const hca_tuning &t) {
        rc = run(t);
        if (rc) return;
        double tmin = DBL_MAX;
        for (int r = 0; r < repeats && rc == HCA_OK; ++r) {
            cudaEventRecord(e0, s);
            rc = run(t);
            cudaEventRecord(e1, s);
            float ms = 0.f;
            if (rc == HCA_OK && (cudaEventSynchronize(e1) != cudaSuccess ||
                                 cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess))
                rc = HCA_ECUDA;
            if (rc == HCA_OK && ms < tmin) tmin = ms;
        }
        if (rc == HCA_OK && tmin < best) {
            best = tmin;
            pick = t;
        }
    };
    for (const hca_tuning &t : candidates(d, dtype)) {
        trial(t);
        if (rc) break;
    }
    if (rc == HCA_OK && pick.path == 2) {
        const hca_tuning base = pick;
        for (int w : {2, 8}) {
            hca_tuning t = base;
            t.cta_warps = w;
            trial(t);
            if (rc) break;
        }
    }
    if (rc == HCA_OK && pick.path == 2 && dtype == HCA_F32) {
        const hca_tuning base = pick;
        for (int h : {8, 16, 32, 64}) {
            if (h == base.tc_handoff) continue;
            hca_tuning t = base;
            t.tc_handoff = h;
            trial(t);
            if (rc) break;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc) return rc;
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        ensure_init();
        g_tune[d] = pick;
    }
    if (out) *out = pick;
    if (best_ms) *best_ms = best;
    return HCA_OK;
}

}  // namespace

hca_tuning tuning_for(int d) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    ensure_init();
    return (d >= 1 && d <= kMaxDim) ? g_tune[d] : default_tuning(d);
}

}  // namespace hca

using namespace hca;

extern "C" int hca_tuning_get(int32_t d, hca_tuning *out) {
    if (d < 1 || d > kMaxDim || !out) return HCA_EINVAL;
    *out = tuning_for(d);
    return HCA_OK;
}

extern "C" int hca_tuning_set(int32_t d, const hca_tuning *t) {
    if (d < 1 || d > kMaxDim) return HCA_EINVAL;
    const hca_tuning v = t ? *t : default_tuning(d);
    if (!valid_tuning(d, v)) return HCA_EINVAL;
    std::lock_guard<std::mutex> lk(g_tune_mu);
    ensure_init();
    g_tune[d] = v;
    return HCA_OK;
}

extern "C" int hca_autotune(const void *d_points, int32_t dtype, int64_t n, int32_t d, double eps,
                            int32_t min_pts, void *stream, int32_t repeats, hca_tuning *out, double *best_ms) {
    // the labels of the trial runs go to a scratch buffer; the arguments are checked by the run
    int rc = check_common(d_points, dtype, n, d, eps, min_pts, d_points);
    if (rc) return rc;
    if (n == 0) return HCA_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    void *lab = nullptr;
    if (pool_alloc(&lab, (size_t)n * 4, s) != cudaSuccess) return HCA_ENOMEM;
    rc = tune_with(d, dtype, s, repeats, [&](const hca_tuning &t) {
        return device_ex_tuned(d_points, dtype, n, d, eps, min_pts, (int32_t *)lab, nullptr, stream, nullptr, 0, t);
    }, out, best_ms);
    pool_free(lab, s);
    cudaStreamSynchronize(s);
    return rc;
}

extern "C" int hca_autotune_batched(const void *d_points, int32_t dtype, int32_t n_sets, const int64_t *offsets,
                                    const int32_t *d_per_set, const double *eps, const int32_t *min_pts,
                                    void *stream, int32_t repeats, hca_tuning *out, double *best_ms) {
    std::vector<SetGroup> groups;
    int rc = group_sets(n_sets, offsets, d_per_set, eps, min_pts, nullptr, nullptr, groups);
    if (rc) return rc;
    const int64_t n = offsets[n_sets];
    rc = check_common(d_points, dtype, n, 1, 1.0, 1, d_points);
    if (rc) return rc;
    if (n == 0) return HCA_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    double total = 0.0;
    for (const SetGroup &g : groups) {
        if (g.n == 0) continue;
        // the labels of the trial runs go to a scratch buffer laid out as the caller's
        void *lab = nullptr;
        if (pool_alloc(&lab, (size_t)n * 4, s) != cudaSuccess) return HCA_ENOMEM;
        hca_tuning pick;
        double ms = 0.0;
        rc = tune_with(g.d, dtype, s, repeats, [&](const hca_tuning &t) {
            return run_group(g, d_points, dtype, (int32_t *)lab, nullptr, s, nullptr, 0, t);
        }, &pick, &ms);
        pool_free(lab, s);
        cudaStreamSynchronize(s);
        if (rc) return rc;
        if (out) out[g.d - 1] = pick;
        total += ms;
    }
    if (best_ms) *best_ms = total;
    return HCA_OK;
}
