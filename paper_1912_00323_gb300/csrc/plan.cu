// Plans (include/hca_dbscan.h: hca_plan_create, hca_plan_create_batched, hca_plan_launch,
// hca_plan_wait, hca_plan_destroy): one clustering call (either neighbour search, with the
// tuning of its d) whose buffers and point extents are fixed up front, captured once into a
// CUDA graph and replayed.
// With the extents declared, the grids, the stencil and the workspace are known before the
// first launch, so the call never waits for the host and the whole launch sequence is one
// graph; a kernel in the graph checks every launch's points against the declared boxes.
#include <stdlib.h>
#include <string.h>

#include <vector>

#include "hca_internal.cuh"

struct hca_plan {
    std::vector<int64_t> off;
    std::vector<double> eps, box_mn, box_mx;
    std::vector<int32_t> min_pts;
    void *ws = nullptr;
    hca::DevCounters *h = nullptr;  // pinned: the counters of the last launch
    void *stage = nullptr;          // pinned: per-set tables the graph copies to the device
    cudaStream_t cap = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
};

namespace {

void release(hca_plan *p) {
    if (!p) return;
    if (p->exec) cudaGraphExecDestroy(p->exec);
    if (p->graph) cudaGraphDestroy(p->graph);
    if (p->ws && p->cap) {
        hca::pool_free(p->ws, p->cap);
        cudaStreamSynchronize(p->cap);
    }
    if (p->cap) cudaStreamDestroy(p->cap);
    if (p->h) cudaFreeHost(p->h);
    if (p->stage) cudaFreeHost(p->stage);
    delete p;
}

int create(hca_plan **out, const void *d_points, int32_t dtype, int32_t n_sets, int64_t n, int32_t d,
           const double *eps, const int32_t *min_pts, const int64_t *offsets, const double *box_min,
           const double *box_max, int32_t *d_labels, uint8_t *d_core) {
    using namespace hca;
    if (!out || !box_min || !box_max || !eps || !min_pts) return HCA_EINVAL;
    *out = nullptr;
    if (d < 1 || d > 64) return HCA_EINVAL;
    int rc = check_common(d_points, dtype, n, d, eps[0], min_pts[0], d_labels);
    if (rc) return rc;
    if (n == 0) return HCA_EINVAL;
    const size_t esz = dtype == HCA_F32 ? 4 : 8;
    if (((uintptr_t)d_points) % esz || ((uintptr_t)d_labels) % 4) return HCA_EINVAL;
    hca_plan *p = new hca_plan();
    const int sets = n_sets > 0 ? n_sets : 1;
    p->eps.assign(eps, eps + sets);
    p->min_pts.assign(min_pts, min_pts + sets);
    p->box_mn.assign(box_min, box_min + (size_t)sets * d);
    p->box_mx.assign(box_max, box_max + (size_t)sets * d);
    if (n_sets > 0) p->off.assign(offsets, offsets + n_sets + 1);
    RunArgs a;
    a.d_points = d_points;
    a.n = n;
    a.d = d;
    a.eps = p->eps[0];
    a.min_pts = p->min_pts[0];
    a.d_labels = d_labels;
    a.d_core = d_core;
    a.tune = tuning_for(d);  // fixed into the graph
    a.box_mn = p->box_mn.data();
    a.box_mx = p->box_mx.data();
    if (n_sets > 0) {
        a.nsets = n_sets;
        a.h_off = p->off.data();
        a.h_eps = p->eps.data();
        a.h_minpts = p->min_pts.data();
    }
    size_t bytes = 0;
    a.ws_query = &bytes;
    rc = dispatch(a, dtype);
    a.ws_query = nullptr;
    const size_t stage_bytes = 4096 + 256 * 3 + (sizeof(int64_t) + sizeof(GridParams) + 16 * (size_t)d) * (sets + 1);
    if (rc == HCA_OK && (cudaStreamCreateWithFlags(&p->cap, cudaStreamNonBlocking) != cudaSuccess ||
                         cudaMallocHost((void **)&p->h, sizeof(DevCounters)) != cudaSuccess ||
                         cudaMallocHost(&p->stage, stage_bytes) != cudaSuccess))
        rc = HCA_ECUDA;
    if (rc == HCA_OK && (pool_alloc(&p->ws, bytes, p->cap) != cudaSuccess || !p->ws)) rc = HCA_ENOMEM;
    if (rc == HCA_OK && cudaStreamSynchronize(p->cap) != cudaSuccess) rc = HCA_ECUDA;
    if (rc == HCA_OK) {
        memset(p->h, 0, sizeof(DevCounters));
        a.ws_ext = p->ws;
        a.ws_ext_bytes = bytes;
        a.h_ext = p->h;
        a.h_stage = p->stage;
        a.deferred = true;
        a.stream = p->cap;
        if (cudaStreamBeginCapture(p->cap, cudaStreamCaptureModeRelaxed) != cudaSuccess) {
            rc = HCA_ECUDA;
        } else {
            rc = dispatch(a, dtype);
            cudaGraph_t g = nullptr;
            const cudaError_t e = cudaStreamEndCapture(p->cap, &g);
            p->graph = g;
            if (rc == HCA_OK && (e != cudaSuccess || !g)) rc = HCA_ECUDA;
            if (rc == HCA_OK && cudaGraphInstantiate(&p->exec, p->graph, 0) != cudaSuccess) rc = HCA_ECUDA;
        }
    }
    cudaGetLastError();
    if (rc != HCA_OK) {
        release(p);
        return rc;
    }
    *out = p;
    return HCA_OK;
}

}  // namespace

extern "C" int hca_plan_create(hca_plan **out, const void *d_points, int32_t dtype, int64_t n, int32_t d,
                               double eps, int32_t min_pts, const double *box_min, const double *box_max,
                               int32_t *d_labels, uint8_t *d_core) {
    return create(out, d_points, dtype, 0, n, d, &eps, &min_pts, nullptr, box_min, box_max, d_labels, d_core);
}

extern "C" int hca_plan_create_batched(hca_plan **out, const void *d_points, int32_t dtype, int32_t n_sets,
                                       const int64_t *offsets, int32_t d, const double *eps, const int32_t *min_pts,
                                       const double *box_min, const double *box_max, int32_t *d_labels,
                                       uint8_t *d_core) {
    if (n_sets < 1 || !offsets || !eps || !min_pts || offsets[0] != 0) return HCA_EINVAL;
    for (int32_t i = 0; i < n_sets; ++i) {
        if (offsets[i + 1] < offsets[i]) return HCA_EINVAL;
        if (!(eps[i] > 0.0) || eps[i] != eps[i] || eps[i] > 1.7e308 || min_pts[i] < 1) return HCA_EINVAL;
    }
    return create(out, d_points, dtype, n_sets, offsets[n_sets], d, eps, min_pts, offsets, box_min, box_max,
                  d_labels, d_core);
}

extern "C" int hca_plan_launch(hca_plan *plan, void *stream) {
    if (!plan || !plan->exec) return HCA_EINVAL;
    return cudaGraphLaunch(plan->exec, (cudaStream_t)stream) == cudaSuccess ? HCA_OK : HCA_ECUDA;
}

extern "C" int hca_plan_wait(hca_plan *plan, void *stream, hca_stats *stats) {
    if (!plan || !plan->h) return HCA_EINVAL;
    if (cudaStreamSynchronize((cudaStream_t)stream) != cudaSuccess) return HCA_ECUDA;
    const hca::DevCounters *h = plan->h;
    if (stats) {
        hca_stats z = {};
        *stats = z;
        stats->n_cells = h->n_cells;
        stats->n_pencils = h->n_pencils;
        stats->n_dense_cells = h->n_dense;
        stats->n_core_cells = h->n_core_cells;
        stats->n_core_points = h->n_core;
        stats->n_clusters = h->n_clusters;
        stats->n_noise = h->n_noise;
    }
    if (h->nan_seen) return HCA_EINVAL;
    if (h->status) return (h->status & hca::kErrBox) ? HCA_ERANGE : HCA_EDEVICE;
    return HCA_OK;
}

extern "C" int hca_plan_destroy(hca_plan *plan) {
    if (!plan) return HCA_EINVAL;
    release(plan);
    return HCA_OK;
}
