// Plans (include/hca_dbscan.h: hca_plan_create, hca_plan_create_batched, hca_plan_launch,
// hca_plan_wait, hca_plan_destroy): one clustering call (either neighbour search, with the
// tuning of its d) whose buffers and point extents are fixed up front, captured once into a
// CUDA graph and replayed.
// With the extents declared, the grids, the stencil and the workspace are known before the
// first launch, so the call never waits for the host and the whole launch sequence is one
// graph; a kernel in the graph checks every launch's points against the declared boxes.
// A batched plan with several dimensions holds one part per d group; each part is captured
// into a graph of its own and the plan's graph chains them as child-graph nodes, so one graph
// launch runs them all in order.
#include <stdlib.h>
#include <string.h>

#include <vector>

#include "hca_internal.cuh"

namespace {

struct PlanPart {
    hca::SetGroup g;                 // the part's sets (a single call: one set, nsets = 0)
    bool batched = false;
    size_t ws_bytes = 0;
    void *ws = nullptr;              // pipeline workspace
    void *gbuf = nullptr;            // gathered copy of the part's sets (gather parts only)
    hca::GroupBuffers gb = {};
    hca::DevCounters *h = nullptr;   // pinned: the counters of the last launch
    void *stage = nullptr;           // pinned: per-set tables the graph copies to the device
    int32_t flags = 0;               // HCA_FLAG_* of the captured call (no timing)
    int launches = 0;                // kernels the captured call launches
    int key_bits = 0;                // bits of its cell keys
};

}  // namespace

struct hca_plan {
    std::vector<PlanPart> parts;
    cudaStream_t cap = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
};

namespace {

void release(hca_plan *p) {
    if (!p) return;
    if (p->exec) cudaGraphExecDestroy(p->exec);
    if (p->graph) cudaGraphDestroy(p->graph);
    for (PlanPart &pt : p->parts) {
        if (p->cap) {
            if (pt.ws) hca::pool_free(pt.ws, p->cap);
            if (pt.gbuf) hca::pool_free(pt.gbuf, p->cap);
        }
        if (pt.h) cudaFreeHost(pt.h);
        if (pt.stage) cudaFreeHost(pt.stage);
    }
    if (p->cap) {
        cudaStreamSynchronize(p->cap);
        cudaStreamDestroy(p->cap);
    }
    delete p;
}

hca::RunArgs part_args(const PlanPart &pt, const void *pts, int32_t *lab, uint8_t *core) {
    hca::RunArgs a;
    a.flags = pt.flags;  // hca_plan_create: 0, the default path (FP32 filter, tensor-core tiles)
    a.d_points = pts;
    a.n = pt.g.n;
    a.d = pt.g.d;
    a.eps = pt.g.eps[0];
    a.min_pts = pt.g.min_pts[0];
    a.d_labels = lab;
    a.d_core = core;
    a.tune = hca::tuning_for(pt.g.d);  // fixed into the graph
    a.box_mn = pt.g.box_mn.data();
    a.box_mx = pt.g.box_mx.data();
    if (pt.batched) {
        a.nsets = (int)pt.g.sets.size();
        a.h_off = pt.g.off.data();
        a.h_eps = pt.g.eps.data();
        a.h_minpts = pt.g.min_pts.data();
    }
    return a;
}

// The points, labels and core flags a part's pipeline works on: the caller's buffers at the
// part's offsets, or the part's gathered copy.
void part_buffers(const PlanPart &pt, const void *d_points, int32_t dtype, int32_t *d_labels, uint8_t *d_core,
                  const void **pts, int32_t **lab, uint8_t **core) {
    const size_t esz = dtype == HCA_F32 ? 4 : 8;
    if (pt.g.gather) {
        *pts = pt.gb.points;
        *lab = pt.gb.labels;
        *core = pt.gb.core;
    } else {
        *pts = (const char *)d_points + pt.g.first_elem * esz;
        *lab = d_labels + pt.g.first_point;
        *core = d_core ? d_core + pt.g.first_point : nullptr;
    }
}

int create(hca_plan **out, const void *d_points, int32_t dtype, bool batched, std::vector<hca::SetGroup> &groups,
           int32_t *d_labels, uint8_t *d_core, int32_t flags) {
    using namespace hca;
    hca_plan *p = new hca_plan();
    int rc = HCA_OK;
    if (cudaStreamCreateWithFlags(&p->cap, cudaStreamNonBlocking) != cudaSuccess) {
        p->cap = nullptr;
        release(p);
        return HCA_ECUDA;
    }
    for (SetGroup &g : groups) {
        if (g.n == 0) continue;  // a d whose sets are all empty has nothing to run
        p->parts.emplace_back();
        PlanPart &pt = p->parts.back();
        pt.g = g;
        pt.batched = batched;
        pt.flags = flags & ~HCA_FLAG_TIMING;
    }
    if (p->parts.empty()) {
        release(p);
        return HCA_EINVAL;
    }
    for (PlanPart &pt : p->parts) {
        const size_t sets = pt.g.sets.size();
        if (pt.g.gather) {
            if (pool_alloc(&pt.gbuf, group_gather_bytes(pt.g, dtype, d_core != nullptr), p->cap) != cudaSuccess ||
                !pt.gbuf) {
                rc = HCA_ENOMEM;
                break;
            }
            group_gather_layout(pt.g, dtype, d_core != nullptr, pt.gbuf, pt.gb);
            std::vector<int64_t> t;
            group_table(pt.g, t);
            if (cudaMemcpyAsync(pt.gb.table, t.data(), sizeof(int64_t) * t.size(), cudaMemcpyHostToDevice,
                                p->cap) != cudaSuccess ||
                cudaStreamSynchronize(p->cap) != cudaSuccess) {
                rc = HCA_ECUDA;
                break;
            }
        }
        const void *pts;
        int32_t *lab;
        uint8_t *core;
        part_buffers(pt, d_points, dtype, d_labels, d_core, &pts, &lab, &core);
        RunArgs a = part_args(pt, pts, lab, core);
        a.ws_query = &pt.ws_bytes;
        rc = dispatch(a, dtype);
        if (rc) break;
        const size_t stage_bytes = 4096 + 256 * 3 + (sizeof(int64_t) + sizeof(GridParams) + 16 * (size_t)pt.g.d) * (sets + 1);
        if (cudaMallocHost((void **)&pt.h, sizeof(DevCounters)) != cudaSuccess ||
            cudaMallocHost(&pt.stage, stage_bytes) != cudaSuccess) {
            pt.h = nullptr;
            rc = HCA_ECUDA;
            break;
        }
        memset(pt.h, 0, sizeof(DevCounters));
        if (pool_alloc(&pt.ws, pt.ws_bytes, p->cap) != cudaSuccess || !pt.ws) {
            rc = HCA_ENOMEM;
            break;
        }
    }
    if (rc == HCA_OK && cudaStreamSynchronize(p->cap) != cudaSuccess) rc = HCA_ECUDA;
    // each part is captured into a graph of its own; the plan's graph runs them as a chain of
    // child-graph nodes, so one graph launch runs every part
    if (rc == HCA_OK && cudaGraphCreate(&p->graph, 0) != cudaSuccess) {
        p->graph = nullptr;
        rc = HCA_ECUDA;
    }
    cudaGraphNode_t prev = nullptr;
    for (PlanPart &pt : p->parts) {
        if (rc) break;
        cudaStream_t s = p->cap;
        if (cudaStreamBeginCapture(s, cudaStreamCaptureModeRelaxed) != cudaSuccess) {
            rc = HCA_ECUDA;
            break;
        }
        if (pt.g.gather) group_gather(pt.g, dtype, d_points, pt.gb, s);
        const void *pts;
        int32_t *lab;
        uint8_t *core;
        part_buffers(pt, d_points, dtype, d_labels, d_core, &pts, &lab, &core);
        RunArgs a = part_args(pt, pts, lab, core);
        a.ws_ext = pt.ws;
        a.ws_ext_bytes = pt.ws_bytes;
        a.h_ext = pt.h;
        a.h_stage = pt.stage;
        a.deferred = true;
        a.stream = s;
        a.launches_out = &pt.launches;
        a.key_bits_out = &pt.key_bits;
        rc = dispatch(a, dtype);
        if (rc == HCA_OK && pt.g.gather) group_scatter(pt.g, pt.gb, d_labels, d_core, s);
        cudaGraph_t g = nullptr;
        const cudaError_t e = cudaStreamEndCapture(s, &g);
        if (rc == HCA_OK && (e != cudaSuccess || !g)) rc = HCA_ECUDA;
        cudaGraphNode_t node = nullptr;
        if (rc == HCA_OK &&
            cudaGraphAddChildGraphNode(&node, p->graph, prev ? &prev : nullptr, prev ? 1 : 0, g) != cudaSuccess)
            rc = HCA_ECUDA;
        if (g) cudaGraphDestroy(g);  // the child node holds its own copy
        prev = node;
    }
    if (rc == HCA_OK && cudaGraphInstantiate(&p->exec, p->graph, 0) != cudaSuccess) rc = HCA_ECUDA;
    cudaGetLastError();
    if (rc != HCA_OK) {
        release(p);
        return rc;
    }
    *out = p;
    return HCA_OK;
}

bool valid_box(const double *mn, const double *mx, size_t count) {
    for (size_t i = 0; i < count; ++i)
        if (!(mn[i] <= mx[i]) || mn[i] != mn[i] || mx[i] != mx[i]) return false;
    return true;
}

}  // namespace

namespace hca {

int plan_create_single(hca_plan **out, const void *d_points, int32_t dtype, int64_t n, int32_t d, double eps,
                       int32_t min_pts, const double *box_min, const double *box_max, int32_t *d_labels,
                       uint8_t *d_core, int32_t flags) {
    if (!out) return HCA_EINVAL;
    *out = nullptr;
    if (!box_min || !box_max) return HCA_EINVAL;
    int rc = check_common(d_points, dtype, n, d, eps, min_pts, d_labels);
    if (rc) return rc;
    if (n == 0) return HCA_EINVAL;
    const size_t esz = dtype == HCA_F32 ? 4 : 8;
    if (((uintptr_t)d_points) % esz || ((uintptr_t)d_labels) % 4) return HCA_EINVAL;
    std::vector<SetGroup> groups(1);
    SetGroup &g = groups[0];
    g.d = d;
    g.sets = {0};
    g.off = {0, n};
    g.eps = {eps};
    g.min_pts = {min_pts};
    g.box_mn.assign(box_min, box_min + d);
    g.box_mx.assign(box_max, box_max + d);
    g.far_pts = {0};
    g.far_lab = {0};
    g.n = n;
    return create(out, d_points, dtype, false, groups, d_labels, d_core, flags);
}

}  // namespace hca

extern "C" int hca_plan_create(hca_plan **out, const void *d_points, int32_t dtype, int64_t n, int32_t d,
                               double eps, int32_t min_pts, const double *box_min, const double *box_max,
                               int32_t *d_labels, uint8_t *d_core) {
    return hca::plan_create_single(out, d_points, dtype, n, d, eps, min_pts, box_min, box_max, d_labels, d_core, 0);
}

extern "C" int hca_plan_create_batched(hca_plan **out, const void *d_points, int32_t dtype, int32_t n_sets,
                                       const int64_t *offsets, const int32_t *d_per_set, const double *eps,
                                       const int32_t *min_pts, const double *box_min, const double *box_max,
                                       int32_t *d_labels, uint8_t *d_core) {
    using namespace hca;
    if (!out) return HCA_EINVAL;
    *out = nullptr;
    if (!box_min || !box_max) return HCA_EINVAL;
    std::vector<SetGroup> groups;
    int rc = group_sets(n_sets, offsets, d_per_set, eps, min_pts, box_min, box_max, groups);
    if (rc) return rc;
    size_t nbox = 0;
    for (int32_t s = 0; s < n_sets; ++s) nbox += (size_t)d_per_set[s];
    if (!valid_box(box_min, box_max, nbox)) return HCA_EINVAL;
    const int64_t n = offsets[n_sets];
    if (dtype != HCA_F32 && dtype != HCA_F64) return HCA_EINVAL;
    if (n == 0 || !d_points || !d_labels) return HCA_EINVAL;
    const size_t esz = dtype == HCA_F32 ? 4 : 8;
    if (((uintptr_t)d_points) % esz || ((uintptr_t)d_labels) % 4) return HCA_EINVAL;
    return create(out, d_points, dtype, true, groups, d_labels, d_core, 0);
}

extern "C" int hca_plan_launch(hca_plan *plan, void *stream) {
    if (!plan || !plan->exec) return HCA_EINVAL;
    return cudaGraphLaunch(plan->exec, (cudaStream_t)stream) == cudaSuccess ? HCA_OK : HCA_ECUDA;
}

extern "C" int hca_plan_wait(hca_plan *plan, void *stream, hca_stats *stats) {
    if (!plan || plan->parts.empty()) return HCA_EINVAL;
    if (cudaStreamSynchronize((cudaStream_t)stream) != cudaSuccess) return HCA_ECUDA;
    if (stats) {
        hca_stats z = {};
        *stats = z;
    }
    int rc = HCA_OK;
    for (const PlanPart &pt : plan->parts) {
        const hca::DevCounters *h = pt.h;
        if (stats) {
            stats->n_points += pt.g.n;
            stats->n_cells += h->n_cells;
            stats->n_pencils += h->n_pencils;
            stats->n_dense_cells += h->n_dense;
            stats->n_core_cells += h->n_core_cells;
            stats->n_core_points += h->n_core;
            stats->n_clusters += h->n_clusters;
            stats->n_noise += h->n_noise;
            if (pt.key_bits > stats->key_bits) {
                stats->key_bits = pt.key_bits;
                stats->sort_passes = (pt.key_bits + 7) / 8;
            }
            stats->kernel_launches += pt.launches;
            stats->n_count_chunks += (int64_t)h->work[0];
            stats->n_rep_tests += (int64_t)h->work[1];
            stats->n_rep_hits += (int64_t)h->work[2];
            stats->n_exhaustive_pairs += (int64_t)h->work[3];
            stats->n_exhaustive_chunks += (int64_t)h->work[4];
            stats->n_border_chunks += (int64_t)h->work[5];
            stats->n_tc_tiles += (int64_t)h->work[6];
            stats->n_tc_rechecks += (int64_t)h->work[7];
            stats->n_tc_pairs += (int64_t)h->tc_pairs;
            stats->workspace_bytes += (int64_t)pt.ws_bytes;
        }
        int r = HCA_OK;
        if (h->nan_seen) r = HCA_EINVAL;
        else if (h->status) r = (h->status & hca::kErrBox) ? HCA_ERANGE : HCA_EDEVICE;
        if (rc == HCA_OK) rc = r;
    }
    return rc;
}

extern "C" int hca_plan_destroy(hca_plan *plan) {
    if (!plan) return HCA_EINVAL;
    release(plan);
    return HCA_OK;
}
