// Host orchestration of the high-dimensional path (5 <= d <= 64) for one call.
#pragma once

#include <type_traits>

#include "hd_kernels.cuh"
#include "lowd_run.cuh"
#include "tc_kernels.cuh"

namespace hca {

namespace detail {

// Coarse grid over three projected dimensions with side eps (1 + 2^-10): two points within eps
// differ by at most eps (1 + 2^-50) in every coordinate, and with band coordinates computed in
// FP64 (error tau in band units, tau << 2^-12) they fall in the same or adjacent coarse cells.
inline int make_coarse_grid(bool input_f32, double eps, int min_pts, int64_t n, const double *mn,
                            const double *mx, int flags, GridParams &g, double &tau) {
    memset(&g, 0, sizeof(g));
    g.d = 3;
    g.n = n;
    g.min_pts = (uint32_t)min_pts;
    g.eps2 = eps * eps;
    const double side = eps * (1.0 + ldexp(1.0, -10));
    const double inv = 1.0 / side;
    double range_max = 0.0;
    for (int i = 0; i < 3; ++i) range_max = fmax(range_max, mx[i] - mn[i]);
    if (!isfinite(range_max) || !isfinite(inv)) return HCA_ERANGE;
    tau = (range_max * inv + 1.0) * ldexp(1.0, -51);
    if (tau > ldexp(1.0, -14)) return HCA_ERANGE;
    g.inv_side = inv;
    g.inv_side_f = (float)inv;
    g.bin_fp64 = 1;
    int total = 0;
    for (int i = 0; i < 3; ++i) {
        g.origin[i] = mn[i];
        g.origin_f[i] = (float)mn[i];
        const double cells = floor((mx[i] - mn[i]) * inv * (1.0 + 1e-6)) + 2.0;
        if (!(cells < 2147483648.0)) return HCA_ERANGE;
        g.ncell[i] = (uint32_t)cells;
        uint32_t b = 1;
        while ((1ull << b) < (uint64_t)g.ncell[i]) ++b;
        g.bits[i] = b;
        total += (int)b;
    }
    if (total > 63) return HCA_ERANGE;
    g.key_bits = total;
    int sh = 0;
    for (int i = 2; i >= 0; --i) {
        g.shift[i] = (uint32_t)sh;
        sh += (int)g.bits[i];
    }
    g.prefix_shift = (int)g.bits[2];
    const bool filter = input_f32 && !(flags & HCA_FLAG_FP64_ONLY) && g.eps2 >= ldexp(1.0, -100) &&
                        g.eps2 <= ldexp(1.0, 100);
    if (filter) {
        float lo = (float)(g.eps2 * (1.0 - ldexp(1.0, -16)));
        if ((double)lo > g.eps2 * (1.0 - ldexp(1.0, -16))) lo = nextafterf(lo, 0.f);
        float hi = (float)(g.eps2 * (1.0 + ldexp(1.0, -16)));
        if ((double)hi < g.eps2 * (1.0 + ldexp(1.0, -16))) hi = nextafterf(hi, INFINITY);
        g.lo32 = lo;
        g.hi32 = hi;
    } else {
        g.lo32 = -1.0f;
        g.hi32 = INFINITY;
    }
    g.box_ok = 0;
    return HCA_OK;
}

template <typename Kern>
inline void allow_smem(Kern k, size_t bytes) {
    if (bytes > 48 * 1024) cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

// The tensor-core filter's error bound needs finite FP32 norms and products: d * extent^2 <=
// 2^100 in every dimension and the FP32 filter enabled (eps^2 in [2^-100, 2^100]).
inline bool tc_magnitude_ok(int d, const double *mn, const double *mx, const GridParams &g) {
    if (!(g.lo32 >= 0.0f)) return false;
    for (int i = 0; i < d; ++i) {
        const double ext = mx[i] - mn[i];
        if (!(d * ext * ext <= ldexp(1.0, 100))) return false;
    }
    return true;
}

// Launch shape of the tensor-core kernels: their own shared memory, raised until a fifth CTA
// no longer fits on an SM (each CTA holds 128 of the SM's 512 tensor-memory columns, so four
// resident CTAs never wait in tcgen05.alloc), and the resident CTAs per SM (0: do not use).
template <int DP>
inline int tc_launch_shape(size_t &smem) {
    int dev = 0, sm_bytes = 0, reserved = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sm_bytes, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, dev) != cudaSuccess)
        return 0;
    size_t need = tc::smem_bytes<DP>();
    const size_t floor5 = (size_t)sm_bytes / 5 - (size_t)reserved + 16;  // 5 (floor5 + reserved) > sm_bytes
    if (need < floor5) need = floor5;
    smem = (need + 127) & ~(size_t)127;
    auto setup = [&](auto k) {
        cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        cudaFuncSetAttribute(k, cudaFuncAttributePreferredSharedMemoryCarveout, (int)cudaSharedmemCarveoutMaxShared);
    };
    setup(tc::k_tc_hd<DP, tc::kCount>);
    setup(tc::k_tc_hd<DP, tc::kMerge>);
    setup(tc::k_tc_hd<DP, tc::kLabels>);
    int occ = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, tc::k_tc_hd<DP, tc::kCount>, tc::kTile, smem) !=
            cudaSuccess ||
        occ < 1)
        return 0;
    // CTAs per SM that the shared memory admits (at most 4); more launched than can be resident
    // only wait for a slot, and find the chunk counter exhausted
    const int fit = (int)((size_t)sm_bytes / (smem + (size_t)reserved));
    return fit < 1 ? 0 : (fit > 4 ? 4 : fit);
}

}  // namespace detail

// Rows of a phase (counts, unions, labels) from which a coarse cell goes to the tensor-core
// kernels, whether the first links also run in cells whose unions are on tensor cores, and the
// open count rows at which a tensor-core chunk hands over (from the call's hca_tuning).
struct TcTuning {
    uint32_t min[3];
    uint32_t hook;
    uint32_t handoff;
};

// Workspace offsets of the tensor-core phases.
struct TcOffsets {
    size_t nch, nch2, ch0, ch1, ch2, flags, cx, clist, nclist, clab;
};

inline uint32_t *part_of(char *b, size_t o) { return (uint32_t *)(b + o); }

// The three point phases with tensor-core tiles for the cells holding at least min_rows rows
// of a phase and the CUDA-core kernels for the rest (float input): counts (Definition 2),
// first links + pointer jumping + unions (Definitions 3-5) and labels (Algorithm 4).
template <int DP, typename Mark>
void run_tc_phases(HdView<float, DP> &hv, cudaStream_t s, char *b, int64_t n, int grid_tc, size_t tc_smem,
                   int gpts, int gcell, int hd_block, size_t smem, uint32_t *part, const TcOffsets &o, int nsets,
                   DevCounters *ctr, const TcTuning &tune, Mark &mark, int &launches, cudaEvent_t *tev) {
    // tev (nullable): six events recorded around the three tensor-core launches
    auto tmark = [&](int i) { if (tev) cudaEventRecord(tev[i], s); };
    uint32_t *nch = (uint32_t *)(b + o.nch), *nch2 = (uint32_t *)(b + o.nch2);
    uint32_t *ch0 = (uint32_t *)(b + o.ch0), *ch1 = (uint32_t *)(b + o.ch1), *ch2 = (uint32_t *)(b + o.ch2);
    uint32_t *flags = (uint32_t *)(b + o.flags), *cx = (uint32_t *)(b + o.cx);
    uint32_t *clist = (uint32_t *)(b + o.clist), *nclist = (uint32_t *)(b + o.nclist);
    uint32_t *clab = (uint32_t *)(b + o.clab);
    for (int i = 0; i < 3; ++i) hv.tc_min[i] = tune.min[i];
    hv.tc_hook = tune.hook;
    hv.tc_handoff = tune.handoff;
    hv.cx = cx;
    hv.tc_cnt = clab;   // free until the labels phase
    hv.tc_pos = flags;  // free until the core numbering
    // ---- Definition 2: exact counts over the neighbouring coarse cells ----
    cudaMemsetAsync(hv.cell_core, 0, (size_t)n, s);
    cudaMemsetAsync(hv.core, 0, (size_t)n, s);  // the recount below lists the rows with core = 2
    tc::k_tc_chunks_count<<<gpts, 256, 0, s>>>(hv.cell_start, ctr, tune.min[0], nch);
    exclusive_scan_u32(nch, ch0, n, &ctr->n_cells, &ctr->n_tc_chunks[tc::kCount], part, s, &launches);
    tmark(0);
    tc::k_tc_hd<DP, tc::kCount><<<grid_tc, tc::kTile, tc_smem, s>>>(hv, tc::Tables{ch0, cx, clist, nclist, clab, nullptr});
    // the rows those chunks handed over, in cells with at least kRecountMin of them, counted again
    // from the start, 128 per chunk (cx, clist, nclist, nch2 and ch1 are free until the core
    // numbering); the rest, and what the recount hands over, go to the CUDA-core count
    tc::k_tc_handed_flags<<<gpts, 256, 0, s>>>(hv.core, n, nclist);
    exclusive_scan_u32(nclist, cx, n, nullptr, cx + n, part, s, &launches);
    tc::k_tc_handed_list<<<gpts, 256, 0, s>>>(hv.core, cx, n, clist);
    tc::k_tc_chunks_recount<<<gpts, 256, 0, s>>>(hv.cell_start, cx, ctr, hv.ranges, hv.n_all, tc::kRecountMin, nch2);
    exclusive_scan_u32(nch2, ch1, n, &ctr->n_cells, &ctr->n_tc_recount, part, s, &launches);
    // per listed row: the tallies summed over its windows and the windows done (nch, ch0 and
    // nclist are free once scanned / once the first count is done)
    cudaMemsetAsync(nch, 0, 4 * (size_t)n, s);
    cudaMemsetAsync(ch0, 0, 4 * (size_t)n, s);
    cudaMemsetAsync(nclist, 0, 4 * (size_t)n, s);
    tc::k_tc_hd<DP, tc::kCount><<<grid_tc, tc::kTile, tc_smem, s>>>(
        hv, tc::Tables{ch1, cx, nullptr, nullptr, nullptr, nullptr, nullptr, clist, nch, ch0, nclist});
    tmark(1);
    k_count_hd<float, DP><<<gcell, hd_block, smem, s>>>(hv);
    launches += 7;
    mark(6);
    // core numbering, core and non-core lists, chunk tables of the unions and the labels
    tc::k_tc_core_flags<<<gpts, 256, 0, s>>>(hv.core, n, flags);
    exclusive_scan_u32(flags, cx, n, nullptr, cx + n, part, s, &launches);
    tc::k_tc_partition<<<gpts, 256, 0, s>>>(hv.core, cx, n, clist, nclist);
    // (flags and ch0 are free once cx is scanned and the counts are done: the unions' later
    // windows take them)
    tc::k_tc_chunks_split<<<gpts, 256, 0, s>>>(hv.cell_start, cx, ctr, hv.ranges, hv.n_half, hv.n_all, tune.min[1],
                                               tune.min[2], nch, flags, nch2);
    exclusive_scan_u32(nch, ch1, n, &ctr->n_cells, &ctr->n_tc_chunks[tc::kMerge], part, s, &launches);
    exclusive_scan_u32(nch2, ch2, n, &ctr->n_cells, &ctr->n_tc_chunks[tc::kLabels], part, s, &launches);
    exclusive_scan_u32(flags, ch0, n, &ctr->n_cells, &ctr->n_tc_chunks[3], part, s, &launches);
    launches += 3;
    mark(7);
    // ---- Definitions 3-5: first links, pointer jumping, then the remaining unions ----
    k_uf_init_hd<float, DP><<<gpts, 256, 0, s>>>(hv);
    k_hook_hd<float, DP><<<gcell, hd_block, smem, s>>>(hv);
    for (int r = 0; r < 6; ++r) k_jump_hd<float, DP><<<gpts, 256, 0, s>>>(hv);
    // (nch and nch2 are free once the chunk tables are scanned)
    tc::k_tc_cell_root_clear<<<gpts, 256, 0, s>>>(ctr, nch, nch2);
    tc::k_tc_cell_root<DP><<<gpts, 256, 0, s>>>(hv, nch, nch2);
    tc::k_tc_cell_root_final<<<gpts, 256, 0, s>>>(ctr, nch, nch2);
    tmark(2);
    // window-major items: the first window of every chunk, then the other windows
    tc::k_tc_hd<DP, tc::kMerge><<<grid_tc, tc::kTile, tc_smem, s>>>(hv, tc::Tables{ch1, cx, clist, nclist, clab, nch, ch0});
    tmark(3);
    // the CUDA-core unions take the cells below the threshold; from one core row on every cell
    // with a core point is on the tensor cores and nothing is left for them
    if (tune.min[1] > 1) {
        k_merge_hd<float, DP><<<gcell, hd_block, smem, s>>>(hv);
        ++launches;
    }
    k_compress_hd<float, DP><<<gpts, 256, 0, s>>>(hv);
    launches += 13;
    mark(8);
    // ---- Algorithm 4: canonical ids, core labels, border and noise points ----
    k_comp_min_hd<float, DP><<<gpts, 256, 0, s>>>(hv);
    // the cells below the labels threshold on a second stream beside the tensor-core labels:
    // the two write the labels of disjoint cells
    const detail::SideStream ss = detail::side_stream();
    const bool fork = ss.ok && cudaEventRecord(ss.fork, s) == cudaSuccess &&
                      cudaStreamWaitEvent(ss.s, ss.fork, 0) == cudaSuccess;
    if (fork) k_labels_hd<float, DP><<<gcell, hd_block, smem, ss.s>>>(hv);
    tc::k_tc_core_labels<DP><<<gpts, 256, 0, s>>>(hv, tc::Tables{ch2, cx, clist, nclist, clab, nullptr}, nsets, clab);
    tmark(4);
    tc::k_tc_hd<DP, tc::kLabels><<<grid_tc, tc::kTile, tc_smem, s>>>(hv, tc::Tables{ch2, cx, clist, nclist, clab, nullptr});
    tmark(5);
    if (fork) {
        cudaEventRecord(ss.join, ss.s);
        cudaStreamWaitEvent(s, ss.join, 0);
    } else {
        k_labels_hd<float, DP><<<gcell, hd_block, smem, s>>>(hv);
    }
    launches += 4;
    mark(9);
}

template <typename T, int DP>
int run_hd(const RunArgs &a) {
    using namespace detail;
    cudaStream_t s = a.stream;
    const int64_t n = a.n;
    const int d = a.d;
    int launches = 0;
    int sms = device_sm_count();
    if (sms <= 0) {
        if (!a.ws_query) return HCA_ECUDA;
        sms = 1;  // sizing only: no device needed
    }

    size_t off = 0;
    auto take = [&](size_t bytes) { size_t o = off; off = align_up(off + bytes); return o; };
    int64_t cap_max = 64;
    while (cap_max < 2 * n) cap_max <<= 1;
    const size_t hist_elems = sort_hist_size(n);
    const int64_t scan_max = n > (int64_t)hist_elems ? n : (int64_t)hist_elems;
    const size_t o_ctr = take(sizeof(DevCounters));
    const size_t o_mm = take(sizeof(unsigned long long) * 128);
    const size_t o_ka = take(8 * n), o_kb = take(8 * n), o_ia = take(4 * n), o_ib = take(4 * n);
    const size_t o_hist = take(4 * hist_elems);
    const size_t o_part = take(4 * scan_partials_size(scan_max));
    const size_t o_pts = take(sizeof(T) * DP * (size_t)n);
    const size_t o_flags = take(4 * n), o_excl = take(4 * n);
    const size_t o_cstart = take(4 * (n + 1)), o_ckey = take(8 * n);
    const size_t o_pflags = take(4 * n), o_pexcl = take(4 * n), o_pstart = take(4 * (n + 1));
    const size_t o_hk = take(8 * cap_max), o_hv = take(4 * cap_max);
    const size_t o_core = take(n), o_ccore = take(n);
    const size_t o_parent = take(4 * n), o_cmin = take(4 * n);
    const size_t o_ranges = take(sizeof(uint2) * 9 * (size_t)n);
    const size_t o_nch = take(4 * n), o_choff = take(4 * n);
    const size_t o_blo = take(sizeof(T) * DP * (size_t)n), o_bhi = take(sizeof(T) * DP * (size_t)n);
    const bool batched = a.nsets > 0;
    const int nsets = batched ? a.nsets : 1;
    const size_t o_smm = take(sizeof(unsigned long long) * 2 * 64 * (size_t)nsets);
    const size_t o_gtab = take(sizeof(GridParams) * (size_t)nsets);
    const size_t o_setoff = take(sizeof(int64_t) * ((size_t)nsets + 1));
    // tensor-core phases (float input): chunk tables, core numbering, core / non-core lists
    size_t tc_smem = 0;
    int tc_occ = 0;
    if constexpr (std::is_same<T, float>::value)
        if (!(a.flags & (HCA_FLAG_FP64_ONLY | HCA_FLAG_NO_TENSOR_CORES))) tc_occ = tc_launch_shape<DP>(tc_smem);
    // (a size query counts the tensor-core tables whenever the input and flags allow them)
    const bool tc_allowed = std::is_same<T, float>::value &&
                            !(a.flags & (HCA_FLAG_FP64_ONLY | HCA_FLAG_NO_TENSOR_CORES));
    const size_t tc_n = (tc_occ || (a.ws_query && tc_allowed)) ? (size_t)n : 0;
    const size_t o_tnch = take(4 * tc_n), o_tnch2 = take(4 * tc_n);
    const size_t o_tch0 = take(4 * tc_n), o_tch1 = take(4 * tc_n), o_tch2 = take(4 * tc_n);
    const size_t o_tflags = take(4 * tc_n), o_cx = take(4 * (tc_n + 1));
    const size_t o_clist = take(4 * tc_n), o_nclist = take(4 * tc_n), o_clab = take(4 * tc_n);
    const size_t o_box = take(sizeof(double) * 2 * (size_t)d * nsets);
    bool use_tc = tc_occ > 0;
    const bool boxed = a.box_mn != nullptr;
    const bool own_ws = a.ws_ext == nullptr;
    void *ws = nullptr;
    if (a.ws_query) {  // the layout depends on n, d, the sets and the flags only
        *a.ws_query = off;
        return HCA_OK;
    }
    if (!own_ws) {
        if (!boxed || a.ws_ext_bytes < off) return HCA_EINVAL;
        ws = a.ws_ext;
    } else if (pool_alloc(&ws, off, s) != cudaSuccess || !ws) {
        return HCA_ENOMEM;
    }
    char *b = (char *)ws;
    DevCounters *ctr = (DevCounters *)(b + o_ctr);
    unsigned long long *mm = (unsigned long long *)(b + o_mm);
    DevCounters *h = a.h_ext ? a.h_ext : (a.ws_query ? nullptr : host_counters());
    int rc = HCA_OK;
    bool tc_phases = false;  // the tensor-core split ran every phase

    cudaEvent_t ev[HCA_NUM_STAGES + 1] = {};
    cudaEvent_t tev[6] = {};
    const bool timing = (a.flags & HCA_FLAG_TIMING) && a.stats && !a.deferred;
    if (timing) {
        for (int i = 0; i <= HCA_NUM_STAGES; ++i) cudaEventCreate(&ev[i]);
        for (int i = 0; i < 6; ++i) cudaEventCreate(&tev[i]);
    }
    auto mark = [&](int i) { if (timing) cudaEventRecord(ev[i], s); };

    GridParams g;
    Stencil st;
    double tau = 0.0;
    int3 sel = make_int3(0, 1, 2);
    const int gpts = grid_for(n, 256, sms, 8);
    // CUDA-core chunk kernels: one 32-point chunk per warp, tuning.cta_warps warps per CTA
    const int hd_warps = (a.tune.cta_warps == 2 || a.tune.cta_warps == 8) ? a.tune.cta_warps : kHdWarps;
    const int hd_block = 32 * hd_warps;
    const int gcell = grid_for((n + 31) / 32 + 1, hd_warps, sms, 64 / hd_warps);
    const size_t smem = (size_t)hd_warps * 32 * DP * sizeof(T);
    bool flipped = false;
    std::vector<unsigned long long> hmm(128);
    HdView<T, DP> hv;
    LowdView<float, 3> lv;
    memset(&hv, 0, sizeof(hv));
    memset(&lv, 0, sizeof(lv));
    int sort_bits = 0;
    std::vector<unsigned long long> smm;
    std::vector<GridParams> gsets;
    GridParams *d_gtab = (GridParams *)(b + o_gtab);
    int64_t *d_setoff = (int64_t *)(b + o_setoff);
    unsigned long long *d_smm = (unsigned long long *)(b + o_smm);
    const size_t stage_setoff = 0, stage_gtab = align_up(sizeof(int64_t) * ((size_t)nsets + 1));
    const size_t stage_box = stage_gtab + align_up(sizeof(GridParams) * (size_t)nsets);

    // the coarse grid of one set from its extents: the three dimensions of largest extent
    // (ties: lower index), cells of side eps (1 + 2^-10) over them
    auto grid_of = [&](const double *mn_all, const double *mx_all, double set_eps, int set_minpts, GridParams &gp,
                       double &tau_s) -> int {
        for (int i = 0; i < d; ++i)
            if (!isfinite(mn_all[i]) || !isfinite(mx_all[i]) || mx_all[i] < mn_all[i]) return HCA_EINVAL;
        int pick[3] = {-1, -1, -1};
        for (int k = 0; k < 3; ++k) {
            double best = -1.0;
            for (int i = 0; i < d; ++i) {
                if (i == pick[0] || i == pick[1]) continue;
                const double ext = mx_all[i] - mn_all[i];
                if (ext > best) { best = ext; pick[k] = i; }
            }
        }
        const double mn3[3] = {mn_all[pick[0]], mn_all[pick[1]], mn_all[pick[2]]};
        const double mx3[3] = {mx_all[pick[0]], mx_all[pick[1]], mx_all[pick[2]]};
        const int r = make_coarse_grid(sizeof(T) == 4, set_eps, set_minpts, n, mn3, mx3, a.flags, gp, tau_s);
        if (r) return r;
        if (!tc_magnitude_ok(d, mn_all, mx_all, gp)) use_tc = false;
        for (int k = 0; k < 3; ++k) gp.sel[k] = pick[k];
        return HCA_OK;
    };
    // every set's grid, one key layout for all, the stencil; extents of set si, dimension i
    // from mn_of / mx_of (measured, or a plan's declared boxes)
    auto build_grids = [&](auto mn_of, auto mx_of) -> int {
        double mn_all[64], mx_all[64];
        if (!batched) {
            for (int i = 0; i < d; ++i) {
                mn_all[i] = mn_of(0, i);
                mx_all[i] = mx_of(0, i);
            }
            int r = grid_of(mn_all, mx_all, a.eps, a.min_pts, g, tau);
            if (r) return r;
            sel = make_int3(g.sel[0], g.sel[1], g.sel[2]);
            r = make_stencil(3, a.eps, 1.0 / g.inv_side, tau, st);
            if (r) return r;
            sort_bits = g.key_bits;
            return HCA_OK;
        }
        gsets.resize(nsets);
        std::vector<double> e_eps(nsets), e_side(nsets), e_tau(nsets);
        uint32_t bits[3] = {};
        for (int si = 0; si < nsets; ++si) {
            const bool empty = a.h_off[si + 1] == a.h_off[si];
            for (int i = 0; i < d; ++i) {
                mn_all[i] = empty ? 0.0 : mn_of(si, i);
                mx_all[i] = empty ? 0.0 : mx_of(si, i);
            }
            double tau_s = 0.0;
            const int r = grid_of(mn_all, mx_all, a.h_eps[si], a.h_minpts[si], gsets[si], tau_s);
            if (r) return r;
            e_eps[si] = a.h_eps[si];
            e_side[si] = 1.0 / gsets[si].inv_side;
            e_tau[si] = tau_s;
            for (int i = 0; i < 3; ++i) bits[i] = bits[i] > gsets[si].bits[i] ? bits[i] : gsets[si].bits[i];
        }
        int key_bits = 0, set_bits = 1;
        for (int i = 0; i < 3; ++i) key_bits += (int)bits[i];
        while ((1ll << set_bits) < nsets) ++set_bits;
        if (key_bits + set_bits > 63) return HCA_ERANGE;
        for (GridParams &gp : gsets) {
            int sh = 0;
            for (int i = 2; i >= 0; --i) {
                gp.bits[i] = bits[i];
                gp.shift[i] = (uint32_t)sh;
                sh += (int)bits[i];
            }
            gp.key_bits = key_bits;
            gp.prefix_shift = (int)bits[2];
        }
        g = gsets[0];
        sort_bits = key_bits + set_bits;
        return make_stencil_union(3, e_eps, e_side, e_tau, st);
    };
    auto upload = [&](void *dst, const void *src, size_t bytes, size_t stage_off) {
        if (a.deferred && a.h_stage) {
            memcpy((char *)a.h_stage + stage_off, src, bytes);
            src = (char *)a.h_stage + stage_off;
        }
        cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, s);
    };

    if (!h) { rc = HCA_ECUDA; goto out; }
    if (boxed) {
        rc = build_grids([&](int set, int i) { return a.box_mn[(size_t)set * d + i]; },
                         [&](int set, int i) { return a.box_mx[(size_t)set * d + i]; });
        if (rc) goto out;
    }
    mark(0);
    cudaMemsetAsync(ctr, 0, sizeof(DevCounters), s);
    if (!batched) {
        cudaMemsetAsync(mm, 0xff, sizeof(unsigned long long) * 64, s);
        cudaMemsetAsync(mm + 64, 0, sizeof(unsigned long long) * 64, s);
        k_minmax_rt<T><<<grid_for(n * d, 256, sms, 8), 256, 0, s>>>((const T *)a.d_points, n, d, ctr, mm);
        if (!boxed) cudaMemcpyAsync(hmm.data(), mm, sizeof(unsigned long long) * 128, cudaMemcpyDeviceToHost, s);
    } else {
        cudaMemsetAsync(d_smm, 0xff, sizeof(unsigned long long) * 64 * nsets, s);
        cudaMemsetAsync(d_smm + (size_t)64 * nsets, 0, sizeof(unsigned long long) * 64 * nsets, s);
        upload(d_setoff, a.h_off, sizeof(int64_t) * (nsets + 1), stage_setoff);
        k_minmax_rt_seg<T><<<grid_for(n, 256, sms, 8), 256, 0, s>>>((const T *)a.d_points, n, d, d_setoff, nsets,
                                                                   d_smm, ctr);
        if (!boxed) {
            smm.resize((size_t)2 * 64 * nsets);
            cudaMemcpyAsync(smm.data(), d_smm, sizeof(unsigned long long) * smm.size(), cudaMemcpyDeviceToHost, s);
        }
    }
    ++launches;
    if (boxed) {
        // declared extents: check them on the device, no host round trip
        std::vector<double> boxes((size_t)2 * d * nsets);
        memcpy(boxes.data(), a.box_mn, sizeof(double) * d * nsets);
        memcpy(boxes.data() + (size_t)d * nsets, a.box_mx, sizeof(double) * d * nsets);
        double *d_box = (double *)(b + o_box);
        upload(d_box, boxes.data(), sizeof(double) * boxes.size(), stage_box);
        if (batched) upload(d_gtab, gsets.data(), sizeof(GridParams) * nsets, stage_gtab);
        k_box_check_hd<<<grid_for((int64_t)nsets * d, 256, sms, 1), 256, 0, s>>>(
            d_box, nsets, d, batched ? d_setoff : nullptr, batched ? d_smm : mm, ctr);
        ++launches;
    } else {
        if (cudaMemcpyAsync(h, ctr, sizeof(DevCounters), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess) { rc = HCA_ECUDA; goto out; }
        if (h->nan_seen) { rc = HCA_EINVAL; goto out; }
        if (a.ext_out && !batched)
            for (int i = 0; i < d; ++i) {
                a.ext_out[i] = dec_double(hmm[i]);
                a.ext_out[d + i] = dec_double(hmm[64 + i]);
            }
        if (batched)
            rc = build_grids([&](int set, int i) { return dec_double(smm[(size_t)set * 64 + i]); },
                             [&](int set, int i) { return dec_double(smm[((size_t)nsets + set) * 64 + i]); });
        else
            rc = build_grids([&](int, int i) { return dec_double(hmm[i]); },
                             [&](int, int i) { return dec_double(hmm[64 + i]); });
        if (rc) goto out;
        if (batched) cudaMemcpyAsync(d_gtab, gsets.data(), sizeof(GridParams) * nsets, cudaMemcpyHostToDevice, s);
    }
    mark(1);
    {
        uint32_t *ia = (uint32_t *)(b + o_ia), *ib = (uint32_t *)(b + o_ib);
        uint32_t *hist = (uint32_t *)(b + o_hist), *part = (uint32_t *)(b + o_part);
        const bool use32 = sort_bits <= 32;
        const int gtile = (int)((n + kScanTileElems - 1) / kScanTileElems);  // gather: one block per scan tile
        if (use32) {
            uint32_t *ka = (uint32_t *)(b + o_ka), *kb = (uint32_t *)(b + o_kb);
            if (batched)
                k_bin_proj_seg<T, uint32_t><<<gpts, 256, 0, s>>>((const T *)a.d_points, n, d, d_setoff, nsets, d_gtab,
                                                                 g.key_bits, ka, ia);
            else
                k_bin_proj<T, uint32_t><<<gpts, 256, 0, s>>>((const T *)a.d_points, d, sel, g, ka, ia);
            mark(2);
            flipped = radix_sort_pairs<uint32_t>(ka, ia, kb, ib, n, 0, sort_bits, hist, part, s, &launches, &ctr->status);
            mark(3);
            k_gather_hd<T, DP, uint32_t><<<gtile, 256, 0, s>>>(
                (const T *)a.d_points, d, flipped ? kb : ka, flipped ? ib : ia, n, (T *)(b + o_pts),
                (uint32_t *)(b + o_flags), part);
        } else {
            uint64_t *ka = (uint64_t *)(b + o_ka), *kb = (uint64_t *)(b + o_kb);
            if (batched)
                k_bin_proj_seg<T, uint64_t><<<gpts, 256, 0, s>>>((const T *)a.d_points, n, d, d_setoff, nsets, d_gtab,
                                                                 g.key_bits, ka, ia);
            else
                k_bin_proj<T, uint64_t><<<gpts, 256, 0, s>>>((const T *)a.d_points, d, sel, g, ka, ia);
            mark(2);
            flipped = radix_sort_pairs<uint64_t>(ka, ia, kb, ib, n, 0, sort_bits, hist, part, s, &launches, &ctr->status);
            mark(3);
            k_gather_hd<T, DP, uint64_t><<<gtile, 256, 0, s>>>(
                (const T *)a.d_points, d, flipped ? kb : ka, flipped ? ib : ia, n, (T *)(b + o_pts),
                (uint32_t *)(b + o_flags), part);
        }
        launches += 2;
        // run-length cells: scan of the gather's tile counts, cell ids / starts / keys
        if (use32)
            cells_from_flags<uint32_t>((const uint32_t *)(b + (flipped ? o_kb : o_ka)), (uint32_t *)(b + o_flags), n,
                                       part, &ctr->n_cells, (uint32_t *)(b + o_cstart), (uint64_t *)(b + o_ckey), s,
                                       &launches);
        else
            cells_from_flags<uint64_t>((const uint64_t *)(b + (flipped ? o_kb : o_ka)), (uint32_t *)(b + o_flags), n,
                                       part, &ctr->n_cells, (uint32_t *)(b + o_cstart), (uint64_t *)(b + o_ckey), s,
                                       &launches);
        hv.perm = flipped ? ib : ia;
    }
    mark(4);
    {
        uint32_t *part = (uint32_t *)(b + o_part);
        k_pencil_flags<<<gpts, 256, 0, s>>>((const uint64_t *)(b + o_ckey), g.prefix_shift, ctr,
                                            (uint32_t *)(b + o_pflags));
        exclusive_scan_u32((uint32_t *)(b + o_pflags), (uint32_t *)(b + o_pexcl), n, &ctr->n_cells,
                           &ctr->n_pencils, part, s, &launches);
        k_hash_init<<<grid_for(cap_max, 256, sms, 8), 256, 0, s>>>((uint64_t *)(b + o_hk), ctr);
        k_pencils<<<gpts, 256, 0, s>>>((const uint64_t *)(b + o_ckey), g.prefix_shift,
                                       (const uint32_t *)(b + o_pflags), (const uint32_t *)(b + o_pexcl),
                                       (uint32_t *)(b + o_pstart), (uint64_t *)(b + o_hk),
                                       (uint32_t *)(b + o_hv), ctr);
        lv.g = g;
        lv.gtab = batched ? d_gtab : nullptr;
        lv.cell_key = (const uint64_t *)(b + o_ckey);
        lv.pencil_start = (const uint32_t *)(b + o_pstart);
        lv.hkeys = (uint64_t *)(b + o_hk);
        lv.hvals = (uint32_t *)(b + o_hv);
        lv.ranges = (uint2 *)(b + o_ranges);
        lv.ctr = ctr;
        k_ranges<float, 3><<<grid_for((n / kRangeRun + 1) * (int64_t)st.n_all, 256, sms, 16), 256, 0, s>>>(lv, st);
        k_chunk_counts<<<gpts, 256, 0, s>>>((const uint32_t *)(b + o_cstart), ctr, (uint32_t *)(b + o_nch));
        exclusive_scan_u32((uint32_t *)(b + o_nch), (uint32_t *)(b + o_choff), n, &ctr->n_cells,
                           &ctr->n_chunks, part, s, &launches);
        launches += 5;
    }
    mark(5);
    hv.g = g;
    hv.gtab = batched ? d_gtab : nullptr;
    hv.set_off = batched ? d_setoff : nullptr;
    hv.d = d;
    hv.pts = (const T *)(b + o_pts);
    hv.cell_start = (const uint32_t *)(b + o_cstart);
    hv.cell_key = (const uint64_t *)(b + o_ckey);
    hv.chunk_off = (const uint32_t *)(b + o_choff);
    hv.ranges = (const uint2 *)(b + o_ranges);
    hv.core = (uint8_t *)(b + o_core);
    hv.cell_core = (uint8_t *)(b + o_ccore);
    hv.parent = (uint32_t *)(b + o_parent);
    hv.comp_min = (uint32_t *)(b + o_cmin);
    hv.labels = a.d_labels;
    hv.core_out = a.d_core;
    hv.ctr = ctr;
    hv.n_all = st.n_all;
    hv.n_half = st.n_half;
    hv.box_lo = (T *)(b + o_blo);
    hv.box_hi = (T *)(b + o_bhi);
    // the box of every coarse cell in all d dimensions (point-to-box distance bounds)
    k_cell_box_clear<T, DP><<<grid_for((int64_t)n * DP, 256, sms, 8), 256, 0, s>>>(hv);
    k_cell_box_hd<T, DP><<<grid_for(n / 32 + 1, 8, sms, 16), 256, 0, s>>>(hv);
    k_cell_box_decode<T, DP><<<grid_for((int64_t)n * DP, 256, sms, 8), 256, 0, s>>>(hv);
    launches += 3;
    allow_smem(k_count_hd<T, DP>, smem);
    allow_smem(k_hook_hd<T, DP>, smem);
    allow_smem(k_merge_hd<T, DP>, smem);
    allow_smem(k_labels_hd<T, DP>, smem);
    if constexpr (std::is_same<T, float>::value) {
        if (use_tc && st.n_all <= tc::kMaxRng) {
            run_tc_phases<DP>(hv, s, b, n, sms * tc_occ, tc_smem, gpts, gcell, hd_block, smem, part_of(b, o_part),
                              TcOffsets{o_tnch, o_tnch2, o_tch0, o_tch1, o_tch2, o_tflags, o_cx, o_clist, o_nclist,
                                        o_clab},
                              batched ? nsets : 0, ctr,
                              TcTuning{{(uint32_t)a.tune.tc_min_count, (uint32_t)a.tune.tc_min_merge,
                                        (uint32_t)a.tune.tc_min_labels},
                                       (uint32_t)a.tune.first_links, (uint32_t)a.tune.tc_handoff},
                              mark, launches, timing ? tev : nullptr);
            tc_phases = true;
        }
    }
    if (!tc_phases) {
        // ---- Definition 2: exact counts over the neighbouring coarse cells ----
        cudaMemsetAsync(hv.cell_core, 0, (size_t)n, s);
        k_count_hd<T, DP><<<gcell, hd_block, smem, s>>>(hv);
        ++launches;
        mark(6);
        // (no representative points in this path: every pair of core points is a candidate)
        mark(7);
        // ---- Definitions 3-5: first links, pointer jumping, then the remaining unions ----
        k_uf_init_hd<T, DP><<<gpts, 256, 0, s>>>(hv);
        k_hook_hd<T, DP><<<gcell, hd_block, smem, s>>>(hv);
        for (int r = 0; r < 6; ++r) k_jump_hd<T, DP><<<gpts, 256, 0, s>>>(hv);
        k_merge_hd<T, DP><<<gcell, hd_block, smem, s>>>(hv);
        k_compress_hd<T, DP><<<gpts, 256, 0, s>>>(hv);
        launches += 10;
        mark(8);
        // ---- Algorithm 4: canonical ids, border and noise points ----
        k_comp_min_hd<T, DP><<<gpts, 256, 0, s>>>(hv);
        k_labels_hd<T, DP><<<gcell, hd_block, smem, s>>>(hv);
        launches += 2;
        mark(9);
    }
    if (cudaGetLastError() != cudaSuccess) { rc = HCA_ECUDA; goto out; }
    if (cudaMemcpyAsync(h, ctr, sizeof(DevCounters), cudaMemcpyDeviceToHost, s) != cudaSuccess) {
        rc = HCA_ECUDA;
        goto out;
    }
    if (a.launches_out) *a.launches_out = launches;
    if (a.key_bits_out) *a.key_bits_out = sort_bits;
    if (a.deferred) goto out;  // the caller synchronises and reads the status from h
    if (cudaStreamSynchronize(s) != cudaSuccess) { rc = HCA_ECUDA; goto out; }
    if (boxed && h->nan_seen) { rc = HCA_EINVAL; goto out; }
    if (h->status) { rc = (h->status & kErrBox) ? HCA_ERANGE : HCA_EDEVICE; goto out; }
    if (a.stats) {
        hca_stats *so = a.stats;
        so->n_points = n;
        so->n_cells = h->n_cells;
        so->n_pencils = h->n_pencils;
        so->n_dense_cells = 0;
        so->n_core_points = h->n_core;
        so->n_clusters = h->n_clusters;
        so->n_noise = h->n_noise;
        so->key_bits = sort_bits;
        so->sort_passes = (sort_bits + 7) / 8;
        so->kernel_launches = launches;
        so->n_count_chunks = (int64_t)h->work[0];
        so->n_rep_tests = (int64_t)h->work[1];   // hook-pass chunks in this path
        so->n_rep_hits = (int64_t)h->work[2];    // tiles skipped because every root agreed
        so->n_exhaustive_pairs = (int64_t)h->work[3];
        so->n_exhaustive_chunks = (int64_t)h->work[4];
        so->n_border_chunks = (int64_t)h->work[5];
        so->n_tc_tiles = (int64_t)h->work[6];
        so->n_tc_rechecks = (int64_t)h->work[7];
        so->n_tc_pairs = (int64_t)h->tc_pairs;
        so->workspace_bytes = (int64_t)off;
        for (int i = 0; i < HCA_NUM_STAGES; ++i) {
            float ms = 0.f;
            if (timing) cudaEventElapsedTime(&ms, ev[i], ev[i + 1]);
            so->stage_ms[i] = ms;
        }
        for (int i = 0; i < 3; ++i) {
            float ms = 0.f;
            if (timing && tc_phases) cudaEventElapsedTime(&ms, tev[2 * i], tev[2 * i + 1]);
            so->tc_ms[i] = ms;
        }
    }
out:
    if (timing) {
        for (int i = 0; i <= HCA_NUM_STAGES; ++i)
            if (ev[i]) cudaEventDestroy(ev[i]);
        for (int i = 0; i < 6; ++i)
            if (tev[i]) cudaEventDestroy(tev[i]);
    }
    if (own_ws) pool_free(ws, s);
    if (rc != HCA_OK && !a.deferred) cudaStreamSynchronize(s);
    return rc;
}

}  // namespace hca
