// Host orchestration of the hypercube-stencil path for one call: workspace layout, grid
// parameters, neighbour stencil and the launch sequence of the stage kernels.
#pragma once

#include <math.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "lowd_kernels.cuh"

namespace hca {

namespace detail {

inline size_t align_up(size_t x) { return (x + 255) & ~(size_t)255; }

inline double dec_double(uint64_t e) {
    uint64_t b = (e >> 63) ? (e & 0x7fffffffffffffffull) : ~e;
    double f;
    memcpy(&f, &b, 8);
    return f;
}

// Grid of hypercubes (Algorithm 1).  The side is eps/sqrt(d) (space diagonal eps, Sec. 2)
// shrunk so that a cell stays within eps even after the rounding of the band computation:
// with tau the bound on |computed - exact| of (x - o)/side in cell units, every point of
// cell c has an exact band coordinate in [c - tau, c + 1 + tau), and
//     d * ((1 + 2 tau) side)^2 <= (eps (1 - 2^-20))^2
// keeps the FP64 predicate of every pair in one cell at or below eps^2.
inline int make_grid(int D, bool input_f32, double eps, int min_pts, int64_t n,
                     const double *mn, const double *mx, int flags, GridParams &g, double &tau) {
    memset(&g, 0, sizeof(g));
    g.d = D;
    g.n = n;
    g.min_pts = (uint32_t)min_pts;
    g.eps2 = eps * eps;
    double range_max = 0.0;
    for (int i = 0; i < D; ++i) range_max = fmax(range_max, mx[i] - mn[i]);
    if (!isfinite(range_max)) return HCA_ERANGE;
    const double shrink = 1.0 - ldexp(1.0, -20);
    bool bin32 = input_f32;
    double inv = 0.0;
    for (int attempt = 0; attempt < 64; ++attempt) {
        const double u = bin32 ? ldexp(1.0, -22) : ldexp(1.0, -51);
        inv = sqrt((double)D) / (eps * shrink);
        tau = 0.0;
        for (int it = 0; it < 4; ++it) {
            tau = (range_max * inv + 1.0) * u;
            inv = sqrt((double)D) * (1.0 + 2.0 * tau) / (eps * shrink) * (1.0 + ldexp(1.0, -40));
        }
        if (!isfinite(inv) || inv <= 0.0) return HCA_ERANGE;
        bool ok = false;
        for (int bump = 0; bump < 64 && !ok; ++bump) {
            double inv_used = inv;
            if (bin32) {
                float f = (float)inv;
                if ((double)f < inv) f = nextafterf(f, INFINITY);
                inv_used = (double)f;
                g.inv_side_f = f;
            }
            tau = (range_max * inv_used + 1.0) * u;
            const double side = 1.0 / inv_used;
            const double w = side * (1.0 + 2.0 * tau);
            if ((double)D * w * w <= (eps * shrink) * (eps * shrink)) {
                ok = true;
                inv = inv_used;
            } else {
                inv *= 1.0 + ldexp(1.0, -20);
            }
        }
        if (!ok) return HCA_ERANGE;
        if (bin32 && tau > ldexp(1.0, -8)) {  // too coarse a bound: bin in FP64 instead
            bin32 = false;
            continue;
        }
        break;
    }
    g.inv_side = inv;
    if (!bin32) g.inv_side_f = (float)inv;
    g.bin_fp64 = bin32 ? 0 : 1;
    // cell-box tests in FP32 band units (see box_class)
    const double tmax = range_max * inv + 2.0;
    g.box_ok = tmax < ldexp(1.0, 22) ? 1 : 0;
    g.tau_box = (float)(2.0 * tau + tmax * ldexp(1.0, -22));
    const double eps2_band = eps * eps * inv * inv;
    g.box_full = (float)(eps2_band * (1.0 - ldexp(1.0, -12)));
    g.box_none = (float)(eps2_band * (1.0 + ldexp(1.0, -12)));
    int total = 0;
    for (int i = 0; i < D; ++i) {
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
    for (int i = D - 1; i >= 0; --i) {
        g.shift[i] = (uint32_t)sh;
        sh += (int)g.bits[i];
    }
    g.prefix_shift = (int)g.bits[D - 1];
    // FP32 filter thresholds (guard band 2^-16 relative; valid for eps^2 in [2^-100, 2^100])
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
    return HCA_OK;
}

// Neighbour pencils (the stencil of Sec. 2, "Depth First Search" and "Layering", reached
// exactly): a cell at offset delta can hold a point within eps of a point of the current
// cell only if sum_i gap(|delta_i|)^2 <= eps^2, gap(k) = max(k - 1 - 2 tau, 0) * side.  The
// first d-1 offsets form the pencil offset; along the last coordinate the reach is the
// largest k that still passes.  Entry 0 is the zero pencil offset, then the offsets that are
// lexicographically positive (the upper half, used to visit each pair of cells once), then
// the negative ones.
struct StencilEntry { int off[kMaxD]; int reach; int cls; };

inline void collect_stencil(int D, double eps, double side, double tau, std::vector<StencilEntry> &out);

// Union of the stencils of several grids (batched calls): every pencil offset any grid needs,
// with the largest reach.
inline int make_stencil_union(int D, const std::vector<double> &eps, const std::vector<double> &side,
                              const std::vector<double> &tau, Stencil &st) {
    std::vector<StencilEntry> all;
    for (size_t i = 0; i < eps.size(); ++i) {
        std::vector<StencilEntry> one;
        collect_stencil(D, eps[i], side[i], tau[i], one);
        for (const StencilEntry &e : one) {
            bool found = false;
            for (StencilEntry &a : all) {
                if (memcmp(a.off, e.off, sizeof(a.off)) == 0) {
                    a.reach = a.reach > e.reach ? a.reach : e.reach;
                    found = true;
                    break;
                }
            }
            if (!found) all.push_back(e);
        }
    }
    memset(&st, 0, sizeof(st));
    if ((int)all.size() > kMaxPencils) return HCA_ENOTIMPL;
    int k = 0;
    for (int cls = 0; cls < 3; ++cls) {
        for (const StencilEntry &e : all) {
            if (e.cls != cls) continue;
            for (int i = 0; i < D - 1; ++i) st.off[k][i] = (int8_t)e.off[i];
            st.reach[k] = (int8_t)e.reach;
            ++k;
        }
        if (cls == 1) st.n_half = k;
    }
    st.n_all = k;
    // counting order: by the gap of the offset (the squared distance, in cells, between the
    // cell and the nearest cell of the pencil), then by the sum of |offsets|
    std::vector<int> order(k);
    for (int j = 0; j < k; ++j) order[j] = j;
    auto near_key = [&](int j) {
        int gap = 0, l1 = 0;
        for (int i = 0; i < D - 1; ++i) {
            const int a = st.off[j][i] < 0 ? -st.off[j][i] : st.off[j][i];
            gap += (a > 1 ? a - 1 : 0) * (a > 1 ? a - 1 : 0);
            l1 += a;
        }
        return gap * 1024 + l1;
    };
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return near_key(x) < near_key(y); });
    for (int j = 0; j < k; ++j) st.near[j] = (uint16_t)order[j];
    return HCA_OK;
}

inline int make_stencil(int D, double eps, double side, double tau, Stencil &st) {
    return make_stencil_union(D, std::vector<double>{eps}, std::vector<double>{side}, std::vector<double>{tau}, st);
}

inline void collect_stencil(int D, double eps, double side, double tau, std::vector<StencilEntry> &all) {
    const double bound = eps * eps * (1.0 + ldexp(1.0, -20));
    auto gap2 = [&](int k) {
        double gg = (double)k - 1.0 - 2.0 * tau;
        if (gg < 0.0) gg = 0.0;
        gg *= side;
        return gg * gg;
    };
    int R = 1;
    while (gap2(R + 1) <= bound) ++R;
    const int P = D - 1;
    std::vector<int> delta(P > 0 ? P : 1, -R);
    for (;;) {
        double gp = 0.0;
        bool zero = true;
        int first = 0;
        for (int i = 0; i < P; ++i) {
            int a = delta[i] < 0 ? -delta[i] : delta[i];
            gp += gap2(a);
            if (delta[i] != 0 && zero) { zero = false; first = delta[i]; }
        }
        if (gp <= bound) {
            StencilEntry e;
            memset(&e, 0, sizeof(e));
            for (int i = 0; i < P; ++i) e.off[i] = delta[i];
            int r = 1;
            while (r < R && gp + gap2(r + 1) <= bound) ++r;
            e.reach = r;
            e.cls = zero ? 0 : (first > 0 ? 1 : 2);
            all.push_back(e);
        }
        int i = 0;
        while (i < P && delta[i] == R) delta[i++] = -R;
        if (i >= P) break;
        ++delta[i];
    }
}

struct HostCounters {
    DevCounters *p = nullptr;
    HostCounters() {
        if (cudaMallocHost((void **)&p, sizeof(DevCounters)) != cudaSuccess) p = nullptr;
    }
    ~HostCounters() {
        if (p) cudaFreeHost(p);
    }
};

inline DevCounters *host_counters() {
    thread_local HostCounters hc;
    return hc.p;
}

// A second stream of the calling thread on the current device, with the events that fork work
// onto it from a call's stream and join it back (kept for the thread's lifetime); ok is false
// when they could not be created, and the caller then stays on its own stream.
struct SideStream {
    bool ok = false;
    cudaStream_t s = nullptr;
    cudaEvent_t fork = nullptr, join = nullptr;
};

inline SideStream side_stream() {
    struct Slots {
        SideStream v[64];
        bool tried[64] = {};
    };
    thread_local Slots slots;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return SideStream();
    SideStream &ss = slots.v[dev];
    if (!slots.tried[dev]) {
        slots.tried[dev] = true;
        ss.ok = cudaStreamCreateWithFlags(&ss.s, cudaStreamNonBlocking) == cudaSuccess &&
                cudaEventCreateWithFlags(&ss.fork, cudaEventDisableTiming) == cudaSuccess &&
                cudaEventCreateWithFlags(&ss.join, cudaEventDisableTiming) == cudaSuccess;
    }
    return ss;
}

inline int grid_for(int64_t work, int per_block, int sms, int max_per_sm) {
    int64_t b = (work + per_block - 1) / per_block;
    const int64_t cap = (int64_t)sms * max_per_sm;
    if (b > cap) b = cap;
    if (b < 1) b = 1;
    return (int)b;
}

}  // namespace detail

template <typename T, int D>
int run_lowd(const RunArgs &a) {
    using namespace detail;
    cudaStream_t s = a.stream;
    const int64_t n = a.n;
    constexpr int ndir = RepDirs<D>::value;
    int launches = 0;
    int sms = device_sm_count();
    if (sms <= 0) {
        if (!a.ws_query) return HCA_ECUDA;
        sms = 1;  // sizing only: no device needed
    }

    // ---- workspace layout (one pool allocation) ----
    size_t off = 0;
    auto take = [&](size_t bytes) { size_t o = off; off = align_up(off + bytes); return o; };
    int64_t cap_max = 64;
    while (cap_max < 2 * n) cap_max <<= 1;
    const size_t hist_elems = sort_hist_size(n);
    const int64_t scan_max = n > (int64_t)hist_elems ? n : (int64_t)hist_elems;
    const size_t o_ctr = take(sizeof(DevCounters));
    const size_t o_ka = take(8 * n), o_kb = take(8 * n), o_ia = take(4 * n), o_ib = take(4 * n);
    const size_t o_hist = take(4 * hist_elems);
    const size_t o_part = take(4 * scan_partials_size(scan_max));
    const size_t o_pts = take(sizeof(Pt<T, D>) * n);
    const size_t o_flags = take(4 * n), o_excl = take(4 * n);
    const size_t o_cstart = take(4 * (n + 1)), o_ckey = take(8 * n);
    const size_t o_pflags = take(4 * n), o_pexcl = take(4 * n), o_pstart = take(4 * (n + 1));
    const size_t o_hk = take(8 * cap_max), o_hv = take(4 * cap_max);
    const size_t o_core = take(n), o_ccore = take(n);
    const size_t o_parent = take(4 * n), o_cmin = take(4 * n);
    const size_t o_reps = take(8 * (size_t)n * ndir);
    const bool batched = a.nsets > 0;
    const int nsets = batched ? a.nsets : 1;
    const size_t o_mm = take(sizeof(uint64_t) * 2 * kMaxD * (size_t)nsets);
    const size_t o_gtab = take(sizeof(GridParams) * (size_t)nsets);
    const size_t o_setoff = take(sizeof(int64_t) * ((size_t)nsets + 1));
    const size_t o_box = take(sizeof(double) * 2 * D * (size_t)nsets);
    const size_t main_bytes = off;
    void *ws = nullptr, *ws_ranges = nullptr;
    const bool boxed = a.box_mn != nullptr;
    const bool own_ws = a.ws_ext == nullptr;
    char *b = nullptr;
    DevCounters *ctr = nullptr;
    DevCounters *h = a.h_ext ? a.h_ext : (a.ws_query ? nullptr : host_counters());
    int rc = HCA_OK;
    size_t ranges_bytes = 0;

    cudaEvent_t ev[HCA_NUM_STAGES + 1] = {};
    const bool timing = (a.flags & HCA_FLAG_TIMING) && a.stats && !a.deferred;
    auto mark = [&](int i) { if (timing) cudaEventRecord(ev[i], s); };

    GridParams g;
    Stencil st;
    double tau = 0.0;
    const int gpts = grid_for(n, 256, sms, 8);
    const int gwarp = grid_for(n, 8, sms, 16);
    LowdView<T, D> v;
    memset(&v, 0, sizeof(v));
    bool flipped = false;
    int sort_bits = 0;
    std::vector<GridParams> gsets;
    std::vector<uint64_t> hmm;
    GridParams *d_gtab = nullptr;
    int64_t *d_setoff = nullptr;
    uint64_t *d_mm = nullptr;

    // the grids (one per set, one key layout for all) and the stencil, from the extents of
    // every set: the measured ones, or a plan's declared boxes
    auto build_grids = [&](auto mn_of, auto mx_of) -> int {
        if (!batched) {
            double mn[kMaxD], mx[kMaxD];
            for (int i = 0; i < D; ++i) {
                mn[i] = mn_of(0, i);
                mx[i] = mx_of(0, i);
                if (!isfinite(mn[i]) || !isfinite(mx[i]) || mx[i] < mn[i]) return HCA_EINVAL;
            }
            int r = make_grid(D, sizeof(T) == 4, a.eps, a.min_pts, n, mn, mx, a.flags, g, tau);
            if (r) return r;
            r = make_stencil(D, a.eps, 1.0 / g.inv_side, tau, st);
            if (r) return r;
            sort_bits = g.key_bits;
            return HCA_OK;
        }
        gsets.resize(nsets);
        std::vector<double> e_eps(nsets), e_side(nsets), e_tau(nsets);
        uint32_t bits[kMaxD] = {};
        for (int st_i = 0; st_i < nsets; ++st_i) {
            double mn[kMaxD], mx[kMaxD];
            const bool empty = a.h_off[st_i + 1] == a.h_off[st_i];
            for (int i = 0; i < D; ++i) {
                mn[i] = empty ? 0.0 : mn_of(st_i, i);
                mx[i] = empty ? 0.0 : mx_of(st_i, i);
                if (!isfinite(mn[i]) || !isfinite(mx[i]) || mx[i] < mn[i]) return HCA_EINVAL;
            }
            double tau_s = 0.0;
            const int r = make_grid(D, sizeof(T) == 4, a.h_eps[st_i], a.h_minpts[st_i], n, mn, mx, a.flags,
                                    gsets[st_i], tau_s);
            if (r) return r;
            e_eps[st_i] = a.h_eps[st_i];
            e_side[st_i] = 1.0 / gsets[st_i].inv_side;
            e_tau[st_i] = tau_s;
            for (int i = 0; i < D; ++i) bits[i] = bits[i] > gsets[st_i].bits[i] ? bits[i] : gsets[st_i].bits[i];
        }
        int key_bits = 0, set_bits = 1;
        for (int i = 0; i < D; ++i) key_bits += (int)bits[i];
        while ((1ll << set_bits) < nsets) ++set_bits;
        if (key_bits + set_bits > 63) return HCA_ERANGE;
        for (GridParams &gp : gsets) {
            int sh = 0;
            for (int i = D - 1; i >= 0; --i) {
                gp.bits[i] = bits[i];
                gp.shift[i] = (uint32_t)sh;
                sh += (int)bits[i];
            }
            gp.key_bits = key_bits;
            gp.prefix_shift = (int)bits[D - 1];
        }
        g = gsets[0];
        sort_bits = key_bits + set_bits;
        return make_stencil_union(D, e_eps, e_side, e_tau, st);
    };
    // per-set tables to the device: from pinned staging when the call is deferred (a graph
    // replays the copy), else straight from the host arrays
    auto upload = [&](void *dst, const void *src, size_t bytes, size_t stage_off) {
        if (a.deferred && a.h_stage) {
            memcpy((char *)a.h_stage + stage_off, src, bytes);
            src = (char *)a.h_stage + stage_off;
        }
        cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, s);
    };
    const size_t stage_setoff = 0, stage_gtab = align_up(sizeof(int64_t) * ((size_t)nsets + 1));
    const size_t stage_box = stage_gtab + align_up(sizeof(GridParams) * (size_t)nsets);

    if (!h && !a.ws_query) return HCA_ECUDA;
    if (boxed) {
        rc = build_grids([&](int set, int i) { return a.box_mn[(size_t)set * D + i]; },
                         [&](int set, int i) { return a.box_mx[(size_t)set * D + i]; });
        if (rc) return rc;
        ranges_bytes = sizeof(uint2) * (size_t)n * st.n_all + sizeof(Pt<T, D>) * (size_t)n * ndir + 256;
    }
    if (a.ws_query) {  // plans size their workspace first (declared extents only)
        if (!boxed) {
            // no extents: bound the neighbour ranges with the widest stencil of D, the one of
            // the largest binning error the grid allows (tau = 2^-8) and a side below any side
            // make_grid can choose (eps = 1; a smaller side and more error keep more offsets)
            const double tau_max = ldexp(1.0, -8);
            const double side = (1.0 - ldexp(1.0, -20)) * (1.0 - ldexp(1.0, -10)) /
                                (sqrt((double)D) * (1.0 + 2.0 * tau_max));
            Stencil wide;
            if (make_stencil(D, 1.0, side, tau_max, wide) != HCA_OK) return HCA_ENOTIMPL;
            ranges_bytes = sizeof(uint2) * (size_t)n * wide.n_all + sizeof(Pt<T, D>) * (size_t)n * ndir + 256;
        }
        *a.ws_query = main_bytes + ranges_bytes;
        return HCA_OK;
    }
    if (!own_ws) {
        if (!boxed || a.ws_ext_bytes < main_bytes + ranges_bytes) return HCA_EINVAL;
        ws = a.ws_ext;
        ws_ranges = (char *)a.ws_ext + main_bytes;
    } else {
        if (pool_alloc(&ws, main_bytes + ranges_bytes, s) != cudaSuccess || !ws) return HCA_ENOMEM;
        if (boxed) ws_ranges = (char *)ws + main_bytes;
    }
    b = (char *)ws;
    ctr = (DevCounters *)(b + o_ctr);
    d_gtab = (GridParams *)(b + o_gtab);
    d_setoff = (int64_t *)(b + o_setoff);
    d_mm = (uint64_t *)(b + o_mm);
    if (timing)
        for (int i = 0; i <= HCA_NUM_STAGES; ++i) cudaEventCreate(&ev[i]);

    mark(0);
    cudaMemsetAsync(ctr, 0, sizeof(DevCounters), s);
    cudaMemsetAsync(ctr->minmax_enc, 0xff, sizeof(uint64_t) * kMaxD, s);
    if (!batched) {
        k_minmax<T, D><<<grid_for(n, 256, sms, 2), 256, 0, s>>>((const T *)a.d_points, n, ctr);
    } else {
        cudaMemsetAsync(d_mm, 0xff, sizeof(uint64_t) * kMaxD * nsets, s);
        cudaMemsetAsync(d_mm + (size_t)kMaxD * nsets, 0, sizeof(uint64_t) * kMaxD * nsets, s);
        upload(d_setoff, a.h_off, sizeof(int64_t) * (nsets + 1), stage_setoff);
        k_minmax_seg<T, D><<<grid_for(n, 256, sms, 8), 256, 0, s>>>((const T *)a.d_points, n, d_setoff, nsets,
                                                                  (unsigned long long *)d_mm, ctr);
        if (!boxed) {
            hmm.resize((size_t)2 * kMaxD * nsets);
            cudaMemcpyAsync(hmm.data(), d_mm, sizeof(uint64_t) * hmm.size(), cudaMemcpyDeviceToHost, s);
        }
    }
    ++launches;
    if (boxed) {
        // declared extents: check them on the device, no host round trip
        BoxArgs one;
        memset(&one, 0, sizeof(one));
        double *d_box = nullptr;
        if (!batched) {
            for (int i = 0; i < D; ++i) {
                one.mn[i] = a.box_mn[i];
                one.mx[i] = a.box_mx[i];
            }
        } else {
            std::vector<double> boxes((size_t)2 * D * nsets);
            memcpy(boxes.data(), a.box_mn, sizeof(double) * D * nsets);
            memcpy(boxes.data() + (size_t)D * nsets, a.box_mx, sizeof(double) * D * nsets);
            d_box = (double *)(b + o_box);
            upload(d_box, boxes.data(), sizeof(double) * boxes.size(), stage_box);
            upload(d_gtab, gsets.data(), sizeof(GridParams) * nsets, stage_gtab);
        }
        k_box_check<D><<<grid_for((int64_t)nsets * D, 256, sms, 1), 256, 0, s>>>(
            one, d_box, nsets, d_setoff, (const unsigned long long *)d_mm, ctr);
        ++launches;
    } else {
        if (cudaMemcpyAsync(h, ctr, sizeof(DevCounters), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess) { rc = HCA_ECUDA; goto out; }
        if (h->nan_seen) { rc = HCA_EINVAL; goto out; }
        if (a.ext_out && !batched)
            for (int i = 0; i < D; ++i) {
                a.ext_out[i] = dec_double(h->minmax_enc[i]);
                a.ext_out[D + i] = dec_double(h->minmax_enc[kMaxD + i]);
            }
        if (batched)
            rc = build_grids([&](int set, int i) { return dec_double(hmm[(size_t)set * kMaxD + i]); },
                             [&](int set, int i) { return dec_double(hmm[(size_t)kMaxD * nsets + (size_t)set * kMaxD + i]); });
        else
            rc = build_grids([&](int, int i) { return dec_double(h->minmax_enc[i]); },
                             [&](int, int i) { return dec_double(h->minmax_enc[kMaxD + i]); });
        if (rc) goto out;
        if (batched) cudaMemcpyAsync(d_gtab, gsets.data(), sizeof(GridParams) * nsets, cudaMemcpyHostToDevice, s);
        // neighbour ranges (one (lo, hi) pair per cell and stencil pencil) and the coordinates
        // of the representative points (ndir per cell)
        ranges_bytes = sizeof(uint2) * (size_t)n * st.n_all + sizeof(Pt<T, D>) * (size_t)n * ndir + 256;
        if (pool_alloc(&ws_ranges, ranges_bytes, s) != cudaSuccess || !ws_ranges) {
            rc = HCA_ENOMEM;
            goto out;
        }
    }
    mark(1);
    // ---- Algorithm 1: cell keys; pre-sort (Sec. 2) by a radix sort of (key, index) ----
    {
        uint32_t *ia = (uint32_t *)(b + o_ia), *ib = (uint32_t *)(b + o_ib);
        uint32_t *hist = (uint32_t *)(b + o_hist), *part = (uint32_t *)(b + o_part);
        const bool use32 = sort_bits <= 32;
        const int gtile = (int)((n + kScanTileElems - 1) / kScanTileElems);  // gather: one block per scan tile
        if (use32) {
            uint32_t *ka = (uint32_t *)(b + o_ka), *kb = (uint32_t *)(b + o_kb);
            if (batched)
                k_bin_seg<T, D, uint32_t><<<gpts, 256, 0, s>>>((const T *)a.d_points, n, d_setoff, nsets, d_gtab,
                                                               g.key_bits, ka, ia, ctr->digit_counts, sort_bits);
            else
                k_bin<T, D, uint32_t><<<gpts, 256, 0, s>>>((const T *)a.d_points, g, ka, ia, ctr->digit_counts);
            ++launches;
            mark(2);
            flipped = radix_sort_pairs<uint32_t>(ka, ia, kb, ib, n, 0, sort_bits, hist, part, s, &launches, &ctr->status, ctr->digit_counts);
            mark(3);
            k_gather<T, D, uint32_t><<<gtile, 256, 0, s>>>((const T *)a.d_points, flipped ? kb : ka,
                                                           flipped ? ib : ia, n, (Pt<T, D> *)(b + o_pts),
                                                           (uint32_t *)(b + o_flags), part);
        } else {
            uint64_t *ka = (uint64_t *)(b + o_ka), *kb = (uint64_t *)(b + o_kb);
            if (batched)
                k_bin_seg<T, D, uint64_t><<<gpts, 256, 0, s>>>((const T *)a.d_points, n, d_setoff, nsets, d_gtab,
                                                               g.key_bits, ka, ia, ctr->digit_counts, sort_bits);
            else
                k_bin<T, D, uint64_t><<<gpts, 256, 0, s>>>((const T *)a.d_points, g, ka, ia, ctr->digit_counts);
            ++launches;
            mark(2);
            flipped = radix_sort_pairs<uint64_t>(ka, ia, kb, ib, n, 0, sort_bits, hist, part, s, &launches, &ctr->status, ctr->digit_counts);
            mark(3);
            k_gather<T, D, uint64_t><<<gtile, 256, 0, s>>>((const T *)a.d_points, flipped ? kb : ka,
                                                           flipped ? ib : ia, n, (Pt<T, D> *)(b + o_pts),
                                                           (uint32_t *)(b + o_flags), part);
        }
        ++launches;
        // run-length cells: scan of the gather's tile counts, cell ids / starts / keys
        if (use32)
            cells_from_flags<uint32_t>((const uint32_t *)(b + (flipped ? o_kb : o_ka)), (uint32_t *)(b + o_flags), n,
                                       part, &ctr->n_cells, (uint32_t *)(b + o_cstart), (uint64_t *)(b + o_ckey), s,
                                       &launches);
        else
            cells_from_flags<uint64_t>((const uint64_t *)(b + (flipped ? o_kb : o_ka)), (uint32_t *)(b + o_flags), n,
                                       part, &ctr->n_cells, (uint32_t *)(b + o_cstart), (uint64_t *)(b + o_ckey), s,
                                       &launches);
        v.perm = flipped ? ib : ia;
    }
    mark(4);
    // ---- pencils and their hash table ----
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
        launches += 3;
    }
    v.g = g;
    v.gtab = batched ? d_gtab : nullptr;
    v.set_off = batched ? d_setoff : nullptr;
    v.in = (const T *)a.d_points;
    v.pts = (const Pt<T, D> *)(b + o_pts);
    v.cell_of = (const uint32_t *)(b + o_flags);
    v.cell_start = (const uint32_t *)(b + o_cstart);
    v.cell_key = (const uint64_t *)(b + o_ckey);
    v.pencil_start = (const uint32_t *)(b + o_pstart);
    v.hkeys = (uint64_t *)(b + o_hk);
    v.hvals = (uint32_t *)(b + o_hv);
    v.core = (uint8_t *)(b + o_core);
    v.cell_core = (uint8_t *)(b + o_ccore);
    v.parent = (uint32_t *)(b + o_parent);
    v.reps = (uint64_t *)(b + o_reps);
    v.comp_min = (uint32_t *)(b + o_cmin);
    v.ranges = (uint2 *)ws_ranges;
    v.list_count = (uint32_t *)(b + o_excl);   // the scan scratch of the cell and pencil passes is free now
    v.list_core = (uint32_t *)(b + o_pflags);
    v.list_label = (uint32_t *)(b + o_pexcl);
    v.rep_pts = (Pt<T, D> *)((char *)ws_ranges + align_up(sizeof(uint2) * (size_t)n * st.n_all));
    v.labels = a.d_labels;
    v.core_out = a.d_core;
    v.ctr = ctr;
    // ---- neighbour cells of every cell (stencil pencils -> cell ranges) ----
    k_ranges<T, D><<<grid_for((n / kRangeRun + 1) * (int64_t)st.n_all, 256, sms, 16), 256, 0, s>>>(v, st);
    ++launches;
    mark(5);
    // ---- Definition 2: triage of the cells, then dense cells and exact counts ----
    k_triage<T, D><<<gpts, 256, 0, s>>>(v, st.n_all);
    k_core<T, D><<<gwarp, 256, 0, s>>>(v, st);
    launches += 2;
    // ---- Algorithm 2: representative points and their coordinates (the stage times k_reps
    // alone; the coordinates of boundary-crossing cells are counted with the merge stage) ----
    mark(6);
    k_reps<T, D><<<(unsigned)((n + (int64_t)kRepWin * kRepWarps - 1) / ((int64_t)kRepWin * kRepWarps)),
                   32 * kRepWarps, 0, s>>>(v, n);
    mark(7);
    k_rep_fix<T, D><<<grid_for((n / RepGeom<D>::sub + 1) * ndir, 256, sms, 8), 256, 0, s>>>(v, n);
    launches += 2;
    // ---- Algorithm 3: first links, pointer jumping, then one merge pass over every pair ----
    k_hook<T, D><<<gwarp, 256, 0, s>>>(v, st.n_all, st.n_half);
    for (int r = 0; r < 3; ++r) k_jump<T, D><<<gpts, 256, 0, s>>>(v);
    launches += 4;
    k_merge<T, D><<<gwarp, 256, 0, s>>>(v, st.n_all, st.n_half, 2);
    k_compress<T, D><<<gpts, 256, 0, s>>>(v, 1);
    launches += 2;
    mark(8);
    // ---- Algorithm 4: cluster ids, border and noise ----
    k_comp_min<T, D><<<gpts, 256, 0, s>>>(v);
    {
        // the core points' labels (point-parallel, bandwidth) on a second stream beside the
        // border search (latency-bound, few cells): they write disjoint points
        const SideStream ss = side_stream();
        if (ss.ok && cudaEventRecord(ss.fork, s) == cudaSuccess && cudaStreamWaitEvent(ss.s, ss.fork, 0) == cudaSuccess) {
            k_label_core<T, D><<<gpts, 256, 0, ss.s>>>(v);
            k_labels<T, D><<<gwarp, 256, 0, s>>>(v, st.n_all);
            cudaEventRecord(ss.join, ss.s);
            cudaStreamWaitEvent(s, ss.join, 0);
        } else {
            k_label_core<T, D><<<gpts, 256, 0, s>>>(v);
            k_labels<T, D><<<gwarp, 256, 0, s>>>(v, st.n_all);
        }
    }
    launches += 3;
    mark(9);
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
        hca_stats *st_out = a.stats;
        st_out->n_points = n;
        st_out->n_cells = h->n_cells;
        st_out->n_pencils = h->n_pencils;
        st_out->n_dense_cells = h->n_dense;
        st_out->n_core_cells = h->n_core_cells;
        st_out->workspace_bytes = (int64_t)(main_bytes + ranges_bytes);
        st_out->n_core_points = h->n_core;
        st_out->n_clusters = h->n_clusters;
        st_out->n_noise = h->n_noise;
        st_out->key_bits = sort_bits;
        st_out->sort_passes = (sort_bits + 7) / 8;
        st_out->kernel_launches = launches;
        st_out->n_count_chunks = (int64_t)h->work[0];
        st_out->n_rep_tests = (int64_t)h->work[1];
        st_out->n_rep_hits = (int64_t)h->work[2];
        st_out->n_exhaustive_pairs = (int64_t)h->work[3];
        st_out->n_exhaustive_chunks = (int64_t)h->work[4];
        st_out->n_border_chunks = (int64_t)h->work[5];
        for (int i = 0; i < HCA_NUM_STAGES; ++i) {
            float ms = 0.f;
            if (timing) cudaEventElapsedTime(&ms, ev[i], ev[i + 1]);
            st_out->stage_ms[i] = ms;
        }
    }
out:
    if (timing)
        for (int i = 0; i <= HCA_NUM_STAGES; ++i)
            if (ev[i]) cudaEventDestroy(ev[i]);
    if (!boxed) pool_free(ws_ranges, s);  // with declared extents it is part of ws
    if (own_ws) pool_free(ws, s);
    if (rc != HCA_OK && !a.deferred) cudaStreamSynchronize(s);
    return rc;
}

}  // namespace hca
