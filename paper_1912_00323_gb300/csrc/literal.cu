// hca_dbscan_literal_device: the paper's Algorithms 2-4 as printed, on the GPU, for d <= 4.
//
// An ablation, not DBSCAN: it shows what the printed algorithm computes.  Readings of the
// printed text (the same ones the oracle's literal variant takes):
//   - hypercubes of side exactly eps / sqrt(d) from the per-dimension minimum (Algorithm 1,
//     Sec. 2 "Overlaying Hypercubes"); band index floor((x - min) / side) in double precision;
//   - representative points over all points of a cube (Algorithm 2): for each of the 3^d - 1
//     directions, the point closest to the cube's face, edge or corner in that direction (its
//     "ideal position"), the smallest input index among equally close points;
//   - neighbouring cubes: offsets in [-R, R]^d with R = ceil(sqrt(d)), without the cube itself
//     and the corner cubes (Sec. 2, "Depth First Search"; 20 cubes in 2-D);
//   - two neighbouring cubes belong to one cluster when their representative points of
//     complementary directions are strictly closer than eps (Algorithm 3, "< eps");
//   - every non-empty cube belongs to a cluster: no MINPTS, no noise (Algorithm 4).
// Labels follow the library's canonical rule: the smallest input index of the cluster.
//
// Kernels: min/max (the library's), binning into packed cube keys, the library's radix sort
// and run-length cells, one thread per (cube, direction) for the representatives, one thread
// per (cube, neighbour offset) for the merge (binary search of the neighbour's key among the
// sorted cube keys, lock-free union-find), then the smallest index per component.
#include "lowd_run.cuh"

namespace hca {
namespace {

constexpr int kLitMaxD = 4;

struct LitParams {
    int d;
    int ndir;                 // 3^d - 1
    int noff;                 // neighbour offsets
    double origin[kLitMaxD];
    double side;
    double eps2;
    uint32_t cmax[kLitMaxD];  // largest band index per dimension
    uint32_t shift[kLitMaxD]; // bit position of each band index in the cube key (dimension 0 highest)
};

// Band indices of every point, packed into a key ordered lexicographically by (c_0, ..., c_{d-1}).
template <typename T, typename K>
__global__ void __launch_bounds__(256) k_lit_bin(const T *__restrict__ x, int64_t n, LitParams p,
                                                K *__restrict__ keys, uint32_t *__restrict__ idx) {
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x) {
        uint64_t key = 0;
        for (int i = 0; i < p.d; ++i) {
            const double t = floor(__ddiv_rn(__dsub_rn((double)x[j * p.d + i], p.origin[i]), p.side));
            uint32_t c = t < 0.0 ? 0u : (uint32_t)t;
            if (c > p.cmax[i]) c = p.cmax[i];
            key |= (uint64_t)c << p.shift[i];
        }
        keys[j] = (K)key;
        idx[j] = (uint32_t)j;
    }
}

// First-of-cube flags of the sorted keys, and the flag count of every scan tile.
template <typename K>
__global__ void __launch_bounds__(256) k_lit_flags(const K *__restrict__ keys, int64_t n, uint32_t *__restrict__ flags,
                                                  uint32_t *__restrict__ tile_sums) {
    const int64_t base = (int64_t)blockIdx.x * kScanTileElems;
    uint32_t cnt = 0;
#pragma unroll
    for (int k = 0; k < kScanTileElems / 256; ++k) {
        const int64_t j = base + k * 256 + threadIdx.x;
        if (j < n) {
            const uint32_t f = (j == 0 || keys[j] != keys[j - 1]) ? 1u : 0u;
            flags[j] = f;
            cnt += f;
        }
    }
    uint32_t total;
    block_exclusive_scan<256>(cnt, &total);
    if (threadIdx.x == 0) tile_sums[blockIdx.x] = total;
}

__device__ __forceinline__ void lit_coords(uint64_t key, const LitParams &p, uint32_t *c) {
    for (int i = 0; i < p.d; ++i) {
        const uint32_t bits = (i == 0 ? 64u : p.shift[i - 1]) - p.shift[i];
        c[i] = (uint32_t)((key >> p.shift[i]) & (bits >= 64 ? ~0ull : ((1ull << bits) - 1ull)));
    }
}

// Direction r of the representative table: every delta in {-1, 0, 1}^d but 0, delta_0 varying
// fastest.
__device__ __forceinline__ void lit_dir(int r, int d, int *delta) {
    int total = 1;
    for (int i = 0; i < d; ++i) total *= 3;
    int code = r < (total - 1) / 2 ? r : r + 1;
    for (int i = 0; i < d; ++i) {
        delta[i] = code % 3 - 1;
        code /= 3;
    }
}

// Algorithm 2: per cube and direction, the point closest to the ideal position (squared
// distance over the dimensions the direction constrains, double precision in dimension order);
// points are visited in increasing input index and a later one wins only when strictly closer.
template <typename T>
__global__ void __launch_bounds__(256) k_lit_reps(const T *__restrict__ x, const uint32_t *__restrict__ idx,
                                                 const uint32_t *__restrict__ cell_start,
                                                 const uint64_t *__restrict__ cell_key, const DevCounters *ctr,
                                                 LitParams p, uint32_t *__restrict__ rep) {
    const uint64_t total = (uint64_t)ctr->n_cells * p.ndir;
    for (uint64_t t = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; t < total; t += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t c = (uint32_t)(t / p.ndir);
        const int r = (int)(t % p.ndir);
        int delta[kLitMaxD];
        lit_dir(r, p.d, delta);
        uint32_t cc[kLitMaxD];
        lit_coords(cell_key[c], p, cc);
        double ideal[kLitMaxD];
        for (int i = 0; i < p.d; ++i)
            ideal[i] = __dadd_rn(p.origin[i], __dmul_rn((double)(cc[i] + (delta[i] > 0 ? 1u : 0u)), p.side));
        uint32_t best = 0xffffffffu;
        double best_s = 0.0;
        for (uint32_t k = cell_start[c]; k < cell_start[c + 1]; ++k) {
            const uint32_t q = idx[k];
            double s = 0.0;
            for (int i = 0; i < p.d; ++i) {
                if (delta[i] == 0) continue;
                const double u = __dsub_rn(ideal[i], (double)x[(int64_t)q * p.d + i]);
                s = __dadd_rn(s, __dmul_rn(u, u));
            }
            if (best == 0xffffffffu || s < best_s) {
                best = q;
                best_s = s;
            }
        }
        rep[(uint64_t)c * p.ndir + r] = best;
    }
}

// Cube with key `key` among the sorted cube keys, or ~0.
__device__ __forceinline__ uint32_t lit_lookup(const uint64_t *__restrict__ cell_key, uint32_t C, uint64_t key) {
    uint32_t lo = 0, hi = C;
    while (lo < hi) {
        const uint32_t mid = (lo + hi) >> 1;
        if (__ldg(cell_key + mid) < key) lo = mid + 1; else hi = mid;
    }
    return (lo < C && __ldg(cell_key + lo) == key) ? lo : 0xffffffffu;
}

// Index in the direction table of sign(delta).
__device__ __forceinline__ int lit_dir_index(const int *delta, int d) {
    int code = 0, mul = 1;
    for (int i = 0; i < d; ++i) {
        const int s = delta[i] > 0 ? 1 : (delta[i] < 0 ? -1 : 0);
        code += (s + 1) * mul;
        mul *= 3;
    }
    const int zero = (mul - 1) / 2;
    return code < zero ? code : code - 1;
}

// Algorithm 3: cube a and each neighbour b > a (in key order) are joined when the
// representative of a towards b and the representative of b towards a are strictly closer than
// eps (squared distance in double precision, dimension order).
template <typename T>
__global__ void __launch_bounds__(256) k_lit_merge(const T *__restrict__ x, const uint64_t *__restrict__ cell_key,
                                                  DevCounters *ctr, LitParams p, const int8_t *__restrict__ offs,
                                                  const uint32_t *__restrict__ rep, uint32_t *parent) {
    const uint32_t C = ctr->n_cells;
    const uint64_t total = (uint64_t)C * p.noff;
    for (uint64_t t = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; t < total; t += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t a = (uint32_t)(t / p.noff);
        const int o = (int)(t % p.noff);
        uint32_t ca[kLitMaxD];
        lit_coords(cell_key[a], p, ca);
        int delta[kLitMaxD];
        uint64_t key = 0;
        bool inside = true;
        for (int i = 0; i < p.d; ++i) {
            delta[i] = offs[o * kLitMaxD + i];
            const int64_t cb = (int64_t)ca[i] + delta[i];
            if (cb < 0 || cb > (int64_t)p.cmax[i]) inside = false;
            key |= (uint64_t)(cb < 0 ? 0 : cb) << p.shift[i];
        }
        if (!inside) continue;
        const uint32_t b = lit_lookup(cell_key, C, key);
        if (b == 0xffffffffu || b <= a) continue;
        const int di = lit_dir_index(delta, p.d);
        const uint32_t ra = rep[(uint64_t)a * p.ndir + di];
        const uint32_t rb = rep[(uint64_t)b * p.ndir + (p.ndir - 1 - di)];
        double s = 0.0;
        for (int i = 0; i < p.d; ++i) {
            const double u = __dsub_rn((double)x[(int64_t)ra * p.d + i], (double)x[(int64_t)rb * p.d + i]);
            s = __dadd_rn(s, __dmul_rn(u, u));
        }
        if (s < p.eps2) uf_union(parent, a, b, ctr);
    }
}

__global__ void __launch_bounds__(256) k_lit_uf_init(const DevCounters *ctr, uint32_t *parent, uint32_t *comp_min) {
    const uint32_t C = ctr->n_cells;
    for (uint32_t c = blockIdx.x * blockDim.x + threadIdx.x; c < C; c += gridDim.x * blockDim.x) {
        parent[c] = c;
        comp_min[c] = 0xffffffffu;
    }
}

// Algorithm 4 with the canonical ids: the smallest input index of every component, then every
// point's label.  cell_of and idx are in sorted order.
__global__ void __launch_bounds__(256) k_lit_comp_min(const uint32_t *__restrict__ cell_of, const uint32_t *__restrict__ idx,
                                                     int64_t n, DevCounters *ctr, const uint32_t *parent,
                                                     uint32_t *comp_min) {
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x)
        atomicMin(comp_min + uf_root_readonly(parent, cell_of[j], ctr), idx[j]);
}

__global__ void __launch_bounds__(256) k_lit_labels(const uint32_t *__restrict__ cell_of, const uint32_t *__restrict__ idx,
                                                   int64_t n, DevCounters *ctr, const uint32_t *parent,
                                                   const uint32_t *__restrict__ comp_min, int32_t *labels) {
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x)
        labels[idx[j]] = (int32_t)comp_min[uf_root_readonly(parent, cell_of[j], ctr)];
}

template <typename T, int D>
int run_literal(const T *d_points, int64_t n, double eps, int32_t *d_labels, cudaStream_t s, int *launches_out) {
    using namespace detail;
    const int sms = device_sm_count();
    if (sms <= 0) return HCA_ECUDA;
    int launches = 0;
    LitParams p;
    memset(&p, 0, sizeof(p));
    p.d = D;
    p.ndir = 1;
    for (int i = 0; i < D; ++i) p.ndir *= 3;
    p.ndir -= 1;
    p.side = eps / sqrt((double)D);
    p.eps2 = eps * eps;
    // neighbour offsets: [-R, R]^d without 0 and the corners, R = ceil(sqrt(d))
    const int R = (int)ceil(sqrt((double)D));
    std::vector<int8_t> offs;
    {
        int delta[kLitMaxD];
        for (int i = 0; i < D; ++i) delta[i] = -R;
        for (;;) {
            bool zero = true, corner = true;
            for (int i = 0; i < D; ++i) {
                const int a = delta[i] < 0 ? -delta[i] : delta[i];
                if (a != 0) zero = false;
                if (a != R) corner = false;
            }
            if (!zero && !corner)
                for (int i = 0; i < kLitMaxD; ++i) offs.push_back((int8_t)(i < D ? delta[i] : 0));
            int i = 0;
            while (i < D && delta[i] == R) delta[i++] = -R;
            if (i == D) break;
            ++delta[i];
        }
    }
    p.noff = (int)(offs.size() / kLitMaxD);

    // workspace
    size_t off = 0;
    auto take = [&](size_t bytes) { size_t o = off; off = align_up(off + bytes); return o; };
    const size_t o_ctr = take(sizeof(DevCounters));
    const size_t o_ka = take(8 * n), o_kb = take(8 * n), o_ia = take(4 * n), o_ib = take(4 * n);
    const size_t o_hist = take(4 * sort_hist_size(n));
    const size_t o_part = take(4 * scan_partials_size(n));
    const size_t o_flags = take(4 * n), o_cstart = take(4 * (n + 1)), o_ckey = take(8 * n);
    const size_t o_rep = take(4 * (size_t)n * p.ndir);
    const size_t o_parent = take(4 * n), o_cmin = take(4 * n);
    const size_t o_offs = take(offs.size());
    void *ws = nullptr;
    if (pool_alloc(&ws, off, s) != cudaSuccess || !ws) return HCA_ENOMEM;
    char *b = (char *)ws;
    DevCounters *ctr = (DevCounters *)(b + o_ctr);
    DevCounters *h = host_counters();
    int rc = HCA_OK;
    const int gpts = grid_for(n, 256, sms, 8);
    bool flipped = false;
    cudaMemsetAsync(ctr, 0, sizeof(DevCounters), s);
    cudaMemsetAsync(ctr->minmax_enc, 0xff, sizeof(uint64_t) * kMaxD, s);
    k_minmax<T, D><<<grid_for(n, 256, sms, 2), 256, 0, s>>>(d_points, n, ctr);
    ++launches;
    if (cudaMemcpyAsync(h, ctr, sizeof(DevCounters), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess) {
        rc = HCA_ECUDA;
        goto out;
    }
    if (h->nan_seen) { rc = HCA_EINVAL; goto out; }
    {
        int sh = 0;
        for (int i = D - 1; i >= 0; --i) {
            p.origin[i] = dec_double(h->minmax_enc[i]);
            const double mx = dec_double(h->minmax_enc[kMaxD + i]);
            if (!isfinite(p.origin[i]) || !isfinite(mx)) { rc = HCA_EINVAL; goto out; }
            const double t = floor((mx - p.origin[i]) / p.side);
            if (!(t < 4294967295.0)) { rc = HCA_ERANGE; goto out; }
            p.cmax[i] = (uint32_t)t;
            int bits = 1;
            while (bits < 32 && ((uint64_t)p.cmax[i] >> bits) != 0) ++bits;
            p.shift[i] = (uint32_t)sh;
            sh += bits;
        }
        if (sh > 64) { rc = HCA_ERANGE; goto out; }
        const int key_bits = sh;
        int8_t *d_offs = (int8_t *)(b + o_offs);
        if (cudaMemcpyAsync(d_offs, offs.data(), offs.size(), cudaMemcpyHostToDevice, s) != cudaSuccess) {
            rc = HCA_ECUDA;
            goto out;
        }
        uint32_t *ia = (uint32_t *)(b + o_ia), *ib = (uint32_t *)(b + o_ib);
        uint32_t *hist = (uint32_t *)(b + o_hist), *part = (uint32_t *)(b + o_part);
        const int gtile = (int)((n + kScanTileElems - 1) / kScanTileElems);
        uint32_t *flags = (uint32_t *)(b + o_flags), *cstart = (uint32_t *)(b + o_cstart);
        uint64_t *ckey = (uint64_t *)(b + o_ckey);
        if (key_bits <= 32) {
            uint32_t *ka = (uint32_t *)(b + o_ka), *kb = (uint32_t *)(b + o_kb);
            k_lit_bin<T, uint32_t><<<gpts, 256, 0, s>>>(d_points, n, p, ka, ia);
            flipped = radix_sort_pairs<uint32_t>(ka, ia, kb, ib, n, 0, key_bits, hist, part, s, &launches, &ctr->status);
            const uint32_t *ks = flipped ? kb : ka;
            k_lit_flags<uint32_t><<<gtile, 256, 0, s>>>(ks, n, flags, part);
            cells_from_flags<uint32_t>(ks, flags, n, part, &ctr->n_cells, cstart, ckey, s, &launches);
        } else {
            uint64_t *ka = (uint64_t *)(b + o_ka), *kb = (uint64_t *)(b + o_kb);
            k_lit_bin<T, uint64_t><<<gpts, 256, 0, s>>>(d_points, n, p, ka, ia);
            flipped = radix_sort_pairs<uint64_t>(ka, ia, kb, ib, n, 0, key_bits, hist, part, s, &launches, &ctr->status);
            const uint64_t *ks = flipped ? kb : ka;
            k_lit_flags<uint64_t><<<gtile, 256, 0, s>>>(ks, n, flags, part);
            cells_from_flags<uint64_t>(ks, flags, n, part, &ctr->n_cells, cstart, ckey, s, &launches);
        }
        launches += 2;
        const uint32_t *perm = flipped ? ib : ia;
        uint32_t *rep = (uint32_t *)(b + o_rep), *parent = (uint32_t *)(b + o_parent), *cmin = (uint32_t *)(b + o_cmin);
        k_lit_reps<T><<<grid_for((int64_t)n * p.ndir, 256, sms, 8), 256, 0, s>>>(d_points, perm, cstart, ckey, ctr, p, rep);
        k_lit_uf_init<<<gpts, 256, 0, s>>>(ctr, parent, cmin);
        k_lit_merge<T><<<grid_for((int64_t)n * p.noff, 256, sms, 8), 256, 0, s>>>(d_points, ckey, ctr, p, d_offs, rep,
                                                                                    parent);
        k_lit_comp_min<<<gpts, 256, 0, s>>>(flags, perm, n, ctr, parent, cmin);
        k_lit_labels<<<gpts, 256, 0, s>>>(flags, perm, n, ctr, parent, cmin, d_labels);
        launches += 5;
    }
    if (cudaGetLastError() != cudaSuccess) { rc = HCA_ECUDA; goto out; }
    if (cudaMemcpyAsync(h, ctr, sizeof(DevCounters), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess) {
        rc = HCA_ECUDA;
        goto out;
    }
    if (h->status) rc = HCA_EDEVICE;
    if (launches_out) *launches_out = launches;
out:
    pool_free(ws, s);
    if (rc != HCA_OK) cudaStreamSynchronize(s);
    return rc;
}

}  // namespace
}  // namespace hca

using namespace hca;

extern "C" int hca_dbscan_literal_device(const void *d_points, int32_t dtype, int64_t n, int32_t d, double eps,
                                         int32_t *d_labels, void *stream) {
    if (d < 1 || d > kLitMaxD) return HCA_EINVAL;
    int rc = check_common(d_points, dtype, n, d, eps, 1, d_labels);
    if (rc) return rc;
    if (n == 0) return HCA_OK;
    const size_t esz = dtype == HCA_F32 ? 4 : 8;
    if (((uintptr_t)d_points) % esz || ((uintptr_t)d_labels) % 4) return HCA_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    int launches = 0;
    if (dtype == HCA_F32) {
        const float *x = (const float *)d_points;
        switch (d) {
            case 1: return run_literal<float, 1>(x, n, eps, d_labels, s, &launches);
            case 2: return run_literal<float, 2>(x, n, eps, d_labels, s, &launches);
            case 3: return run_literal<float, 3>(x, n, eps, d_labels, s, &launches);
            default: return run_literal<float, 4>(x, n, eps, d_labels, s, &launches);
        }
    }
    const double *x = (const double *)d_points;
    switch (d) {
        case 1: return run_literal<double, 1>(x, n, eps, d_labels, s, &launches);
        case 2: return run_literal<double, 2>(x, n, eps, d_labels, s, &launches);
        case 3: return run_literal<double, 3>(x, n, eps, d_labels, s, &launches);
        default: return run_literal<double, 4>(x, n, eps, d_labels, s, &launches);
    }
}
