// Kernels of the hypercube-stencil path (1 <= d <= 4), templated on the coordinate type T
// (float or double) and the dimension D.
//
// Data layout in device memory after the sort (all arrays indexed in "cell order", the
// order of the sorted cell keys; ties keep input order):
//   pts[j]          the j-th point, padded to 1/2/4/4 coordinates (16-byte rows for d = 3)
//   perm[j]         its input index
//   cell_of[j]      its cell id;  cells are numbered in key order
//   cell_start[c]   first j of cell c (cell_start[C] = n);  cell_key[c] its packed key
//   pencil_start[p] first cell of pencil p; a pencil is a maximal run of cells that share
//                   every coordinate but the last, so its cells are consecutive in key order
//   hash            pencil key -> pencil id (open addressing, linear probing)
//   core[j], cell_core[c], parent[c] (union-find), reps[c * ndir + r], comp_min[c]
#pragma once

#include <float.h>

#include "hca_internal.cuh"

namespace hca {

template <typename T, int D>
struct LowdView {
    GridParams g;
    const T *in;                  // input points, row-major n x D
    const Pt<T, D> *pts;          // sorted, padded
    const uint32_t *perm;
    const uint32_t *cell_of;
    const uint32_t *cell_start;
    const uint64_t *cell_key;
    const uint32_t *pencil_start;
    uint64_t *hkeys;
    uint32_t *hvals;
    uint8_t *core;
    uint8_t *cell_core;
    uint32_t *parent;
    uint64_t *reps;
    uint32_t *comp_min;
    int32_t *labels;              // output, input order
    uint8_t *core_out;            // optional output, input order
    DevCounters *ctr;
};

// ------------------------------------------------------------------------------------------
// Small helpers
// ------------------------------------------------------------------------------------------

__device__ __forceinline__ uint64_t enc_double(double f) {
    uint64_t b = (uint64_t)__double_as_longlong(f);
    return (b >> 63) ? ~b : (b | 0x8000000000000000ull);
}

__device__ __forceinline__ uint64_t mix64(uint64_t x) {
    x ^= x >> 30;
    x *= 0xbf58476d1ce4e5b9ull;
    x ^= x >> 27;
    x *= 0x94d049bb133111ebull;
    x ^= x >> 31;
    return x;
}

__device__ __forceinline__ int global_warp() {
    return (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5);
}
__device__ __forceinline__ int total_warps() { return (int)((gridDim.x * (int64_t)blockDim.x) >> 5); }
__device__ __forceinline__ int lane_id() { return threadIdx.x & 31; }

__device__ __forceinline__ void set_error(DevCounters *ctr, uint32_t bit) {
    atomicOr(&ctr->status, bit);
}

// Number of representative directions kept per cell: all 3^D - 1 for D <= 3 (Sec. 2), the
// 2D axis directions for D = 4.
template <int D>
struct RepDirs {
    static constexpr int value = (D == 1) ? 2 : (D == 2) ? 8 : (D == 3) ? 26 : 2 * D;
};

// Direction index of sign(delta) and of its complement -sign(delta).
template <int D>
__device__ __forceinline__ int rep_dir_of(const int *delta) {
    if (D <= 3) {
        int code = 0, mul = 1;
#pragma unroll
        for (int i = 0; i < D; ++i) {
            int s = delta[i] > 0 ? 1 : (delta[i] < 0 ? -1 : 0);
            code += (s + 1) * mul;
            mul *= 3;
        }
        const int zero = (mul - 1) / 2;
        return code < zero ? code : code - 1;
    } else {
        int best = 0, mag = -1;
#pragma unroll
        for (int i = 0; i < D; ++i) {
            int a = delta[i] < 0 ? -delta[i] : delta[i];
            if (a > mag) { mag = a; best = i; }
        }
        return 2 * best + (delta[best] > 0 ? 1 : 0);
    }
}
template <int D>
__device__ __forceinline__ int rep_dir_complement(int r) {
    return (D <= 3) ? (RepDirs<D>::value - 1 - r) : (r ^ 1);
}

// ------------------------------------------------------------------------------------------
// The predicate dist(p, q) <= eps (Definition 1), decided exactly as
// fl64(sum_i (p_i - q_i)^2) <= fl64(eps^2), summed in dimension order without fused
// multiply-add.  For float input an FP32 sum with fused multiply-add decides every pair
// outside a relative guard band of 2^-16 around eps^2 (its error is below (D+2) 2^-24 of
// the sum), and the pairs inside the band are decided by the FP64 sum.
// ------------------------------------------------------------------------------------------

template <int D>
__device__ __forceinline__ bool le_exact(const Pt<float, D> &a, const Pt<float, D> &b, double eps2) {
    double s = 0.0;
#pragma unroll
    for (int i = 0; i < D; ++i) {
        double t = __dsub_rn((double)a.x[i], (double)b.x[i]);
        s = __dadd_rn(s, __dmul_rn(t, t));
    }
    return s <= eps2;
}
template <int D>
__device__ __forceinline__ bool le_exact(const Pt<double, D> &a, const Pt<double, D> &b, double eps2) {
    double s = 0.0;
#pragma unroll
    for (int i = 0; i < D; ++i) {
        double t = __dsub_rn(a.x[i], b.x[i]);
        s = __dadd_rn(s, __dmul_rn(t, t));
    }
    return s <= eps2;
}

template <int D>
__device__ __forceinline__ bool within_eps(const Pt<float, D> &a, const Pt<float, D> &b,
                                           const GridParams &g) {
    float s = 0.f;
#pragma unroll
    for (int i = 0; i < D; ++i) {
        float t = __fsub_rn(a.x[i], b.x[i]);
        s = __fmaf_rn(t, t, s);
    }
    if (s < g.lo32) return true;
    if (s > g.hi32) return false;
    return le_exact<D>(a, b, g.eps2);
}
template <int D>
__device__ __forceinline__ bool within_eps(const Pt<double, D> &a, const Pt<double, D> &b,
                                           const GridParams &g) {
    return le_exact<D>(a, b, g.eps2);
}

template <typename T, int D>
__device__ __forceinline__ Pt<T, D> shfl_pt(const Pt<T, D> &p, int src) {
    Pt<T, D> r;
#pragma unroll
    for (int i = 0; i < D; ++i) r.x[i] = __shfl_sync(0xffffffffu, p.x[i], src);
#pragma unroll
    for (int i = D; i < PadDim<T, D>::value; ++i) r.x[i] = T(0);
    return r;
}

template <typename T, int D>
__device__ __forceinline__ Pt<T, D> zero_pt() {
    Pt<T, D> r;
#pragma unroll
    for (int i = 0; i < PadDim<T, D>::value; ++i) r.x[i] = T(0);
    return r;
}

// ------------------------------------------------------------------------------------------
// Cell keys and the pencil hash table
// ------------------------------------------------------------------------------------------

template <int D>
__device__ __forceinline__ void unpack_key(uint64_t key, const GridParams &g, int *c) {
#pragma unroll
    for (int i = 0; i < D; ++i) c[i] = (int)((key >> g.shift[i]) & ((1ull << g.bits[i]) - 1ull));
}

__device__ __forceinline__ uint32_t hash_lookup(const uint64_t *hkeys, const uint32_t *hvals,
                                                uint32_t mask, uint64_t key) {
    uint32_t h = (uint32_t)mix64(key) & mask;
    for (uint32_t it = 0; it <= mask; ++it) {
        uint64_t k = __ldg(hkeys + h);
        if (k == key) return __ldg(hvals + h);
        if (k == kEmptyKey) return 0xffffffffu;
        h = (h + 1) & mask;
    }
    return 0xffffffffu;
}

// Cell range [lo, hi) of the neighbours of cell `a` (coordinates ac) in stencil pencil k.
// half: for the zero offset only cells after `a` along the last coordinate.
template <typename T, int D>
__device__ __forceinline__ bool pencil_range(const LowdView<T, D> &v, const Stencil &st, int k,
                                             const int *ac, bool half, uint32_t &lo, uint32_t &hi) {
    const GridParams &g = v.g;
    uint64_t pkey = 0;
#pragma unroll
    for (int i = 0; i < D - 1; ++i) {
        int c = ac[i] + (int)st.off[k][i];
        if (c < 0 || c >= (int)g.ncell[i]) return false;
        pkey |= (uint64_t)c << (g.shift[i] - g.prefix_shift);
    }
    const uint32_t p = hash_lookup(v.hkeys, v.hvals, v.ctr->hash_mask, pkey);
    if (p == 0xffffffffu) return false;
    uint32_t ps = v.pencil_start[p], pe = v.pencil_start[p + 1];
    const int r = st.reach[k];
    int llo = ac[D - 1] - r, lhi = ac[D - 1] + r;
    if (half && k == 0) llo = ac[D - 1] + 1;
    if (llo < 0) llo = 0;
    if (lhi > (int)g.ncell[D - 1] - 1) lhi = (int)g.ncell[D - 1] - 1;
    if (llo > lhi) return false;
    const uint64_t base = (D > 1) ? (pkey << g.prefix_shift) : 0ull;
    const uint64_t klo = base | (uint64_t)llo, khi = base | (uint64_t)lhi;
    // lower bound of klo, then upper bound of khi, inside the pencil
    uint32_t a = ps, b = pe;
    while (a < b) {
        uint32_t m = (a + b) >> 1;
        if (__ldg(v.cell_key + m) < klo) a = m + 1; else b = m;
    }
    lo = a;
    b = pe;
    while (a < b) {
        uint32_t m = (a + b) >> 1;
        if (__ldg(v.cell_key + m) <= khi) a = m + 1; else b = m;
    }
    hi = a;
    return lo < hi;
}

// ------------------------------------------------------------------------------------------
// Union-find over cells (lock-free; the root of a set is its smallest cell id)
// ------------------------------------------------------------------------------------------

__device__ __forceinline__ uint32_t uf_find(uint32_t *parent, uint32_t x, DevCounters *ctr) {
    uint32_t it = 0;
    uint32_t p = __ldcg(parent + x);
    while (p != x) {
        uint32_t gp = __ldcg(parent + p);
        if (gp != p) parent[x] = gp;  // path halving: gp is an ancestor of x
        x = p;
        p = gp;
        if (++it > kLoopLimit) { set_error(ctr, kErrLoop); break; }
    }
    return x;
}

__device__ __forceinline__ void uf_union(uint32_t *parent, uint32_t a, uint32_t b, DevCounters *ctr) {
    for (uint32_t it = 0; it < kLoopLimit; ++it) {
        a = uf_find(parent, a, ctr);
        b = uf_find(parent, b, ctr);
        if (a == b) return;
        if (a > b) { uint32_t t = a; a = b; b = t; }
        uint32_t old = atomicCAS(parent + b, b, a);  // hook the larger root under the smaller
        if (old == b) return;
    }
    set_error(ctr, kErrLoop);
}

// ------------------------------------------------------------------------------------------
// Stage kernels
// ------------------------------------------------------------------------------------------

// Origin shift (Sec. 2): per-dimension min and max, plus a NaN check.
template <typename T, int D>
__global__ void __launch_bounds__(256) k_minmax(const T *__restrict__ in, int64_t n, DevCounters *ctr) {
    double mn[D], mx[D];
#pragma unroll
    for (int i = 0; i < D; ++i) { mn[i] = DBL_MAX; mx[i] = -DBL_MAX; }
    bool nan = false;
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n;
         j += (int64_t)gridDim.x * blockDim.x) {
#pragma unroll
        for (int i = 0; i < D; ++i) {
            double x = (double)in[j * D + i];
            nan |= (x != x);
            mn[i] = fmin(mn[i], x);
            mx[i] = fmax(mx[i], x);
        }
    }
#pragma unroll
    for (int i = 0; i < D; ++i) {
        for (int o = 16; o; o >>= 1) {
            mn[i] = fmin(mn[i], __shfl_xor_sync(0xffffffffu, mn[i], o));
            mx[i] = fmax(mx[i], __shfl_xor_sync(0xffffffffu, mx[i], o));
        }
    }
    nan = __any_sync(0xffffffffu, nan);
    if (lane_id() == 0) {
        uint64_t *mm = reinterpret_cast<uint64_t *>(ctr->minmax_enc);
#pragma unroll
        for (int i = 0; i < D; ++i) {
            atomicMin((unsigned long long *)&mm[i], (unsigned long long)enc_double(mn[i]));
            atomicMax((unsigned long long *)&mm[kMaxD + i], (unsigned long long)enc_double(mx[i]));
        }
        if (nan) atomicOr(&ctr->nan_seen, 1u);
    }
}

// Algorithm 1: band index of every coordinate, c_i = floor((x_i - o_i) / side), packed into a
// key whose order is lexicographic in (c_0, ..., c_{d-1}).
template <typename T, int D, typename K>
__global__ void __launch_bounds__(256) k_bin(const T *__restrict__ in, GridParams g,
                                            K *__restrict__ keys, uint32_t *__restrict__ idx) {
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < g.n;
         j += (int64_t)gridDim.x * blockDim.x) {
        uint64_t key = 0;
#pragma unroll
        for (int i = 0; i < D; ++i) {
            const T x = in[j * D + i];
            uint32_t c;
            if (sizeof(T) == 4 && !g.bin_fp64) {
                float t = __fmul_rn(__fsub_rn((float)x, g.origin_f[i]), g.inv_side_f);
                c = (uint32_t)floorf(t);
            } else {
                double t = __dmul_rn(__dsub_rn((double)x, g.origin[i]), g.inv_side);
                c = (uint32_t)floor(t);
            }
            if (c > g.ncell[i] - 1) c = g.ncell[i] - 1;
            key |= (uint64_t)c << g.shift[i];
        }
        keys[j] = (K)key;
        idx[j] = (uint32_t)j;
    }
}

// Gather the points into cell order and flag the first point of every cell.
template <typename T, int D, typename K>
__global__ void __launch_bounds__(256) k_gather(const T *__restrict__ in, const K *__restrict__ keys,
                                               const uint32_t *__restrict__ idx, int64_t n,
                                               Pt<T, D> *__restrict__ pts, uint32_t *__restrict__ flags) {
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n;
         j += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t o = idx[j];
        Pt<T, D> p = zero_pt<T, D>();
#pragma unroll
        for (int i = 0; i < D; ++i) p.x[i] = in[(int64_t)o * D + i];
        pts[j] = p;
        flags[j] = (j == 0 || keys[j] != keys[j - 1]) ? 1u : 0u;
    }
}

// Run-length cells: cell id of every point, first point and key of every cell.
template <typename K>
__global__ void __launch_bounds__(256) k_cells(const K *__restrict__ keys, uint32_t *flags_cell_of,
                                              const uint32_t *__restrict__ excl, int64_t n,
                                              uint32_t *__restrict__ cell_start,
                                              uint64_t *__restrict__ cell_key) {
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n;
         j += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t f = flags_cell_of[j];
        const uint32_t c = excl[j] + f - 1u;
        flags_cell_of[j] = c;
        if (f) {
            cell_start[c] = (uint32_t)j;
            cell_key[c] = (uint64_t)keys[j];
        }
        if (j == n - 1) cell_start[c + 1] = (uint32_t)n;
    }
}

// First cell of every pencil (cells sharing all coordinates but the last).
static __global__ void __launch_bounds__(256) k_pencil_flags(const uint64_t *__restrict__ cell_key,
                                                     int prefix_shift, const DevCounters *ctr,
                                                     uint32_t *__restrict__ pflags) {
    const uint32_t C = ctr->n_cells;
    for (uint32_t c = blockIdx.x * blockDim.x + threadIdx.x; c < C; c += gridDim.x * blockDim.x)
        pflags[c] = (c == 0 || (cell_key[c] >> prefix_shift) != (cell_key[c - 1] >> prefix_shift)) ? 1u : 0u;
}

// Clear the used part of the hash table (capacity = power of two >= 2 P).
static __global__ void __launch_bounds__(256) k_hash_init(uint64_t *__restrict__ hkeys, DevCounters *ctr) {
    const uint32_t P = ctr->n_pencils;
    uint32_t cap = 64;
    while (cap < 2u * P) cap <<= 1;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < cap; i += gridDim.x * blockDim.x)
        hkeys[i] = kEmptyKey;
    if (blockIdx.x == 0 && threadIdx.x == 0) ctr->hash_mask = cap - 1;
}

static __global__ void __launch_bounds__(256) k_pencils(const uint64_t *__restrict__ cell_key,
                                                int prefix_shift, const uint32_t *__restrict__ pflags,
                                                const uint32_t *__restrict__ pexcl,
                                                uint32_t *__restrict__ pencil_start,
                                                uint64_t *hkeys, uint32_t *hvals, DevCounters *ctr) {
    const uint32_t C = ctr->n_cells;
    const uint32_t mask = ctr->hash_mask;
    for (uint32_t c = blockIdx.x * blockDim.x + threadIdx.x; c < C; c += gridDim.x * blockDim.x) {
        if (c == C - 1) pencil_start[pexcl[c] + pflags[c]] = C;
        if (!pflags[c]) continue;
        const uint32_t p = pexcl[c];
        pencil_start[p] = c;
        const uint64_t key = cell_key[c] >> prefix_shift;
        uint32_t h = (uint32_t)mix64(key) & mask;
        bool placed = false;
        for (uint32_t it = 0; it <= mask; ++it) {
            unsigned long long prev = atomicCAS((unsigned long long *)(hkeys + h),
                                                (unsigned long long)kEmptyKey, (unsigned long long)key);
            if (prev == kEmptyKey || prev == key) {
                hvals[h] = p;
                placed = true;
                break;
            }
            h = (h + 1) & mask;
        }
        if (!placed) set_error(ctr, kErrHashFull);
    }
}

// Definition 2 with the hypercube shortcut: a cell holding >= MINPTS points is core as a
// whole (its diagonal is at most eps); every point of another cell is counted exactly over
// its own cell and the neighbour cells, stopping once it reaches MINPTS.  One warp per cell;
// candidate points are held one per lane and every point of the cell is compared against
// them with a warp ballot.  Also initialises the per-cell union-find, reps and labels.
template <typename T, int D>
__global__ void __launch_bounds__(256) k_core(LowdView<T, D> v, Stencil st_in) {
    __shared__ Stencil st;
    for (int i = threadIdx.x; i < (int)(sizeof(Stencil) / 4); i += blockDim.x)
        reinterpret_cast<uint32_t *>(&st)[i] = reinterpret_cast<const uint32_t *>(&st_in)[i];
    __syncthreads();
    constexpr int ndir = RepDirs<D>::value;
    const uint32_t C = v.ctr->n_cells;
    const uint32_t min_pts = v.g.min_pts;
    const int lane = lane_id();
    uint32_t dense_cells = 0;
    for (uint32_t A = global_warp(); A < C; A += total_warps()) {
        const uint32_t s = v.cell_start[A], e = v.cell_start[A + 1], m = e - s;
        if (lane == 0) {
            v.parent[A] = A;
            v.comp_min[A] = kNoLabel;
        }
        if (m >= min_pts) {
            for (uint32_t i = s + lane; i < e; i += 32) v.core[i] = 1;
            for (int r = lane; r < ndir; r += 32) v.reps[(int64_t)A * ndir + r] = ~0ull;
            if (lane == 0) v.cell_core[A] = 1;
            ++dense_cells;
            continue;
        }
        int ac[D];
        unpack_key<D>(v.cell_key[A], v.g, ac);
        bool any_core = false;
        for (uint32_t base = s; base < e; base += 32) {
            const uint32_t i = base + lane;
            const bool have = i < e;
            const Pt<T, D> pa = have ? v.pts[i] : zero_pt<T, D>();
            const int nA = (int)min(32u, e - base);
            uint32_t cnt = m;
            bool all_done = false;
            for (int k0 = 0; k0 < st.n_all && !all_done; k0 += 32) {
                const int k = k0 + lane;
                uint32_t lo = 0, hi = 0;
                const bool ok = k < st.n_all && pencil_range<T, D>(v, st, k, ac, false, lo, hi);
                const uint32_t qlo = ok ? v.cell_start[lo] : 0u, qhi = ok ? v.cell_start[hi] : 0u;
                unsigned rm = __ballot_sync(0xffffffffu, ok);
                while (rm && !all_done) {
                    const int L = __ffs(rm) - 1;
                    rm &= rm - 1;
                    const uint32_t q0 = __shfl_sync(0xffffffffu, qlo, L);
                    const uint32_t q1 = __shfl_sync(0xffffffffu, qhi, L);
                    // the zero offset's range contains this cell: skip its points
                    for (int part = 0; part < 2 && !all_done; ++part) {
                        const uint32_t a0 = part == 0 ? q0 : max(q0, e);
                        const uint32_t a1 = part == 0 ? min(q1, s) : q1;
                        for (uint32_t qb = a0; qb < a1 && !all_done; qb += 32) {
                            const uint32_t q = qb + lane;
                            const bool vq = q < a1;
                            const Pt<T, D> pq = vq ? v.pts[q] : zero_pt<T, D>();
                            for (int jj = 0; jj < nA; ++jj) {
                                const Pt<T, D> aj = shfl_pt<T, D>(pa, jj);
                                const bool hit = vq && within_eps<D>(aj, pq, v.g);
                                const unsigned b = __ballot_sync(0xffffffffu, hit);
                                if (lane == jj) cnt += __popc(b);
                            }
                            all_done = __all_sync(0xffffffffu, !have || cnt >= min_pts);
                        }
                    }
                }
            }
            const bool is_core = have && cnt >= min_pts;
            if (have) v.core[i] = is_core ? 1 : 0;
            any_core |= __any_sync(0xffffffffu, is_core);
        }
        if (any_core)
            for (int r = lane; r < ndir; r += 32) v.reps[(int64_t)A * ndir + r] = ~0ull;
        if (lane == 0) v.cell_core[A] = any_core ? 1 : 0;
    }
    if (lane == 0 && dense_cells) atomicAdd(&v.ctr->n_dense, dense_cells);
}

// Algorithm 2: for every cell with core points and every direction delta, the core point
// nearest to the ideal position (the face / edge / corner of the cube in direction delta),
// measured in cell units.  Ties go to the smaller sorted index.  Point-parallel; a warp
// whose points share one cell reduces before its atomic.
template <typename T, int D>
__global__ void __launch_bounds__(256) k_reps(LowdView<T, D> v) {
    constexpr int ndir = RepDirs<D>::value;
    const int64_t n = v.g.n;
    const int lane = lane_id();
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31); base < n; base += stride) {
        const int64_t j = base + lane;
        const bool valid = j < n && v.core[j];
        const uint32_t c = valid ? v.cell_of[j] : 0xffffffffu;
        float u[D];
        if (valid) {
            const Pt<T, D> p = v.pts[j];
            int cc[D];
            unpack_key<D>(v.cell_key[c], v.g, cc);
#pragma unroll
            for (int i = 0; i < D; ++i) {
                if (sizeof(T) == 4) {
                    float t = ((float)p.x[i] - v.g.origin_f[i]) * v.g.inv_side_f;
                    u[i] = t - (float)cc[i];
                } else {
                    double t = ((double)p.x[i] - v.g.origin[i]) * v.g.inv_side;
                    u[i] = (float)(t - (double)cc[i]);
                }
            }
        } else {
#pragma unroll
            for (int i = 0; i < D; ++i) u[i] = 0.f;
        }
        const unsigned vm = __ballot_sync(0xffffffffu, valid);
        if (!vm) continue;
        const uint32_t c0 = __shfl_sync(0xffffffffu, c, __ffs(vm) - 1);
        const bool uniform = __all_sync(0xffffffffu, !valid || c == c0);
#pragma unroll 1
        for (int r = 0; r < ndir; ++r) {
            float dist = 0.f;
            if (D <= 3) {
                int code = r < (ndir / 2) ? r : r + 1;
#pragma unroll
                for (int i = 0; i < D; ++i) {
                    int s = code % 3 - 1;
                    code /= 3;
                    float w = s > 0 ? 1.f - u[i] : (s < 0 ? u[i] : 0.f);
                    dist = fmaf(w, w, dist);
                }
            } else {
                const int i = r >> 1;
                float ui = 0.f;
#pragma unroll
                for (int t = 0; t < D; ++t) if (t == i) ui = u[t];
                float w = (r & 1) ? 1.f - ui : ui;
                dist = w * w;
            }
            uint64_t val = valid ? (((uint64_t)__float_as_uint(dist) << 32) | (uint64_t)(uint32_t)j) : ~0ull;
            if (uniform) {
#pragma unroll
                for (int o = 16; o; o >>= 1) {
                    uint64_t other = __shfl_xor_sync(0xffffffffu, val, o);
                    val = other < val ? other : val;
                }
                if (lane == 0) atomicMin((unsigned long long *)&v.reps[(int64_t)c0 * ndir + r], (unsigned long long)val);
            } else if (valid) {
                atomicMin((unsigned long long *)&v.reps[(int64_t)c * ndir + r], (unsigned long long)val);
            }
        }
    }
}

// Does some core point of cell A lie within eps of some core point of cell B?  Warp-wide,
// early exit on the first pair.
template <typename T, int D>
__device__ bool warp_core_pair(const LowdView<T, D> &v, uint32_t A, uint32_t B) {
    const int lane = lane_id();
    const uint32_t sa = v.cell_start[A], ea = v.cell_start[A + 1];
    const uint32_t sb = v.cell_start[B], eb = v.cell_start[B + 1];
    for (uint32_t ia = sa; ia < ea; ia += 32) {
        const uint32_t i = ia + lane;
        const bool va = i < ea && v.core[i];
        if (!__any_sync(0xffffffffu, va)) continue;
        const Pt<T, D> pa = va ? v.pts[i] : zero_pt<T, D>();
        for (uint32_t jb = sb; jb < eb; jb += 32) {
            const uint32_t j = jb + lane;
            const bool vb = j < eb && v.core[j];
            const unsigned bm = __ballot_sync(0xffffffffu, vb);
            if (!bm) continue;
            const Pt<T, D> pb = vb ? v.pts[j] : zero_pt<T, D>();
            unsigned rem = bm;
            while (rem) {
                const int t = __ffs(rem) - 1;
                rem &= rem - 1;
                const Pt<T, D> q = shfl_pt<T, D>(pb, t);
                if (__any_sync(0xffffffffu, va && within_eps<D>(pa, q, v.g))) return true;
            }
        }
    }
    return false;
}

// Algorithm 3: merge every pair of neighbouring cells that hold core points and have a core
// pair within eps.  Each unordered pair is visited once (upper half of the stencil).  The
// complementary representative points are tested first; a hit settles the pair, a miss falls
// back to the exhaustive core x core test.  Pairs already in one set are skipped.
template <typename T, int D>
__global__ void __launch_bounds__(256) k_merge(LowdView<T, D> v, Stencil st_in) {
    __shared__ Stencil st;
    for (int i = threadIdx.x; i < (int)(sizeof(Stencil) / 4); i += blockDim.x)
        reinterpret_cast<uint32_t *>(&st)[i] = reinterpret_cast<const uint32_t *>(&st_in)[i];
    __syncthreads();
    constexpr int ndir = RepDirs<D>::value;
    const uint32_t C = v.ctr->n_cells;
    const int lane = lane_id();
    for (uint32_t A = global_warp(); A < C; A += total_warps()) {
        if (!v.cell_core[A]) continue;
        int ac[D];
        unpack_key<D>(v.cell_key[A], v.g, ac);
        for (int k0 = 0; k0 < st.n_half; k0 += 32) {
            const int k = k0 + lane;
            uint32_t lo = 0, hi = 0;
            const bool ok = k < st.n_half && pencil_range<T, D>(v, st, k, ac, true, lo, hi);
            unsigned rm = __ballot_sync(0xffffffffu, ok);
            while (rm) {
                const int L = __ffs(rm) - 1;
                rm &= rm - 1;
                const uint32_t c0 = __shfl_sync(0xffffffffu, lo, L);
                const uint32_t c1 = __shfl_sync(0xffffffffu, hi, L);
                for (uint32_t cb = c0; cb < c1; cb += 32) {
                    const uint32_t B = cb + lane;
                    bool pending = B < c1 && v.cell_core[B];
                    if (pending && uf_find(v.parent, A, v.ctr) == uf_find(v.parent, B, v.ctr)) pending = false;
                    if (pending) {
                        int bc[D], delta[D];
                        unpack_key<D>(v.cell_key[B], v.g, bc);
#pragma unroll
                        for (int i = 0; i < D; ++i) delta[i] = bc[i] - ac[i];
                        const int ra = rep_dir_of<D>(delta);
                        const int rb = rep_dir_complement<D>(ra);
                        const uint32_t pa = (uint32_t)v.reps[(int64_t)A * ndir + ra];
                        const uint32_t pb = (uint32_t)v.reps[(int64_t)B * ndir + rb];
                        if (within_eps<D>(v.pts[pa], v.pts[pb], v.g)) {
                            uf_union(v.parent, A, B, v.ctr);
                            pending = false;
                        }
                    }
                    unsigned need = __ballot_sync(0xffffffffu, pending);
                    while (need) {
                        const int t = __ffs(need) - 1;
                        need &= need - 1;
                        const uint32_t B2 = __shfl_sync(0xffffffffu, B, t);
                        bool same = false;
                        if (lane == 0) same = uf_find(v.parent, A, v.ctr) == uf_find(v.parent, B2, v.ctr);
                        same = __shfl_sync(0xffffffffu, same, 0);
                        if (same) continue;
                        if (warp_core_pair<T, D>(v, A, B2) && lane == 0) uf_union(v.parent, A, B2, v.ctr);
                    }
                }
            }
        }
    }
}

// Flatten the union-find: parent[c] = root for every cell with core points; count roots.
template <typename T, int D>
__global__ void __launch_bounds__(256) k_compress(LowdView<T, D> v) {
    const uint32_t C = v.ctr->n_cells;
    uint32_t roots = 0;
    for (uint32_t c = blockIdx.x * blockDim.x + threadIdx.x; c < C; c += gridDim.x * blockDim.x) {
        if (!v.cell_core[c]) continue;
        const uint32_t r = uf_find(v.parent, c, v.ctr);
        v.parent[c] = r;
        roots += (r == c);
    }
    for (int o = 16; o; o >>= 1) roots += __shfl_xor_sync(0xffffffffu, roots, o);
    if (lane_id() == 0 && roots) atomicAdd(&v.ctr->n_clusters, roots);
}

// Canonical cluster id (Algorithm 4 numbers clusters in traversal order; the fixed rule
// here is the smallest input index among the cluster's core points).
template <typename T, int D>
__global__ void __launch_bounds__(256) k_comp_min(LowdView<T, D> v) {
    const int64_t n = v.g.n;
    const int lane = lane_id();
    uint32_t ncore = 0;
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31); base < n;
         base += (int64_t)gridDim.x * blockDim.x) {
        const int64_t j = base + lane;
        const bool valid = j < n && v.core[j];
        const uint32_t r = valid ? v.parent[v.cell_of[j]] : 0xffffffffu;
        uint32_t val = valid ? v.perm[j] : kNoLabel;
        const unsigned vm = __ballot_sync(0xffffffffu, valid);
        if (!vm) continue;
        ncore += (lane == 0) ? __popc(vm) : 0u;
        const uint32_t r0 = __shfl_sync(0xffffffffu, r, __ffs(vm) - 1);
        if (__all_sync(0xffffffffu, !valid || r == r0)) {
            for (int o = 16; o; o >>= 1) val = min(val, __shfl_xor_sync(0xffffffffu, val, o));
            if (lane == 0) atomicMin(&v.comp_min[r0], val);
        } else if (valid) {
            atomicMin(&v.comp_min[r], val);
        }
    }
    if (lane == 0 && ncore) atomicAdd(&v.ctr->n_core, ncore);
}

// Algorithm 4 and Definition 5 with the canonical rule: core points take their cluster id;
// a non-core point takes the smallest id among the clusters of the core points within eps
// (the core points of its own cell qualify without a test, the cell's diagonal being at most
// eps), else -1.  One warp per cell; writes labels in input order.
template <typename T, int D>
__global__ void __launch_bounds__(256) k_labels(LowdView<T, D> v, Stencil st_in) {
    __shared__ Stencil st;
    for (int i = threadIdx.x; i < (int)(sizeof(Stencil) / 4); i += blockDim.x)
        reinterpret_cast<uint32_t *>(&st)[i] = reinterpret_cast<const uint32_t *>(&st_in)[i];
    __syncthreads();
    const uint32_t C = v.ctr->n_cells;
    const int lane = lane_id();
    uint32_t noise = 0;
    for (uint32_t A = global_warp(); A < C; A += total_warps()) {
        const uint32_t s = v.cell_start[A], e = v.cell_start[A + 1];
        const bool hasc = v.cell_core[A];
        const uint32_t clA = hasc ? v.comp_min[v.parent[A]] : kNoLabel;
        int ac[D];
        unpack_key<D>(v.cell_key[A], v.g, ac);
        for (uint32_t base = s; base < e; base += 32) {
            const uint32_t i = base + lane;
            const bool have = i < e;
            const bool isc = have && v.core[i];
            uint32_t best = clA;
            bool search = have && !isc;
            const int nA = (int)min(32u, e - base);
            if (__any_sync(0xffffffffu, search)) {
                const Pt<T, D> pa = have ? v.pts[i] : zero_pt<T, D>();
                for (int k0 = 0; k0 < st.n_all; k0 += 32) {
                    const int k = k0 + lane;
                    uint32_t lo = 0, hi = 0;
                    const bool ok = k < st.n_all && pencil_range<T, D>(v, st, k, ac, false, lo, hi);
                    unsigned rm = __ballot_sync(0xffffffffu, ok);
                    while (rm) {
                        const int L = __ffs(rm) - 1;
                        rm &= rm - 1;
                        const uint32_t c0 = __shfl_sync(0xffffffffu, lo, L);
                        const uint32_t c1 = __shfl_sync(0xffffffffu, hi, L);
                        for (uint32_t cb = c0; cb < c1; cb += 32) {
                            // current worst best among searching lanes
                            uint32_t worst = search ? best : 0u;
                            for (int o = 16; o; o >>= 1) worst = max(worst, __shfl_xor_sync(0xffffffffu, worst, o));
                            const uint32_t B = cb + lane;
                            const bool vb = B < c1 && B != A && v.cell_core[B];
                            const uint32_t clB = vb ? v.comp_min[v.parent[B]] : kNoLabel;
                            unsigned cm = __ballot_sync(0xffffffffu, vb && clB < worst);
                            while (cm) {
                                const int t = __ffs(cm) - 1;
                                cm &= cm - 1;
                                const uint32_t B2 = __shfl_sync(0xffffffffu, B, t);
                                const uint32_t cl2 = __shfl_sync(0xffffffffu, clB, t);
                                bool want = search && best > cl2;
                                if (!__any_sync(0xffffffffu, want)) continue;
                                const uint32_t sb = v.cell_start[B2], eb = v.cell_start[B2 + 1];
                                for (uint32_t qb = sb; qb < eb; qb += 32) {
                                    const uint32_t q = qb + lane;
                                    const bool vq = q < eb && v.core[q];
                                    const Pt<T, D> pq = vq ? v.pts[q] : zero_pt<T, D>();
                                    for (int jj = 0; jj < nA; ++jj) {
                                        if (!__shfl_sync(0xffffffffu, want, jj)) continue;
                                        const Pt<T, D> aj = shfl_pt<T, D>(pa, jj);
                                        const bool hit = vq && within_eps<D>(aj, pq, v.g);
                                        if (__any_sync(0xffffffffu, hit) && lane == jj) {
                                            best = cl2;
                                            want = false;
                                        }
                                    }
                                    if (!__any_sync(0xffffffffu, want)) break;
                                }
                            }
                        }
                    }
                }
            }
            if (have) {
                const int32_t lab = best == kNoLabel ? -1 : (int32_t)best;
                const uint32_t o = v.perm[i];
                v.labels[o] = lab;
                if (v.core_out) v.core_out[o] = isc ? 1 : 0;
                noise += lab < 0;
            }
        }
    }
    for (int o = 16; o; o >>= 1) noise += __shfl_xor_sync(0xffffffffu, noise, o);
    if (lane == 0 && noise) atomicAdd(&v.ctr->n_noise, noise);
}

}  // namespace hca
