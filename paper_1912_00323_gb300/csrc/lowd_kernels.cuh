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
//   ranges[c * n_all + k]  cells [lo, hi) of stencil pencil k around cell c
//   core[j], cell_core[c], parent[c] (union-find), reps[c * ndir + r], comp_min[c]
#pragma once

#include <float.h>

#include "block_scan.cuh"
#include "hca_internal.cuh"

namespace hca {

template <typename T, int D>
struct LowdView {
    GridParams g;                 // key layout, and the parameters of a single-instance call
    const GridParams *gtab;       // batched calls: parameters of every set (same key layout)
    const int64_t *set_off;       // batched calls: first point of every set (n_sets + 1)
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
    Pt<T, D> *rep_pts;            // coordinates of reps[c * ndir + r]
    uint32_t *comp_min;
    uint2 *ranges;                // [cell * n_all + k]: neighbour cells [lo, hi) in pencil k
    uint32_t *list_count;         // cells whose points k_core decides (ctr->n_list[0])
    uint32_t *list_core;          // cells holding a core point (ctr->n_list[1])
    uint32_t *list_label;         // cells holding a non-core point that may have a core neighbour (ctr->n_list[2])
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

__device__ __forceinline__ double dec_double_dev(uint64_t e) {
    const uint64_t b = (e >> 63) ? (e & 0x7fffffffffffffffull) : ~e;
    return __longlong_as_double((long long)b);
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

// The next work item for this warp from a per-kernel counter (warp-uniform): cells and chunks
// differ in cost by orders of magnitude, so they are handed out dynamically.
__device__ __forceinline__ uint32_t next_chunk(uint32_t *counter) {
    uint32_t t = 0;
    if (lane_id() == 0) t = atomicAdd(counter, 1u);
    return __shfl_sync(0xffffffffu, t, 0);
}

// Items [0, N) to warps in batches of kItemBatch taken from counter ctr->lowd_next[slot] (one
// item at a time: the label list is short, so batches left most warps idle).
constexpr uint32_t kItemBatch = 1;
#define LOWD_FOR_EACH(v, X, N, slot)                                                                  \
    for (uint32_t b_ = next_chunk(&(v).ctr->lowd_next[slot]) * kItemBatch; b_ < (N);                \
         b_ = next_chunk(&(v).ctr->lowd_next[slot]) * kItemBatch)                                   \
        for (uint32_t X = b_, xe_ = min(b_ + kItemBatch, (uint32_t)(N)); X < xe_; ++X)

// Batched calls put the set id above the cell key bits; cells never mix sets.
template <typename V>
__device__ __forceinline__ uint32_t set_of_key(const V &v, uint64_t key) {
    return v.gtab ? (uint32_t)(key >> v.g.key_bits) : 0u;
}
template <typename V>
__device__ __forceinline__ const GridParams &params_of(const V &v, uint32_t set) {
    return v.gtab ? v.gtab[set] : v.g;
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

// First position in [a, e) of a pencil's cells (keys ascending) whose key is not below kt
// (Upper: above kt).  A few linear steps first, since the bounds of consecutive cells of a
// pencil move little, then a binary search over the rest.
template <bool Upper>
__device__ __forceinline__ uint32_t key_bound_from(const uint64_t *__restrict__ ck, uint32_t a, uint32_t e,
                                                   uint64_t kt) {
#pragma unroll
    for (int step = 0; step < 4; ++step) {
        if (a >= e) return a;
        const uint64_t x = __ldg(ck + a);
        if (Upper ? (x > kt) : (x >= kt)) return a;
        ++a;
    }
    uint32_t b = e;
    while (a < b) {
        const uint32_t m = (a + b) >> 1;
        const uint64_t x = __ldg(ck + m);
        if (Upper ? (x <= kt) : (x < kt)) a = m + 1;
        else b = m;
    }
    return a;
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

// Root of x without writing: used once merging is over, where a path-halving write could
// overwrite another thread's flattened parent[c] = root with an intermediate ancestor.
__device__ __forceinline__ uint32_t uf_root_readonly(const uint32_t *parent, uint32_t x, DevCounters *ctr) {
    uint32_t it = 0;
    uint32_t p = __ldcg(parent + x);
    while (p != x) {
        x = p;
        p = __ldcg(parent + x);
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
// Cell boxes and flattened neighbour lists
// ------------------------------------------------------------------------------------------

// Band coordinates of a point, t_i = (x_i - o_i) / side, in the arithmetic of the binning.
template <typename T, int D>
__device__ __forceinline__ void band_coords(const Pt<T, D> &p, const GridParams &g, float *t) {
#pragma unroll
    for (int i = 0; i < D; ++i) {
        if (sizeof(T) == 4 && !g.bin_fp64)
            t[i] = __fmul_rn(__fsub_rn((float)p.x[i], g.origin_f[i]), g.inv_side_f);
        else
            t[i] = (float)__dmul_rn(__dsub_rn((double)p.x[i], g.origin[i]), g.inv_side);
    }
}

// Where can the points of cell cb lie relative to eps of a point with band coordinates t?
// 0: every point of the cell is farther than eps; 2: every point is within eps; 1: unknown.
// The cell is widened by tau_box band units, which bounds the binning error of both the
// point and the cell's points plus the FP32 error of this test; the thresholds carry a
// relative margin of 2^-12, far above the FP32 error of the sums, so the answer agrees with
// the exact predicate whenever it is 0 or 2.
template <int D>
__device__ __forceinline__ int box_class(const float *t, const int *cb, const GridParams &g) {
    if (!g.box_ok) return 1;
    float mn = 0.f, mx = 0.f;
#pragma unroll
    for (int i = 0; i < D; ++i) {
        const float lo = (float)cb[i] - g.tau_box, hi = (float)cb[i] + 1.0f + g.tau_box;
        const float gap = fmaxf(fmaxf(lo - t[i], t[i] - hi), 0.f);
        const float far = fmaxf(fabsf(t[i] - lo), fabsf(t[i] - hi));
        mn = fmaf(gap, gap, mn);
        mx = fmaf(far, far, mx);
    }
    if (mn > g.box_none) return 0;
    if (mx < g.box_full) return 2;
    return 1;
}

// Per lane a cell range [lo, lo + len); inclusive prefix sums of the lengths across the warp
// let the warp walk all cells of up to 32 ranges, 32 at a time.
struct LaneRanges {
    uint32_t lo, len, incl, total;
};

__device__ __forceinline__ LaneRanges lane_ranges(uint32_t lo, uint32_t hi) {
    LaneRanges r;
    r.lo = lo;
    r.len = hi > lo ? hi - lo : 0u;
    uint32_t v = r.len;
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t t = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += t;
    }
    r.incl = v;
    r.total = __shfl_sync(0xffffffffu, v, 31);
    return r;
}

// Cell at flattened position f (< total).  Every lane of the warp must call it.
__device__ __forceinline__ uint32_t flat_cell(const LaneRanges &r, uint32_t f) {
    int k = 0;
#pragma unroll
    for (int step = 16; step >= 1; step >>= 1) {
        const uint32_t v = __shfl_sync(0xffffffffu, r.incl, k + step - 1);
        if (v <= f) k += step;
    }
    const uint32_t excl = __shfl_sync(0xffffffffu, r.incl - r.len, k);
    const uint32_t lo = __shfl_sync(0xffffffffu, r.lo, k);
    return lo + (f - excl);
}

template <typename T, int D>
__device__ __forceinline__ void load_stencil(Stencil &st, const Stencil &st_in) {
    for (int i = threadIdx.x; i < (int)(sizeof(Stencil) / 4); i += blockDim.x)
        reinterpret_cast<uint32_t *>(&st)[i] = reinterpret_cast<const uint32_t *>(&st_in)[i];
    __syncthreads();
}

__device__ __forceinline__ void add_counter(unsigned long long *ctr, uint32_t v) {
    v = __reduce_add_sync(0xffffffffu, v);
    if ((threadIdx.x & 31) == 0 && v) atomicAdd(ctr, (unsigned long long)v);
}

// ------------------------------------------------------------------------------------------
// Stage kernels
// ------------------------------------------------------------------------------------------

// Points per thread step of the streaming kernels (min/max, binning): the fewest consecutive
// points whose bytes are a multiple of 16, so a thread reads them with 16-byte loads.
template <typename T, int D>
struct VecPts {
    static constexpr int bytes = D * (int)sizeof(T);
    static constexpr int pts = bytes % 16 == 0 ? 1 : (bytes % 8 == 0 ? 2 : 4);
    static constexpr int vec = pts * bytes / 16;  // 16-byte loads per step
};

// Coordinates of points [j0, j0 + P) (P = VecPts::pts) into x[P * D]: 16-byte loads when the
// whole group is in range and `vec_ok` (the input is 16-byte aligned), else element loads;
// points past n read as zero.
template <typename T, int D>
__device__ __forceinline__ void load_pts(const T *__restrict__ in, int64_t j0, int64_t n, bool vec_ok,
                                         T (&x)[VecPts<T, D>::pts * D]) {
    constexpr int P = VecPts<T, D>::pts, V = VecPts<T, D>::vec;
    if (vec_ok && j0 + P <= n) {
        const float4 *src = reinterpret_cast<const float4 *>(in + j0 * D);
        union {
            float4 v[V];
            T e[P * D];
        } u;
#pragma unroll
        for (int k = 0; k < V; ++k) u.v[k] = __ldg(src + k);
#pragma unroll
        for (int k = 0; k < P * D; ++k) x[k] = u.e[k];
    } else {
#pragma unroll
        for (int k = 0; k < P * D; ++k) x[k] = j0 + k / D < n ? in[j0 * D + k] : T(0);
    }
}

// Origin shift (Sec. 2): per-dimension min and max in the input's own precision, plus a NaN
// check.  Each thread step reads VecPts::pts consecutive points with 16-byte loads.
template <typename T, int D>
__global__ void __launch_bounds__(256) k_minmax(const T *__restrict__ in, int64_t n, DevCounters *ctr) {
    constexpr int P = VecPts<T, D>::pts;
    T mn[D], mx[D];
#pragma unroll
    for (int i = 0; i < D; ++i) {
        mn[i] = sizeof(T) == 4 ? (T)FLT_MAX : (T)DBL_MAX;
        mx[i] = -mn[i];
    }
    bool nan = false;
    const bool vec_ok = ((uintptr_t)in & 15u) == 0;
    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c * P < n;
         c += (int64_t)gridDim.x * blockDim.x) {
        T x[P * D];
        load_pts<T, D>(in, c * P, n, vec_ok, x);
#pragma unroll
        for (int t = 0; t < P; ++t) {
            if (c * P + t >= n) continue;
#pragma unroll
            for (int i = 0; i < D; ++i) {
                const T v = x[t * D + i];
                nan |= (v != v);
                mn[i] = v < mn[i] ? v : mn[i];
                mx[i] = v > mx[i] ? v : mx[i];
            }
        }
    }
#pragma unroll
    for (int i = 0; i < D; ++i) {
        for (int o = 16; o; o >>= 1) {
            const T a = __shfl_xor_sync(0xffffffffu, mn[i], o), b = __shfl_xor_sync(0xffffffffu, mx[i], o);
            mn[i] = a < mn[i] ? a : mn[i];
            mx[i] = b > mx[i] ? b : mx[i];
        }
    }
    nan = __any_sync(0xffffffffu, nan);
    // one atomic per block and dimension (per-warp atomics on the same few words serialise)
    __shared__ T smn[8][D], smx[8][D];
    __shared__ int snan;
    const int warp = threadIdx.x >> 5;
    if (threadIdx.x == 0) snan = 0;
    __syncthreads();
    if (lane_id() == 0) {
#pragma unroll
        for (int i = 0; i < D; ++i) { smn[warp][i] = mn[i]; smx[warp][i] = mx[i]; }
        if (nan) snan = 1;
    }
    __syncthreads();
    if (threadIdx.x < D) {
        const int i = threadIdx.x;
        T a = smn[0][i], b = smx[0][i];
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w) {
            a = smn[w][i] < a ? smn[w][i] : a;
            b = smx[w][i] > b ? smx[w][i] : b;
        }
        uint64_t *mm = ctr->minmax_enc;
        atomicMin((unsigned long long *)&mm[i], (unsigned long long)enc_double((double)a));
        atomicMax((unsigned long long *)&mm[kMaxD + i], (unsigned long long)enc_double((double)b));
    }
    if (threadIdx.x == 0 && snan) atomicOr(&ctr->nan_seen, 1u);
}

// Algorithm 1: band index of every coordinate, c_i = floor((x_i - o_i) / side), packed into a
// key whose order is lexicographic in (c_0, ..., c_{d-1}).  Each thread step bins
// VecPts::pts consecutive points read with 16-byte loads and stores their keys and indices
// together.
template <typename T, int D, typename K>
__global__ void __launch_bounds__(256) k_bin(const T *__restrict__ in, GridParams g,
                                            K *__restrict__ keys, uint32_t *__restrict__ idx,
                                            uint32_t *__restrict__ digit_counts) {
    constexpr int P = VecPts<T, D>::pts;
    // digit counts of every radix pass, for the sort that follows
    __shared__ uint32_t h[8][256];
    const int passes = (g.key_bits + 7) / 8;
    for (int i = threadIdx.x; i < 8 * 256; i += blockDim.x) (&h[0][0])[i] = 0;
    __syncthreads();
    const bool vec_ok = ((uintptr_t)in & 15u) == 0;
    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c * P < g.n;
         c += (int64_t)gridDim.x * blockDim.x) {
        const int64_t j0 = c * P;
        T x[P * D];
        load_pts<T, D>(in, j0, g.n, vec_ok, x);
        K kk[P];
#pragma unroll
        for (int t = 0; t < P; ++t) {
            uint64_t key = 0;
#pragma unroll
            for (int i = 0; i < D; ++i) {
                uint32_t cc;
                if (sizeof(T) == 4 && !g.bin_fp64) {
                    float u = __fmul_rn(__fsub_rn((float)x[t * D + i], g.origin_f[i]), g.inv_side_f);
                    cc = (uint32_t)floorf(u);
                } else {
                    double u = __dmul_rn(__dsub_rn((double)x[t * D + i], g.origin[i]), g.inv_side);
                    cc = (uint32_t)floor(u);
                }
                if (cc > g.ncell[i] - 1) cc = g.ncell[i] - 1;
                key |= (uint64_t)cc << g.shift[i];
            }
            kk[t] = (K)key;
            if (j0 + t < g.n)
                for (int p = 0; p < passes; ++p) atomicAdd(&h[p][(uint32_t)(key >> (8 * p)) & 0xffu], 1u);
        }
        if (j0 + P <= g.n && sizeof(K) * P == 16) {
            // P keys (16 bytes) and P indices at once
            if (sizeof(K) == 4) {
                *reinterpret_cast<uint4 *>(keys + j0) =
                    make_uint4((uint32_t)kk[0], (uint32_t)kk[P > 1 ? 1 : 0], (uint32_t)kk[P > 2 ? 2 : 0],
                               (uint32_t)kk[P > 3 ? 3 : 0]);
                *reinterpret_cast<uint4 *>(idx + j0) =
                    make_uint4((uint32_t)j0, (uint32_t)j0 + 1u, (uint32_t)j0 + 2u, (uint32_t)j0 + 3u);
            } else {
                *reinterpret_cast<ulonglong2 *>(keys + j0) =
                    make_ulonglong2((unsigned long long)kk[0], (unsigned long long)kk[P > 1 ? 1 : 0]);
                *reinterpret_cast<uint2 *>(idx + j0) = make_uint2((uint32_t)j0, (uint32_t)j0 + 1u);
            }
        } else {
#pragma unroll
            for (int t = 0; t < P; ++t) {
                if (j0 + t < g.n) {
                    keys[j0 + t] = kk[t];
                    idx[j0 + t] = (uint32_t)(j0 + t);
                }
            }
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < passes * 256; i += blockDim.x) {
        const uint32_t c = (&h[0][0])[i];
        if (c) atomicAdd(&digit_counts[i], c);
    }
}

// Gather the points into cell order and flag the first point of every cell; one block per
// tile of kScanTileElems points, whose flag count goes to tile_sums[block] for the run-length
// cells that follow (cells_from_flags).
template <typename T, int D, typename K>
__global__ void __launch_bounds__(256) k_gather(const T *__restrict__ in, const K *__restrict__ keys,
                                               const uint32_t *__restrict__ idx, int64_t n,
                                               Pt<T, D> *__restrict__ pts, uint32_t *__restrict__ flags,
                                               uint32_t *__restrict__ tile_sums) {
    const int64_t base = (int64_t)blockIdx.x * kScanTileElems;
    uint32_t cnt = 0;
#pragma unroll
    for (int k = 0; k < kScanTileElems / 256; ++k) {
        const int64_t j = base + k * 256 + threadIdx.x;
        if (j < n) {
            const uint32_t o = idx[j];
            Pt<T, D> p = zero_pt<T, D>();
#pragma unroll
            for (int i = 0; i < D; ++i) p.x[i] = in[(int64_t)o * D + i];
            pts[j] = p;
            const uint32_t f = (j == 0 || keys[j] != keys[j - 1]) ? 1u : 0u;
            flags[j] = f;
            cnt += f;
        }
    }
    uint32_t total;
    block_exclusive_scan<256>(cnt, &total);
    if (threadIdx.x == 0) tile_sums[blockIdx.x] = total;
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

// Neighbour cells of every cell, once: for cell c and stencil pencil k the range of cells
// [lo, hi) of that pencil within reach along the last coordinate.  One thread per run of
// kRangeRun consecutive cells and stencil pencil k.  Consecutive cells mostly share their
// pencil (all coordinates but the last), so the thread looks the neighbour pencil up in the
// hash table once per pencil of its run; along a pencil the last coordinate increases, so
// both ends of the neighbour range only move forward and are found from the previous cell's.
constexpr uint32_t kRangeRun = 4;

template <typename T, int D>
__global__ void __launch_bounds__(256) k_ranges(LowdView<T, D> v, Stencil st_in) {
    __shared__ Stencil st;
    load_stencil<T, D>(st, st_in);
    const uint32_t C = v.ctr->n_cells;
    const int na = st.n_all;
    const uint64_t total = (uint64_t)((C + kRangeRun - 1) / kRangeRun) * na;
    const uint64_t last_mask = (1ull << v.g.bits[D - 1]) - 1ull;
    for (uint64_t idx = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; idx < total;
         idx += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t c0 = (uint32_t)(idx / na) * kRangeRun;
        const int k = (int)(idx % na);
        const uint32_t c1 = min(c0 + kRangeRun, C);
        const int reach = st.reach[k];
        uint64_t pcur = ~0ull, base = 0;
        uint32_t qe = 0, lo = 0, hi = 0;
        int nlast = 0;
        bool ok = false;
        for (uint32_t c = c0; c < c1; ++c) {
            const uint64_t key = v.cell_key[c];
            const uint64_t pref = key >> v.g.prefix_shift;  // set id and all coordinates but the last
            if (pref != pcur) {
                // the neighbour pencil of this cell's pencil at offset k
                pcur = pref;
                int ac[D];
                unpack_key<D>(key, v.g, ac);
                const uint32_t set = set_of_key(v, key);
                const GridParams &g = params_of(v, set);
                uint64_t pkey = v.gtab ? (uint64_t)set << (g.key_bits - g.prefix_shift) : 0ull;
                ok = true;
#pragma unroll
                for (int i = 0; i < D - 1; ++i) {
                    const int cc = ac[i] + (int)st.off[k][i];
                    if (cc < 0 || cc >= (int)g.ncell[i]) ok = false;
                    pkey |= (uint64_t)(cc & ((1 << g.bits[i]) - 1)) << (g.shift[i] - g.prefix_shift);
                }
                const uint32_t q = ok ? hash_lookup(v.hkeys, v.hvals, v.ctr->hash_mask, pkey) : 0xffffffffu;
                ok = q != 0xffffffffu;
                lo = hi = ok ? v.pencil_start[q] : 0u;
                qe = ok ? v.pencil_start[q + 1] : 0u;
                base = pkey << g.prefix_shift;
                nlast = (int)g.ncell[D - 1];
            }
            uint2 out = make_uint2(0u, 0u);
            if (ok) {
                const int a = (int)(key & last_mask);
                const int llo = max(a - reach, 0), lhi = min(a + reach, nlast - 1);
                lo = key_bound_from<false>(v.cell_key, lo, qe, base | (uint64_t)llo);
                hi = key_bound_from<true>(v.cell_key, max(hi, lo), qe, base | (uint64_t)lhi);
                if (lo < hi) out = make_uint2(lo, hi);
            }
            v.ranges[(uint64_t)c * na + k] = out;
        }
    }
}

// Append val to a work list when pred holds (warp-aggregated; every lane of the warp calls).
__device__ __forceinline__ void warp_push(uint32_t *list, uint32_t *count, bool pred, uint32_t val) {
    const unsigned m = __ballot_sync(0xffffffffu, pred);
    if (!m) return;
    const int leader = __ffs(m) - 1, lane = lane_id();
    uint32_t base = 0;
    if (lane == leader) base = atomicAdd(count, (uint32_t)__popc(m));
    base = __shfl_sync(0xffffffffu, base, leader);
    if (pred) list[base + __popc(m & ((1u << lane) - 1u))] = val;
}

// A warp's pending entries of a work list, one per lane, appended 32 at a time (one atomic per
// 32 entries instead of one per entry).  Every call is warp-uniform.
struct WarpList {
    uint32_t pending = 0, val = 0;  // lane i holds entry i while i < pending
    __device__ __forceinline__ void add(uint32_t *list, uint32_t *count, uint32_t x) {
        if (lane_id() == (int)pending) val = x;
        if (++pending == 32u) flush(list, count);
    }
    __device__ __forceinline__ void flush(uint32_t *list, uint32_t *count) {
        if (!pending) return;
        uint32_t base = 0;
        if (lane_id() == 0) base = atomicAdd(count, pending);
        base = __shfl_sync(0xffffffffu, base, 0);
        if (lane_id() < (int)pending) list[base + lane_id()] = val;
        pending = 0;
    }
};

// Cell triage before Definition 2, one thread per cell.  Initialises the union-find and
// cluster-id slots.  A cell of at least MINPTS points (core as a whole) and a cell whose
// stencil neighbourhood holds at least MINPTS points go on the list k_core counts.  In any
// other cell no point can reach MINPTS (every point within eps of it lies in the stencil
// cells), so all its points are non-core here; if no other cell lies within reach they are
// noise and get label -1 at once, else the cell goes on the label list.
template <typename T, int D>
__global__ void __launch_bounds__(256) k_triage(LowdView<T, D> v, int n_all) {
    const uint32_t C = v.ctr->n_cells;
    uint32_t noise = 0;
    const uint32_t stride = gridDim.x * blockDim.x;
    for (uint32_t base = blockIdx.x * blockDim.x + (threadIdx.x & ~31u); base < C; base += stride) {
        const uint32_t A = base + lane_id();
        bool to_count = false, to_label = false;
        if (A < C) {
            const uint32_t s = v.cell_start[A], e = v.cell_start[A + 1], m = e - s;
            const uint64_t key = v.cell_key[A];
            const uint32_t set = set_of_key(v, key);
            const uint32_t min_pts = params_of(v, set).min_pts;
            v.parent[A] = A;
            v.comp_min[A] = kNoLabel;
            if (m >= min_pts) {
                to_count = true;
            } else {
                uint32_t reach_pts = 0, reach_cells = 0;
#pragma unroll 8
                for (int k = 0; k < n_all; ++k) {
                    const uint2 rg = v.ranges[(uint64_t)A * n_all + k];
                    if (rg.y > rg.x) {
                        reach_cells += rg.y - rg.x;
                        reach_pts += v.cell_start[rg.y] - v.cell_start[rg.x];
                    }
                }
                if (reach_pts >= min_pts) {
                    to_count = true;
                } else {
                    v.cell_core[A] = 0;
                    for (uint32_t i = s; i < e; ++i) v.core[i] = 0;
                    if (reach_cells <= 1) {  // only the cell itself
                        for (uint32_t i = s; i < e; ++i) {
                            const uint32_t o = v.perm[i];
                            v.labels[o] = -1;
                            if (v.core_out) v.core_out[o] = 0;
                        }
                        noise += m;
                    } else {
                        to_label = true;
                    }
                }
            }
        }
        warp_push(v.list_count, &v.ctr->n_list[0], to_count, A);
        warp_push(v.list_label, &v.ctr->n_list[2], to_label, A);
    }
    noise = __reduce_add_sync(0xffffffffu, noise);
    if (lane_id() == 0 && noise) atomicAdd(&v.ctr->n_noise, noise);
}

// Definition 2 with the hypercube shortcut: a cell holding >= MINPTS points is core as a
// whole (its diagonal is at most eps); every point of another cell (fewer than MINPTS points)
// is counted exactly over its own cell and the neighbour cells, stopping once it reaches
// MINPTS.  One warp per cell of the triage's count list.  The neighbour cells are walked 32 at
// a time, one per lane; for each open point of the cell every lane classifies its cell's box
// against the point: a box wholly within eps adds the cell's size (warp sum), one wholly
// beyond eps is dropped, and the remaining cells are compared point by point with a warp
// ballot.  Also initialises the representative slots of cells with core points and fills the
// lists of cells with core points (merging) and with non-core points (labels).
template <typename T, int D>
__global__ void __launch_bounds__(256) k_core(LowdView<T, D> v, Stencil st_in) {
    __shared__ Stencil st;
    load_stencil<T, D>(st, st_in);
    const int n_all = st.n_all;
    const int lane = lane_id();
    uint32_t dense_cells = 0, core_cells = 0, chunks = 0;
    WarpList lcore, llabel;
    const uint32_t NL = v.ctr->n_list[0];
    for (uint32_t w = global_warp(); w < NL; w += total_warps()) {
        const uint32_t A = v.list_count[w];
        const GridParams &G = params_of(v, set_of_key(v, v.cell_key[A]));
        const uint32_t min_pts = G.min_pts;
        const uint32_t s = v.cell_start[A], e = v.cell_start[A + 1], m = e - s;
        if (m >= min_pts) {
            for (uint32_t i = s + lane; i < e; i += 32) v.core[i] = 1;
            for (int r = lane; r < RepDirs<D>::value; r += 32) v.reps[(uint64_t)A * RepDirs<D>::value + r] = ~0ull;
            if (lane == 0) v.cell_core[A] = 1;
            lcore.add(v.list_core, &v.ctr->n_list[1], A);
            ++dense_cells;
            ++core_cells;
            continue;
        }
        bool any_core = false, any_noncore = false;
        for (uint32_t base = s; base < e; base += 32) {
            const uint32_t i = base + lane;
            const bool have = i < e;
            const Pt<T, D> pa = have ? v.pts[i] : zero_pt<T, D>();
            float ta[D];
            band_coords<T, D>(pa, G, ta);
            uint32_t cnt = m;  // the own cell: every point within eps
            unsigned open = __ballot_sync(0xffffffffu, have && cnt < min_pts);
            for (int g0 = 0; g0 < n_all && open; g0 += 32) {
                const int k = g0 + lane;  // pencils nearest first: most points settle early
                const uint2 rg = k < n_all ? v.ranges[(uint64_t)A * n_all + st.near[k]] : make_uint2(0u, 0u);
                const LaneRanges lr = lane_ranges(rg.x, rg.y);
                for (uint32_t f0 = 0; f0 < lr.total && open; f0 += 32) {
                    const uint32_t f = f0 + lane;
                    const uint32_t B = flat_cell(lr, f < lr.total ? f : 0u);
                    const bool okb = f < lr.total && B != A;
                    const uint32_t bs = okb ? v.cell_start[B] : 0u;
                    const uint32_t be = okb ? v.cell_start[B + 1] : 0u;
                    int cb[D];
                    unpack_key<D>(okb ? v.cell_key[B] : 0ull, v.g, cb);
                    unsigned rem = open;
                    while (rem) {
                        const int jj = __ffs(rem) - 1;
                        rem &= rem - 1;
                        float tj[D];
#pragma unroll
                        for (int k2 = 0; k2 < D; ++k2) tj[k2] = __shfl_sync(0xffffffffu, ta[k2], jj);
                        const int cls = okb ? box_class<D>(tj, cb, G) : 0;
                        uint32_t full = cls == 2 ? be - bs : 0u;
                        full = __reduce_add_sync(0xffffffffu, full);
                        uint32_t cj = __shfl_sync(0xffffffffu, cnt, jj) + full;
                        unsigned partial = __ballot_sync(0xffffffffu, cls == 1);
                        if (partial && cj < min_pts) {
                            const Pt<T, D> aj = shfl_pt<T, D>(pa, jj);
                            while (partial && cj < min_pts) {
                                const int t = __ffs(partial) - 1;
                                partial &= partial - 1;
                                const uint32_t ps = __shfl_sync(0xffffffffu, bs, t);
                                const uint32_t pe = __shfl_sync(0xffffffffu, be, t);
                                if (pe - ps <= 32) {  // most cells: one chunk
                                    const uint32_t q = ps + lane;
                                    const bool hit = q < pe && within_eps<D>(aj, v.pts[q], G);
                                    cj += __popc(__ballot_sync(0xffffffffu, hit));
                                    ++chunks;
                                    continue;
                                }
                                for (uint32_t qb = ps; qb < pe && cj < min_pts; qb += 128) {
                                    // four chunks of candidates in flight
                                    Pt<T, D> q4[4];
#pragma unroll
                                    for (int u = 0; u < 4; ++u) {
                                        const uint32_t q = qb + 32 * u + lane;
                                        q4[u] = q < pe ? v.pts[q] : zero_pt<T, D>();
                                    }
#pragma unroll
                                    for (int u = 0; u < 4; ++u) {
                                        const uint32_t q = qb + 32 * u + lane;
                                        const bool hit = q < pe && within_eps<D>(aj, q4[u], G);
                                        cj += __popc(__ballot_sync(0xffffffffu, hit));
                                    }
                                    ++chunks;
                                }
                            }
                        }
                        if (lane == jj) cnt = cj;
                        if (cj >= min_pts) open &= ~(1u << jj);
                    }
                }
            }
            const bool is_core = have && cnt >= min_pts;
            if (have) v.core[i] = is_core ? 1 : 0;
            any_core |= __any_sync(0xffffffffu, is_core);
            any_noncore |= __any_sync(0xffffffffu, have && !is_core);
        }
        if (any_core)
            for (int r = lane; r < RepDirs<D>::value; r += 32) v.reps[(uint64_t)A * RepDirs<D>::value + r] = ~0ull;
        if (lane == 0) v.cell_core[A] = any_core ? 1 : 0;
        if (any_core) lcore.add(v.list_core, &v.ctr->n_list[1], A);
        if (any_noncore) llabel.add(v.list_label, &v.ctr->n_list[2], A);
        core_cells += any_core ? 1u : 0u;
    }
    lcore.flush(v.list_core, &v.ctr->n_list[1]);
    llabel.flush(v.list_label, &v.ctr->n_list[2]);
    if (lane == 0 && dense_cells) atomicAdd(&v.ctr->n_dense, dense_cells);
    if (lane == 0 && core_cells) atomicAdd(&v.ctr->n_core_cells, core_cells);
    add_counter(&v.ctr->work[0], lane == 0 ? chunks : 0u);
}

// Algorithm 2: for every cell with core points and every direction delta, the core point
// nearest to the ideal position of delta, and that point's coordinates (rep_pts).
// The points are in cell order, so the pass walks them in windows of kRepWin consecutive
// points, one warp per window: every load of a window is issued at once (point, core flag,
// cell id, then the cell key), which keeps the pass a stream over the sorted points.  Lane r
// of a group of `width` lanes takes direction r and scans the group's core points in order,
// keeping the nearest per run of one cell (ties: the first in cell order).  A cell that lies
// wholly inside the scanned range gets its representatives and their coordinates by plain
// stores; a cell that crosses a range boundary combines its pieces by 64-bit atomicMin of
// (distance bits, sorted index) (non-negative float bits order like the floats) and gets its
// coordinates from k_rep_fix.  The representative only decides which pair a merge tests
// first, never a label.
constexpr uint32_t kRepWin = 128;     // points per warp window
constexpr int kRepWarps = 4;          // warps per block

template <int NDIR>
struct RepWidth {  // lanes per direction group: the power of two >= NDIR
    static constexpr int value = NDIR <= 2 ? 2 : NDIR <= 4 ? 4 : NDIR <= 8 ? 8 : NDIR <= 16 ? 16 : 32;
};

template <int D>
struct RepGeom {
    static constexpr int ndir = RepDirs<D>::value;
    static constexpr int width = RepWidth<ndir>::value;
    static constexpr int groups = 32 / width;
    static constexpr uint32_t sub = kRepWin / groups;  // points scanned by one group
};

// Bits of the 32-point slice `it` of a window that fall in group g's range [g sub, (g+1) sub).
template <int D>
__device__ __forceinline__ unsigned rep_group_bits(int it, int g) {
    constexpr int sub = (int)RepGeom<D>::sub;
    const int lo = max(g * sub - 32 * it, 0), hi = min((g + 1) * sub - 32 * it, 32);
    if (hi <= lo) return 0u;
    const unsigned upto = hi == 32 ? 0xffffffffu : ((1u << hi) - 1u);
    return upto & ~((1u << lo) - 1u);
}

template <typename T, int D>
__global__ void __launch_bounds__(32 * kRepWarps) k_reps(LowdView<T, D> v, int64_t n) {
    using Geo = RepGeom<D>;
    constexpr int ndir = Geo::ndir;
    constexpr int kPer = (int)(kRepWin / 32);
    __shared__ float2 s_lh[kRepWarps][kRepWin][D];    // (lo2, hi2) of every dimension
    __shared__ Pt<T, D> s_pt[kRepWarps][kRepWin];
    __shared__ uint32_t s_cell[kRepWarps][kRepWin + 2];  // cell ids of points w0 - 1 .. w0 + kRepWin
    const int lane = lane_id(), wib = threadIdx.x >> 5;
    const int64_t w0 = ((int64_t)blockIdx.x * kRepWarps + wib) * kRepWin;
    if (w0 >= n) return;
    // ---- loads: cell ids, core flags and points of the window, then the cells' keys ----
    uint32_t cid[kPer];
    uint8_t cf[kPer];
    Pt<T, D> pp[kPer];
#pragma unroll
    for (int it = 0; it < kPer; ++it) {
        const int64_t j = w0 + lane + 32 * it;
        const bool in = j < n;
        cid[it] = in ? v.cell_of[j] : 0xffffffffu;
        cf[it] = in ? v.core[j] : (uint8_t)0;
        pp[it] = in ? v.pts[j] : zero_pt<T, D>();
    }
    if (lane == 0) s_cell[wib][0] = w0 > 0 ? v.cell_of[w0 - 1] : 0xffffffffu;
    if (lane == 1) s_cell[wib][kRepWin + 1] = w0 + kRepWin < n ? v.cell_of[w0 + kRepWin] : 0xffffffffu;
    uint64_t key[kPer];
#pragma unroll
    for (int it = 0; it < kPer; ++it) key[it] = cf[it] ? v.cell_key[cid[it]] : 0ull;
    unsigned cmask[kPer];
#pragma unroll
    for (int it = 0; it < kPer; ++it) {
        const int p = lane + 32 * it;
        s_cell[wib][p + 1] = cid[it];
        cmask[it] = __ballot_sync(0xffffffffu, cf[it] != 0);
        if (cf[it]) {
            const GridParams &G = params_of(v, set_of_key(v, key[it]));
            int ac[D];
            unpack_key<D>(key[it], G, ac);
            float u[D];
            band_coords<T, D>(pp[it], G, u);
#pragma unroll
            for (int k = 0; k < D; ++k) {
                const float x = u[k] - (float)ac[k];
                s_lh[wib][p][k] = make_float2(x * x, (1.f - x) * (1.f - x));
            }
            s_pt[wib][p] = pp[it];
        }
    }
    __syncwarp();
    // ---- scan: lane r of group g takes direction r over the group's points.  The squared
    // distance of a point at cell-local position x to the ideal position of direction delta
    // (the face / edge / corner of the cube, Sec. 2) sums (1 - x_i)^2 over the dimensions with
    // delta_i = +1 and x_i^2 over those with delta_i = -1: weights whi / wlo of the lane ----
    const int g = lane / Geo::width, r = lane % Geo::width;
    const bool active = r < ndir;
    float wlo[D], whi[D];
#pragma unroll
    for (int k = 0; k < D; ++k) {
        wlo[k] = 0.f;
        whi[k] = 0.f;
    }
    if (active) {
        if (D <= 3) {
            int code = r < (ndir / 2) ? r : r + 1;
#pragma unroll
            for (int k = 0; k < D; ++k) {
                const int sgn = code % 3 - 1;
                code /= 3;
                if (sgn > 0) whi[k] = 1.f;
                if (sgn < 0) wlo[k] = 1.f;
            }
        } else {
#pragma unroll
            for (int k = 0; k < D; ++k)
                if (k == (r >> 1)) {
                    if (r & 1) whi[k] = 1.f;
                    else wlo[k] = 1.f;
                }
        }
    }
    // cells of the points just before and just after the group's range: a run of either
    // cell continues outside the range
    const uint32_t cprev = s_cell[wib][g * Geo::sub], cnext = s_cell[wib][(g + 1) * Geo::sub + 1];
    uint32_t cur = 0xffffffffu;
    float best = FLT_MAX;
    int bp = 0;
    auto flush = [&]() {
        if (!active) return;
        const uint64_t slot = (uint64_t)cur * ndir + r;
        const uint64_t val = ((uint64_t)__float_as_uint(best) << 32) | (uint32_t)(w0 + bp);
        if (cur == cprev || cur == cnext) {
            atomicMin((unsigned long long *)&v.reps[slot], (unsigned long long)val);
        } else {
            v.reps[slot] = val;
            v.rep_pts[slot] = s_pt[wib][bp];
        }
    };
#pragma unroll
    for (int it = 0; it < kPer; ++it) {
        unsigned mm = cmask[it] & rep_group_bits<D>(it, g);
        while (mm) {
            const int p = 32 * it + __ffs(mm) - 1;
            mm &= mm - 1;
            const uint32_t c = s_cell[wib][p + 1];
            if (c != cur) {
                if (cur != 0xffffffffu) flush();
                cur = c;
                best = FLT_MAX;
            }
            float dd = 0.f;
#pragma unroll
            for (int i = 0; i < D; ++i) {
                const float2 lh = s_lh[wib][p][i];
                dd = __fmaf_rn(wlo[i], lh.x, dd);
                dd = __fmaf_rn(whi[i], lh.y, dd);
            }
            if (dd < best) {
                best = dd;
                bp = p;
            }
        }
    }
    if (cur != 0xffffffffu) flush();
}

// Coordinates of the representatives of the cells that cross a scan-range boundary of
// k_reps (their pieces were combined by atomicMin): one thread per (boundary, direction).
// A cell that crosses several boundaries is written several times with the same values.
template <typename T, int D>
__global__ void __launch_bounds__(256) k_rep_fix(LowdView<T, D> v, int64_t n) {
    using Geo = RepGeom<D>;
    constexpr int ndir = Geo::ndir;
    const int64_t nb = (n + Geo::sub - 1) / Geo::sub;
    for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < nb * ndir;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int64_t j = (idx / ndir) * Geo::sub;
        const int r = (int)(idx % ndir);
        if (j == 0 || j >= n) continue;
        const uint32_t c = v.cell_of[j];
        if (c != v.cell_of[j - 1] || !v.cell_core[c]) continue;
        const uint64_t slot = (uint64_t)c * ndir + r;
        v.rep_pts[slot] = v.pts[(uint32_t)v.reps[slot]];
    }
}

// Does some core point of cell A lie within eps of some core point of cell B?  Warp-wide
// with early exit.  Only points that can reach the other cell's box take part; a core point
// whose distance to the whole other box is below eps settles it at once (B holds core points).
template <typename T, int D>
__device__ bool warp_core_pair(const LowdView<T, D> &v, uint32_t A, uint32_t B, const int *ac,
                               const int *bc, uint32_t &chunks, const GridParams &G) {
    const int lane = lane_id();
    const uint32_t sa = v.cell_start[A], ea = v.cell_start[A + 1];
    const uint32_t sb = v.cell_start[B], eb = v.cell_start[B + 1];
    for (uint32_t ia = sa; ia < ea; ia += 32) {
        const uint32_t i = ia + lane;
        bool va = i < ea && v.core[i];
        const Pt<T, D> pa = va ? v.pts[i] : zero_pt<T, D>();
        int cls = 0;
        if (va) {
            float t[D];
            band_coords<T, D>(pa, G, t);
            cls = box_class<D>(t, bc, G);
        }
        if (__any_sync(0xffffffffu, cls == 2)) return true;
        va = cls != 0;
        if (!__any_sync(0xffffffffu, va)) continue;
        for (uint32_t jb = sb; jb < eb; jb += 32) {
            const uint32_t j = jb + lane;
            bool vb = j < eb && v.core[j];
            const Pt<T, D> pb = vb ? v.pts[j] : zero_pt<T, D>();
            if (vb) {
                float t[D];
                band_coords<T, D>(pb, G, t);
                vb = box_class<D>(t, ac, G) != 0;
            }
            const unsigned bm = __ballot_sync(0xffffffffu, vb);
            if (!bm) continue;
            ++chunks;
            unsigned rem = bm;
            while (rem) {
                const int t = __ffs(rem) - 1;
                rem &= rem - 1;
                const Pt<T, D> q = shfl_pt<T, D>(pb, t);
                if (__any_sync(0xffffffffu, va && within_eps<D>(pa, q, G))) return true;
            }
        }
    }
    return false;
}

// First links between cells (Algorithm 3's merging condition, tested on the complementary
// representative points): every cell with core points links to the first neighbour cell of
// lower index whose representative pair is within eps.  One plain store per cell and every
// link points to a lower index, so the links form a forest whose trees lie inside clusters;
// pointer jumping flattens it and the merge passes then join the trees.
template <typename T, int D>
__global__ void __launch_bounds__(256) k_hook(LowdView<T, D> v, int n_all, int n_half) {
    constexpr int ndir = RepDirs<D>::value;
    const int lane = lane_id();
    const uint32_t NL = v.ctr->n_list[1];
    for (uint32_t w = global_warp(); w < NL; w += total_warps()) {
        const uint32_t A = v.list_core[w];
        int ac[D];
        const uint64_t akey = v.cell_key[A];
        unpack_key<D>(akey, v.g, ac);
        const GridParams &G = params_of(v, set_of_key(v, akey));
        bool linked = false;
        for (int g0 = 0; g0 < n_all && !linked; g0 += 32) {
            const int k = g0 + lane;
            uint2 rg = k < n_all ? v.ranges[(uint64_t)A * n_all + k] : make_uint2(0u, 0u);
            if (k == 0) rg.y = min(rg.y, A);          // own pencil: cells before A
            else if (k < n_half) rg.y = rg.x;         // upper-half pencils hold only cells after A
            const LaneRanges lr = lane_ranges(rg.x, rg.y);
            for (uint32_t f0 = 0; f0 < lr.total && !linked; f0 += 32) {
                const uint32_t f = f0 + lane;
                const uint32_t B = flat_cell(lr, f < lr.total ? f : 0u);
                const uint64_t bkey = f < lr.total ? v.cell_key[B] : 0ull;  // loaded with the core flag
                bool hit = f < lr.total && v.cell_core[B];
                if (hit) {
                    int bc[D], delta[D];
                    unpack_key<D>(bkey, v.g, bc);
#pragma unroll
                    for (int i = 0; i < D; ++i) delta[i] = bc[i] - ac[i];
                    const int ra = rep_dir_of<D>(delta);
                    const int rb = rep_dir_complement<D>(ra);
                    hit = within_eps<D>(v.rep_pts[(uint64_t)A * ndir + ra], v.rep_pts[(uint64_t)B * ndir + rb], G);
                }
                const unsigned hm = __ballot_sync(0xffffffffu, hit);
                if (hm) {
                    const uint32_t target = __shfl_sync(0xffffffffu, B, __ffs(hm) - 1);
                    if (lane == 0) v.parent[A] = target;
                    linked = true;
                }
            }
        }
    }
}

// One round of pointer jumping over cells with core points: parent[c] = parent[parent[c]].
template <typename T, int D>
__global__ void __launch_bounds__(256) k_jump(LowdView<T, D> v) {
    const uint32_t C = v.ctr->n_cells;
    for (uint32_t c = blockIdx.x * blockDim.x + threadIdx.x; c < C; c += gridDim.x * blockDim.x) {
        if (!v.cell_core[c]) continue;
        const uint32_t p = __ldcg(v.parent + c);
        const uint32_t gp = __ldcg(v.parent + p);
        if (gp != p) v.parent[c] = gp;
    }
}

// Algorithm 3: merge every pair of neighbouring cells that hold core points and have a core
// pair within eps.  Each unordered pair is visited once (upper half of the stencil).  Pass 0
// takes the cells at Chebyshev offset 1, pass 1 the rest, pass 2 all of them; a pair already in
// one set (after the first links and pointer jumping, most pairs of a cluster) is skipped.  The complementary
// representative points are tested first (Algorithm 3); a miss falls back to the exhaustive
// core x core test.  Lanes walk the flattened list of candidate cells of one cell.
template <typename T, int D>
__global__ void __launch_bounds__(256) k_merge(LowdView<T, D> v, int n_all, int n_half, int pass) {
    constexpr int ndir = RepDirs<D>::value;
    const int lane = lane_id();
    uint32_t rep_tests = 0, rep_hits = 0, exhaustive = 0, chunks = 0;
    const uint32_t NL = v.ctr->n_list[1];
    for (uint32_t w = global_warp(); w < NL; w += total_warps()) {
        const uint32_t A = v.list_core[w];
        int ac[D];
        const uint64_t akey = v.cell_key[A];
        unpack_key<D>(akey, v.g, ac);
        const GridParams &G = params_of(v, set_of_key(v, akey));
        for (int g0 = 0; g0 < n_half; g0 += 32) {
            const int k = g0 + lane;
            uint2 rg = k < n_half ? v.ranges[(uint64_t)A * n_all + k] : make_uint2(0u, 0u);
            if (k == 0 && rg.x < A + 1) rg.x = min(A + 1, rg.y);  // own pencil: cells after A
            const LaneRanges lr = lane_ranges(rg.x, rg.y);
            for (uint32_t f0 = 0; f0 < lr.total; f0 += 32) {
                const uint32_t f = f0 + lane;
                const uint32_t B = flat_cell(lr, f < lr.total ? f : 0u);
                const uint64_t bkey = f < lr.total ? v.cell_key[B] : 0ull;  // loaded with the core flag
                bool pending = f < lr.total && v.cell_core[B];
                int bc[D], delta[D];
                if (pending) {
                    unpack_key<D>(bkey, v.g, bc);
                    int cheb = 0;
#pragma unroll
                    for (int i = 0; i < D; ++i) {
                        delta[i] = bc[i] - ac[i];
                        cheb = max(cheb, abs(delta[i]));
                    }
                    pending = pass == 2 || (pass == 0) == (cheb <= 1);
                }
                if (pending && uf_find(v.parent, A, v.ctr) == uf_find(v.parent, B, v.ctr)) pending = false;
                if (pending) {
                    const int ra = rep_dir_of<D>(delta);
                    const int rb = rep_dir_complement<D>(ra);
                    ++rep_tests;
                    if (within_eps<D>(v.rep_pts[(uint64_t)A * ndir + ra], v.rep_pts[(uint64_t)B * ndir + rb], G)) {
                        uf_union(v.parent, A, B, v.ctr);
                        pending = false;
                        ++rep_hits;
                    }
                }
                unsigned need = __ballot_sync(0xffffffffu, pending);
                while (need) {
                    const int t = __ffs(need) - 1;
                    need &= need - 1;
                    const uint32_t B2 = __shfl_sync(0xffffffffu, B, t);
                    int bc2[D];
#pragma unroll
                    for (int i = 0; i < D; ++i) bc2[i] = __shfl_sync(0xffffffffu, bc[i], t);
                    bool same = false;
                    if (lane == 0) same = uf_find(v.parent, A, v.ctr) == uf_find(v.parent, B2, v.ctr);
                    same = __shfl_sync(0xffffffffu, same, 0);
                    if (same) continue;
                    ++exhaustive;
                    if (warp_core_pair<T, D>(v, A, B2, ac, bc2, chunks, G) && lane == 0)
                        uf_union(v.parent, A, B2, v.ctr);
                }
            }
        }
    }
    add_counter(&v.ctr->work[1], rep_tests);
    add_counter(&v.ctr->work[2], rep_hits);
    add_counter(&v.ctr->work[3], lane == 0 ? exhaustive : 0u);
    add_counter(&v.ctr->work[4], lane == 0 ? chunks : 0u);
}

// Flatten the union-find: parent[c] = root for every cell with core points; count roots.
// The only writes are parent[c] = root, so every pointer ends at its root.
template <typename T, int D>
__global__ void __launch_bounds__(256) k_compress(LowdView<T, D> v, int count_roots) {
    const uint32_t C = v.ctr->n_cells;
    uint32_t roots = 0;
    for (uint32_t c = blockIdx.x * blockDim.x + threadIdx.x; c < C; c += gridDim.x * blockDim.x) {
        if (!v.cell_core[c]) continue;
        const uint32_t r = uf_root_readonly(v.parent, c, v.ctr);
        v.parent[c] = r;
        roots += (r == c);
    }
    roots = __reduce_add_sync(0xffffffffu, roots);
    if (count_roots && lane_id() == 0 && roots) atomicAdd(&v.ctr->n_clusters, roots);
}

// Canonical cluster id (Algorithm 4 numbers clusters in traversal order; the fixed rule
// here is the smallest input index among the cluster's core points).  The radix sort is
// stable and starts from input order, so inside a cell the points keep their input order and
// the first core point of a cell holds the cell's smallest core index: one atomicMin per cell
// with core points.
template <typename T, int D>
__global__ void __launch_bounds__(256) k_comp_min(LowdView<T, D> v) {
    const uint32_t NL = v.ctr->n_list[1];
    for (uint32_t w = blockIdx.x * blockDim.x + threadIdx.x; w < NL; w += gridDim.x * blockDim.x) {
        const uint32_t A = v.list_core[w];
        const uint32_t e = v.cell_start[A + 1];
        uint32_t i = v.cell_start[A];
        while (i < e && !v.core[i]) ++i;
        if (i < e) atomicMin(&v.comp_min[v.parent[A]], v.perm[i]);
    }
}

// Cluster ids of core points, point-parallel (a cell can hold tens of thousands of points);
// also counts the core points.
template <typename T, int D>
__global__ void __launch_bounds__(256) k_label_core(LowdView<T, D> v) {
    const int64_t n = v.g.n;
    const int lane = lane_id();
    uint32_t ncore = 0;
    for (int64_t jb = blockIdx.x * (int64_t)blockDim.x + (threadIdx.x & ~31); jb < n;
         jb += (int64_t)gridDim.x * blockDim.x) {
        const int64_t j = jb + lane;
        const bool isc = j < n && v.core[j];
        ncore += __popc(__ballot_sync(0xffffffffu, isc));
        if (!isc) continue;
        const uint32_t o = v.perm[j];
        const uint32_t c = v.cell_of[j];
        const uint32_t base = v.gtab ? (uint32_t)v.set_off[set_of_key(v, v.cell_key[c])] : 0u;
        v.labels[o] = (int32_t)(v.comp_min[v.parent[c]] - base);
        if (v.core_out) v.core_out[o] = 1;
    }
    if (lane == 0 && ncore) atomicAdd(&v.ctr->n_core, ncore);
}

// Algorithm 4 and Definition 5 with the canonical rule: core points take their cluster id;
// a non-core point takes the smallest id among the clusters of the core points within eps
// (the core points of its own cell qualify without a test, the cell's diagonal being at most
// eps), else -1.  One warp per cell; the neighbour cells that hold core points and a smaller
// id are walked 32 at a time, one per lane; for each searching point a cell whose box lies
// wholly within eps settles that point at once (warp minimum), one wholly beyond eps is
// dropped, and the others are compared point by point.  Writes labels in input order.
template <typename T, int D>
__global__ void __launch_bounds__(256, 4) k_labels(LowdView<T, D> v, int n_all) {
    const int lane = lane_id();
    uint32_t noise = 0, chunks = 0;
    const uint32_t NL = v.ctr->n_list[2];
    LOWD_FOR_EACH(v, X, NL, 4) {
        const uint32_t A = v.list_label[X];
        const uint32_t s = v.cell_start[A], e = v.cell_start[A + 1];
        const uint64_t akey = v.cell_key[A];
        const uint32_t aset = set_of_key(v, akey);
        const GridParams &G = params_of(v, aset);
        if (e - s >= G.min_pts) continue;  // dense: every point is core (k_label_core)
        const uint32_t base_label = v.gtab ? (uint32_t)v.set_off[aset] : 0u;
        const bool hasc = v.cell_core[A];
        const uint32_t clA = hasc ? v.comp_min[v.parent[A]] : kNoLabel;
        for (uint32_t base = s; base < e; base += 32) {
            const uint32_t i = base + lane;
            const bool have = i < e;
            const bool isc = have && v.core[i];
            uint32_t best = clA;
            unsigned search = __ballot_sync(0xffffffffu, have && !isc);
            if (search) {
                const Pt<T, D> pa = have ? v.pts[i] : zero_pt<T, D>();
                float ta[D];
                band_coords<T, D>(pa, G, ta);
                for (int g0 = 0; g0 < n_all; g0 += 32) {
                    const int k = g0 + lane;
                    const uint2 rg = k < n_all ? v.ranges[(uint64_t)A * n_all + k] : make_uint2(0u, 0u);
                    const LaneRanges lr = lane_ranges(rg.x, rg.y);
                    for (uint32_t f0 = 0; f0 < lr.total; f0 += 32) {
                        const uint32_t f = f0 + lane;
                        const uint32_t B = flat_cell(lr, f < lr.total ? f : 0u);
                        const bool okb = f < lr.total && B != A && v.cell_core[B];
                        const uint32_t clB = okb ? v.comp_min[v.parent[B]] : kNoLabel;
                        if (!__any_sync(0xffffffffu, okb)) continue;
                        const uint32_t bs = okb ? v.cell_start[B] : 0u;
                        const uint32_t be = okb ? v.cell_start[B + 1] : 0u;
                        int cb[D];
                        unpack_key<D>(okb ? v.cell_key[B] : 0ull, v.g, cb);
                        unsigned rem = search;
                        while (rem) {
                            const int jj = __ffs(rem) - 1;
                            rem &= rem - 1;
                            uint32_t bj = __shfl_sync(0xffffffffu, best, jj);
                            const bool cand = okb && clB < bj;
                            if (!__any_sync(0xffffffffu, cand)) continue;
                            float tj[D];
#pragma unroll
                            for (int k2 = 0; k2 < D; ++k2) tj[k2] = __shfl_sync(0xffffffffu, ta[k2], jj);
                            const int cls = cand ? box_class<D>(tj, cb, G) : 0;
                            uint32_t m2 = cls == 2 ? clB : kNoLabel;
                            m2 = __reduce_min_sync(0xffffffffu, m2);
                            bj = min(bj, m2);
                            unsigned partial = __ballot_sync(0xffffffffu, cls == 1 && clB < bj);
                            if (partial) {
                                const Pt<T, D> aj = shfl_pt<T, D>(pa, jj);
                                while (partial) {
                                    const int t = __ffs(partial) - 1;
                                    partial &= partial - 1;
                                    const uint32_t cl2 = __shfl_sync(0xffffffffu, clB, t);
                                    if (cl2 >= bj) continue;
                                    const uint32_t ps = __shfl_sync(0xffffffffu, bs, t);
                                    const uint32_t pe = __shfl_sync(0xffffffffu, be, t);
                                    if (pe - ps <= 32) {  // most cells: one chunk
                                        const uint32_t q = ps + lane;
                                        const bool hit = q < pe && v.core[q] && within_eps<D>(aj, v.pts[q], G);
                                        ++chunks;
                                        if (__any_sync(0xffffffffu, hit)) bj = cl2;
                                        continue;
                                    }
                                    for (uint32_t qb = ps; qb < pe; qb += 128) {
                                        Pt<T, D> q4[4];
                                        bool c4[4];
#pragma unroll
                                        for (int u = 0; u < 4; ++u) {
                                            const uint32_t q = qb + 32 * u + lane;
                                            c4[u] = q < pe && v.core[q];
                                            q4[u] = q < pe ? v.pts[q] : zero_pt<T, D>();
                                        }
                                        bool hit = false;
#pragma unroll
                                        for (int u = 0; u < 4; ++u) hit |= c4[u] && within_eps<D>(aj, q4[u], G);
                                        ++chunks;
                                        if (__any_sync(0xffffffffu, hit)) {
                                            bj = cl2;
                                            break;
                                        }
                                    }
                                }
                            }
                            if (lane == jj) best = bj;
                        }
                    }
                }
            }
            if (have && !isc) {
                const int32_t lab = best == kNoLabel ? -1 : (int32_t)(best - base_label);
                const uint32_t o = v.perm[i];
                v.labels[o] = lab;
                if (v.core_out) v.core_out[o] = 0;
                noise += lab < 0;
            }
        }
    }
    noise = __reduce_add_sync(0xffffffffu, noise);
    if (lane == 0 && noise) atomicAdd(&v.ctr->n_noise, noise);
    add_counter(&v.ctr->work[5], lane == 0 ? chunks : 0u);
}


// ------------------------------------------------------------------------------------------
// Batched calls: per-set origin shift and binning
// ------------------------------------------------------------------------------------------

__device__ __forceinline__ uint32_t set_of_point(const int64_t *set_off, int nsets, int64_t j) {
    int lo = 0, hi = nsets;  // last s with set_off[s] <= j
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (__ldg(set_off + mid) <= j) lo = mid; else hi = mid;
    }
    return (uint32_t)lo;
}

// Declared extents of a plan (one set: box in `single`, measured extents in ctr->minmax_enc;
// sets: boxes and measured extents per set in `mm`, set-major): a measured minimum below or
// maximum above the box, or a NaN, sets status bit kErrBox.
struct BoxArgs {
    double mn[kMaxD], mx[kMaxD];
};
template <int D>
__global__ void __launch_bounds__(256) k_box_check(BoxArgs single, const double *__restrict__ boxes, int nsets,
                                                  const int64_t *__restrict__ set_off,
                                                  const unsigned long long *__restrict__ mm, DevCounters *ctr) {
    if (blockIdx.x == 0 && threadIdx.x == 0 && ctr->nan_seen) atomicOr(&ctr->status, kErrBox);
    if (!boxes) {
        if (blockIdx.x != 0 || threadIdx.x >= D) return;
        const int i = threadIdx.x;
        const uint64_t *enc = ctr->minmax_enc;
        if (dec_double_dev(enc[i]) < single.mn[i] || dec_double_dev(enc[kMaxD + i]) > single.mx[i])
            atomicOr(&ctr->status, kErrBox);
        return;
    }
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < (int64_t)nsets * D;
         k += (int64_t)gridDim.x * blockDim.x) {
        const int set = (int)(k / D), i = (int)(k % D);
        if (set_off[set + 1] == set_off[set]) continue;
        const double lo = dec_double_dev(mm[(size_t)set * kMaxD + i]);
        const double hi = dec_double_dev(mm[(size_t)kMaxD * nsets + (size_t)set * kMaxD + i]);
        if (lo < boxes[(size_t)set * D + i] || hi > boxes[(size_t)(nsets + set) * D + i])
            atomicOr(&ctr->status, kErrBox);
    }
}

// Per-set min / max of every dimension for a batched call (set s = points [set_off[s],
// set_off[s + 1]), d values each; mm[s * stride + i] and mm[(nsets + s) * stride + i] receive
// the order-preserving codes of the minimum and maximum of dimension i).  Each warp takes a
// contiguous run of points, so it crosses few set boundaries: lanes hold running minima and
// maxima of fixed dimensions (lane % d, for d <= 32 and 32 / d points per step; dimensions
// lane and lane + 32 for larger d), and the warp folds them into the set's words with one
// atomic per dimension at each set boundary and at the end of its run.
template <typename T>
__device__ __forceinline__ void seg_minmax(const T *__restrict__ in, int64_t n, int d, const int64_t *set_off,
                                           int nsets, unsigned long long *mm, int stride, DevCounters *ctr) {
    const int lane = lane_id();
    const int64_t warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t per = (n + warps - 1) / warps;
    const int64_t j0 = gw * per, j1 = min(n, j0 + per);
    const int g = d <= 32 ? 32 / d : 1;   // points per step
    const int dim = d <= 32 ? lane % d : lane;
    const int slot = d <= 32 ? lane / d : 0;
    const bool lane_on = slot < g;
    const T big = sizeof(T) == 4 ? (T)FLT_MAX : (T)DBL_MAX;
    bool nan = false;
    if (j0 < j1) {
        uint32_t set = set_of_point(set_off, nsets, j0);
        int64_t next = __ldg(set_off + set + 1);
        T mn0 = big, mx0 = -big, mn1 = big, mx1 = -big;
        bool any = false;
        auto flush = [&]() {
            if (!any) return;
            if (d <= 32) {
                // fold the point slots of each dimension into lanes 0 .. d - 1
                for (int k = 1; k < g; ++k) {
                    const T a = __shfl_sync(0xffffffffu, mn0, min(lane + k * d, 31));
                    const T b = __shfl_sync(0xffffffffu, mx0, min(lane + k * d, 31));
                    if (lane < d) {
                        mn0 = a < mn0 ? a : mn0;
                        mx0 = b > mx0 ? b : mx0;
                    }
                }
                if (lane < d) {
                    atomicMin(&mm[(uint64_t)set * stride + lane], (unsigned long long)enc_double((double)mn0));
                    atomicMax(&mm[((uint64_t)nsets + set) * stride + lane], (unsigned long long)enc_double((double)mx0));
                }
            } else {
                if (lane < d) {
                    atomicMin(&mm[(uint64_t)set * stride + lane], (unsigned long long)enc_double((double)mn0));
                    atomicMax(&mm[((uint64_t)nsets + set) * stride + lane], (unsigned long long)enc_double((double)mx0));
                }
                if (lane + 32 < d) {
                    atomicMin(&mm[(uint64_t)set * stride + lane + 32], (unsigned long long)enc_double((double)mn1));
                    atomicMax(&mm[((uint64_t)nsets + set) * stride + lane + 32],
                              (unsigned long long)enc_double((double)mx1));
                }
            }
            mn0 = big; mx0 = -big; mn1 = big; mx1 = -big;
            any = false;
        };
        for (int64_t j = j0; j < j1;) {
            while (j >= next) {  // warp-uniform: the run enters the next non-empty set
                flush();
                ++set;
                next = __ldg(set_off + set + 1);
            }
            const int64_t stop = min(j1, next);
            if (stop - j >= 4 * g) {
                // four full steps, their loads in flight together
                T x0[4], x1[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int64_t p = j + u * g + slot;
                    x0[u] = lane_on && (d <= 32 || lane < d) ? __ldg(in + p * d + dim) : (T)0;
                    x1[u] = d > 32 && lane + 32 < d ? __ldg(in + p * d + lane + 32) : (T)0;
                }
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    if (lane_on && (d <= 32 || lane < d)) {
                        nan |= (x0[u] != x0[u]);
                        mn0 = x0[u] < mn0 ? x0[u] : mn0;
                        mx0 = x0[u] > mx0 ? x0[u] : mx0;
                    }
                    if (d > 32 && lane + 32 < d) {
                        nan |= (x1[u] != x1[u]);
                        mn1 = x1[u] < mn1 ? x1[u] : mn1;
                        mx1 = x1[u] > mx1 ? x1[u] : mx1;
                    }
                }
                any = true;
                j += 4 * g;
                continue;
            }
            const int take = (int)min((int64_t)g, stop - j);
            const int64_t p = j + slot;
            if (lane_on && slot < take) {
                if (d <= 32) {
                    const T x = __ldg(in + p * d + dim);
                    nan |= (x != x);
                    mn0 = x < mn0 ? x : mn0;
                    mx0 = x > mx0 ? x : mx0;
                } else {
                    if (lane < d) {
                        const T x = __ldg(in + p * d + lane);
                        nan |= (x != x);
                        mn0 = x < mn0 ? x : mn0;
                        mx0 = x > mx0 ? x : mx0;
                    }
                    if (lane + 32 < d) {
                        const T x = __ldg(in + p * d + lane + 32);
                        nan |= (x != x);
                        mn1 = x < mn1 ? x : mn1;
                        mx1 = x > mx1 ? x : mx1;
                    }
                }
            }
            any = true;
            j += take;
        }
        flush();
    }
    if (__any_sync(0xffffffffu, nan) && lane == 0) atomicOr(&ctr->nan_seen, 1u);
}

template <typename T, int D>
__global__ void __launch_bounds__(256) k_minmax_seg(const T *__restrict__ in, int64_t n, const int64_t *set_off,
                                                   int nsets, unsigned long long *mm, DevCounters *ctr) {
    seg_minmax<T>(in, n, D, set_off, nsets, mm, kMaxD, ctr);
}

// Algorithm 1 per set, with the set id above the cell key bits.
template <typename T, int D, typename K>
__global__ void __launch_bounds__(256) k_bin_seg(const T *__restrict__ in, int64_t n, const int64_t *set_off,
                                                int nsets, const GridParams *gtab, int key_bits,
                                                K *__restrict__ keys, uint32_t *__restrict__ idx,
                                                uint32_t *__restrict__ digit_counts, int total_bits) {
    __shared__ uint32_t h[8][256];
    const int passes = (total_bits + 7) / 8;
    for (int i = threadIdx.x; i < 8 * 256; i += blockDim.x) (&h[0][0])[i] = 0;
    __syncthreads();
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n;
         j += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t set = set_of_point(set_off, nsets, j);
        const GridParams &g = gtab[set];
        uint64_t key = (uint64_t)set << key_bits;
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
        for (int p = 0; p < passes; ++p) atomicAdd(&h[p][(uint32_t)(key >> (8 * p)) & 0xffu], 1u);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < passes * 256; i += blockDim.x) {
        const uint32_t c = (&h[0][0])[i];
        if (c) atomicAdd(&digit_counts[i], c);
    }
}

}  // namespace hca
