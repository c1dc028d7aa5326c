// Kernels of the high-dimensional path (5 <= d <= 64), templated on the coordinate type T and
// the padded row width DP (8, 16, 32 or 64 >= d; the padding coordinates are zero and add
// exact zeros to every distance).
//
// In d dimensions the hypercubes of side eps/sqrt(d) (Sec. 2, Algorithm 1) hold about one point
// each on spread data and their neighbour block (2 ceil(sqrt d) + 1)^d (Sec. 2, "Depth First
// Search") is astronomically large, so the neighbour search uses a coarse grid instead: cells
// of side >= eps over the three dimensions of largest extent.  Two points within eps differ by
// at most eps in every coordinate, so they lie in the same or adjacent coarse cells (the 3x3x3
// block).  The coarse cells are binned, sorted, run-length encoded, hashed and given neighbour
// ranges by the same kernels as the hypercube path (D = 3 on the projected coordinates).  The
// clustering itself then works on points: exact counts with early exit at MINPTS
// (Definition 2), union-find over core points (Definitions 3-5) and the canonical labels.
//
// Layout: pts[j * DP + i] (cell order, zero padded), perm[j], cell_start/cell_key/ranges of
// the coarse cells, core[j], parent[j] and comp_min[j] over points.
#pragma once

#include <type_traits>

#include "lowd_kernels.cuh"

namespace hca {

template <typename T, int DP>
struct HdView {
    GridParams g;                 // coarse grid on the projected dimensions; eps2, lo32, hi32, min_pts, n
    const GridParams *gtab;       // batched calls: parameters of every set (same key layout)
    const int64_t *set_off;       // batched calls: first point of every set
    int d;
    const T *pts;                 // sorted, n x DP
    const uint32_t *perm;
    const uint32_t *cell_start;
    const uint32_t *chunk_off;    // first 32-point chunk of each coarse cell
    const uint64_t *cell_key;
    const uint2 *ranges;
    uint8_t *core;
    uint8_t *cell_core;
    uint32_t *parent;
    uint32_t *comp_min;
    int32_t *labels;
    uint8_t *core_out;
    DevCounters *ctr;
    int n_all, n_half;
    // cells left to the tensor-core kernels (float input): those with at least tc_min[phase] rows
    // of a phase (counts, unions, labels; 0: none); cx = exclusive scan of the core flags, for
    // the per-cell core counts; tc_hook: first links also in cells whose unions run there
    uint32_t tc_min[3];
    uint32_t tc_hook;
    uint32_t tc_handoff;  // open count rows at which a tensor-core chunk hands over
    const uint32_t *cx;
    // rows the tensor-core count handed over: count so far and candidate-stream position
    uint32_t *tc_cnt;
    uint32_t *tc_pos;
    // per coarse cell, the smallest and largest coordinate of its points in every dimension
    // (DP values each): a point farther than eps from a cell's box is farther than eps from
    // every point of the cell
    T *box_lo;
    T *box_hi;
};

constexpr int kHdWarps = 4;     // warps per block in the point kernels of this path (default)
constexpr int kHdMaxWarps = 8;  // most warps per block a tuning may choose

// dist(a, q) <= eps with a in shared memory and q in registers (same exact predicate and FP32
// guard band as the hypercube path; summation in dimension order).
template <int DP>
__device__ __forceinline__ bool hd_within(const float *a, const float (&q)[DP], const GridParams &g) {
    float s = 0.f;
#pragma unroll
    for (int i = 0; i < DP; i += 4) {
        // the sum of squares only grows (fma of a square into a non-negative sum rounds to at
        // least the sum), so a partial sum above hi32 already decides the pair: when every
        // lane of the warp is there, the rest of the dimensions are skipped
        if (i == DP / 2 && s > g.hi32) return false;
        const float4 av = *reinterpret_cast<const float4 *>(a + i);
        float t = __fsub_rn(av.x, q[i]);     s = __fmaf_rn(t, t, s);
        t = __fsub_rn(av.y, q[i + 1]);       s = __fmaf_rn(t, t, s);
        t = __fsub_rn(av.z, q[i + 2]);       s = __fmaf_rn(t, t, s);
        t = __fsub_rn(av.w, q[i + 3]);       s = __fmaf_rn(t, t, s);
    }
    if (s < g.lo32) return true;
    if (s > g.hi32) return false;
    double e = 0.0;
#pragma unroll
    for (int i = 0; i < DP; ++i) {
        const double t = __dsub_rn((double)a[i], (double)q[i]);
        e = __dadd_rn(e, __dmul_rn(t, t));
    }
    return e <= g.eps2;
}
template <int DP>
__device__ __forceinline__ bool hd_within(const double *a, const double (&q)[DP], const GridParams &g) {
    double e = 0.0;
#pragma unroll
    for (int i = 0; i < DP; ++i) {
        const double t = __dsub_rn(a[i], q[i]);
        e = __dadd_rn(e, __dmul_rn(t, t));
    }
    return e <= g.eps2;
}

// True when the point a (DP coordinates) is provably farther than eps from every point of the
// box [lo, hi]: the squared distance to the box, sum_i max(lo_i - a_i, a_i - hi_i, 0)^2, is a
// lower bound of the squared distance to any point inside.  float: summed in FP32 (each term
// and the sum within (DP + 2) 2^-24 of exact) against hi32 = eps^2 (1 + 2^-16) rounded up, so a
// box it calls far is farther than eps in exact arithmetic and in the FP64 predicate (when the
// FP32 filter is off, hi32 is infinite and no box is called far); double: summed in FP64
// against eps^2 (1 + 2^-40).
template <int DP>
__device__ __forceinline__ bool box_far(const float *a, const float *lo, const float *hi, const GridParams &g) {
    float s = 0.f;
#pragma unroll
    for (int i = 0; i < DP; i += 4) {
        const float4 av = *reinterpret_cast<const float4 *>(a + i);
        const float4 l = __ldg(reinterpret_cast<const float4 *>(lo + i));
        const float4 h = __ldg(reinterpret_cast<const float4 *>(hi + i));
        float t = fmaxf(fmaxf(__fsub_rn(l.x, av.x), __fsub_rn(av.x, h.x)), 0.f); s = __fmaf_rn(t, t, s);
        t = fmaxf(fmaxf(__fsub_rn(l.y, av.y), __fsub_rn(av.y, h.y)), 0.f);       s = __fmaf_rn(t, t, s);
        t = fmaxf(fmaxf(__fsub_rn(l.z, av.z), __fsub_rn(av.z, h.z)), 0.f);       s = __fmaf_rn(t, t, s);
        t = fmaxf(fmaxf(__fsub_rn(l.w, av.w), __fsub_rn(av.w, h.w)), 0.f);       s = __fmaf_rn(t, t, s);
    }
    return s > g.hi32;
}
template <int DP>
__device__ __forceinline__ bool box_far(const double *a, const double *lo, const double *hi, const GridParams &g) {
    double s = 0.0;
#pragma unroll
    for (int i = 0; i < DP; ++i) {
        const double t = fmax(fmax(__dsub_rn(__ldg(lo + i), a[i]), __dsub_rn(a[i], __ldg(hi + i))), 0.0);
        s = __fma_rn(t, t, s);
    }
    return s > g.eps2 * (1.0 + 0x1p-40);
}

template <typename T, int DP>
__device__ __forceinline__ void hd_load(const T *pts, uint32_t j, bool valid, T (&q)[DP]) {
    if (sizeof(T) == 4) {
        const float4 *src = reinterpret_cast<const float4 *>(pts + (uint64_t)j * DP);
#pragma unroll
        for (int i = 0; i < DP / 4; ++i) {
            const float4 v4 = valid ? src[i] : make_float4(0.f, 0.f, 0.f, 0.f);
            q[4 * i] = v4.x; q[4 * i + 1] = v4.y; q[4 * i + 2] = v4.z; q[4 * i + 3] = v4.w;
        }
    } else {
        const double2 *src = reinterpret_cast<const double2 *>(pts + (uint64_t)j * DP);
#pragma unroll
        for (int i = 0; i < DP / 2; ++i) {
            const double2 v2 = valid ? src[i] : make_double2(0.0, 0.0);
            q[2 * i] = v2.x; q[2 * i + 1] = v2.y;
        }
    }
}

// Declared extents of a plan against the measured ones (encoded min of dimension i of set s at
// mm[s * 64 + i], max at mm[(nsets + s) * 64 + i]; boxes: mins [s * d + i], maxes
// [(nsets + s) * d + i]): a point outside its box, or a NaN, sets status bit kErrBox.
static __global__ void __launch_bounds__(256) k_box_check_hd(const double *__restrict__ boxes, int nsets, int d,
                                                            const int64_t *__restrict__ set_off,
                                                            const unsigned long long *__restrict__ mm,
                                                            DevCounters *ctr) {
    if (blockIdx.x == 0 && threadIdx.x == 0 && ctr->nan_seen) atomicOr(&ctr->status, kErrBox);
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < (int64_t)nsets * d;
         k += (int64_t)gridDim.x * blockDim.x) {
        const int set = (int)(k / d), i = (int)(k % d);
        if (set_off && set_off[set + 1] == set_off[set]) continue;
        const double lo = dec_double_dev(mm[(size_t)set * 64 + i]);
        const double hi = dec_double_dev(mm[((size_t)nsets + set) * 64 + i]);
        if (lo < boxes[(size_t)set * d + i] || hi > boxes[((size_t)nsets + set) * d + i])
            atomicOr(&ctr->status, kErrBox);
    }
}

// Per-dimension min / max of row-major n x d input (origin shift, Sec. 2).  Each thread keeps
// one dimension (the stride is a multiple of d).
template <typename T>
__global__ void __launch_bounds__(256) k_minmax_rt(const T *__restrict__ in, int64_t n, int d, DevCounters *ctr,
                                                  unsigned long long *mm /* [2 * 64] */) {
    // each thread walks one dimension (a stride that is a multiple of d), four independent
    // loads in flight; the block folds its threads per dimension in shared memory, then one
    // global atomic per block and dimension
    __shared__ unsigned long long smn[64], smx[64];
    __shared__ int snan;
    for (int i = threadIdx.x; i < 64; i += blockDim.x) {
        smn[i] = ~0ull;
        smx[i] = 0ull;
    }
    if (threadIdx.x == 0) snan = 0;
    __syncthreads();
    const int64_t total = n * d;
    const int64_t threads = (int64_t)gridDim.x * blockDim.x;
    const int64_t stride = (threads / d) * d;
    const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (tid < stride) {
        T mn[4], mx[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            mn[u] = sizeof(T) == 4 ? (T)FLT_MAX : (T)DBL_MAX;
            mx[u] = -mn[u];
        }
        bool nan = false;
        int64_t e = tid;
        for (; e + 3 * stride < total; e += 4 * stride) {
            T x[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) x[u] = __ldg(in + e + u * stride);
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                nan |= (x[u] != x[u]);
                mn[u] = x[u] < mn[u] ? x[u] : mn[u];
                mx[u] = x[u] > mx[u] ? x[u] : mx[u];
            }
        }
        for (; e < total; e += stride) {
            const T x = __ldg(in + e);
            nan |= (x != x);
            mn[0] = x < mn[0] ? x : mn[0];
            mx[0] = x > mx[0] ? x : mx[0];
        }
#pragma unroll
        for (int u = 1; u < 4; ++u) {
            mn[0] = mn[u] < mn[0] ? mn[u] : mn[0];
            mx[0] = mx[u] > mx[0] ? mx[u] : mx[0];
        }
        const int dim = (int)(tid % d);
        atomicMin(&smn[dim], (unsigned long long)enc_double((double)mn[0]));
        atomicMax(&smx[dim], (unsigned long long)enc_double((double)mx[0]));
        if (nan) snan = 1;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < d; i += blockDim.x) {
        if (smn[i] != ~0ull) atomicMin(&mm[i], smn[i]);
        if (smx[i] != 0ull) atomicMax(&mm[64 + i], smx[i]);
    }
    if (threadIdx.x == 0 && snan) atomicOr(&ctr->nan_seen, 1u);
}

// Coarse cell keys from the three projected dimensions (Algorithm 1 on a grid of side >= eps).
template <typename T, typename K>
__global__ void __launch_bounds__(256) k_bin_proj(const T *__restrict__ in, int d, int3 sel, GridParams g,
                                                 K *__restrict__ keys, uint32_t *__restrict__ idx) {
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < g.n;
         j += (int64_t)gridDim.x * blockDim.x) {
        const int dims[3] = {sel.x, sel.y, sel.z};
        uint64_t key = 0;
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            const double t = __dmul_rn(__dsub_rn((double)in[j * d + dims[i]], g.origin[i]), g.inv_side);
            uint32_t c = (uint32_t)floor(t);
            if (c > g.ncell[i] - 1) c = g.ncell[i] - 1;
            key |= (uint64_t)c << g.shift[i];
        }
        keys[j] = (K)key;
        idx[j] = (uint32_t)j;
    }
}

// Gather the points into cell order, padded to DP coordinates, and flag the first point of
// every coarse cell; one block per tile of kScanTileElems rows, DP / 4 threads per row (four
// coordinates each, one vector store), the tile's flag count to tile_sums[block].
template <typename T, int DP, typename K>
__global__ void __launch_bounds__(256) k_gather_hd(const T *__restrict__ in, int d, const K *__restrict__ keys,
                                                  const uint32_t *__restrict__ idx, int64_t n,
                                                  T *__restrict__ pts, uint32_t *__restrict__ flags,
                                                  uint32_t *__restrict__ tile_sums) {
    constexpr int G = DP / 4;          // threads per row
    constexpr int R = 256 / G;         // rows per step of the block
    const int g = threadIdx.x % G, r0 = threadIdx.x / G;
    const int64_t base = (int64_t)blockIdx.x * kScanTileElems;
    uint32_t cnt = 0;
#pragma unroll 4
    for (int k = 0; k < kScanTileElems / R; ++k) {
        const int64_t j = base + (int64_t)k * R + r0;
        if (j < n) {
            const uint32_t o = idx[j];
            const T *src = in + (int64_t)o * d;
            T x[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) x[u] = 4 * g + u < d ? src[4 * g + u] : T(0);
            T *dst = pts + j * DP + 4 * g;
            if (sizeof(T) == 4) {
                *reinterpret_cast<float4 *>(dst) = make_float4((float)x[0], (float)x[1], (float)x[2], (float)x[3]);
            } else {
                reinterpret_cast<double2 *>(dst)[0] = make_double2((double)x[0], (double)x[1]);
                reinterpret_cast<double2 *>(dst)[1] = make_double2((double)x[2], (double)x[3]);
            }
            if (g == 0) {
                const uint32_t f = (j == 0 || keys[j] != keys[j - 1]) ? 1u : 0u;
                flags[j] = f;
                cnt += f;
            }
        }
    }
    uint32_t total;
    block_exclusive_scan<256>(cnt, &total);
    if (threadIdx.x == 0) tile_sums[blockIdx.x] = total;
}

template <typename T, int DP>
__device__ __forceinline__ void stage_rows(T *rows, const T *pts, uint32_t base, uint32_t e) {
    // rows: 32 x DP for this warp; lane L copies row L
    const int lane = threadIdx.x & 31;
    const uint32_t i = base + lane;
    T q[DP];
    hd_load<T, DP>(pts, i, i < e, q);
    if (sizeof(T) == 4) {
        float4 *dst = reinterpret_cast<float4 *>(rows + lane * DP);
#pragma unroll
        for (int k = 0; k < DP / 4; ++k)
            dst[k] = make_float4((float)q[4 * k], (float)q[4 * k + 1], (float)q[4 * k + 2], (float)q[4 * k + 3]);
    } else {
#pragma unroll
        for (int k = 0; k < DP; ++k) rows[lane * DP + k] = q[k];
    }
    __syncwarp();
}

// Work is scheduled in chunks of 32 consecutive points of one coarse cell (a coarse cell can
// hold a whole cluster, so one warp per cell would leave the largest cell to a single warp).
// chunk_off[c] = first chunk of cell c (exclusive scan of ceil(size / 32)).
static __global__ void __launch_bounds__(256) k_chunk_counts(const uint32_t *__restrict__ cell_start,
                                                     const DevCounters *ctr, uint32_t *__restrict__ nch) {
    const uint32_t C = ctr->n_cells;
    for (uint32_t c = blockIdx.x * blockDim.x + threadIdx.x; c < C; c += gridDim.x * blockDim.x)
        nch[c] = (cell_start[c + 1] - cell_start[c] + 31u) / 32u;
}

// Cell of chunk t (upper bound in chunk_off, minus one).  Warp-uniform.
__device__ __forceinline__ uint32_t chunk_cell(const uint32_t *chunk_off, uint32_t C, uint32_t t) {
    uint32_t lo = 0, hi = C;
    while (hi - lo > 1) {
        const uint32_t mid = (lo + hi) >> 1;
        if (__ldg(chunk_off + mid) <= t) lo = mid; else hi = mid;
    }
    return lo;
}

// Box of every coarse cell in three launches: clear, accumulate over 32-point chunks (one
// warp per chunk, so a large cell is spread over many warps), decode.  Coordinates are
// accumulated as order-preserving unsigned integers (sign bit flipped for x >= 0, every bit
// for x < 0), so min / max of the codes is min / max of the values and the warps of one cell
// combine with atomicMin / atomicMax.
template <typename T>
struct BoxCode {
    typedef typename std::conditional<sizeof(T) == 4, uint32_t, unsigned long long>::type U;
    static __device__ __forceinline__ U enc(T x) {
        if (sizeof(T) == 4) {
            const uint32_t u = __float_as_uint((float)x);
            return (U)(u ^ ((uint32_t)((int32_t)u >> 31) | 0x80000000u));
        } else {
            const unsigned long long u = (unsigned long long)__double_as_longlong((double)x);
            return (U)(u ^ ((unsigned long long)((long long)u >> 63) | 0x8000000000000000ull));
        }
    }
    static __device__ __forceinline__ T dec(U c) {
        if (sizeof(T) == 4) {
            const uint32_t u = (uint32_t)c;
            return (T)__uint_as_float(u ^ ((u >> 31) ? 0x80000000u : 0xffffffffu));
        } else {
            const unsigned long long u = (unsigned long long)c;
            return (T)__longlong_as_double((long long)(u ^ ((u >> 63) ? 0x8000000000000000ull : ~0ull)));
        }
    }
    static __device__ __forceinline__ U warp_min(U v) {
        if (sizeof(T) == 4) return (U)__reduce_min_sync(0xffffffffu, (uint32_t)v);
        for (int o = 16; o; o >>= 1) {
            const U t = __shfl_xor_sync(0xffffffffu, v, o);
            v = t < v ? t : v;
        }
        return v;
    }
    static __device__ __forceinline__ U warp_max(U v) {
        if (sizeof(T) == 4) return (U)__reduce_max_sync(0xffffffffu, (uint32_t)v);
        for (int o = 16; o; o >>= 1) {
            const U t = __shfl_xor_sync(0xffffffffu, v, o);
            v = t > v ? t : v;
        }
        return v;
    }
};

template <typename T, int DP>
__global__ void __launch_bounds__(256) k_cell_box_clear(HdView<T, DP> v) {
    typedef typename BoxCode<T>::U U;
    const uint64_t m = (uint64_t)v.ctr->n_cells * DP;
    U *lo = reinterpret_cast<U *>(v.box_lo), *hi = reinterpret_cast<U *>(v.box_hi);
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < m; i += (uint64_t)gridDim.x * blockDim.x) {
        lo[i] = ~(U)0;
        hi[i] = (U)0;
    }
}

template <typename T, int DP>
__global__ void __launch_bounds__(256) k_cell_box_hd(HdView<T, DP> v) {
    typedef BoxCode<T> BC;
    typedef typename BC::U U;
    constexpr int E = DP > 32 ? DP / 32 : 1;  // dimensions per lane in the atomics
    const int lane = lane_id();
    const uint32_t C = v.ctr->n_cells, NC = v.ctr->n_chunks;
    const uint32_t warps = (gridDim.x * blockDim.x) >> 5;
    U *lo = reinterpret_cast<U *>(v.box_lo), *hi = reinterpret_cast<U *>(v.box_hi);
    for (uint32_t t = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; t < NC; t += warps) {
        const uint32_t A = chunk_cell(v.chunk_off, C, t);
        const uint32_t e = v.cell_start[A + 1], base = v.cell_start[A] + 32u * (t - v.chunk_off[A]);
        const uint32_t p = base + lane;
        const bool valid = p < e;
        U mn[E], mx[E];
#pragma unroll
        for (int k = 0; k < E; ++k) {
            mn[k] = ~(U)0;
            mx[k] = (U)0;
        }
#pragma unroll
        for (int g0 = 0; g0 < DP; g0 += 4) {
            T x[4];
            if (sizeof(T) == 4) {
                const float4 f = valid ? __ldg(reinterpret_cast<const float4 *>(v.pts + (uint64_t)p * DP + g0))
                                       : make_float4(0.f, 0.f, 0.f, 0.f);
                x[0] = (T)f.x; x[1] = (T)f.y; x[2] = (T)f.z; x[3] = (T)f.w;
            } else {
#pragma unroll
                for (int i = 0; i < 4; ++i) x[i] = valid ? __ldg(v.pts + (uint64_t)p * DP + g0 + i) : (T)0;
            }
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const U c = BC::enc(x[i]);
                const U a = BC::warp_min(valid ? c : ~(U)0);
                const U b = BC::warp_max(valid ? c : (U)0);
                if (lane == ((g0 + i) & 31)) {
                    mn[(g0 + i) >> 5] = a;
                    mx[(g0 + i) >> 5] = b;
                }
            }
        }
        if (lane < DP) {
#pragma unroll
            for (int k = 0; k < E; ++k) {
                atomicMin(lo + (uint64_t)A * DP + lane + 32 * k, mn[k]);
                atomicMax(hi + (uint64_t)A * DP + lane + 32 * k, mx[k]);
            }
        }
    }
}

template <typename T, int DP>
__global__ void __launch_bounds__(256) k_cell_box_decode(HdView<T, DP> v) {
    typedef BoxCode<T> BC;
    typedef typename BC::U U;
    const uint64_t m = (uint64_t)v.ctr->n_cells * DP;
    U *lo = reinterpret_cast<U *>(v.box_lo), *hi = reinterpret_cast<U *>(v.box_hi);
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < m; i += (uint64_t)gridDim.x * blockDim.x) {
        v.box_lo[i] = BC::dec(lo[i]);
        v.box_hi[i] = BC::dec(hi[i]);
    }
}

#define HD_FOR_EACH_CHUNK(v, A, base, e, slot)                                                \
    const uint32_t C_ = (v).ctr->n_cells, NC_ = (v).ctr->n_chunks;                           \
    for (uint32_t t_ = next_chunk(&(v).ctr->hd_next[slot]); t_ < NC_;                        \
         t_ = next_chunk(&(v).ctr->hd_next[slot]))                                           \
        for (uint32_t A = chunk_cell((v).chunk_off, C_, t_), once_ = 1; once_; once_ = 0)    \
            for (uint32_t e = (v).cell_start[A + 1],                                         \
                          base = (v).cell_start[A] + 32u * (t_ - (v).chunk_off[A]), o2_ = 1; \
                 o2_; o2_ = 0)

// Definition 2: |N_eps(p)| >= MINPTS, counted over the 27 neighbouring coarse cells (the own
// point included), stopping once every point of the chunk has reached MINPTS.  The chunk's
// points are staged in shared memory, candidates stream through the lanes, and each open
// point is compared with a warp ballot.
template <typename T, int DP>
__global__ void __launch_bounds__(32 * kHdMaxWarps) k_count_hd(HdView<T, DP> v) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *rows = reinterpret_cast<T *>(smem_raw) + (threadIdx.x >> 5) * 32 * DP;
    const int lane = lane_id();
    uint32_t chunks = 0;
    HD_FOR_EACH_CHUNK(v, A, base, e, 0) {
        // a cell counted on the tensor cores leaves here only the rows it handed over (core = 2)
        const bool tc_cell = v.tc_min[0] && e - v.cell_start[A] >= v.tc_min[0];
        const bool have = base + lane < e && (!tc_cell || v.core[base + lane] == 2);
        unsigned open = __ballot_sync(0xffffffffu, have);
        if (!open) continue;
        const GridParams &G = params_of(v, set_of_key(v, v.cell_key[A]));
        const uint32_t min_pts = G.min_pts;
        stage_rows<T, DP>(rows, v.pts, base, e);
        uint32_t cnt = 0, skip = 0;
        if (tc_cell) {  // resume where the tensor-core count stopped (same candidate order)
            if (have) cnt = v.tc_cnt[base + lane];
            skip = __shfl_sync(0xffffffffu, have ? v.tc_pos[base + lane] : 0u, __ffs(open) - 1);
        }
        for (int g0 = 0; g0 < v.n_all && open; g0 += 32) {
            const int k = g0 + lane;
            const uint2 rg = k < v.n_all ? v.ranges[(uint64_t)A * v.n_all + k] : make_uint2(0u, 0u);
            // the cells of a pencil range, one at a time: a cell whose box is farther than eps
            // from every open row adds nothing to their counts and is passed over
            for (int kk = 0; kk < 32 && open; ++kk) {
                const uint32_t lo = __shfl_sync(0xffffffffu, rg.x, kk);
                const uint32_t hi = __shfl_sync(0xffffffffu, rg.y, kk);
                for (uint32_t B = lo; B < hi && open; ++B) {
                    uint32_t q0 = v.cell_start[B];
                    const uint32_t q1 = v.cell_start[B + 1];
                    if (skip) {  // positions count every point of the stream (the tensor-core order)
                        if (skip >= q1 - q0) {
                            skip -= q1 - q0;
                            continue;
                        }
                        q0 += skip;
                        skip = 0;
                    }
                    const unsigned near = open & __ballot_sync(0xffffffffu,
                        !box_far<DP>(rows + lane * DP, v.box_lo + (uint64_t)B * DP, v.box_hi + (uint64_t)B * DP, G));
                    if (!near) continue;
                    for (uint32_t qb = q0; qb < q1 && open; qb += 32) {
                        const uint32_t q = qb + lane;
                        T qv[DP];
                        hd_load<T, DP>(v.pts, q, q < q1, qv);
                        ++chunks;
                        unsigned rem = open & near;
                        while (rem) {
                            const int jj = __ffs(rem) - 1;
                            rem &= rem - 1;
                            const unsigned hits = __ballot_sync(0xffffffffu, q < q1 && hd_within<DP>(rows + jj * DP, qv, G));
                            if (lane == jj) cnt += __popc(hits);
                        }
                        open &= __ballot_sync(0xffffffffu, have && cnt < min_pts);
                    }
                }
            }
        }
        const bool is_core = have && cnt >= min_pts;
        if (have) v.core[base + lane] = is_core ? 1 : 0;
        if (__any_sync(0xffffffffu, is_core) && lane == 0) v.cell_core[A] = 1;
        __syncwarp();
    }
    add_counter(&v.ctr->work[0], lane == 0 ? chunks : 0u);
}

// Union-find over points: parent[j] = j for every point.
template <typename T, int DP>
__global__ void __launch_bounds__(256) k_uf_init_hd(HdView<T, DP> v) {
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < v.g.n; j += (int64_t)gridDim.x * blockDim.x) {
        v.parent[j] = (uint32_t)j;
        v.comp_min[j] = kNoLabel;
    }
}

// First links of the core graph (Definitions 3-5): every core point p hooks to the first core
// point q < p within eps that the scan meets (p keeps itself when there is none).  Each link
// is an edge of the graph and points to a smaller index, so the links form a forest whose
// trees lie inside clusters; the union pass that follows joins the trees.  The links only
// shorten that pass (it tests every pair itself), so a chunk stops looking after
// kHookBlocks candidate blocks: a point with no lower neighbour (the first point of every
// cluster) would otherwise make its warp read the whole lower half of its neighbourhood.
constexpr uint32_t kHookBlocks = 16;
template <typename T, int DP>
__global__ void __launch_bounds__(32 * kHdMaxWarps) k_hook_hd(HdView<T, DP> v) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *rows = reinterpret_cast<T *>(smem_raw) + (threadIdx.x >> 5) * 32 * DP;
    const int lane = lane_id();
    uint32_t chunks = 0;
    HD_FOR_EACH_CHUNK(v, A, base, e, 1) {
        if (v.tc_min[1] && !v.tc_hook && v.cx[e] - v.cx[v.cell_start[A]] >= v.tc_min[1]) continue;
        const uint32_t p = base + lane;
        unsigned open = __ballot_sync(0xffffffffu, p < e && v.core[p]);
        if (!open) continue;
        const GridParams &G = params_of(v, set_of_key(v, v.cell_key[A]));
        stage_rows<T, DP>(rows, v.pts, base, e);
        uint32_t chunks_here = 0;
        for (int g0 = 0; g0 < v.n_all && open; g0 += 32) {
            const int k = g0 + lane;
            const uint2 rg = k < v.n_all ? v.ranges[(uint64_t)A * v.n_all + k] : make_uint2(0u, 0u);
            for (int kk = 0; kk < 32 && open; ++kk) {
                const uint32_t lo = __shfl_sync(0xffffffffu, rg.x, kk);
                const uint32_t hi = __shfl_sync(0xffffffffu, rg.y, kk);
                if (lo >= hi) continue;
                const uint32_t q0 = v.cell_start[lo];
                const uint32_t q1 = min(v.cell_start[hi], base + 31u);  // only q < p can link
                for (uint32_t qb = q0; qb < q1 && open; qb += 32) {
                    const uint32_t q = qb + lane;
                    const bool qc = q < q1 && v.core[q];
                    if (!__any_sync(0xffffffffu, qc)) continue;
                    if (++chunks_here > kHookBlocks) {
                        open = 0;
                        break;
                    }
                    T qv[DP];
                    hd_load<T, DP>(v.pts, q, qc, qv);
                    ++chunks;
                    unsigned rem = open;
                    while (rem) {
                        const int jj = __ffs(rem) - 1;
                        rem &= rem - 1;
                        const bool hit = qc && q < base + jj && hd_within<DP>(rows + jj * DP, qv, G);
                        const unsigned hm = __ballot_sync(0xffffffffu, hit);
                        if (hm) {
                            if (lane == jj) v.parent[base + jj] = qb + (uint32_t)(__ffs(hm) - 1);
                            open &= ~(1u << jj);
                        }
                    }
                }
            }
        }
        __syncwarp();
    }
    add_counter(&v.ctr->work[1], lane == 0 ? chunks : 0u);
}

// One round of pointer jumping over core points: parent[p] = parent[parent[p]].
template <typename T, int DP>
__global__ void __launch_bounds__(256) k_jump_hd(HdView<T, DP> v) {
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < v.g.n; j += (int64_t)gridDim.x * blockDim.x) {
        if (!v.core[j]) continue;
        const uint32_t p = __ldcg(v.parent + j);
        const uint32_t gp = __ldcg(v.parent + p);
        if (gp != p) v.parent[j] = gp;
    }
}

// Definitions 3-5, remaining edges: every pair of core points within eps of the upper half of
// the neighbourhood (the own pencil from this chunk on) whose trees differ is joined
// (lock-free union-find, root = smallest index).  A 32 x 32 tile whose core points all share
// one root is skipped without loading coordinates.
template <typename T, int DP>
__global__ void __launch_bounds__(32 * kHdMaxWarps) k_merge_hd(HdView<T, DP> v) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *rows = reinterpret_cast<T *>(smem_raw) + (threadIdx.x >> 5) * 32 * DP;
    const int lane = lane_id();
    uint32_t chunks = 0, tests = 0, skipped = 0;
    HD_FOR_EACH_CHUNK(v, A, base, e, 2) {
        if (!v.cell_core[A]) continue;
        if (v.tc_min[1] && v.cx[e] - v.cx[v.cell_start[A]] >= v.tc_min[1]) continue;  // tensor-core cell
        const uint32_t p = base + lane;
        const bool pc = p < e && v.core[p];
        const unsigned amask = __ballot_sync(0xffffffffu, pc);
        if (!amask) continue;
        const GridParams &G = params_of(v, set_of_key(v, v.cell_key[A]));
        stage_rows<T, DP>(rows, v.pts, base, e);
        uint32_t rp = pc ? uf_find(v.parent, p, v.ctr) : 0xffffffffu;
        for (int g0 = 0; g0 < v.n_half; g0 += 32) {
            const int k = g0 + lane;
            uint2 rg = k < v.n_half ? v.ranges[(uint64_t)A * v.n_all + k] : make_uint2(0u, 0u);
            if (k == 0) rg.x = A;  // own pencil: this cell and the ones after it
            for (int kk = 0; kk < 32; ++kk) {
                const uint32_t lo = __shfl_sync(0xffffffffu, rg.x, kk);
                const uint32_t hi = __shfl_sync(0xffffffffu, rg.y, kk);
                if (lo >= hi) continue;
                // own pencil: start at this chunk (earlier points pair with it from their side)
                const uint32_t q0 = (g0 + kk == 0) ? max(v.cell_start[lo], base) : v.cell_start[lo];
                const uint32_t q1 = v.cell_start[hi];
                for (uint32_t qb = q0; qb < q1; qb += 32) {
                    const uint32_t q = qb + lane;
                    const bool qc = q < q1 && v.core[q];
                    if (!__any_sync(0xffffffffu, qc)) continue;
                    uint32_t rq = qc ? uf_find(v.parent, q, v.ctr) : 0xfffffffeu;
                    const uint32_t r0 = __shfl_sync(0xffffffffu, rp, __ffs(amask) - 1);
                    if (__all_sync(0xffffffffu, (!pc || rp == r0) && (!qc || rq == r0))) {
                        ++skipped;
                        continue;
                    }
                    T qv[DP];
                    hd_load<T, DP>(v.pts, q, qc, qv);
                    ++chunks;
                    unsigned rem = amask;
                    while (rem) {
                        const int jj = __ffs(rem) - 1;
                        rem &= rem - 1;
                        const uint32_t pj = base + jj;
                        const uint32_t rj = __shfl_sync(0xffffffffu, rp, jj);
                        const bool need = qc && q > pj && rq != rj;
                        if (!__any_sync(0xffffffffu, need)) continue;
                        ++tests;
                        const bool hit = need && hd_within<DP>(rows + jj * DP, qv, G);
                        if (hit) uf_union(v.parent, pj, q, v.ctr);
                        if (__any_sync(0xffffffffu, hit)) {
                            // roots moved: refresh every lane so later pairs of the tile skip
                            rq = qc ? uf_find(v.parent, q, v.ctr) : 0xfffffffeu;
                            rp = pc ? uf_find(v.parent, p, v.ctr) : 0xffffffffu;
                        }
                    }
                }
            }
        }
        __syncwarp();
    }
    add_counter(&v.ctr->work[4], lane == 0 ? chunks : 0u);
    add_counter(&v.ctr->work[3], lane == 0 ? tests : 0u);
    add_counter(&v.ctr->work[2], lane == 0 ? skipped : 0u);
}

// Flatten the point union-find (read-only finds), count roots, canonical ids.
template <typename T, int DP>
__global__ void __launch_bounds__(256) k_compress_hd(HdView<T, DP> v) {
    uint32_t roots = 0;
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < v.g.n; j += (int64_t)gridDim.x * blockDim.x) {
        if (!v.core[j]) continue;
        const uint32_t r = uf_root_readonly(v.parent, (uint32_t)j, v.ctr);
        v.parent[j] = r;
        roots += (r == (uint32_t)j);
    }
    roots = __reduce_add_sync(0xffffffffu, roots);
    if (lane_id() == 0 && roots) atomicAdd(&v.ctr->n_clusters, roots);
}

template <typename T, int DP>
__global__ void __launch_bounds__(256) k_comp_min_hd(HdView<T, DP> v) {
    const int64_t n = v.g.n;
    const int lane = lane_id();
    uint32_t ncore = 0;
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31); base < n;
         base += (int64_t)gridDim.x * blockDim.x) {
        const int64_t j = base + lane;
        const bool valid = j < n && v.core[j];
        const uint32_t r = valid ? v.parent[j] : 0xffffffffu;
        uint32_t val = valid ? v.perm[j] : kNoLabel;
        const unsigned vm = __ballot_sync(0xffffffffu, valid);
        if (!vm) continue;
        ncore += (lane == 0) ? __popc(vm) : 0u;
        const uint32_t r0 = __shfl_sync(0xffffffffu, r, __ffs(vm) - 1);
        if (__all_sync(0xffffffffu, !valid || r == r0)) {
            val = __reduce_min_sync(0xffffffffu, val);
            if (lane == 0) atomicMin(&v.comp_min[r0], val);
        } else if (valid) {
            atomicMin(&v.comp_min[r], val);
        }
    }
    if (lane == 0 && ncore) atomicAdd(&v.ctr->n_core, ncore);
}

// Algorithm 4 / Definition 5 with the canonical rule, over points: core points take their
// cluster id, a non-core point the smallest id among its core neighbours, else -1.
template <typename T, int DP>
__global__ void __launch_bounds__(32 * kHdMaxWarps) k_labels_hd(HdView<T, DP> v) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *rows = reinterpret_cast<T *>(smem_raw) + (threadIdx.x >> 5) * 32 * DP;
    const int lane = lane_id();
    uint32_t noise = 0, chunks = 0;
    HD_FOR_EACH_CHUNK(v, A, base, e, 3) {
        if (v.tc_min[2]) {  // non-core rows of a tensor-core cell: labelled there
            const uint32_t s0 = v.cell_start[A];
            if (e - s0 - (v.cx[e] - v.cx[s0]) >= v.tc_min[2]) continue;
        }
        {
            const uint32_t aset = set_of_key(v, v.cell_key[A]);
            const GridParams &G = params_of(v, aset);
            const uint32_t base_label = v.gtab ? (uint32_t)v.set_off[aset] : 0u;
            const uint32_t p = base + lane;
            const bool have = p < e;
            const bool isc = have && v.core[p];
            uint32_t best = isc ? v.comp_min[v.parent[p]] : kNoLabel;
            const unsigned smask = __ballot_sync(0xffffffffu, have && !isc);
            if (smask) {
                stage_rows<T, DP>(rows, v.pts, base, e);
                for (int g0 = 0; g0 < v.n_all; g0 += 32) {
                    const int k = g0 + lane;
                    const uint2 rg = k < v.n_all ? v.ranges[(uint64_t)A * v.n_all + k] : make_uint2(0u, 0u);
                    for (int kk = 0; kk < 32; ++kk) {
                        const uint32_t lo = __shfl_sync(0xffffffffu, rg.x, kk);
                        const uint32_t hi = __shfl_sync(0xffffffffu, rg.y, kk);
                        for (uint32_t B = lo; B < hi; ++B) {
                            // a cell whose box is farther than eps from every row is passed over
                            const unsigned near = smask & __ballot_sync(0xffffffffu,
                                !box_far<DP>(rows + lane * DP, v.box_lo + (uint64_t)B * DP,
                                             v.box_hi + (uint64_t)B * DP, G));
                            if (!near) continue;
                            const uint32_t q0 = v.cell_start[B], q1 = v.cell_start[B + 1];
                            for (uint32_t qb = q0; qb < q1; qb += 32) {
                                const uint32_t q = qb + lane;
                                const bool qc = q < q1 && v.core[q];
                                if (!__any_sync(0xffffffffu, qc)) continue;
                                const uint32_t lq = qc ? v.comp_min[v.parent[q]] : kNoLabel;
                                T qv[DP];
                                hd_load<T, DP>(v.pts, q, qc, qv);
                                ++chunks;
                                unsigned rem = near;
                                while (rem) {
                                    const int jj = __ffs(rem) - 1;
                                    rem &= rem - 1;
                                    const uint32_t bj = __shfl_sync(0xffffffffu, best, jj);
                                    const bool need = qc && lq < bj;
                                    if (!__any_sync(0xffffffffu, need)) continue;
                                    uint32_t cand = (need && hd_within<DP>(rows + jj * DP, qv, G)) ? lq : kNoLabel;
                                    cand = __reduce_min_sync(0xffffffffu, cand);
                                    if (lane == jj && cand < best) best = cand;
                                }
                            }
                        }
                    }
                }
                __syncwarp();
            }
            if (have) {
                const int32_t lab = best == kNoLabel ? -1 : (int32_t)(best - base_label);
                const uint32_t o = v.perm[p];
                v.labels[o] = lab;
                if (v.core_out) v.core_out[o] = isc ? 1 : 0;
                noise += lab < 0;
            }
        }
    }
    noise = __reduce_add_sync(0xffffffffu, noise);
    if (lane == 0 && noise) atomicAdd(&v.ctr->n_noise, noise);
    add_counter(&v.ctr->work[5], lane == 0 ? chunks : 0u);
}


// Batched calls: per-set min / max of every dimension (mm[set * 64 + i] min encodings,
// mm[(nsets + set) * 64 + i] max encodings), by seg_minmax.
template <typename T>
__global__ void __launch_bounds__(256) k_minmax_rt_seg(const T *__restrict__ in, int64_t n, int d,
                                                      const int64_t *set_off, int nsets,
                                                      unsigned long long *mm, DevCounters *ctr) {
    seg_minmax<T>(in, n, d, set_off, nsets, mm, 64, ctr);
}

// Batched calls: coarse cell keys with the set id above them; each set projects on its own
// three dimensions (GridParams::sel).
template <typename T, typename K>
__global__ void __launch_bounds__(256) k_bin_proj_seg(const T *__restrict__ in, int64_t n, int d,
                                                     const int64_t *set_off, int nsets, const GridParams *gtab,
                                                     int key_bits, K *__restrict__ keys, uint32_t *__restrict__ idx) {
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n;
         j += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t set = set_of_point(set_off, nsets, j);
        const GridParams &g = gtab[set];
        uint64_t key = (uint64_t)set << key_bits;
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            const double t = __dmul_rn(__dsub_rn((double)in[j * d + g.sel[i]], g.origin[i]), g.inv_side);
            uint32_t c = (uint32_t)floor(t);
            if (c > g.ncell[i] - 1) c = g.ncell[i] - 1;
            key |= (uint64_t)c << g.shift[i];
        }
        keys[j] = (K)key;
        idx[j] = (uint32_t)j;
    }
}

}  // namespace hca
