// LSD radix sort of (key, uint32 value) pairs, 8 bits per pass.
//
// Each pass: (1) every block counts the digits of its tile of 2048 keys into a per-block
// histogram, stored digit-major; (2) an exclusive scan of that array gives every
// (digit, block) its first output position; (3) every block re-reads its tile, ranks each
// key stably among the keys of its tile with the same digit (warp match + per-warp digit
// counters, then an exclusive scan across warps), and scatters.  Stability across passes
// makes the result a stable sort by the whole bit range.
#include "block_scan.cuh"
#include "hca_internal.cuh"

namespace hca {

namespace {

constexpr int kSortThreads = 256;
constexpr int kSortWarps = kSortThreads / 32;
constexpr int kSortItems = 8;   // per lane: a warp covers 256 consecutive keys
constexpr int kSortTile = kSortThreads * kSortItems;
constexpr int kRadix = 256;

template <typename K>
__global__ void __launch_bounds__(kSortThreads) k_sort_hist(const K *__restrict__ keys, int64_t n,
                                                            int shift, int mask_bits,
                                                            uint32_t *__restrict__ hist, int nb) {
    __shared__ uint32_t h[kRadix];
    for (int i = threadIdx.x; i < kRadix; i += kSortThreads) h[i] = 0;
    __syncthreads();
    const uint32_t mask = (1u << mask_bits) - 1u;
    const int64_t base = (int64_t)blockIdx.x * kSortTile;
#pragma unroll 4
    for (int k = 0; k < kSortItems; ++k) {
        const int64_t i = base + (int64_t)k * kSortThreads + threadIdx.x;
        const bool valid = i < n;
        const uint32_t dg = valid ? ((uint32_t)(keys[i] >> shift) & mask) : (uint32_t)kRadix;
        // aggregate equal digits of the warp into one shared-memory atomic
        const unsigned peers = __match_any_sync(0xffffffffu, dg);
        if (valid && (threadIdx.x & 31) == __ffs(peers) - 1) atomicAdd(&h[dg], __popc(peers));
    }
    __syncthreads();
    for (int i = threadIdx.x; i < kRadix; i += kSortThreads) hist[(int64_t)i * nb + blockIdx.x] = h[i];
}

// Scatter of one pass.  Keys are ranked stably inside the tile, written to shared memory in
// digit order, and then copied out so that consecutive threads write consecutive positions of
// each digit's output run (coalesced stores).
template <typename K>
__global__ void __launch_bounds__(kSortThreads) k_sort_scatter(
    const K *__restrict__ keys_in, const uint32_t *__restrict__ vals_in, K *__restrict__ keys_out,
    uint32_t *__restrict__ vals_out, int64_t n, int shift, int mask_bits,
    const uint32_t *__restrict__ offsets, int nb) {
    extern __shared__ __align__(16) unsigned char sm[];
    uint32_t(*whist)[kRadix] = reinterpret_cast<uint32_t(*)[kRadix]>(sm);  // [warps][digits]
    uint32_t *lstart = reinterpret_cast<uint32_t *>(sm) + kSortWarps * kRadix;
    uint32_t *goff = lstart + kRadix;
    K *skeys = reinterpret_cast<K *>(goff + kRadix);
    uint32_t *svals = reinterpret_cast<uint32_t *>(skeys + kSortTile);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t mask = (1u << mask_bits) - 1u;
    for (int i = threadIdx.x; i < kSortWarps * kRadix; i += kSortThreads) (&whist[0][0])[i] = 0;
    __syncthreads();

    const int64_t tbase = (int64_t)blockIdx.x * kSortTile;
    const int64_t wbase = tbase + (int64_t)warp * (32 * kSortItems);
    K k[kSortItems];
    uint32_t v[kSortItems];
    uint32_t rank[kSortItems];
#pragma unroll
    for (int r = 0; r < kSortItems; ++r) {
        const int64_t i = wbase + r * 32 + lane;
        const bool valid = i < n;
        k[r] = valid ? keys_in[i] : K(0);
        v[r] = valid ? vals_in[i] : 0u;
        const uint32_t dg = valid ? ((uint32_t)(k[r] >> shift) & mask) : (uint32_t)kRadix;
        const unsigned peers = __match_any_sync(0xffffffffu, dg);
        const uint32_t before = valid ? whist[warp][dg] : 0u;
        __syncwarp();
        if (valid && lane == __ffs(peers) - 1) whist[warp][dg] = before + __popc(peers);
        __syncwarp();
        rank[r] = before + __popc(peers & ((1u << lane) - 1u));
    }
    __syncthreads();
    // per digit: exclusive prefix across warps, the tile's count, and the global offset
    uint32_t total = 0;
    {
        const int dg = threadIdx.x;  // kSortThreads == kRadix
#pragma unroll
        for (int w = 0; w < kSortWarps; ++w) {
            const uint32_t t = whist[w][dg];
            whist[w][dg] = total;
            total += t;
        }
        goff[dg] = offsets[(int64_t)dg * nb + blockIdx.x];
    }
    uint32_t tile_count;
    const uint32_t ls = block_exclusive_scan<kSortThreads>(total, &tile_count);
    lstart[threadIdx.x] = ls;
    __syncthreads();
#pragma unroll
    for (int r = 0; r < kSortItems; ++r) {
        const int64_t i = wbase + r * 32 + lane;
        if (i < n) {
            const uint32_t dg = (uint32_t)(k[r] >> shift) & mask;
            const uint32_t lpos = lstart[dg] + whist[warp][dg] + rank[r];
            skeys[lpos] = k[r];
            svals[lpos] = v[r];
        }
    }
    __syncthreads();
    for (uint32_t i = threadIdx.x; i < tile_count; i += kSortThreads) {
        const K key = skeys[i];
        const uint32_t dg = (uint32_t)(key >> shift) & mask;
        const uint32_t gpos = goff[dg] + (i - lstart[dg]);
        keys_out[gpos] = key;
        vals_out[gpos] = svals[i];
    }
}

template <typename K>
constexpr size_t scatter_smem() {
    return sizeof(uint32_t) * (kSortWarps * kRadix + 2 * kRadix) + (sizeof(K) + sizeof(uint32_t)) * kSortTile;
}

}  // namespace

size_t sort_hist_size(int64_t n) {
    int64_t nb = (n + kSortTile - 1) / kSortTile;
    if (nb < 1) nb = 1;
    return (size_t)(nb * kRadix);
}

template <typename K>
bool radix_sort_pairs(K *keys, uint32_t *vals, K *keys_alt, uint32_t *vals_alt, int64_t n,
                      int begin_bit, int end_bit, uint32_t *hist, uint32_t *partials,
                      cudaStream_t s, int *launches) {
    if (n <= 1 || end_bit <= begin_bit) return false;
    const int nb = (int)((n + kSortTile - 1) / kSortTile);
    static_assert(kSortThreads == kRadix, "one thread per digit in the scatter's digit scan");
    if (scatter_smem<K>() > 48 * 1024)
        cudaFuncSetAttribute(k_sort_scatter<K>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)scatter_smem<K>());
    bool flipped = false;
    K *kin = keys, *kout = keys_alt;
    uint32_t *vin = vals, *vout = vals_alt;
    for (int shift = begin_bit; shift < end_bit; shift += 8) {
        const int bits = (end_bit - shift) < 8 ? (end_bit - shift) : 8;
        k_sort_hist<K><<<nb, kSortThreads, 0, s>>>(kin, n, shift, bits, hist, nb);
        exclusive_scan_u32(hist, hist, (int64_t)nb * kRadix, nullptr, nullptr, partials, s, launches);
        k_sort_scatter<K><<<nb, kSortThreads, scatter_smem<K>(), s>>>(kin, vin, kout, vout, n, shift, bits, hist, nb);
        if (launches) *launches += 2;
        K *tk = kin; kin = kout; kout = tk;
        uint32_t *tv = vin; vin = vout; vout = tv;
        flipped = !flipped;
    }
    return flipped;
}

template bool radix_sort_pairs<uint32_t>(uint32_t *, uint32_t *, uint32_t *, uint32_t *, int64_t,
                                         int, int, uint32_t *, uint32_t *, cudaStream_t, int *);
template bool radix_sort_pairs<uint64_t>(uint64_t *, uint32_t *, uint64_t *, uint32_t *, int64_t,
                                         int, int, uint32_t *, uint32_t *, cudaStream_t, int *);

}  // namespace hca
