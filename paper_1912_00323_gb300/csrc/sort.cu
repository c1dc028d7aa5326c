// LSD radix sort of (key, uint32 value) pairs, 8 bits per pass, one kernel per pass.
//
// A first kernel counts the digits of every pass over all keys (the counts do not depend on
// the order, so one read of the keys serves all passes); a caller that produced the keys may
// pass these counts in instead.  Each pass kernel then takes a tile
// of 4096 keys, ranks every key stably among the keys of its tile with the same digit (warp
// match + per-warp digit counters + an exclusive scan across warps), learns how many keys of
// each digit the earlier tiles hold by decoupled look-back, and scatters the tile through
// shared memory in digit order so that the global stores of each digit run are coalesced.
//
// Look-back: a tile publishes, per digit, first its own count (state AGG) and then the count of
// all tiles up to and including itself (state PREFIX).  A tile reads its predecessors'
// words from the nearest one backwards, adding AGG values until it meets a PREFIX.  Tiles take
// their index from an atomic ticket in the order they start, so a tile only ever waits on
// tiles that are already running; every wait is bounded (kSpinLimit), and a wait that runs
// out sets the caller's status word instead of hanging.  Each status word packs
// (epoch, state, count) into 64 bits so flag and value are read and written together; the
// epoch (pass number + 1) makes words left by an earlier pass invisible.
#include "block_scan.cuh"
#include "hca_internal.cuh"

namespace hca {

namespace {

constexpr int kSortThreads = 256;
constexpr int kSortWarps = kSortThreads / 32;
constexpr int kSortItems = 16;  // per lane: a warp covers 512 consecutive keys
constexpr int kSortTile = kSortThreads * kSortItems;
constexpr int kRadix = kSortRadix;
constexpr int kMaxPasses = kSortMaxPasses;
static_assert(kSortTile == kSortTileKeys, "tile size shared with the scratch sizing");
constexpr uint32_t kSpinLimit = 1u << 24;
constexpr uint64_t kStateAgg = 1, kStatePrefix = 2;

__device__ __forceinline__ uint64_t os_pack(uint32_t epoch, uint64_t state, uint32_t value) {
    return ((uint64_t)(epoch * 4u + (uint32_t)state) << 32) | value;
}

// Digit counts of every pass: ghist[p * 256 + digit].
template <typename K>
__global__ void __launch_bounds__(kSortThreads) k_os_hist(const K *__restrict__ keys, int64_t n, int begin_bit,
                                                         int end_bit, uint32_t *__restrict__ ghist) {
    __shared__ uint32_t h[kMaxPasses][kRadix];
    for (int i = threadIdx.x; i < kMaxPasses * kRadix; i += kSortThreads) (&h[0][0])[i] = 0;
    __syncthreads();
    const int passes = (end_bit - begin_bit + 7) / 8;
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < n; base += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = base + threadIdx.x;
        const bool valid = i < n;
        const K key = valid ? keys[i] : K(0);
        if (valid) {
            for (int p = 0; p < passes; ++p) {
                const int shift = begin_bit + 8 * p;
                const int bits = min(8, end_bit - shift);
                atomicAdd(&h[p][(uint32_t)(key >> shift) & ((1u << bits) - 1u)], 1u);
            }
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < passes * kRadix; i += kSortThreads) {
        const uint32_t c = (&h[0][0])[i];
        if (c) atomicAdd(&ghist[i], c);
    }
}

// One pass: rank, look back, scatter.
template <typename K>
__global__ void __launch_bounds__(kSortThreads) k_os_pass(
    const K *__restrict__ keys_in, const uint32_t *__restrict__ vals_in, K *__restrict__ keys_out,
    uint32_t *__restrict__ vals_out, int64_t n, int shift, int mask_bits,
    const uint32_t *__restrict__ ghist_pass, unsigned long long *status, uint32_t *ticket, uint32_t epoch,
    uint32_t *err) {
    extern __shared__ __align__(16) unsigned char sm[];
    uint32_t(*whist)[kRadix] = reinterpret_cast<uint32_t(*)[kRadix]>(sm);  // [warps][digits]
    uint32_t *lstart = reinterpret_cast<uint32_t *>(sm) + kSortWarps * kRadix;
    uint32_t *goff = lstart + kRadix;
    uint32_t *tile_id = goff + kRadix;
    K *skeys = reinterpret_cast<K *>(tile_id + 4);
    uint32_t *svals = reinterpret_cast<uint32_t *>(skeys + kSortTile);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t mask = (1u << mask_bits) - 1u;
    for (int i = threadIdx.x; i < kSortWarps * kRadix; i += kSortThreads) (&whist[0][0])[i] = 0;
    if (threadIdx.x == 0) tile_id[0] = atomicAdd(ticket, 1u);
    __syncthreads();
    const uint32_t tile = tile_id[0];

    const int64_t tbase = (int64_t)tile * kSortTile;
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
    const int dg = threadIdx.x;  // kSortThreads == kRadix: one thread per digit
    uint32_t count = 0;
#pragma unroll
    for (int w = 0; w < kSortWarps; ++w) {
        const uint32_t t = whist[w][dg];
        whist[w][dg] = count;
        count += t;
    }
    // decoupled look-back over the earlier tiles, per digit
    volatile unsigned long long *st = status;
    uint32_t excl = 0;
    if (tile == 0) {
        st[dg] = os_pack(epoch, kStatePrefix, count);
    } else {
        st[(uint64_t)tile * kRadix + dg] = os_pack(epoch, kStateAgg, count);
        // read eight predecessors per round trip, nearest first; stop at the first PREFIX, and
        // re-read from the first word that is not published yet
        int64_t j = (int64_t)tile - 1;
        uint32_t spins = 0;
        bool done = false;
        while (!done && j >= 0) {
            uint64_t w[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) w[u] = (j - u >= 0) ? st[(uint64_t)(j - u) * kRadix + dg] : 0ull;
            int u = 0;
            for (; u < 8 && j - u >= 0; ++u) {
                const uint32_t hi = (uint32_t)(w[u] >> 32);
                if ((hi >> 2) != epoch || (hi & 3u) == 0u) break;   // not published yet
                excl += (uint32_t)w[u];
                if ((hi & 3u) == kStatePrefix) { done = true; break; }
            }
            if (done) break;
            if (u < 8 && j - u >= 0) {                               // wait on tile j - u
                if (++spins > kSpinLimit) {
                    atomicOr(err, 2u);
                    break;
                }
            }
            j -= u;
        }
        st[(uint64_t)tile * kRadix + dg] = os_pack(epoch, kStatePrefix, excl + count);
    }
    // global start of this digit: exclusive scan of the pass's digit counts
    uint32_t total_unused;
    const uint32_t gdig = block_exclusive_scan<kSortThreads>(ghist_pass[dg], &total_unused);
    goff[dg] = gdig + excl;
    uint32_t tile_count;
    lstart[dg] = block_exclusive_scan<kSortThreads>(count, &tile_count);
    __syncthreads();
#pragma unroll
    for (int r = 0; r < kSortItems; ++r) {
        const int64_t i = wbase + r * 32 + lane;
        if (i < n) {
            const uint32_t d = (uint32_t)(k[r] >> shift) & mask;
            const uint32_t lpos = lstart[d] + whist[warp][d] + rank[r];
            skeys[lpos] = k[r];
            svals[lpos] = v[r];
        }
    }
    __syncthreads();
    for (uint32_t i = threadIdx.x; i < tile_count; i += kSortThreads) {
        const K key = skeys[i];
        const uint32_t d = (uint32_t)(key >> shift) & mask;
        const uint32_t gpos = goff[d] + (i - lstart[d]);
        keys_out[gpos] = key;
        vals_out[gpos] = svals[i];
    }
}

template <typename K>
constexpr size_t pass_smem() {
    return sizeof(uint32_t) * (kSortWarps * kRadix + 2 * kRadix + 4) + (sizeof(K) + sizeof(uint32_t)) * kSortTile;
}

int64_t sort_tiles(int64_t n) { return sort_tiles_for(n); }

}  // namespace

uint32_t *sort_status_word(uint32_t *hist, int64_t n) {
    return hist + 2 * sort_tiles(n) * kRadix + kMaxPasses * kRadix + kMaxPasses;
}

template <typename K>
bool radix_sort_pairs(K *keys, uint32_t *vals, K *keys_alt, uint32_t *vals_alt, int64_t n,
                      int begin_bit, int end_bit, uint32_t *hist, uint32_t *partials,
                      cudaStream_t s, int *launches, uint32_t *err_out, const uint32_t *digit_counts) {
    (void)partials;
    if (n <= 1 || end_bit <= begin_bit) return false;
    static_assert(kSortThreads == kRadix, "one thread per digit in the pass kernel");
    const int nb = (int)sort_tiles(n);
    const int passes = (end_bit - begin_bit + 7) / 8;
    unsigned long long *status = reinterpret_cast<unsigned long long *>(hist);  // 8-byte aligned
    uint32_t *ghist = hist + 2 * (size_t)nb * kRadix;
    uint32_t *tickets = ghist + kMaxPasses * kRadix;
    uint32_t *err = err_out ? err_out : sort_status_word(hist, n);
    cudaMemsetAsync(hist, 0, sizeof(uint32_t) * sort_hist_size(n), s);
    if (digit_counts) {
        ghist = const_cast<uint32_t *>(digit_counts);
    } else {
        k_os_hist<K><<<nb < 1216 ? nb : 1216, kSortThreads, 0, s>>>(keys, n, begin_bit, end_bit, ghist);
        if (launches) *launches += 1;
    }
    if (pass_smem<K>() > 48 * 1024)
        cudaFuncSetAttribute(k_os_pass<K>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)pass_smem<K>());
    bool flipped = false;
    K *kin = keys, *kout = keys_alt;
    uint32_t *vin = vals, *vout = vals_alt;
    for (int p = 0; p < passes; ++p) {
        const int shift = begin_bit + 8 * p;
        const int bits = (end_bit - shift) < 8 ? (end_bit - shift) : 8;
        k_os_pass<K><<<nb, kSortThreads, pass_smem<K>(), s>>>(kin, vin, kout, vout, n, shift, bits,
                                                              ghist + p * kRadix, status, tickets + p,
                                                              (uint32_t)(p + 1), err);
        K *tk = kin; kin = kout; kout = tk;
        uint32_t *tv = vin; vin = vout; vout = tv;
        flipped = !flipped;
    }
    if (launches) *launches += passes;
    return flipped;
}

template bool radix_sort_pairs<uint32_t>(uint32_t *, uint32_t *, uint32_t *, uint32_t *, int64_t,
                                         int, int, uint32_t *, uint32_t *, cudaStream_t, int *, uint32_t *,
                                         const uint32_t *);
template bool radix_sort_pairs<uint64_t>(uint64_t *, uint32_t *, uint64_t *, uint32_t *, int64_t,
                                         int, int, uint32_t *, uint32_t *, cudaStream_t, int *, uint32_t *,
                                         const uint32_t *);

}  // namespace hca
