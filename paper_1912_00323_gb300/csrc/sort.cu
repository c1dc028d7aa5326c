// LSD radix sort of (key, uint32 value) pairs, 8 bits per pass, one kernel per pass.
//
// A first kernel counts the digits of every pass over all keys (the counts do not depend on
// the order, so one read of the keys serves all passes); a caller that produced the keys may
// pass these counts in instead.  Each pass kernel then takes a tile of 13,312 keys (1024
// threads x 13), ranks every key stably among the keys of its tile with the same digit (the
// lanes of a warp with one digit found by a match instruction or by shared-memory OR masks,
// per-warp digit counters, an exclusive scan across warps), publishes the tile's digit
// counts, scatters the tile through shared memory in digit order, learns how many keys of each
// digit the earlier tiles hold by decoupled look-back, and writes the digit runs out with
// coalesced stores.
//
// Tile size.  A tile is one CTA per SM (its shared memory holds the whole tile), so at two
// million keys the ~150 tiles all run at once.  With every tile running together a published
// prefix reaches the later tiles only through their own reads, so the look-back reads 64
// predecessors per round trip (four thread quarters of 16 words per digit): the last tile of
// two million keys needs three round trips instead of the dozens that a 4096-key tile with a
// few words per trip needed.
//
// Up to kFullSumTiles tiles (about 3.4 million keys) a tile instead sums the published counts
// of all earlier tiles (eight loads in flight per thread, no prefix published): with every
// tile running at once no prefix would be there to shorten the look-back anyway.
//
// Look-back: a tile publishes, per digit, first its own count (state AGG) and then the count of
// all tiles up to and including itself (state PREFIX).  A tile reads its predecessors'
// words from the nearest one backwards, adding AGG values until it meets a PREFIX.  Tiles take
// their index from an atomic ticket in the order they start, so a tile only ever waits on
// tiles that are already running; every wait is bounded (kSpinLimit), and a wait that runs
// out sets the caller's status word instead of hanging.  Each status word packs
// (epoch, state, count) into 64 bits so flag and value are read and written together; the
// epoch (pass number + 1) makes words left by an earlier pass invisible.  Words are tile-major
// (the 256 digits of one tile are consecutive), so a warp reads 32 digits of a tile in one
// coalesced 256-byte access.
#include "block_scan.cuh"
#include "hca_internal.cuh"

namespace hca {

namespace {

constexpr int kSortThreads = 1024;
constexpr int kSortWarps = kSortThreads / 32;
constexpr int kSortItems = 13;  // per lane: a warp covers 416 consecutive keys
constexpr int kSortTile = kSortThreads * kSortItems;
constexpr int kRadix = kSortRadix;
constexpr int kMaxPasses = kSortMaxPasses;
constexpr int kQuarters = kSortThreads / kRadix;  // threads per digit in the look-back
constexpr int kLbWords = 16;                      // predecessors per thread per round trip
constexpr int kHistThreads = 256;
static_assert(kSortTile == kSortTileKeys, "tile size shared with the scratch sizing");
static_assert(kQuarters * kRadix == kSortThreads, "whole quarters of digits");
constexpr uint32_t kSpinLimit = 1u << 24;
// Up to this many tiles a tile sums the counts of all earlier tiles instead of the decoupled
// look-back (at two million keys all ~150 tiles run at once, so the look-back finds no
// published prefix and reads the same words over three round trips)
constexpr int kFullSumTiles = 256;
constexpr uint64_t kStateAgg = 1, kStatePrefix = 2;

__device__ __forceinline__ uint64_t os_pack(uint32_t epoch, uint64_t state, uint32_t value) {
    return ((uint64_t)(epoch * 4u + (uint32_t)state) << 32) | value;
}

// Digit counts of every pass: ghist[p * 256 + digit].
template <typename K>
__global__ void __launch_bounds__(kHistThreads) k_os_hist(const K *__restrict__ keys, int64_t n, int begin_bit,
                                                         int end_bit, uint32_t *__restrict__ ghist) {
    __shared__ uint32_t h[kMaxPasses][kRadix];
    for (int i = threadIdx.x; i < kMaxPasses * kRadix; i += kHistThreads) (&h[0][0])[i] = 0;
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
    for (int i = threadIdx.x; i < passes * kRadix; i += kHistThreads) {
        const uint32_t c = (&h[0][0])[i];
        if (c) atomicAdd(&ghist[i], c);
    }
}

// Shared memory of a pass (dynamic, 16-byte aligned).
template <typename K>
struct PassSmem {
    uint32_t whist[kSortWarps][kRadix];   // per-warp digit counts, then per-warp digit offsets
    uint32_t part[kQuarters][kRadix];     // counts of warps [8q, 8q + 8), per digit
    uint32_t lstart[kRadix];              // first position of each digit in the tile
    uint32_t goff[kRadix];                // global position of the tile's first key of each digit
    uint32_t lb_sum[kQuarters][kRadix];   // look-back: AGG sum of a quarter's window
    uint32_t lb_used[kQuarters][kRadix];  // predecessors the quarter consumed
    uint32_t lb_kind[kQuarters][kRadix];  // 0 window read through, 1 met a PREFIX, 2 met an unpublished word
    int32_t lb_next[kRadix];              // nearest predecessor not yet added, per digit (-1: done)
    uint32_t tile_id, pad[3];
    union {
        uint32_t wmask[kSortWarps][kRadix];  // ranking: per-warp lane masks of each digit
        K keys[kSortTile];                   // then: the tile in digit order
    };
    uint32_t vals[kSortTile];
};
static_assert(sizeof(uint32_t) * kSortWarps * kRadix <= sizeof(uint32_t) * kSortTile, "masks fit the key array");

// One pass: rank within the tile, publish the tile's digit counts, scatter the tile into
// shared memory in digit order, look back for the counts of the earlier tiles, write out.
template <typename K>
__global__ void __launch_bounds__(kSortThreads, 1) k_os_pass(
    const K *__restrict__ keys_in, const uint32_t *__restrict__ vals_in, K *__restrict__ keys_out,
    uint32_t *__restrict__ vals_out, int64_t n, int shift, int mask_bits,
    const uint32_t *__restrict__ ghist_pass, unsigned long long *status, uint32_t *ticket, uint32_t epoch,
    uint32_t *err, bool full_sum) {
    extern __shared__ __align__(16) unsigned char sm_raw[];
    PassSmem<K> &S = *reinterpret_cast<PassSmem<K> *>(sm_raw);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int dg = threadIdx.x & (kRadix - 1), q = threadIdx.x / kRadix;
    const uint32_t mask = (1u << mask_bits) - 1u;
    for (int i = threadIdx.x; i < kSortWarps * kRadix; i += kSortThreads) {
        (&S.whist[0][0])[i] = 0;
        (&S.wmask[0][0])[i] = 0;
    }
    if (threadIdx.x == 0) S.tile_id = atomicAdd(ticket, 1u);
    __syncthreads();
    const uint32_t tile = S.tile_id;

    const int64_t tbase = (int64_t)tile * kSortTile;
    const int64_t wbase = tbase + (int64_t)warp * (32 * kSortItems);
    K k[kSortItems];
    uint32_t v[kSortItems];
    uint32_t rank2[(kSortItems + 1) / 2];  // rank within the warp's digit run, two 16-bit ranks per word
    static_assert(32 * kSortItems < 65536, "16-bit ranks");
#pragma unroll
    for (int r = 0; r < kSortItems; ++r) {
        const int64_t i = wbase + r * 32 + lane;
        k[r] = i < n ? keys_in[i] : K(0);
    }
    // ranks within the warp; the values are loaded meanwhile (needed only for the scatter)
#pragma unroll
    for (int r = 0; r < kSortItems; ++r) {
        const int64_t i = wbase + r * 32 + lane;
        const bool valid = i < n;
        v[r] = valid ? vals_in[i] : 0u;
        const uint32_t d = valid ? ((uint32_t)(k[r] >> shift) & mask) : (uint32_t)kRadix;
        // the lanes holding the same digit: a match instruction when lane 0's digit recurs
        // often (few distinct digits), else one shared-memory OR per lane into the warp's
        // digit masks (many distinct digits, where the match instruction is slow)
        const uint32_t d0 = __shfl_sync(0xffffffffu, d, 0);
        const bool use_match = __popc(__ballot_sync(0xffffffffu, d == d0)) >= 4;
        unsigned peers = 0u;
        if (use_match) {
            peers = __match_any_sync(0xffffffffu, d);
        } else {
            if (valid) atomicOr(&S.wmask[warp][d], 1u << lane);
            __syncwarp();
            if (valid) peers = S.wmask[warp][d];
        }
        const uint32_t before = valid ? S.whist[warp][d] : 0u;
        __syncwarp();
        if (valid && lane == __ffs(peers) - 1) {
            S.whist[warp][d] = before + __popc(peers);
            if (!use_match) S.wmask[warp][d] = 0u;  // clean for the next key
        }
        __syncwarp();
        const uint32_t rk = before + __popc(peers & ((1u << lane) - 1u));
        if (r & 1) rank2[r >> 1] |= rk << 16;
        else rank2[r >> 1] = rk;
    }
    __syncthreads();
    // per digit: the count of each quarter's eight warps, then per-warp exclusive offsets
    {
        uint32_t c = 0;
#pragma unroll
        for (int w = 0; w < kSortWarps / kQuarters; ++w) c += S.whist[q * (kSortWarps / kQuarters) + w][dg];
        S.part[q][dg] = c;
    }
    __syncthreads();
    uint32_t count = 0;  // the tile's count of digit dg
    {
        uint32_t base = 0;
#pragma unroll
        for (int qq = 0; qq < kQuarters; ++qq) {
            const uint32_t c = S.part[qq][dg];
            base += qq < q ? c : 0u;
            count += c;
        }
#pragma unroll
        for (int w = 0; w < kSortWarps / kQuarters; ++w) {
            uint32_t &h = S.whist[q * (kSortWarps / kQuarters) + w][dg];
            const uint32_t t = h;
            h = base;
            base += t;
        }
    }
    // publish this tile's count of the digit at once, so later tiles can read past it
    volatile unsigned long long *st = status;
    if (q == 0) st[(uint64_t)tile * kRadix + dg] = os_pack(epoch, tile == 0 ? kStatePrefix : kStateAgg, count);
    // local and global digit starts (the global one from the pass's digit counts)
    uint32_t tile_count, total_unused;
    const uint32_t lst = block_exclusive_scan<kSortThreads>(q == 0 ? count : 0u, &tile_count);
    const uint32_t gdig = block_exclusive_scan<kSortThreads>(q == 0 ? ghist_pass[dg] : 0u, &total_unused);
    if (q == 0) {
        S.lstart[dg] = lst;
        S.lb_next[dg] = (int32_t)tile - 1;
    }
    __syncthreads();
    // the tile in digit order in shared memory (frees the key registers before the look-back)
#pragma unroll
    for (int r = 0; r < kSortItems; ++r) {
        const int64_t i = wbase + r * 32 + lane;
        if (i < n) {
            const uint32_t d = (uint32_t)(k[r] >> shift) & mask;
            const uint32_t lpos = S.lstart[d] + S.whist[warp][d] + ((rank2[r >> 1] >> (16 * (r & 1))) & 0xffffu);
            S.keys[lpos] = k[r];
            S.vals[lpos] = v[r];
        }
    }
    // decoupled look-back over the earlier tiles: per round trip, quarter q of digit dg reads
    // the 16 predecessors [j - 16 q - 15, j - 16 q] (j = nearest not yet added), adds the AGG
    // counts from its nearest down to the first PREFIX (included) or unpublished word
    // (excluded); the quarter-0 thread then joins the quarters in order.  Bounded wait.
    uint32_t excl = 0, spins = 0;
    int32_t next = (int32_t)tile - 1;  // quarter 0: nearest predecessor not yet added (-1: done)
    if (full_sum) {
        // few tiles: sum every earlier tile's own count (quarter q takes the tiles q, q + 4, ...,
        // eight loads in flight); no inclusive prefix is published or read.  Bounded waits.
        uint32_t sum = 0;
        for (int32_t i0 = q; i0 < (int32_t)tile; i0 += kQuarters * 8) {
            unsigned long long w[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int32_t i = i0 + kQuarters * u;
                w[u] = i < (int32_t)tile ? st[(uint64_t)i * kRadix + dg] : os_pack(epoch, kStateAgg, 0u);
            }
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int32_t i = i0 + kQuarters * u;
                uint32_t tries = 0;
                while (((uint32_t)(w[u] >> 34)) != epoch || ((uint32_t)(w[u] >> 32) & 3u) == 0u) {
                    if (++tries > kSpinLimit) {
                        atomicOr(err, 2u);
                        break;
                    }
                    w[u] = st[(uint64_t)i * kRadix + dg];
                }
                sum += (uint32_t)w[u];
            }
        }
        S.lb_sum[q][dg] = sum;
        __syncthreads();
        if (q == 0)
#pragma unroll
            for (int qq = 0; qq < kQuarters; ++qq) excl += S.lb_sum[qq][dg];
        next = -1;
    }
    while (!full_sum) {
        const int32_t j = S.lb_next[dg];
        if (j >= 0) {
            const int32_t hi = j - kLbWords * q;
            unsigned long long w[kLbWords];
#pragma unroll
            for (int u = 0; u < kLbWords; ++u)
                w[u] = hi - u >= 0 ? st[(uint64_t)(hi - u) * kRadix + dg] : 0ull;
            uint32_t sum = 0, used = 0, kind = 0;
#pragma unroll
            for (int u = 0; u < kLbWords; ++u) {
                if (kind != 0 || hi - u < 0) continue;
                const uint32_t h32 = (uint32_t)(w[u] >> 32);
                if ((h32 >> 2) != epoch || (h32 & 3u) == 0u) {
                    kind = 2;
                    continue;
                }
                sum += (uint32_t)w[u];
                ++used;
                if ((h32 & 3u) == kStatePrefix) kind = 1;
            }
            S.lb_sum[q][dg] = sum;
            S.lb_used[q][dg] = used;
            S.lb_kind[q][dg] = kind;
        }
        __syncthreads();
        if (q == 0 && j >= 0) {
            int32_t nj = j;
            bool done = false, stalled = false;
#pragma unroll
            for (int qq = 0; qq < kQuarters; ++qq) {
                if (done || stalled) continue;
                excl += S.lb_sum[qq][dg];
                nj -= (int32_t)S.lb_used[qq][dg];
                const uint32_t kind = S.lb_kind[qq][dg];
                if (kind == 1 || nj < 0) done = true;
                else if (kind == 2) stalled = true;
            }
            if (stalled && ++spins > kSpinLimit) {
                atomicOr(err, 2u);
                done = true;
            }
            next = done ? -1 : nj;
            S.lb_next[dg] = next;
        }
        // every digit done: the quarter-0 threads decide, read after this barrier
        if (__syncthreads_and(q != 0 || next < 0)) break;
    }
    if (q == 0) {
        if (tile > 0 && !full_sum) st[(uint64_t)tile * kRadix + dg] = os_pack(epoch, kStatePrefix, excl + count);
        S.goff[dg] = gdig + excl;
    }
    __syncthreads();
    for (uint32_t i = threadIdx.x; i < tile_count; i += kSortThreads) {
        const K key = S.keys[i];
        const uint32_t d = (uint32_t)(key >> shift) & mask;
        const uint32_t gpos = S.goff[d] + (i - S.lstart[d]);
        keys_out[gpos] = key;
        vals_out[gpos] = S.vals[i];
    }
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
        const int64_t hb = (n + kHistThreads - 1) / kHistThreads;
        k_os_hist<K><<<hb < 1216 ? (int)hb : 1216, kHistThreads, 0, s>>>(keys, n, begin_bit, end_bit, ghist);
        if (launches) *launches += 1;
    }
    const size_t smem = sizeof(PassSmem<K>);
    cudaFuncSetAttribute(k_os_pass<K>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    bool flipped = false;
    K *kin = keys, *kout = keys_alt;
    uint32_t *vin = vals, *vout = vals_alt;
    for (int p = 0; p < passes; ++p) {
        const int shift = begin_bit + 8 * p;
        const int bits = (end_bit - shift) < 8 ? (end_bit - shift) : 8;
        k_os_pass<K><<<nb, kSortThreads, smem, s>>>(kin, vin, kout, vout, n, shift, bits, ghist + p * kRadix,
                                                    status, tickets + p, (uint32_t)(p + 1), err,
                                                    nb <= kFullSumTiles);
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
