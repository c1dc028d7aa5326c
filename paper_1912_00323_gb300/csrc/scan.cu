// Device-wide exclusive prefix sum of uint32 (reduce, scan of tile sums, scan-and-apply), and
// the run-length cells of sorted cell keys from first-of-cell flags whose tile sums the gather
// kernels produce (scan of tile sums, scan-and-apply with the cell tables written in place).
#include "block_scan.cuh"
#include "hca_internal.cuh"

namespace hca {

namespace {

constexpr int kScanThreads = 256;
constexpr int kScanItems = 8;
constexpr int kScanTile = kScanThreads * kScanItems;
static_assert(kScanTile == kScanTileElems, "tile size shared with the gather kernels");

__device__ __forceinline__ int64_t scan_len(int64_t m_max, const uint32_t *m_dev) {
    if (!m_dev) return m_max;
    int64_t m = (int64_t)*m_dev;
    return m < m_max ? m : m_max;
}

__global__ void __launch_bounds__(kScanThreads) k_scan_reduce(const uint32_t *in, int64_t m_max,
                                                              const uint32_t *m_dev,
                                                              uint32_t *partials) {
    const int64_t m = scan_len(m_max, m_dev);
    const int64_t base = (int64_t)blockIdx.x * kScanTile;
    uint32_t s = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        int64_t i = base + k * kScanThreads + threadIdx.x;
        if (i < m) s += in[i];
    }
    uint32_t total;
    block_exclusive_scan<kScanThreads>(s, &total);
    if (threadIdx.x == 0) partials[blockIdx.x] = total;
}

// One block scans the nb tile sums in place (exclusive); total -> partials[nb] and *total.
__global__ void __launch_bounds__(1024) k_scan_partials(uint32_t *partials, int64_t nb,
                                                        uint32_t *total) {
    uint32_t carry = 0;
    for (int64_t b0 = 0; b0 < nb; b0 += 1024) {
        int64_t i = b0 + threadIdx.x;
        uint32_t v = i < nb ? partials[i] : 0u;
        uint32_t t;
        uint32_t ex = block_exclusive_scan<1024>(v, &t);
        if (i < nb) partials[i] = carry + ex;
        carry += t;
    }
    if (threadIdx.x == 0) {
        partials[nb] = carry;
        if (total) *total = carry;
    }
}

__global__ void __launch_bounds__(kScanThreads) k_scan_apply(const uint32_t *in, uint32_t *out,
                                                             int64_t m_max,
                                                             const uint32_t *m_dev,
                                                             const uint32_t *partials) {
    __shared__ uint32_t tile[kScanTile];
    const int64_t m = scan_len(m_max, m_dev);
    const int64_t base = (int64_t)blockIdx.x * kScanTile;
    if (base >= m) return;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        int64_t i = base + k * kScanThreads + threadIdx.x;
        tile[k * kScanThreads + threadIdx.x] = i < m ? in[i] : 0u;
    }
    __syncthreads();
    uint32_t v[kScanItems];
    uint32_t s = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        v[k] = tile[threadIdx.x * kScanItems + k];
        s += v[k];
    }
    uint32_t total;
    uint32_t run = block_exclusive_scan<kScanThreads>(s, &total) + partials[blockIdx.x];
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        tile[threadIdx.x * kScanItems + k] = run;
        run += v[k];
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        int64_t i = base + k * kScanThreads + threadIdx.x;
        if (i < m) out[i] = tile[k * kScanThreads + threadIdx.x];
    }
}

// Per tile: exclusive prefix of the flags (tile offset from the scanned tile sums) -> cell id
// of every point, first point and key of every cell, the end of the last cell.
template <typename K>
__global__ void __launch_bounds__(kScanThreads) k_cells_apply(const K *__restrict__ keys, uint32_t *flags_cell_of,
                                                              int64_t n, const uint32_t *__restrict__ partials,
                                                              uint32_t *__restrict__ cell_start,
                                                              uint64_t *__restrict__ cell_key) {
    __shared__ uint32_t tile[kScanTile];
    const int64_t base = (int64_t)blockIdx.x * kScanTile;
    if (base >= n) return;
    uint32_t f[kScanItems];
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        const int64_t i = base + k * kScanThreads + threadIdx.x;
        f[k] = i < n ? flags_cell_of[i] : 0u;
        tile[k * kScanThreads + threadIdx.x] = f[k];
    }
    __syncthreads();
    uint32_t v[kScanItems];
    uint32_t sum = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        v[k] = tile[threadIdx.x * kScanItems + k];
        sum += v[k];
    }
    uint32_t total;
    uint32_t run = block_exclusive_scan<kScanThreads>(sum, &total) + partials[blockIdx.x];
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        tile[threadIdx.x * kScanItems + k] = run;
        run += v[k];
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        const int64_t i = base + k * kScanThreads + threadIdx.x;
        if (i < n) {
            const uint32_t c = tile[k * kScanThreads + threadIdx.x] + f[k] - 1u;
            flags_cell_of[i] = c;
            if (f[k]) {
                cell_start[c] = (uint32_t)i;
                cell_key[c] = (uint64_t)keys[i];
            }
            if (i == n - 1) cell_start[c + 1] = (uint32_t)n;
        }
    }
}

}  // namespace

template <typename K>
void cells_from_flags(const K *keys, uint32_t *flags_cell_of, int64_t n, uint32_t *partials, uint32_t *n_cells,
                      uint32_t *cell_start, uint64_t *cell_key, cudaStream_t s, int *launches) {
    int64_t nb = (n + kScanTile - 1) / kScanTile;
    if (nb == 0) nb = 1;
    k_scan_partials<<<1, 1024, 0, s>>>(partials, nb, n_cells);
    k_cells_apply<K><<<(unsigned)nb, kScanThreads, 0, s>>>(keys, flags_cell_of, n, partials, cell_start, cell_key);
    if (launches) *launches += 2;
}

template void cells_from_flags<uint32_t>(const uint32_t *, uint32_t *, int64_t, uint32_t *, uint32_t *, uint32_t *,
                                         uint64_t *, cudaStream_t, int *);
template void cells_from_flags<uint64_t>(const uint64_t *, uint32_t *, int64_t, uint32_t *, uint32_t *, uint32_t *,
                                         uint64_t *, cudaStream_t, int *);

size_t scan_partials_size(int64_t m_max) {
    return (size_t)((m_max + kScanTile - 1) / kScanTile) + 2;
}

void exclusive_scan_u32(const uint32_t *in, uint32_t *out, int64_t m_max, const uint32_t *m_dev,
                        uint32_t *total, uint32_t *partials, cudaStream_t s, int *launches) {
    int64_t nb = (m_max + kScanTile - 1) / kScanTile;
    if (nb == 0) nb = 1;
    k_scan_reduce<<<(unsigned)nb, kScanThreads, 0, s>>>(in, m_max, m_dev, partials);
    k_scan_partials<<<1, 1024, 0, s>>>(partials, nb, total);
    k_scan_apply<<<(unsigned)nb, kScanThreads, 0, s>>>(in, out, m_max, m_dev, partials);
    if (launches) *launches += 3;
}

}  // namespace hca
