// Device-wide exclusive prefix sum of uint32 (reduce, scan of tile sums, scan-and-apply).
// Used for the run-length encoding of sorted cell keys and pencils, and for the radix
// sort's digit offsets.
#include "block_scan.cuh"
#include "hca_internal.cuh"

namespace hca {

namespace {

constexpr int kScanThreads = 256;
constexpr int kScanItems = 8;
constexpr int kScanTile = kScanThreads * kScanItems;

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

}  // namespace

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
