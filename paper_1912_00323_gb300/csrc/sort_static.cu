// hca_radix_sort_pairs_noalloc: the radix sort of hca_radix_sort_pairs with its scratch in a
// fixed device array of this library instead of memory allocated per call.
//
// Some callers cannot allocate device memory while they run: a loop with a fixed memory
// budget set at start-up, a host framework whose allocator owns all device memory, or code
// that must not risk the device-wide synchronisation cudaMalloc / cudaFree can cause.  This
// entry point takes the caller's keys and values and uses only the array below.
//
// The array is a file-scope __device__ variable: every GPU on which the library is loaded
// holds its HCA_SORT_NOALLOC_MAX_PAIRS * 12 bytes (plus look-back space, about 3.3 MiB in all)
// until the process exits.  In host code its name is only a stand-in: the device address is
// looked up once per device with cudaGetSymbolAddress, by the first call on that device.
#include <mutex>

#include "hca_internal.cuh"

namespace hca {
namespace {

constexpr int64_t kMaxPairs = HCA_SORT_NOALLOC_MAX_PAIRS;
constexpr size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }
// sort scratch words for kMaxPairs: look-back words (2 per 2048-key tile and digit), digit
// counts of up to 8 passes, tickets and a status word
constexpr size_t kHistElems = 2 * ((kMaxPairs + 2047) / 2048) * 256 + 8 * 256 + 10;
constexpr size_t kPartElems = ((kMaxPairs > (int64_t)kHistElems ? kMaxPairs : (int64_t)kHistElems) + 2047) / 2048 + 2;
constexpr size_t kOffVals = align256(sizeof(uint64_t) * kMaxPairs);
constexpr size_t kOffHist = kOffVals + align256(sizeof(uint32_t) * kMaxPairs);
constexpr size_t kOffPart = kOffHist + align256(sizeof(uint32_t) * kHistElems);
constexpr size_t kScratchBytes = kOffPart + align256(sizeof(uint32_t) * kPartElems);

__device__ __align__(256) unsigned char g_sort_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void *g_scratch_addr[kMaxDevices] = {};

// Device address of g_sort_scratch on the current device (looked up once per device).
int scratch_address(void **out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return HCA_ECUDA;
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_scratch_addr[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_sort_scratch) != cudaSuccess || !p) return HCA_ECUDA;
        g_scratch_addr[dev] = p;
    }
    *out = g_scratch_addr[dev];
    return HCA_OK;
}

}  // namespace
}  // namespace hca

using namespace hca;

extern "C" int hca_radix_sort_pairs_noalloc(void *d_keys, uint32_t *d_vals, int64_t n,
                                            int32_t key_bytes, int32_t begin_bit, int32_t end_bit,
                                            void *stream) {
    if (n < 0) return HCA_EINVAL;
    if (key_bytes != 4 && key_bytes != 8) return HCA_EINVAL;
    if (begin_bit < 0 || end_bit <= begin_bit || end_bit > 8 * key_bytes) return HCA_EINVAL;
    if (n > kMaxPairs) return HCA_ETOOLARGE;
    if (n > 0 && (!d_keys || !d_vals)) return HCA_EINVAL;
    if (((uintptr_t)d_keys) % key_bytes || ((uintptr_t)d_vals) % 4) return HCA_EINVAL;
    if (n <= 1) return HCA_OK;
    const size_t hist_need = sort_hist_size(n);
    if (hist_need > kHistElems ||
        scan_partials_size(n > (int64_t)hist_need ? n : (int64_t)hist_need) > kPartElems)
        return HCA_ETOOLARGE;
    void *base = nullptr;
    int rc = scratch_address(&base);
    if (rc) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    char *b = (char *)base;
    uint32_t *valt = (uint32_t *)(b + kOffVals);
    uint32_t *hist = (uint32_t *)(b + kOffHist);
    uint32_t *part = (uint32_t *)(b + kOffPart);
    // The sort clears its counters, tickets and look-back words itself at the start of every
    // call; every other scratch word is written before it is read, so nothing left by an
    // earlier call is used.
    bool flipped;
    if (key_bytes == 4)
        flipped = radix_sort_pairs<uint32_t>((uint32_t *)d_keys, d_vals, (uint32_t *)b, valt, n,
                                             begin_bit, end_bit, hist, part, s, nullptr);
    else
        flipped = radix_sort_pairs<uint64_t>((uint64_t *)d_keys, d_vals, (uint64_t *)b, valt, n,
                                             begin_bit, end_bit, hist, part, s, nullptr);
    rc = HCA_OK;
    if (flipped) {
        if (cudaMemcpyAsync(d_keys, b, (size_t)n * key_bytes, cudaMemcpyDeviceToDevice, s) != cudaSuccess ||
            cudaMemcpyAsync(d_vals, valt, (size_t)n * 4, cudaMemcpyDeviceToDevice, s) != cudaSuccess)
            rc = HCA_ECUDA;
    }
    uint32_t status = 0;
    if (cudaMemcpyAsync(&status, sort_status_word(hist, n), sizeof(status), cudaMemcpyDeviceToHost, s) != cudaSuccess)
        rc = HCA_ECUDA;
    if (cudaGetLastError() != cudaSuccess) rc = HCA_ECUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) rc = HCA_ECUDA;
    if (rc == HCA_OK && status) rc = HCA_EDEVICE;
    return rc;
}
