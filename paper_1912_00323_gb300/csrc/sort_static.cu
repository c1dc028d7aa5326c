// hca_radix_sort_pairs_noalloc: the radix sort of hca_radix_sort_pairs with its scratch in a
// fixed device array of this library instead of memory allocated per call.
//
// Some callers cannot allocate device memory while they run: a loop with a fixed memory
// budget set at start-up, a host framework whose allocator owns all device memory, or code
// that must not risk the device-wide synchronisation cudaMalloc / cudaFree can cause.  This
// entry point takes the caller's keys and values and uses only the array below.
//
// The array is a file-scope __device__ variable: every GPU on which the library is loaded
// holds it until the process exits.  Its size follows the sort's own geometry: the
// alternate keys and values of HCA_SORT_NOALLOC_MAX_PAIRS pairs (12 bytes each, 3 MiB) and
// the look-back words, digit counts, tickets and status word of that many pairs (about
// 48 KiB with the sort's 13,312-key tiles).  In host code its name is only a stand-in: its device address
// is looked up with cudaGetSymbolAddress, with the device current, the first time a call
// runs in a CUDA context of that device (normally once per device; again after
// cudaDeviceReset, which destroys the context the cached address belongs to).
#include <mutex>

#include "hca_internal.cuh"

namespace hca {

// The unique id of the calling thread's current CUDA context (0 when none is current or the
// driver does not provide the query).  Driver entry points are found through the runtime, so
// the library does not link the driver library itself.
typedef int (*ctx_get_current_t)(void **);
typedef int (*ctx_get_id_t)(void *, unsigned long long *);

unsigned long long current_context_id() {
    static ctx_get_current_t get_current = nullptr;
    static ctx_get_id_t get_id = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) ==
                cudaSuccess && q == cudaDriverEntryPointSuccess)
            get_current = (ctx_get_current_t)f;
        f = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_id = (ctx_get_id_t)f;
    });
    if (!get_current || !get_id) return 0;
    void *ctx = nullptr;
    unsigned long long id = 0;
    if (get_current(&ctx) != 0 || !ctx || get_id(ctx, &id) != 0) return 0;
    return id;
}

namespace {

constexpr int64_t kMaxPairs = HCA_SORT_NOALLOC_MAX_PAIRS;
constexpr size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }
constexpr size_t kHistElems = sort_hist_elems(kMaxPairs);
constexpr size_t kOffVals = align256(sizeof(uint64_t) * kMaxPairs);
constexpr size_t kOffHist = kOffVals + align256(sizeof(uint32_t) * kMaxPairs);
constexpr size_t kScratchBytes = kOffHist + align256(sizeof(uint32_t) * kHistElems);

__device__ __align__(256) unsigned char g_sort_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
struct ScratchSlot {
    unsigned long long ctx_id;
    void *addr;
};
ScratchSlot g_slot[kMaxDevices] = {};

// Device address of g_sort_scratch in the current context of the current device.  The
// look-up runs once per context; a context whose id cannot be read is looked up every call.
int scratch_address(void **out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return HCA_ECUDA;
    std::lock_guard<std::mutex> lk(g_mu);
    unsigned long long id = current_context_id();
    ScratchSlot &slot = g_slot[dev];
    if (id == 0 || slot.ctx_id != id || !slot.addr) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_sort_scratch) != cudaSuccess || !p) return HCA_ECUDA;
        if (id == 0) id = current_context_id();  // the look-up may have created the context
        slot.ctx_id = id;
        slot.addr = p;
    }
    *out = slot.addr;
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
    if (sort_hist_size(n) > kHistElems) return HCA_ETOOLARGE;
    void *base = nullptr;
    int rc = scratch_address(&base);
    if (rc) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    char *b = (char *)base;
    uint32_t *valt = (uint32_t *)(b + kOffVals);
    uint32_t *hist = (uint32_t *)(b + kOffHist);
    // The sort clears its counters, tickets and look-back words itself at the start of every
    // call; every other scratch word is written before it is read, so nothing left by an
    // earlier call is used.
    bool flipped;
    if (key_bytes == 4)
        flipped = radix_sort_pairs<uint32_t>((uint32_t *)d_keys, d_vals, (uint32_t *)b, valt, n,
                                             begin_bit, end_bit, hist, nullptr, s, nullptr);
    else
        flipped = radix_sort_pairs<uint64_t>((uint64_t *)d_keys, d_vals, (uint64_t *)b, valt, n,
                                             begin_bit, end_bit, hist, nullptr, s, nullptr);
    rc = HCA_OK;
    if (flipped) {
        if (cudaMemcpyAsync(d_keys, b, (size_t)n * key_bytes, cudaMemcpyDeviceToDevice, s) != cudaSuccess ||
            cudaMemcpyAsync(d_vals, valt, (size_t)n * 4, cudaMemcpyDeviceToDevice, s) != cudaSuccess)
            rc = HCA_ECUDA;
    }
    // the look-back status word is read back, so every call waits for its sort on `stream`
    uint32_t status = 0;
    if (cudaMemcpyAsync(&status, sort_status_word(hist, n), sizeof(status), cudaMemcpyDeviceToHost, s) != cudaSuccess)
        rc = HCA_ECUDA;
    if (cudaGetLastError() != cudaSuccess) rc = HCA_ECUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) rc = HCA_ECUDA;
    if (rc == HCA_OK && status) rc = HCA_EDEVICE;
    return rc;
}
