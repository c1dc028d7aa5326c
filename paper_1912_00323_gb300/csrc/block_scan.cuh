// Warp- and block-level prefix sums used by the scan and sort kernels.
#pragma once

#include <stdint.h>

namespace hca {

__device__ __forceinline__ uint32_t warp_inclusive_scan(uint32_t v) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t t = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += t;
    }
    return v;
}

// Exclusive scan of one value per thread across a block of NT threads (NT a multiple of 32,
// at most 1024).  Returns the thread's exclusive prefix; *total gets the block sum.  Every
// thread of the block must call it; it synchronises the block.
template <int NT>
__device__ __forceinline__ uint32_t block_exclusive_scan(uint32_t v, uint32_t *total) {
    __shared__ uint32_t warp_sums[NT / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t inc = warp_inclusive_scan(v);
    if (lane == 31) warp_sums[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        uint32_t w = lane < NT / 32 ? warp_sums[lane] : 0u;
        w = warp_inclusive_scan(w);
        if (lane < NT / 32) warp_sums[lane] = w;
    }
    __syncthreads();
    uint32_t prefix = warp ? warp_sums[warp - 1] : 0u;
    *total = warp_sums[NT / 32 - 1];
    __syncthreads();
    return prefix + inc - v;
}

}  // namespace hca
