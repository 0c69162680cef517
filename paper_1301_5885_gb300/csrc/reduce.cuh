// reduce.cuh -- deterministic block and grid reductions (no floating-point atomics).
#pragma once

#include "pb_internal.cuh"

namespace pb {

// Sum of v over the block, returned in thread 0 (other threads get garbage).
// The order of additions is fixed by the block size, so results are reproducible.
template <int BS>
__device__ __forceinline__ double block_sum(double v) {
    __shared__ double s_warp[BS / 32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    __syncthreads();            // s_warp may still be read by a previous call
    if (lane == 0) s_warp[wid] = v;
    __syncthreads();
    double t = 0.0;
    if (threadIdx.x == 0) {
#pragma unroll
        for (int w = 0; w < BS / 32; ++w) t += s_warp[w];
    }
    return t;
}

// Called by every thread of every block after thread 0 wrote this block's
// partial(s).  Returns true in every thread of the one block that arrives last;
// that block may then read all partials (with __ldcg) and must reset *counter.
__device__ __forceinline__ bool last_block_arrived(unsigned int *counter, unsigned int nblocks) {
    __shared__ int s_last;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) s_last = (atomicAdd(counter, 1u) == nblocks - 1);
    __syncthreads();
    if (s_last) __threadfence();
    return s_last != 0;
}

}  // namespace pb
