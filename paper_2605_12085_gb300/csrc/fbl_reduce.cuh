// Deterministic block reductions for the FP64 line-search sums.
//
// Each thread holds an FP32 partial over a handful of elements; a warp adds
// its 32 partials in FP32 with a fixed shuffle tree, converts to FP64, and the
// block adds its warps in FP64 in warp order.  The per-block results go to a
// partials array that launch_reduce sums in a fixed order, so every sum is
// bit-reproducible run to run (no atomics).
#pragma once

#include <cuda_runtime.h>

namespace fbl {

__device__ __forceinline__ float warp_sum_f32(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

// Sum of NC FP32 values over a block of NT threads, in FP64; the result is
// valid in thread 0 (linear thread index).  Must be called by every thread.
template <int NT, int NC>
__device__ __forceinline__ void block_sum_f64(const float (&v)[NC], double (&out)[NC]) {
    static_assert(NT % 32 == 0 && NT <= 1024, "block size");
    constexpr int NW = NT / 32;
    __shared__ double sm[NC][NW];
    const int tid = threadIdx.x + blockDim.x * (threadIdx.y + blockDim.y * threadIdx.z);
    const int lane = tid & 31, wid = tid >> 5;
#pragma unroll
    for (int c = 0; c < NC; ++c) {
        float w = warp_sum_f32(v[c]);
        if (lane == 0) sm[c][wid] = (double)w;
    }
    __syncthreads();
    if (tid == 0) {
#pragma unroll
        for (int c = 0; c < NC; ++c) {
            double s = 0.0;
#pragma unroll
            for (int q = 0; q < NW; ++q) s += sm[c][q];
            out[c] = s;
        }
    }
}

}  // namespace fbl
