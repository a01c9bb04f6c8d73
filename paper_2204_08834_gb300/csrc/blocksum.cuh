// blocksum.cuh - per-CTA partial sums of the x passes (added up across CTAs by k_finalize).
#pragma once
#include <cuda_runtime.h>

namespace {

// Block sums into part[bi * 3 + q] (bi = blockIdx.x unless given) of the partials a (FP64, reduced only when
// HAS_A), b and c (FP32, reduced in FP32 within each warp, only when HAS_B / HAS_C); absent
// partials are written as 0.  Warp values are added in FP64 by warp 0.  Per thread this costs
// 5 FP64 adds for a and none for b, c (FP64 instructions run on GB300's narrow FP64 pipe).
template <bool HAS_A, bool HAS_B, bool HAS_C>
__device__ void block_sum_abc(double a, float b, float c, double* __restrict__ part, int bi = -1) {
    if (bi < 0) bi = blockIdx.x;
    __shared__ double red[3][32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        if (HAS_A) a += __shfl_xor_sync(0xffffffffu, a, o);
        if (HAS_B) b += __shfl_xor_sync(0xffffffffu, b, o);
        if (HAS_C) c += __shfl_xor_sync(0xffffffffu, c, o);
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    if (lane == 0) {
        red[0][wid] = HAS_A ? a : 0.0;
        red[1][wid] = HAS_B ? (double)b : 0.0;
        red[2][wid] = HAS_C ? (double)c : 0.0;
    }
    __syncthreads();
    if (wid == 0) {
        double x = lane < nw ? red[0][lane] : 0.0;
        double y = lane < nw ? red[1][lane] : 0.0;
        double z = lane < nw ? red[2][lane] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            x += __shfl_down_sync(0xffffffffu, x, o);
            y += __shfl_down_sync(0xffffffffu, y, o);
            z += __shfl_down_sync(0xffffffffu, z, o);
        }
        if (lane == 0) {
            part[bi * 3 + 0] = x;
            part[bi * 3 + 1] = y;
            part[bi * 3 + 2] = z;
        }
    }
}

}  // namespace
