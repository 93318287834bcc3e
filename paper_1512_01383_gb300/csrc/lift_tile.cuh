// Per-tile helpers shared by the step kernels (pdhg_step.cu) and the
// cluster-resident iteration (resident.cu): the thread -> (pixel, interval)
// split of a 256-thread tile, the exact row of a pixel, and the per-pixel
// segmented scan over the block.
#pragma once

#include <cuda_runtime.h>

#include "lift_params.h"

namespace lift {

__device__ __forceinline__ void split_thread(const LiftParams &P, int tid, int &lp, int &i)
{
    // (tid + 0.5) / k is at least 0.5/k away from an integer; the float
    // product is exact to far better than that for tid < 256, k <= 64
    lp = __float2int_rz((static_cast<float>(tid) + 0.5f) * P.inv_k);
    i = tid - lp * P.k;
}

__device__ __forceinline__ int pixel_row(const LiftParams &P, int pix)
{
    return static_cast<int>((static_cast<unsigned long long>(pix) * P.wmul) >> P.wshift);
}

// Row within its slice of a global row index z*H + y (volumes).
__device__ __forceinline__ int row_in_slice(const LiftParams &P, int row)
{
    const int zz = static_cast<int>((static_cast<unsigned long long>(row) * P.hmul) >> P.hshift);
    return row - zz * P.H;
}

// Inclusive prefix sum of `val` over the thread's pixel segment
// [seg, seg + k) of the block, and the segment's total.  Every thread of the
// block must call it (it contains a barrier); threads outside any pixel pass
// val = 0 and a segment of their own.
struct SegScan {
    float incl, total;
};

__device__ __forceinline__ SegScan block_segmented_scan(float val, int seg, int k, int tid,
                                                        bool active, float *s_in, float *s_last)
    // s_in: one float per thread; s_last: one float per warp
{
    const int lane = tid & 31, warp = tid >> 5;
    const int wbase = warp << 5;
    const int start = seg > wbase ? seg - wbase : 0;   // first lane of my segment in this warp
    float x = val;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const float y = __shfl_up_sync(0xffffffffu, x, off);
        if (lane - off >= start) x += y;
    }
    s_in[tid] = x;
    if (lane == 31) s_last[warp] = x;
    __syncthreads();
    SegScan r{0.0f, 0.0f};
    if (!active) return r;
    // a segment (k <= 64 records) spans at most three warps: add the in-warp
    // totals of the earlier warps it covers, in straight-line code
    const int sw = seg >> 5;
    float carry = 0.0f;
    if (sw < warp) {
        carry = s_last[warp - 1];
        if (sw < warp - 1) carry += s_last[warp - 2];
    }
    r.incl = x + carry;
    const int e = seg + k - 1, ew = e >> 5;
    float ce = 0.0f;
    if (sw < ew) {
        ce = s_last[sw];
        if (sw + 1 < ew) ce += s_last[sw + 1];
    }
    r.total = s_in[e] + ce;
    return r;
}

}  // namespace lift
