// Block-level helpers shared by the walk kernels.
#pragma once

#include <cuda_runtime.h>

#include "gfk_device.cuh"
#include "gfk_types.h"

namespace gfk {

// Instance owning this block (blocks of an instance are contiguous).
__device__ __forceinline__ int block_instance(const BlockMap& bm, int blk) {
    int inst = 0;
    for (int i = 1; i < bm.n_inst; ++i)
        if (blk >= bm.begin[i]) inst = i;
    return inst;
}

// Log-weight shift of the block: floor of the block's largest log-weight
// (integer-valued, so the cross-block merge meets few distinct factors
// e^{c_b - C}); `red` holds kMaxWarps doubles of shared memory.  Returns 0 when
// every thread passed -inf (no live walker in the block).
__device__ __forceinline__ double block_max_shift(double v, double* red) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nwarps = blockDim.x >> 5;
    v = warp_max(v);
    if (lane == 0) red[warp] = v;
    __syncthreads();
    double m = red[0];
    for (int w = 1; w < nwarps; ++w) m = fmax(m, red[w]);
    __syncthreads();
    return isfinite(m) ? floor(m) : 0.0;
}

// Per-thread event counters folded into the instance's global counters.
__device__ __forceinline__ void flush_counters(unsigned long long* counters, int inst,
                                               unsigned n_nonfinite, unsigned n_node,
                                               unsigned n_coal) {
    unsigned v[kNumCounters] = {n_nonfinite, n_node, n_coal};
#pragma unroll
    for (int j = 0; j < kNumCounters; ++j) {
        unsigned s = warp_sum(v[j]);
        if ((threadIdx.x & 31) == 0 && s != 0)
            atomicAdd(&counters[inst * kNumCounters + j], (unsigned long long)s);
    }
}

}  // namespace gfk
