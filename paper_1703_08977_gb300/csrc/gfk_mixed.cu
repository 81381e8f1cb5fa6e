// Host launchers of the mixed-precision walk (kernels in gfk_mixed.cuh).  The
// Gaussian-noise kernels are instantiated here, the Bernoulli ones in
// gfk_mixed_bern.cu, so the two compile in parallel.
#include <cuda_runtime.h>

#include <cstring>

#include "gfk_mixed.cuh"

namespace gfk {

extern template void launch_walk_mixed_n<1>(int kind, int wpt, int threads, int nblk, int blk0,
                                            int grid, const InstDev* insts, const BlockMap& bm,
                                            const StateMixed& st, uint32_t step0, int nsteps,
                                            PartialRec* part, unsigned long long* counters,
                                            const TrialHost* one_trial, int ee_on,
                                            cudaStream_t stream, bool run);

__global__ void fill_angle_table_kernel(float2* __restrict__ cs) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < kAngleGrid) cs[k] = angle_cs_entry((uint32_t)k);
}

cudaError_t fill_angle_table(float2* cs, cudaStream_t stream) {
    fill_angle_table_kernel<<<kAngleGrid / 256, 256, 0, stream>>>(cs);
    return cudaGetLastError();
}

cudaError_t launch_init_mixed(int kind, int threads, int nblk, const InstDev* insts,
                              const BlockMap& bm, const StateMixed& st, PartialRec* part,
                              unsigned long long* counters, cudaStream_t stream) {
    if (kind == 0)
        init_mixed_kernel<0><<<nblk, threads, 0, stream>>>(insts, bm, st, part, nblk, counters);
    else if (kind == 1)
        init_mixed_kernel<1><<<nblk, threads, 0, stream>>>(insts, bm, st, part, nblk, counters);
    else
        init_mixed_kernel<2><<<nblk, threads, 0, stream>>>(insts, bm, st, part, nblk, counters);
    return cudaGetLastError();
}

cudaError_t launch_walk_mixed(int kind, int noise, int wpt, int threads, int nblk, int blk0,
                              int grid, const InstDev* insts, const BlockMap& bm,
                              const StateMixed& st, uint32_t step0, int nsteps, PartialRec* part,
                              unsigned long long* counters, const TrialHost* one_trial,
                              int ee_on, cudaStream_t stream) {
    if (noise == GFK_NOISE_BERNOULLI)
        launch_walk_mixed_n<1>(kind, wpt, threads, nblk, blk0, grid, insts, bm, st, step0, nsteps,
                               part, counters, one_trial, ee_on, stream, true);
    else
        launch_walk_mixed_n<0>(kind, wpt, threads, nblk, blk0, grid, insts, bm, st, step0, nsteps,
                               part, counters, one_trial, ee_on, stream, true);
    return cudaGetLastError();
}

cudaError_t prepare_walk_mixed(int kind, int noise, int wpt, int threads, bool one_trial) {
    TrialHost dummy;
    std::memset(&dummy, 0, sizeof(dummy));
    BlockMap bm;
    std::memset(&bm, 0, sizeof(bm));
    StateMixed st{};
    const TrialHost* t = one_trial ? &dummy : nullptr;
    if (noise == GFK_NOISE_BERNOULLI)
        launch_walk_mixed_n<1>(kind, wpt, threads, 0, 0, 0, nullptr, bm, st, 0u, 0, nullptr,
                               nullptr, t, 0, nullptr, false);
    else
        launch_walk_mixed_n<0>(kind, wpt, threads, 0, 0, 0, nullptr, bm, st, 0u, 0, nullptr,
                               nullptr, t, 0, nullptr, false);
    return cudaGetLastError();
}

}  // namespace gfk
