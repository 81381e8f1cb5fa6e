// The Bernoulli-noise instantiations of the mixed-precision walk kernels
// (gfk_mixed.cuh), compiled apart from the Gaussian ones.
#include "gfk_mixed.cuh"

namespace gfk {

template void launch_walk_mixed_n<1>(int kind, int wpt, int threads, int nblk, int blk0,
                                     int grid, const InstDev* insts, const BlockMap& bm,
                                     const StateMixed& st, uint32_t step0, int nsteps,
                                     PartialRec* part, unsigned long long* counters,
                                     const TrialHost* one_trial, int ee_on, cudaStream_t stream,
                                     bool run);

}  // namespace gfk
