// Host launchers of the GFK kernels (defined beside their kernels), called by
// the C ABI layer.  Each queues its kernels on `stream` and returns
// cudaGetLastError(); `kind` is the trial kind (2 = per-block dispatch).
#pragma once

#include <cuda_runtime.h>

#include "gfk_types.h"

namespace gfk {
cudaError_t launch_init_fp64(int kind, int threads, int nblk, const InstDev* insts,
                             const BlockMap& bm, const StateF64& st, PartialRec* part,
                             unsigned long long* counters, cudaStream_t stream);
// noise: gfk_noise of the context (selects the kernel instantiation)
cudaError_t launch_walk_fp64(int kind, int noise, int threads, int nblk, const InstDev* insts,
                             const BlockMap& bm, const StateF64& st, uint32_t step0, int nsteps,
                             PartialRec* part, unsigned long long* counters, cudaStream_t stream);
// The Box-Muller angle table of the mixed path (kAngleGrid float2 pairs of
// cos, sin; see angle_cs_entry), written on `stream`.
cudaError_t fill_angle_table(float2* cs, cudaStream_t stream);
cudaError_t launch_init_mixed(int kind, int threads, int nblk, const InstDev* insts,
                              const BlockMap& bm, const StateMixed& st, PartialRec* part,
                              unsigned long long* counters, cudaStream_t stream);
// kind: 0 / 1 the trial family, 2 both in one launch (or any trial function
// with Jastrow polynomial terms), 3 orbital pairs whose orbitals all lack the
// r and z prefactor terms (mixed_walk_kind).
// one_trial: when the launch covers a single instance, its trial function (and
// ee_on); the kernel then takes it as a launch argument.  NULL otherwise.
// nblk: all blocks of the context (the records' stride); the launch runs
// blocks blk0 .. blk0 + grid - 1 of them.
cudaError_t launch_walk_mixed(int kind, int noise, int wpt, int threads, int nblk, int blk0,
                              int grid, const InstDev* insts, const BlockMap& bm,
                              const StateMixed& st, uint32_t step0, int nsteps, PartialRec* part,
                              unsigned long long* counters, const TrialHost* one_trial,
                              int ee_on, cudaStream_t stream);
// The mixed walk's kind for these trial functions.  The specialised kinds 0,
// 1 and 3 are compiled for trial functions without Jastrow polynomial terms,
// so a set with any c_k != 0 takes the per-block dispatch (2).  Otherwise 3
// when every one is an orbital-pair function whose orbitals have no r or z
// prefactor terms (c1 = cz = 0 in every used term), else `kind` unchanged.
inline int mixed_walk_kind(int kind, const TrialHost* trials, int n) {
    for (int i = 0; i < n; ++i)
        for (int k = 0; k < 4; ++k)
            if (trials[i].ck[k] != 0.0) return 2;
    if (kind != GFK_TRIAL_ORBITAL_PAIRS) return kind;
    for (int i = 0; i < n; ++i)
        for (int k = 0; k < trials[i].nterms; ++k)
            for (int e = 0; e < 2; ++e)
                if (trials[i].c1[k][e] != 0.0 || trials[i].cz[k][e] != 0.0) return kind;
    return 3;
}

// Sets what the mixed walk kernel of this launch shape needs before it can be
// launched (the shared-memory opt-in of 512-thread blocks); called before a
// stream capture, where it could not happen.
cudaError_t prepare_walk_mixed(int kind, int noise, int wpt, int threads, bool one_trial);
// W and P are merged as double-doubles (compensated) on both paths
cudaError_t launch_reduce_rows(const PartialRec* part, int nblk, const BlockMap& bm, int rows,
                               SeriesRow* series, int64_t series_cap, int64_t row_base,
                               cudaStream_t stream);
cudaError_t launch_finalize(const SeriesRow* rows, int64_t n, double n0, double* e, double* lnz,
                            double* ess, cudaStream_t stream);
cudaError_t launch_export(bool mixed, const StateF64& s64, const StateMixed& smx, int64_t off,
                          int64_t n, double* x6, double* logw, uint8_t* alive,
                          cudaStream_t stream);
cudaError_t launch_adjoint_f64(const InstDev* inst, int64_t n, int S, int K, int loss_kind,
                               const double* ckpt, double* seg, const double* pos_final,
                               const double* logw_final, double* ew, double* part_max,
                               double* part_sums, double* part_theta, void* term, double* grad,
                               cudaStream_t stream);
// traj: the forward's whole trajectory (StateMixed::traj), or NULL to
// recompute the segments from the checkpoints
cudaError_t launch_adjoint_f32(const InstDev* inst, int64_t n, int S, int K, int loss_kind,
                               const float* ckpt, float* seg, const float* traj,
                               const float* pos_final,
                               const double* logw_final, double* ew, double* part_max,
                               double* part_sums, double* part_theta, void* term, double* grad,
                               cudaStream_t stream);
}  // namespace gfk
