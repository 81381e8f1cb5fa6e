// Adjoint sweep, FP32 instantiation (the mixed path's positions and trial
// arithmetic; the parameter adjoint is summed in FP64).  Compiled with the
// same flags as the mixed walk kernel, so recomputed positions match it.
#include "gfk_adjoint.cuh"

namespace gfk {

cudaError_t launch_adjoint_f32(const InstDev* inst, int64_t n, int S, int K, int loss_kind,
                               const float* ckpt, float* seg, const float* traj,
                               const float* pos_final,
                               const double* logw_final, double* ew, double* part_max,
                               double* part_sums, double* part_theta, void* term, double* grad,
                               cudaStream_t stream) {
    return adj_run<float>(inst, n, S, K, loss_kind, ckpt, seg, traj, pos_final, logw_final, ew, part_max,
                          part_sums, part_theta, (AdjTerminal*)term, grad, stream);
}

}  // namespace gfk
