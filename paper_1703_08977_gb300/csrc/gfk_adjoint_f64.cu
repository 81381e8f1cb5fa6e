// Adjoint sweep, FP64 instantiation.  Compiled with --fmad=false like the FP64
// walk kernel, so the recomputed positions round exactly as the forward's.
#include "gfk_adjoint.cuh"

namespace gfk {

cudaError_t launch_adjoint_f64(const InstDev* inst, int64_t n, int S, int K, int loss_kind,
                               const double* ckpt, double* seg, const double* pos_final,
                               const double* logw_final, double* ew, double* part_max,
                               double* part_sums, double* part_theta, void* term, double* grad,
                               cudaStream_t stream) {
    return adj_run<double>(inst, n, S, K, loss_kind, ckpt, seg, nullptr, pos_final, logw_final, ew, part_max,
                           part_sums, part_theta, (AdjTerminal*)term, grad, stream);
}

}  // namespace gfk
