// FP64 walk: every operation of the GFK step in double precision.
//
// This translation unit is compiled with --fmad=false so that no multiply-add
// is fused: the arithmetic then rounds like a plain sequential evaluation.
//
// One thread advances one walker for a whole chunk of steps with its state in
// registers.  Per step (the discretised Eq. 4 with the drifted diffusion under
// it):
//   xi       <- six N(0,1) from one Philox4x32-10 block (radii and angles),
//               or (NOISE = 1) six signs +-1 from the walker's Superduper generator
//   X        <- X + b(X) dt + sqrt(dt) xi                       (Euler-Maruyama)
//   b, E_L   <- trial function at the new X
//   node     :  sign psi changed (or psi = 0) -> walker killed
//   logw     <- logw - (E_L - E_T) dt                           (right-point rule)
//   sums     :  w = e^{logw - c}, block sums of w, w E_L, w^2, w E_L^2, alive
// The per-step sums of each warp go to a shared-memory ring of kRing steps;
// every kRing steps the block adds its warps in FP64 and writes one PartialRec
// per step, and the block shift c is refreshed to the block's largest logw.
#include <cuda_runtime.h>

#include "gfk_block.cuh"
#include "gfk_device.cuh"
#include "gfk_launch.h"
#include "gfk_types.h"

namespace gfk {

// The debug build's check of a walker's slot in the state planes (true in the
// release build).
__device__ __forceinline__ bool f64_slot_ok(const StateF64& st, int64_t slot) {
    return GFK_DBG_OK(st.x + slot, sizeof(double), kDbgState) &&
           GFK_DBG_OK(st.x + 5 * st.stride + slot, sizeof(double), kDbgState) &&
           GFK_DBG_OK(st.logw + slot, sizeof(double), kDbgState) &&
           GFK_DBG_OK(st.sgn + slot, 1, kDbgState);
}

template <int KIND>
__global__ void __launch_bounds__(kMaxThreads)
init_fp64_kernel(const InstDev* __restrict__ insts, BlockMap bm, StateF64 st,
                 PartialRec* __restrict__ part, int nblk,
                 unsigned long long* __restrict__ counters) {
    __shared__ TrialDev<double> s_trial;
    __shared__ double s_red[5][kMaxWarps];
    const int blk = blockIdx.x;
    const int inst = block_instance(bm, blk);
    const InstDev& I = insts[inst];
    if (threadIdx.x == 0) load_trial<double>(I.trial, I.ee_on, s_trial);
    __syncthreads();

    const int64_t id = (int64_t)(blk - bm.begin[inst]) * blockDim.x + threadIdx.x;
    const bool valid = id < I.n;
    double q[5] = {0, 0, 0, 0, 0};
    unsigned n_nonfinite = 0, n_node = 0;
    if (valid) {
        const int64_t slot = I.off + id;
        double xi[6], x[6];
        uint32_t words[6];
        init_words(I.id0 + (uint32_t)id, I.stream, I.k0, I.k1, words);
        normals6_f64(words, xi);
#pragma unroll
        for (int d = 0; d < 6; ++d) x[d] = I.sigma * xi[d];
        EvalOut<double> ev;
        eval_trial<KIND, double>(s_trial, x, ev);
        int sg = ev.sign;
        double logw = 0.0;
        if (sg == 0) {
            ++n_node;
        } else if (!eval_finite(ev)) {
            sg = 0;
            ++n_nonfinite;
        }
        if (sg == 0) {
            logw = -INFINITY;
        } else {
            q[0] = 1.0;
            q[1] = ev.el;
            q[2] = 1.0;
            q[3] = ev.el * ev.el;
            q[4] = 1.0;
        }
        if (f64_slot_ok(st, slot)) {
#pragma unroll
            for (int d = 0; d < 6; ++d) st.x[d * st.stride + slot] = x[d];
            st.logw[slot] = logw;
            st.sgn[slot] = (int8_t)sg;
        }
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < 5; ++k) {
        double v = warp_sum(q[k]);
        if (lane == 0) s_red[k][warp] = v;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double r[5] = {0, 0, 0, 0, 0};
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w)
            for (int k = 0; k < 5; ++k) r[k] += s_red[k][w];
        PartialRec rec;
        rec.c = 0.0;
        rec.W = r[0]; rec.P = r[1]; rec.Q = r[2]; rec.R = r[3]; rec.n = r[4];
        if (GFK_DBG_OK(part + blk, sizeof(PartialRec), kDbgRecord)) part[blk] = rec;
    }
    flush_counters(counters, inst, n_nonfinite, n_node, 0u);
}

template <int KIND, int NOISE>
__global__ void __launch_bounds__(kMaxThreads)
walk_fp64_kernel(const InstDev* __restrict__ insts, BlockMap bm, StateF64 st,
                 uint32_t step0, int nsteps, PartialRec* __restrict__ part, int nblk,
                 unsigned long long* __restrict__ counters) {
    __shared__ TrialDev<double> s_trial;
    __shared__ double s_ring[kRing][5][kMaxWarps];
    __shared__ double s_red[kMaxWarps];
    const int blk = blockIdx.x;
    const int inst = block_instance(bm, blk);
    const InstDev& I = insts[inst];
    if (threadIdx.x == 0) load_trial<double>(I.trial, I.ee_on, s_trial);
    __syncthreads();
    TrialDev<double> t_local;
    if (KIND == 0) t_local = s_trial;
    const TrialDev<double>& t = (KIND == 0) ? t_local : s_trial;

    const double dt = I.dt, sdt = I.sqrt_dt, et = I.e_trial;
    const uint32_t k0 = I.k0, k1 = I.k1, stream = I.stream;
    const int64_t id = (int64_t)(blk - bm.begin[inst]) * blockDim.x + threadIdx.x;
    const bool valid = id < I.n;
    const int64_t slot = I.off + id;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nwarps = blockDim.x >> 5;

    double x[6] = {0, 0, 0, 0, 0, 0};
    double logw = -INFINITY;
    int sg = 0;
    if (valid && f64_slot_ok(st, slot)) {
#pragma unroll
        for (int d = 0; d < 6; ++d) x[d] = st.x[d * st.stride + slot];
        logw = st.logw[slot];
        sg = st.sgn[slot];
    }
    EvalOut<double> ev;
    if (sg != 0) eval_trial<KIND, double>(t, x, ev);
    uint32_t lcg = NOISE == 1 ? superduper_at(I.id0 + (uint32_t)id, stream, k0, k1, step0) : 0u;
    unsigned n_nonfinite = 0, n_node = 0, n_coal = 0;
    double c = block_max_shift(sg != 0 ? logw : -INFINITY, s_red);

    for (int s = 0; s < nsteps; ++s) {
        const uint32_t step = step0 + (uint32_t)s;
        double q[5] = {0, 0, 0, 0, 0};
        if (sg != 0) {
            double xi[6];
            if (NOISE == 1) {
                bernoulli6<double>(lcg, xi);
            } else {
                uint32_t words[6];
                move_words(I.id0 + (uint32_t)id, step, stream, k0, k1, words);
                normals6_f64(words, xi);
            }
#pragma unroll
            for (int d = 0; d < 6; ++d) x[d] = x[d] + ev.b[d] * dt + sdt * xi[d];
            eval_trial<KIND, double>(t, x, ev);
            if (ev.rmin < 1e-10) ++n_coal;
            // a non-finite position is a non-finite kill, then a sign change a
            // node kill, then a non-finite drift or local energy
            bool node = ev.sign != sg;
            if (node) node = finite_(((x[0] + x[1]) + (x[2] + x[3])) + (x[4] + x[5]));
            if (node) {
                sg = 0;
                logw = -INFINITY;
                ++n_node;
            } else if (!eval_finite(ev)) {
                sg = 0;
                logw = -INFINITY;
                ++n_nonfinite;
            } else {
                logw = logw - (ev.el - et) * dt;
                double w = exp(logw - c);
                double we = w * ev.el;
                q[0] = w;
                q[1] = we;
                q[2] = w * w;
                q[3] = we * ev.el;
                q[4] = 1.0;
            }
        }
        const int r = s % kRing;
#pragma unroll
        for (int k = 0; k < 5; ++k) {
            double v = warp_sum(q[k]);
            if (lane == 0) s_ring[r][k][warp] = v;
        }
        if (r == kRing - 1 || s == nsteps - 1) {
            __syncthreads();
            const int rows = r + 1;
            if ((int)threadIdx.x < rows) {
                const int rr = threadIdx.x;
                double acc[5] = {0, 0, 0, 0, 0};
                for (int w = 0; w < nwarps; ++w)
#pragma unroll
                    for (int k = 0; k < 5; ++k) acc[k] += s_ring[rr][k][w];
                PartialRec rec;
                rec.c = c;
                rec.W = acc[0]; rec.P = acc[1]; rec.Q = acc[2]; rec.R = acc[3]; rec.n = acc[4];
                PartialRec* dst = part + (int64_t)(s - r + rr) * nblk + blk;
                if (GFK_DBG_OK(dst, sizeof(PartialRec), kDbgRecord)) *dst = rec;
            }
            c = block_max_shift(sg != 0 ? logw : -INFINITY, s_red);
        }
    }
    if (valid && f64_slot_ok(st, slot)) {
#pragma unroll
        for (int d = 0; d < 6; ++d) st.x[d * st.stride + slot] = x[d];
        st.logw[slot] = logw;
        st.sgn[slot] = (int8_t)sg;
    }
    flush_counters(counters, inst, n_nonfinite, n_node, n_coal);
}

// Host launchers (called from the C ABI layer).
cudaError_t launch_init_fp64(int kind, int threads, int nblk, const InstDev* insts,
                             const BlockMap& bm, const StateF64& st, PartialRec* part,
                             unsigned long long* counters, cudaStream_t stream) {
    if (kind == 0)
        init_fp64_kernel<0><<<nblk, threads, 0, stream>>>(insts, bm, st, part, nblk, counters);
    else if (kind == 1)
        init_fp64_kernel<1><<<nblk, threads, 0, stream>>>(insts, bm, st, part, nblk, counters);
    else
        init_fp64_kernel<2><<<nblk, threads, 0, stream>>>(insts, bm, st, part, nblk, counters);
    return cudaGetLastError();
}

template <int NOISE>
static void launch_walk_fp64_n(int kind, int threads, int nblk, const InstDev* insts,
                               const BlockMap& bm, const StateF64& st, uint32_t step0,
                               int nsteps, PartialRec* part, unsigned long long* counters,
                               cudaStream_t stream) {
    if (kind == 0)
        walk_fp64_kernel<0, NOISE><<<nblk, threads, 0, stream>>>(insts, bm, st, step0, nsteps,
                                                                 part, nblk, counters);
    else if (kind == 1)
        walk_fp64_kernel<1, NOISE><<<nblk, threads, 0, stream>>>(insts, bm, st, step0, nsteps,
                                                                 part, nblk, counters);
    else
        walk_fp64_kernel<2, NOISE><<<nblk, threads, 0, stream>>>(insts, bm, st, step0, nsteps,
                                                                 part, nblk, counters);
}

cudaError_t launch_walk_fp64(int kind, int noise, int threads, int nblk, const InstDev* insts,
                             const BlockMap& bm, const StateF64& st, uint32_t step0, int nsteps,
                             PartialRec* part, unsigned long long* counters,
                             cudaStream_t stream) {
    if (noise == GFK_NOISE_BERNOULLI)
        launch_walk_fp64_n<1>(kind, threads, nblk, insts, bm, st, step0, nsteps, part, counters,
                              stream);
    else
        launch_walk_fp64_n<0>(kind, threads, nblk, insts, bm, st, step0, nsteps, part, counters,
                              stream);
    return cudaGetLastError();
}

}  // namespace gfk
