// Mixed-precision walk: FP32 positions, drift, local energy and normals; FP64
// log-weights and FP64 population sums above the warp.
//
// Each thread advances WPT walkers (ids tid, tid + T, ... within the block's
// range, so every load and store is coalesced) for a whole chunk of steps with
// the state in registers.  Per step and walker (the discretised Eq. 4 and the
// drifted diffusion under it):
//   xi     <- six N(0,1): Philox4x32-10 words (three blocks serve two moves),
//             FP32 Box-Muller; or (NOISE = 1) six signs +-1 from the walker's
//             Superduper generator, skipped ahead to the launch's first move
//   X      <- X + (b dt + sqrt(dt) xi)   (FP32, the increment formed first;
//             Bernoulli: X + ((b dt +- s_lo) +- s), gfk_device.cuh)
//   b, E_L <- trial function at X in the cusp-cancelled form (FP32)
//   node   :  sign psi changed or psi = 0 -> killed
//   S      <- S + (E_L - E_T)            (FP32 Kahan sum since the last fold)
//   w      =  2^{(d - S dt) log2 e}      (d = FP64 base minus the warp's shift)
// Every kRing steps the FP32 sums are folded into the FP64 base,
//   L <- L - (S + kRing (E_T,fp32 - E_T)) dt            (FP64),
// the warp's shift c is reset to the floor of its largest L and d = (float)(L - c).
// Per step each lane stages its (w, w E_L, w^2, w E_L^2) in shared memory and
// the warp counts its live walkers; every fourth step the warp adds the staged
// columns in FP32.  Every kRing steps, after one block barrier, the block
// rescales each warp's sums to the block's largest shift and adds them in FP64,
// writing one PartialRec per step; a deferred kernel merges the blocks.  The
// FP32 constants (dt, sqrt(dt), the Box-Muller radius constant, E_T) come from
// the host (gfk_mixed_consts.h), chosen so that the diffusion matches the drift.
#pragma once

#include <cuda_runtime.h>

#include <cstring>

#include "gfk_block.cuh"
#include "gfk_device.cuh"
#include "gfk_launch.h"
#include "gfk_types.h"

namespace gfk {

__device__ __forceinline__ float ex2_approx(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__device__ __forceinline__ void store_mixed(const StateMixed& st, int64_t slot, const float x[6],
                                            double logw, int sg) {
    const long long bits = __double_as_longlong(logw);
    st.p0[slot] = make_float4(x[0], x[1], x[2], x[3]);
    st.p1[slot] = make_float4(x[4], x[5], __int_as_float((int)(bits & 0xffffffffLL)),
                              __int_as_float((int)(bits >> 32)));
    st.sgn[slot] = (int8_t)sg;
}

__device__ __forceinline__ void load_mixed(const StateMixed& st, int64_t slot, float x[6],
                                           double& logw, int& sg) {
    const float4 a = st.p0[slot];
    const float4 b = st.p1[slot];
    x[0] = a.x; x[1] = a.y; x[2] = a.z; x[3] = a.w; x[4] = b.x; x[5] = b.y;
    const long long lo = (unsigned)__float_as_int(b.z);
    const long long hi = (long long)__float_as_int(b.w);
    logw = __longlong_as_double((hi << 32) | lo);
    sg = st.sgn[slot];
}

template <int KIND>
__global__ void __launch_bounds__(kMaxThreads)
init_mixed_kernel(const InstDev* __restrict__ insts, BlockMap bm, StateMixed st,
                  PartialRec* __restrict__ part, int nblk,
                  unsigned long long* __restrict__ counters) {
    __shared__ TrialDev<float> s_trial;
    __shared__ double s_red[5][kMaxWarps];
    const int blk = blockIdx.x;
    const int inst = block_instance(bm, blk);
    const InstDev& I = insts[inst];
    if (threadIdx.x == 0) load_trial<float>(I.trial, I.ee_on, s_trial);
    __syncthreads();
    const int T = blockDim.x;
    double q[5] = {0, 0, 0, 0, 0};
    unsigned n_nonfinite = 0, n_node = 0;
    for (int k = 0; k < bm.wpt; ++k) {
        const int64_t id = (int64_t)(blk - bm.begin[inst]) * T * bm.wpt + (int64_t)k * T + threadIdx.x;
        if (id >= I.n) continue;
        // the initial positions are drawn in FP64, exactly as on the FP64 path,
        // then rounded: both paths start from the same population
        double xi[6];
        uint32_t words[6];
        init_words(I.id0 + (uint32_t)id, I.stream, I.k0, I.k1, words);
        normals6_f64(words, xi);
        float x[6];
#pragma unroll
        for (int d = 0; d < 6; ++d) x[d] = (float)(I.sigma * xi[d]);
        EvalOut<float> ev;
        eval_trial<KIND, float>(s_trial, x, ev);
        int sg = ev.sign;
        if (sg == 0) {
            ++n_node;
        } else if (!eval_finite(ev)) {
            sg = 0;
            ++n_nonfinite;
        }
        double logw = -INFINITY;
        if (sg != 0) {
            logw = 0.0;
            q[0] += 1.0;
            q[1] += (double)ev.el;
            q[2] += 1.0;
            q[3] += (double)ev.el * (double)ev.el;
            q[4] += 1.0;
        }
        store_mixed(st, I.off + id, x, logw, sg);
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
        for (int w = 0; w < (T >> 5); ++w)
            for (int k = 0; k < 5; ++k) r[k] += s_red[k][w];
        PartialRec rec;
        rec.c = 0.0;
        rec.W = r[0]; rec.P = r[1]; rec.Q = r[2]; rec.R = r[3]; rec.n = r[4];
        part[blk] = rec;
    }
    flush_counters(counters, inst, n_nonfinite, n_node, 0u);
}

// PARAM: every instance the launch covers has the same trial function, which
// arrives as the kernel argument tk (constant-bank operands, no shared-memory
// loads, no registers); otherwise each block loads its instance's trial into
// shared memory (kind 0 then copies its 16 parameters into registers).  The
// launcher uses PARAM for the orbital-pair kinds only: it speeds them up by
// ~11 % and slows the kind-0 walk by ~2 % against the register copy.
template <int KIND, int WPT, int NOISE, bool PARAM, bool CKPT = false>
__global__ void __launch_bounds__(kMaxThreads)
walk_mixed_kernel(const InstDev* __restrict__ insts, BlockMap bm, StateMixed st,
                  uint32_t step0, int nsteps, PartialRec* __restrict__ part, int nblk,
                  unsigned long long* __restrict__ counters, int blk0,
                  const __grid_constant__ TrialDev<float> tk) {
    __shared__ TrialDev<float> s_trial;
    // the per-warp log-weight shift each ring buffer's window used
    __shared__ double s_shift[2][kMaxWarps];
    // dynamic shared memory (walk_smem_bytes):
    //   ring  [2][kRing][4][nwarps] float:  per-warp sums (W, P, Q, R), double-buffered
    //   cnt   [2][kRing][nwarps] unsigned:   per-warp alive counts
    //   stage [nwarps][16][kStageStride] float: each lane's four sums of up to four moves
    extern __shared__ float s_dyn[];
    const int blk = blockIdx.x + blk0;       // a launch may cover a range of blocks
    const int inst = block_instance(bm, blk);
    const InstDev& I = insts[inst];
    if (!PARAM && threadIdx.x == 0) load_trial<float>(I.trial, I.ee_on, s_trial);
    __syncthreads();
    TrialDev<float> t_local;
    if (!PARAM && KIND == 0) t_local = s_trial;
    const TrialDev<float>& t = PARAM ? tk : ((KIND == 0) ? t_local : s_trial);
    // the specialised kinds run trial functions without Jastrow polynomial
    // terms only (mixed_walk_kind); the per-block dispatch handles the rest
    constexpr int kPoly = KIND == 2 ? -1 : 0;

    // FP32 time step, noise scale and radius constant chosen on the host so the
    // diffusion matches the drift, and the other derived constants, all formed
    // on the host (gfk_mixed_consts.h)
    const float dt = I.dt_f32, sdt = I.sdt_f32, sdt_lo = I.sdt_lo, r2_fix = I.r2_fix;
    const float et = I.et_f32;
    const double dt64 = I.dt;
    const double et_fix = I.et_fix;          // per-move E_T rounding, restored at each fold
    constexpr float kLog2e = 1.4426950408889634f;
    const float dt_log2e = I.dt_log2e;
    const uint32_t k0 = I.k0, k1 = I.k1;
    const int T = blockDim.x;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nwarps = T >> 5;
    float* const s_ring = s_dyn;
    unsigned* const s_cnt = reinterpret_cast<unsigned*>(s_dyn + 2 * kRing * 4 * nwarps);
    float* const s_stage = s_dyn + 2 * kRing * 5 * nwarps + warp * 16 * kStageStride;

    PhiloxPre pre[WPT];
    uint32_t carry[WPT][2];      // tag-1 words 2-3 of the even move, used by the odd one
    uint32_t lcg[WPT];           // Bernoulli mode: generator state before this move
    int64_t slot[WPT];
    bool valid[WPT];
    float x[WPT][6], b[WPT][6];
    double L[WPT];
    float dsh[WPT], S[WPT], comp[WPT];   // dsh: (L - c) log2(e), formed at each fold
    int sg[WPT];
#pragma unroll
    for (int k = 0; k < WPT; ++k) {
        const int64_t id = (int64_t)(blk - bm.begin[inst]) * T * WPT + (int64_t)k * T + threadIdx.x;
        valid[k] = id < I.n;
        if (NOISE == 0) {
            pre[k] = philox_pre(I.id0 + (uint32_t)id, I.stream, k0, k1);
            lcg[k] = 0u;
        } else {
            lcg[k] = superduper_at(I.id0 + (uint32_t)id, I.stream, k0, k1, step0);
        }
        carry[k][0] = carry[k][1] = 0u;
        slot[k] = I.off + id;
        sg[k] = 0;
        L[k] = -INFINITY;
#pragma unroll
        for (int d = 0; d < 6; ++d) { x[k][d] = 0.f; b[k][d] = 0.f; }
        if (valid[k]) load_mixed(st, slot[k], x[k], L[k], sg[k]);
        if (sg[k] != 0) {
            EvalOut<float> ev;
            eval_trial<KIND, float, PARAM, kPoly>(t, x[k], ev);
#pragma unroll
            for (int d = 0; d < 6; ++d) b[k][d] = ev.b[d];
        }
        S[k] = 0.f;
        comp[k] = 0.f;
    }
    unsigned n_nonfinite = 0, n_node = 0, n_coal = 0;
    // per-warp shift: the warp's largest log-weight (0 if the warp has none alive)
    double lmax = -INFINITY;
#pragma unroll
    for (int k = 0; k < WPT; ++k)
        if (sg[k] != 0) lmax = fmax(lmax, L[k]);
    double c = warp_max(lmax);
    c = isfinite(c) ? floor(c) : 0.0;      // integer-valued shift
#pragma unroll
    for (int k = 0; k < WPT; ++k) dsh[k] = sg[k] != 0 ? (float)(L[k] - c) * kLog2e : 0.f;
    int fold_len = 0;
    int buf = 0;

    for (int s = 0; s < nsteps; ++s) {
        const uint32_t step = step0 + (uint32_t)s;
        float q0 = 0.f, q1 = 0.f, q2 = 0.f, q3 = 0.f;
        unsigned na = 0;
        // Gaussian noise: the normals of all WPT walkers first (the Philox
        // words under one even / odd branch), so the moves that follow are one
        // branch-free stretch (+2.4 % against drawing each walker's words in
        // its own iteration); the Bernoulli steps, branch-free already, are
        // drawn per walker (0.6 % faster there).  Every walker slot runs the
        // same instructions (dead or past the end included) so the compiler
        // can interleave the WPT walkers; only the commit of the new state is
        // predicated.
        float xi[WPT][6], xlo[WPT][6];
        if (NOISE == 0) {
            uint32_t words[WPT][6];
            pair_move_words_all<WPT>(pre, carry, step, s == 0, k0, k1, words);
#pragma unroll
            for (int k = 0; k < WPT; ++k) normals6_f32(words[k], xi[k], r2_fix);
        }
#pragma unroll
        for (int k = 0; k < WPT; ++k) {
            const bool alive = sg[k] != 0;
            float xn[6];
            if (NOISE == 1)
                bernoulli6_steps(lcg[k], sdt, sdt_lo, xi[k], xlo[k]);   // +-sdt, +-sdt_lo
#pragma unroll
            for (int d = 0; d < 6; ++d)
                xn[d] = NOISE == 1 ? move_bern_f32(x[k][d], b[k][d], xi[k][d], xlo[k][d], dt)
                                   : move_gauss_f32(x[k][d], b[k][d], xi[k][d], dt, sdt);
            EvalOut<float> ev;
            eval_trial<KIND, float, PARAM, kPoly>(t, xn, ev);
            // a non-finite position is a non-finite kill, then a sign change a
            // node kill, then a non-finite drift or local energy (the position
            // test runs every move, without a branch: +0.4 to +1.3 % against
            // testing it only after a sign change, bitwise the same)
            const bool node = (ev.sign != sg[k]) &
                              finite_(((xn[0] + xn[1]) + (xn[2] + xn[3])) + (xn[4] + xn[5]));
            const bool fin = eval_finite(ev);
            const bool stay = alive && !node && fin;
            n_coal += (alive && ev.rmin < 1e-5f) ? 1u : 0u;
            n_node += (alive && node) ? 1u : 0u;
            n_nonfinite += (alive && !node && !fin) ? 1u : 0u;
#pragma unroll
            for (int d = 0; d < 6; ++d) {
                x[k][d] = alive ? xn[d] : x[k][d];      // a walker killed now stays here
                b[k][d] = ev.b[d];                      // read only while the walker lives
            }
            sg[k] = stay ? sg[k] : 0;
            // Kahan: S accumulates E_L - E_T since the last fold
            const float el = stay ? ev.el : et;
            const float y = (el - et) - comp[k];
            const float tsum = S[k] + y;
            comp[k] = (tsum - S[k]) - y;
            S[k] = tsum;
            const float w = stay ? ex2_approx(fmaf(-S[k], dt_log2e, dsh[k])) : 0.f;
            const float we = w * el;
            q0 += w;
            q1 += we;
            q2 += w * w;
            q3 += we * el;
            na += stay ? 1u : 0u;
        }
        // the lane's four sums go to the warp's staging rows (column = move of
        // the group x 4 + quantity); every fourth move, and at the end of a
        // window, the warp adds the columns up (half a column per lane, the
        // halves joined by one shuffle) and writes them to the ring
        const int m4 = s & 3;
        s_stage[(m4 * 4 + 0) * kStageStride + lane] = q0;
        s_stage[(m4 * 4 + 1) * kStageStride + lane] = q1;
        s_stage[(m4 * 4 + 2) * kStageStride + lane] = q2;
        s_stage[(m4 * 4 + 3) * kStageStride + lane] = q3;
        na = __reduce_add_sync(0xffffffffu, na);
        const int r = s % kRing;
        if (lane == 0) s_cnt[(buf * kRing + r) * nwarps + warp] = na;
        if (m4 == 3 || r == kRing - 1 || s == nsteps - 1) {
            __syncwarp();
            const int col = lane & 15, half = lane >> 4;
            const bool staged = (col >> 2) <= m4;
            float v = 0.f;
            if (staged) {
                const float* src = s_stage + col * kStageStride + 16 * half;
                float a0 = 0.f, a1 = 0.f, a2 = 0.f, a3 = 0.f;
#pragma unroll
                for (int t = 0; t < 16; t += 4) {
                    a0 += src[t];
                    a1 += src[t + 1];
                    a2 += src[t + 2];
                    a3 += src[t + 3];
                }
                v = (a0 + a1) + (a2 + a3);
            }
            v += __shfl_xor_sync(0xffffffffu, v, 16);
            if (half == 0 && staged)
                s_ring[((buf * kRing + r - m4 + (col >> 2)) * 4 + (col & 3)) * nwarps + warp] = v;
            __syncwarp();                        // the staging rows are rewritten next move
        }
        ++fold_len;
        if (r == kRing - 1 || s == nsteps - 1) {
            if (lane == 0) s_shift[buf][warp] = c;
            // fold the FP32 increments into the FP64 base; new per-warp shift
            lmax = -INFINITY;
#pragma unroll
            for (int k = 0; k < WPT; ++k) {
                if (sg[k] != 0) {
                    L[k] = L[k] - (((double)S[k] - (double)comp[k]) + (double)fold_len * et_fix) * dt64;
                    lmax = fmax(lmax, L[k]);
                } else {
                    L[k] = -INFINITY;
                }
                S[k] = 0.f;
                comp[k] = 0.f;
            }
            fold_len = 0;
            c = warp_max(lmax);
            c = isfinite(c) ? floor(c) : 0.0;
#pragma unroll
            for (int k = 0; k < WPT; ++k) dsh[k] = sg[k] != 0 ? (float)(L[k] - c) * kLog2e : 0.f;
            // position checkpoint (StateMixed::ckpt) after move step; compiled
            // into the gradient's forward kernels only (CKPT), since the extra
            // code at the fold slowed the other walks by up to 1.7 %
            if (CKPT) {
                const uint32_t done = step + 1u;
                const uint32_t j = done / (uint32_t)st.ckpt_every;
                if (done % (uint32_t)st.ckpt_every == 0u && j >= 1u && j < (uint32_t)st.ckpt_count) {
                    float4* base = st.ckpt + (int64_t)j * 2 * st.ckpt_slots;
#pragma unroll
                    for (int k = 0; k < WPT; ++k) {
                        if (!valid[k]) continue;
                        base[slot[k]] = make_float4(x[k][0], x[k][1], x[k][2], x[k][3]);
                        base[st.ckpt_slots + slot[k]] = make_float4(x[k][4], x[k][5], 0.f, 0.f);
                    }
                }
            }
            // one barrier per window: the other buffer takes the next window,
            // and nobody writes this one again before the next barrier
            __syncthreads();
            const int rows = r + 1;
            if ((int)threadIdx.x < rows) {
                const int rr = threadIdx.x;
                double cb = -INFINITY;
                const unsigned* cnt = s_cnt + (buf * kRing + rr) * nwarps;
                const float* ring = s_ring + (buf * kRing + rr) * 4 * nwarps;
                for (int w = 0; w < nwarps; ++w)
                    if (cnt[w] != 0u) cb = fmax(cb, s_shift[buf][w]);
                double acc[4] = {0, 0, 0, 0};
                unsigned n_alive = 0;
                if (isfinite(cb)) {
                    for (int w = 0; w < nwarps; ++w) {
                        const unsigned nw = cnt[w];
                        if (nw == 0u) continue;
                        n_alive += nw;
                        // warp shift relative to the block's: exact in FP64, then
                        // the factor in FP32 (it multiplies FP32 warp sums)
                        const float f = ex2_approx((float)(s_shift[buf][w] - cb) * kLog2e);
#pragma unroll
                        for (int k = 0; k < 4; ++k) {
                            const float fk = k == 2 ? f * f : f;
                            acc[k] += (double)(ring[k * nwarps + w] * fk);
                        }
                    }
                } else {
                    cb = 0.0;
                }
                PartialRec rec;
                rec.c = cb;
                rec.W = acc[0]; rec.P = acc[1]; rec.Q = acc[2]; rec.R = acc[3];
                rec.n = (double)n_alive;
                part[(int64_t)(s - r + rr) * nblk + blk] = rec;
            }
            buf ^= 1;
        }
    }
#pragma unroll
    for (int k = 0; k < WPT; ++k)
        if (valid[k]) store_mixed(st, slot[k], x[k], sg[k] != 0 ? L[k] : -INFINITY, sg[k]);
    flush_counters(counters, inst, n_nonfinite, n_node, n_coal);
}

// Dynamic shared memory of the walk kernel for `threads` threads per block.
static size_t walk_smem_bytes(int threads) {
    const size_t nwarps = (size_t)threads / 32;
    return 4 * (2 * kRing * 5 * nwarps + nwarps * 16 * kStageStride);
}

// run = false only prepares the kernel (the shared-memory opt-in), so that it
// can happen before a stream capture rather than inside it.
template <typename K>
static void launch_walk(K kernel, int nblk, int blk0, int grid, int threads, cudaStream_t stream,
                        const InstDev* insts, const BlockMap& bm, const StateMixed& st,
                        uint32_t step0, int nsteps, PartialRec* part,
                        unsigned long long* counters, const TrialDev<float>& tk, bool run) {
    const size_t smem = walk_smem_bytes(threads);
    if (smem > 48 * 1024)       // above the default limit (512-thread blocks): opt in
        cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (run)
        kernel<<<grid, threads, smem, stream>>>(insts, bm, st, step0, nsteps, part, nblk,
                                                counters, blk0, tk);
}

template <int KIND, int NOISE, bool PARAM, bool CKPT = false>
static void launch_walk_mixed_k(int wpt, int threads, int nblk, int blk0, int grid,
                                const InstDev* insts,
                                const BlockMap& bm, const StateMixed& st, uint32_t step0,
                                int nsteps, PartialRec* part, unsigned long long* counters,
                                const TrialDev<float>& tk, cudaStream_t stream, bool run) {
    switch (wpt) {
        case 1:
            launch_walk(walk_mixed_kernel<KIND, 1, NOISE, PARAM, CKPT>, nblk, blk0, grid, threads, stream,
                        insts, bm, st, step0, nsteps, part, counters, tk, run);
            break;
        case 2:
            launch_walk(walk_mixed_kernel<KIND, 2, NOISE, PARAM, CKPT>, nblk, blk0, grid, threads, stream,
                        insts, bm, st, step0, nsteps, part, counters, tk, run);
            break;
        default:
            launch_walk(walk_mixed_kernel<KIND, 4, NOISE, PARAM, CKPT>, nblk, blk0, grid, threads, stream,
                        insts, bm, st, step0, nsteps, part, counters, tk, run);
            break;
    }
}

template <int NOISE>
void launch_walk_mixed_n(int kind, int wpt, int threads, int nblk, int blk0, int grid,
                         const InstDev* insts,
                                const BlockMap& bm, const StateMixed& st, uint32_t step0,
                                int nsteps, PartialRec* part, unsigned long long* counters,
                                const TrialHost* one_trial, int ee_on, cudaStream_t stream,
                                bool run) {
    TrialDev<float> tk;
    std::memset(&tk, 0, sizeof(tk));
    if (one_trial) load_trial<float>(*one_trial, ee_on, tk);
    if (st.ckpt != nullptr) {
        // gfk_grad's forward: kind 0, or the per-block dispatch for a trial
        // function with Jastrow polynomial terms
        if (kind == 0)
            launch_walk_mixed_k<0, NOISE, false, true>(wpt, threads, nblk, blk0, grid, insts, bm, st,
                                                       step0, nsteps, part, counters, tk, stream, run);
        else
            launch_walk_mixed_k<2, NOISE, false, true>(wpt, threads, nblk, blk0, grid, insts, bm, st,
                                                       step0, nsteps, part, counters, tk, stream, run);
        return;
    }
    if (one_trial && kind == 1)
        launch_walk_mixed_k<1, NOISE, true>(wpt, threads, nblk, blk0, grid, insts, bm, st, step0, nsteps,
                                            part, counters, tk, stream, run);
    else if (one_trial && kind == 3)
        launch_walk_mixed_k<3, NOISE, true>(wpt, threads, nblk, blk0, grid, insts, bm, st, step0, nsteps,
                                            part, counters, tk, stream, run);
    else if (kind == 3)
        launch_walk_mixed_k<3, NOISE, false>(wpt, threads, nblk, blk0, grid, insts, bm, st, step0, nsteps,
                                             part, counters, tk, stream, run);
    else if (kind == 0)
        launch_walk_mixed_k<0, NOISE, false>(wpt, threads, nblk, blk0, grid, insts, bm, st, step0, nsteps,
                                             part, counters, tk, stream, run);
    else if (kind == 1)
        launch_walk_mixed_k<1, NOISE, false>(wpt, threads, nblk, blk0, grid, insts, bm, st, step0, nsteps,
                                             part, counters, tk, stream, run);
    else
        launch_walk_mixed_k<2, NOISE, false>(wpt, threads, nblk, blk0, grid, insts, bm, st, step0, nsteps,
                                             part, counters, tk, stream, run);
}

}  // namespace gfk
