// Mixed-precision walk: FP32 positions, drift, local energy and normals; FP64
// log-weights and FP64 population sums above the warp.
//
// Each thread advances WPT walkers (ids tid, tid + T, ... within the block's
// range, so every load and store is coalesced) for a whole chunk of steps with
// the state in registers.  Per step and walker (the discretised Eq. 4 and the
// drifted diffusion under it):
//   xi     <- six N(0,1): one Philox4x32-10 block per move, FP32 Box-Muller; or (NOISE = 1) six signs +-1 from the walker's
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
#include <type_traits>

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

// The debug build's check of a walker's slot in the state planes (true in the
// release build).
__device__ __forceinline__ bool mixed_slot_ok(const StateMixed& st, int64_t slot) {
    return GFK_DBG_OK(st.p0 + slot, sizeof(float4), kDbgState) &&
           GFK_DBG_OK(st.p1 + slot, sizeof(float4), kDbgState) &&
           GFK_DBG_OK(st.sgn + slot, 1, kDbgState);
}

__device__ __forceinline__ void store_mixed(const StateMixed& st, int64_t slot, const float x[6],
                                            double logw, int sg) {
    if (!mixed_slot_ok(st, slot)) return;
    const long long bits = __double_as_longlong(logw);
    st.p0[slot] = make_float4(x[0], x[1], x[2], x[3]);
    st.p1[slot] = make_float4(x[4], x[5], __int_as_float((int)(bits & 0xffffffffLL)),
                              __int_as_float((int)(bits >> 32)));
    st.sgn[slot] = (int8_t)sg;
}

// Positions of walker i after global move m in the trajectory planes
// (StateMixed::traj).  Streaming stores: the adjoint reads them back once,
// long after the walk has moved on.
__device__ __forceinline__ void store_traj(const StateMixed& st, uint32_t m, int64_t i,
                                           float x0, float x1, float x2, float x3, float x4,
                                           float x5) {
    float* pl = st.traj + (int64_t)m * 6 * st.traj_stride;
    if (!GFK_DBG_OK(reinterpret_cast<float4*>(pl) + i, sizeof(float4), kDbgPositions) ||
        !GFK_DBG_OK(reinterpret_cast<float2*>(pl + 4 * st.traj_stride) + i, sizeof(float2),
                    kDbgPositions))
        return;
    __stcs(reinterpret_cast<float4*>(pl) + i, make_float4(x0, x1, x2, x3));
    __stcs(reinterpret_cast<float2*>(pl + 4 * st.traj_stride) + i, make_float2(x4, x5));
}

__device__ __forceinline__ void load_mixed(const StateMixed& st, int64_t slot, float x[6],
                                           double& logw, int& sg) {
    if (!mixed_slot_ok(st, slot)) {
        for (int d = 0; d < 6; ++d) x[d] = 0.f;
        logw = -INFINITY;
        sg = 0;
        return;
    }
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
        if (GFK_DBG_OK(part + blk, sizeof(PartialRec), kDbgRecord)) part[blk] = rec;
    }
    flush_counters(counters, inst, n_nonfinite, n_node, 0u);
}

// PARAM: every instance the launch covers has the same trial function, which
// arrives as the kernel argument tk (constant-bank operands, no shared-memory
// loads, no registers); otherwise each block loads its instance's trial into
// shared memory (kind 0 then copies its parameters into registers).  The
// launcher uses PARAM whenever the launch covers one trial function, except
// for kind 0 with Bernoulli noise (kind 0, Gaussian noise, two packed walkers
// per thread: +0.9 %, 9.34 -> 9.26 ms per 1024-move launch of 2^20 walkers;
// Bernoulli noise: -1.0 %, 5.58 -> 5.63 ms; the orbital-pair kinds: +11 %).
//
// Lanes: the thread's walkers are evaluated in groups of two, the two lanes of
// a float2 (gfk_lanes.cuh: packed FP32 instructions, one issue slot for both
// walkers); with one walker per thread the same code runs on plain floats.
// Walker k of the thread is lane k % 2 of group k / 2.  Every walker moves on
// every step whether it is alive or not (no per-lane selects on the
// positions); a walker killed by a move has its position, a log-weight of
// -inf and a zero sign stored at that move, and only walkers alive at the end
// store their state then.
//
// CKPT: the gradient's forward.  It writes the position checkpoints
// (StateMixed::ckpt) at its folds, or the whole trajectory (StateMixed::traj)
// at every move, whichever of the two is set.
// Offset (floats) in a warp's staging area of the float4 of lane 16 half +
// lane15 for move m4 of a group of four.  The half-planes are padded so that
// the column sums' reads, which take one quantity of one move and half of the
// lanes per warp lane, fall in 32 distinct banks (8 m4 + 4 half + quantity).
__device__ __forceinline__ int stage_offset(int m4, int half, int lane15) {
    return m4 * kStageMove + half * kStageHalf + 4 * lane15;
}

template <int KIND, int WPT, int NOISE, bool PARAM, bool CKPT = false>
__global__ void __launch_bounds__(WPT == 4 ? kMaxThreadsWpt4 : kMaxThreads)
walk_mixed_kernel(const InstDev* __restrict__ insts, BlockMap bm, StateMixed st,
                  uint32_t step0, int nsteps, PartialRec* __restrict__ part, int nblk,
                  unsigned long long* __restrict__ counters, int blk0,
                  const __grid_constant__ TrialDev<float> tk) {
    using L = typename std::conditional<WPT == 1, float, float2>::type;
    constexpr int LW = LaneCount<L>::value;       // walkers per lane group
    constexpr int NG = WPT / LW;                   // lane groups per thread
    __shared__ TrialDev<float> s_trial;
    // the per-warp log-weight shift each ring buffer's window used
    __shared__ double s_shift[2][kMaxWarps];
    // dynamic shared memory (walk_smem_bytes):
    //   ring  [2][kRing][4][nwarps] float:  per-warp sums (W, P, Q, R), double-buffered
    //   cnt   [2][kRing][nwarps] unsigned:   per-warp alive counts
    //   stage [nwarps][4][2][kStageHalf] float: each lane's four sums of up to four
    //         moves, as one float4 per lane and move (stage_offset)
    //   angle [kAngleGrid] float2: Gaussian noise: the Box-Muller angle table
    extern __shared__ __align__(16) float s_dyn[];
    const int blk = blockIdx.x + blk0;       // a launch may cover a range of blocks
    const int inst = block_instance(bm, blk);
    const InstDev& I = insts[inst];
    if (!PARAM && threadIdx.x == 0) load_trial<float>(I.trial, I.ee_on, s_trial);
    float2* const s_cs = reinterpret_cast<float2*>(
        s_dyn + (2 * kRing * 5 + 4 * kStageMove) * (blockDim.x >> 5));
    if (NOISE == 0) {
        const float2* __restrict__ src = I.angle_cs;
        for (int i = threadIdx.x; i < kAngleGrid; i += blockDim.x) s_cs[i] = src[i];
    }
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
    const float r2_fix = I.r2_fix;
    const L dtL = splat<L>(I.dt_f32), sdtL = splat<L>(I.sdt_f32);
    const float sdt = I.sdt_f32, sdt_lo = I.sdt_lo;
    const float et = I.et_f32;
    const L etL = splat<L>(et);
    const double dt64 = I.dt;
    const double et_fix = I.et_fix;          // per-move E_T rounding, restored at each fold
    constexpr float kLog2e = 1.4426950408889634f;
    const L dtl2eL = splat<L>(I.dt_log2e);
    const uint32_t k0 = I.k0, k1 = I.k1;
    const int T = blockDim.x;
    const int lane_id = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nwarps = T >> 5;
    float* const s_ring = s_dyn;
    unsigned* const s_cnt = reinterpret_cast<unsigned*>(s_dyn + 2 * kRing * 4 * nwarps);
    float* const s_stage = s_dyn + 2 * kRing * 5 * nwarps + warp * 4 * kStageMove;

    PhiloxPre pre[WPT];
    uint32_t lcg[WPT];           // Bernoulli mode: generator state before this move
    int64_t slot[WPT];
    bool valid[WPT];
    double Lw[WPT];              // FP64 log-weight base
    int sg[WPT];
    L x[NG][6], b[NG][6];
    L S[NG], comp[NG], dsh[NG];  // dsh: (L - c) log2(e), formed at each fold (-inf: dead)
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
        slot[k] = I.off + id;
        sg[k] = 0;
        Lw[k] = -INFINITY;
        float xk[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        if (valid[k]) load_mixed(st, slot[k], xk, Lw[k], sg[k]);
        if (CKPT && st.traj != nullptr && step0 == 0u && valid[k])
            store_traj(st, 0u, slot[k] - I.off, xk[0], xk[1], xk[2], xk[3], xk[4], xk[5]);
#pragma unroll
        for (int d = 0; d < 6; ++d) set_lane(x[k / LW][d], k % LW, xk[d]);
    }
#pragma unroll
    for (int g = 0; g < NG; ++g) {
        // the drift at the start (unused by walkers that are dead)
        EvalLanes<L> ev;
        eval_lanes<KIND, L, PARAM, kPoly>(t, x[g], ev);
#pragma unroll
        for (int d = 0; d < 6; ++d) b[g][d] = ev.b[d];
        S[g] = splat<L>(0.f);
        comp[g] = splat<L>(0.f);
    }
    unsigned n_nonfinite = 0, n_node = 0, n_coal = 0;
    // per-warp shift: the warp's largest log-weight (0 if the warp has none alive)
    double lmaxw = -INFINITY;
#pragma unroll
    for (int k = 0; k < WPT; ++k)
        if (sg[k] != 0) lmaxw = fmax(lmaxw, Lw[k]);
    double c = warp_max(lmaxw);
    c = isfinite(c) ? floor(c) : 0.0;      // integer-valued shift
    // a dead walker's shift is -inf, so its weight 2^(-inf) is exactly 0
    // (its Kahan sum stays finite: its local energy is replaced by E_T)
    unsigned na_t = 0;             // the thread's walkers alive
#pragma unroll
    for (int k = 0; k < WPT; ++k) {
        set_lane(dsh[k / LW], k % LW, sg[k] != 0 ? (float)(Lw[k] - c) * kLog2e : -INFINITY);
        na_t += sg[k] != 0 ? 1u : 0u;
    }
    int fold_len = 0;
    int buf = 0;

    // One move of every walker of the thread from its increments xi (and the
    // Bernoulli steps' sub-ulp parts xlo), then its sums to the warp's staging
    // area and the warp's alive count to the ring.
    auto advance = [&](int s, L (&xi)[NG][6], L (&xlo)[NG][6]) {
        L q[4];
#pragma unroll
        for (int g = 0; g < NG; ++g) {
            if (NOISE == 1) {
#pragma unroll
                for (int j = 0; j < LW; ++j) {
                    float st6[6], lo6[6];
                    bernoulli6_steps(lcg[g * LW + j], sdt, sdt_lo, st6, lo6);   // +-sdt, +-sdt_lo
#pragma unroll
                    for (int d = 0; d < 6; ++d) {
                        set_lane(xi[g][d], j, st6[d]);
                        set_lane(xlo[g][d], j, lo6[d]);
                    }
                }
            }
            L xn[6];
#pragma unroll
            for (int d = 0; d < 6; ++d)
                xn[d] = NOISE == 1 ? move_bern_lanes(x[g][d], b[g][d], xi[g][d], xlo[g][d], dtL)
                                   : move_gauss_lanes(x[g][d], b[g][d], xi[g][d], dtL, sdtL);
            if (CKPT && st.traj != nullptr) {
                // the whole trajectory (gfk_grad's forward): every walker's
                // position after this move, dead ones included (the adjoint
                // skips walkers whose final weight is zero)
#pragma unroll
                for (int j = 0; j < LW; ++j)
                    if (valid[g * LW + j])
                        store_traj(st, step0 + (uint32_t)s + 1u, slot[g * LW + j] - I.off,
                                   lane_at(xn[0], j), lane_at(xn[1], j), lane_at(xn[2], j),
                                   lane_at(xn[3], j), lane_at(xn[4], j), lane_at(xn[5], j));
            }
            EvalLanes<L> ev;
            eval_lanes<KIND, L, PARAM, kPoly>(t, xn, ev);
            // A walker dies on a sign change of psi (or a psi of exactly 0) or
            // on a non-finite drift or local energy.  An infinite or NaN
            // coordinate needs no test of its own here: every evaluation forms
            // its directions from x rsqrt(s), s the squared distance, which is
            // NaN for such a coordinate, so the drift is NaN too.  The position
            // decides only how a kill is counted (a non-finite position is a
            // non-finite kill, then a sign change a node kill, then the rest),
            // which the rare branch below works out once per dead walker.
            const L fs = eval_check_sum(ev);
            L el = ev.el;
            // the coalescence diagnostic: walkers alive before the move that
            // land within 1e-5 bohr of a nucleus or of the other electron
            // (rare: counted per lane only when some lane of the thread did)
            float rm = lane_at(ev.rmin, 0);
#pragma unroll
            for (int j = 1; j < LW; ++j) rm = fminf(rm, lane_at(ev.rmin, j));
            if (rm < 1e-5f) {
#pragma unroll
                for (int j = 0; j < LW; ++j)
                    n_coal += (sg[g * LW + j] != 0 && lane_at(ev.rmin, j) < 1e-5f) ? 1u : 0u;
            }
            bool stay[LW];
#pragma unroll
            for (int j = 0; j < LW; ++j) {
                const int k = g * LW + j;
                const bool alive = sg[k] != 0;
                const bool flip = ev.sign[j] != sg[k];
                stay[j] = alive && !flip && finite_(lane_at(fs, j));
                if (alive && !stay[j]) {
                    // killed by this move: counted, and it stays here (stored now)
                    float xk[6];
#pragma unroll
                    for (int d = 0; d < 6; ++d) xk[d] = lane_at(xn[d], j);
                    const float xs = ladd(ladd(ladd(xk[0], xk[1]), ladd(xk[2], xk[3])),
                                          ladd(xk[4], xk[5]));
                    if (flip && finite_(xs)) ++n_node;
                    else ++n_nonfinite;
                    if (valid[k]) store_mixed(st, slot[k], xk, -INFINITY, 0);
                    sg[k] = 0;
                    set_lane(dsh[g], j, -INFINITY);
                    --na_t;
                }
                if (!stay[j]) set_lane(el, j, et);
            }
#pragma unroll
            for (int d = 0; d < 6; ++d) {
                x[g][d] = xn[d];
                b[g][d] = ev.b[d];
            }
            // Kahan: S accumulates E_L - E_T since the last fold
            const L y = lsub(lsub(el, etL), comp[g]);
            const L tsum = ladd(S[g], y);
            comp[g] = lsub(lsub(tsum, S[g]), y);
            S[g] = tsum;
            const L w = lex2(lfma(lneg(S[g]), dtl2eL, dsh[g]));   // 0 for the dead
            const L we = lmul(w, el);
            const L ww = lmul(w, w);
            const L wee = lmul(we, el);
            if (g == 0) {
                q[0] = w; q[1] = we; q[2] = ww; q[3] = wee;
            } else {
                q[0] = ladd(q[0], w); q[1] = ladd(q[1], we);
                q[2] = ladd(q[2], ww); q[3] = ladd(q[3], wee);
            }
        }
        // the thread's four sums (over its walkers: the lanes added last)
        float qs[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            float v = lane_at(q[u], 0);
#pragma unroll
            for (int j = 1; j < LW; ++j) v = v + lane_at(q[u], j);
            qs[u] = v;
        }
        // the lane's four sums go to the warp's staging area as one float4
        // (stage_offset: move of the group of four, half-warp, lane); every
        // fourth move, and at the end of a window, the warp adds each quantity
        // of each move over the lanes (half of the lanes per warp lane, the
        // halves joined by one shuffle) and writes the sums to the ring
        const int m4 = s & 3;
        *reinterpret_cast<float4*>(s_stage + stage_offset(m4, lane_id >> 4, lane_id & 15)) =
            make_float4(qs[0], qs[1], qs[2], qs[3]);
        const unsigned na = __reduce_add_sync(0xffffffffu, na_t);
        const int r = s % kRing;
        if (lane_id == 0) s_cnt[(buf * kRing + r) * nwarps + warp] = na;
        ++fold_len;
    };
    // After move s: the warp's column sums every fourth move, and the fold and
    // the block's records at the end of each kRing-move window.
    auto after = [&](int s) {
        const int m4 = s & 3;
        const int r = s % kRing;
        if (m4 == 3 || r == kRing - 1 || s == nsteps - 1) {
            __syncwarp();
            const int col = lane_id & 15, half = lane_id >> 4;
            const bool staged = (col >> 2) <= m4;
            float v = 0.f;
            if (staged) {
                // quantity col & 3 of move col >> 2, lanes 16 half + u
                const float* src = s_stage + stage_offset(col >> 2, half, 0) + (col & 3);
                float a0 = 0.f, a1 = 0.f, a2 = 0.f, a3 = 0.f;
#pragma unroll
                for (int u = 0; u < 16; u += 4) {
                    a0 += src[4 * u];
                    a1 += src[4 * (u + 1)];
                    a2 += src[4 * (u + 2)];
                    a3 += src[4 * (u + 3)];
                }
                v = (a0 + a1) + (a2 + a3);
            }
            v += __shfl_xor_sync(0xffffffffu, v, 16);
            if (half == 0 && staged)
                s_ring[((buf * kRing + r - m4 + (col >> 2)) * 4 + (col & 3)) * nwarps + warp] = v;
            __syncwarp();                        // the staging area is rewritten next move
        }
        if (r == kRing - 1 || s == nsteps - 1) {
            if (lane_id == 0) s_shift[buf][warp] = c;
            // fold the FP32 increments into the FP64 base; new per-warp shift
            lmaxw = -INFINITY;
#pragma unroll
            for (int k = 0; k < WPT; ++k) {
                const float Sk = lane_at(S[k / LW], k % LW), ck = lane_at(comp[k / LW], k % LW);
                if (sg[k] != 0) {
                    Lw[k] = Lw[k] - (((double)Sk - (double)ck) + (double)fold_len * et_fix) * dt64;
                    lmaxw = fmax(lmaxw, Lw[k]);
                } else {
                    Lw[k] = -INFINITY;
                }
            }
#pragma unroll
            for (int g = 0; g < NG; ++g) {
                S[g] = splat<L>(0.f);
                comp[g] = splat<L>(0.f);
            }
            fold_len = 0;
            c = warp_max(lmaxw);
            c = isfinite(c) ? floor(c) : 0.0;
#pragma unroll
            for (int k = 0; k < WPT; ++k)
                set_lane(dsh[k / LW], k % LW, sg[k] != 0 ? (float)(Lw[k] - c) * kLog2e : -INFINITY);
            // position checkpoint (StateMixed::ckpt) after move s, in the
            // gradient's forward kernels (CKPT) when it is set.  Walkers that are
            // dead by then keep moving and write meaningless positions, which the
            // adjoint never reads (their final weight is zero).
            if (CKPT && st.ckpt != nullptr) {
                const uint32_t done = step0 + (uint32_t)s + 1u;
                const uint32_t jc = done / (uint32_t)st.ckpt_every;
                if (done % (uint32_t)st.ckpt_every == 0u && jc >= 1u && jc < (uint32_t)st.ckpt_count) {
                    float4* base = st.ckpt + (int64_t)jc * 2 * st.ckpt_slots;
#pragma unroll
                    for (int k = 0; k < WPT; ++k) {
                        if (!valid[k]) continue;
                        if (!GFK_DBG_OK(base + slot[k], sizeof(float4), kDbgPositions) ||
                            !GFK_DBG_OK(base + st.ckpt_slots + slot[k], sizeof(float4),
                                        kDbgPositions))
                            continue;
                        const int g = k / LW, j = k % LW;
                        base[slot[k]] = make_float4(lane_at(x[g][0], j), lane_at(x[g][1], j),
                                                    lane_at(x[g][2], j), lane_at(x[g][3], j));
                        base[st.ckpt_slots + slot[k]] =
                            make_float4(lane_at(x[g][4], j), lane_at(x[g][5], j), 0.f, 0.f);
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
                        for (int u = 0; u < 4; ++u) {
                            const float fk = u == 2 ? f * f : f;
                            acc[u] += (double)(ring[u * nwarps + w] * fk);
                        }
                    }
                } else {
                    cb = 0.0;
                }
                PartialRec rec;
                rec.c = cb;
                rec.W = acc[0]; rec.P = acc[1]; rec.Q = acc[2]; rec.R = acc[3];
                rec.n = (double)n_alive;
                PartialRec* dst = part + (int64_t)(s - r + rr) * nblk + blk;
                if (GFK_DBG_OK(dst, sizeof(PartialRec), kDbgRecord)) *dst = rec;
            }
            buf ^= 1;
        }
    };

    int s = 0;
    if (NOISE == 0) {
        // Gaussian noise: two moves per iteration.  Each move's Philox block is
        // drawn without a branch, and the second move's words and normals are
        // independent of the first move's arithmetic, which the scheduler can
        // interleave with them.  s is even after the first move of a pair, so
        // there is no column sum, fold or end of launch between the two.
        for (; s + 1 < nsteps; s += 2) {
            uint32_t wa[WPT][6], wb[WPT][6];
            move_words_all<WPT>(pre, step0 + (uint32_t)s, k0, k1, wa);
            move_words_all<WPT>(pre, step0 + (uint32_t)s + 1u, k0, k1, wb);
            L xa[NG][6], xb[NG][6], xlo[NG][6];
#pragma unroll
            for (int g = 0; g < NG; ++g) {
                normals6_lanes<L>(&wa[g * LW], xa[g], r2_fix, s_cs);
                normals6_lanes<L>(&wb[g * LW], xb[g], r2_fix, s_cs);
            }
            advance(s, xa, xlo);
            advance(s + 1, xb, xlo);
            after(s + 1);
        }
    }
    for (; s < nsteps; ++s) {
        const uint32_t step = step0 + (uint32_t)s;
        // Gaussian noise: the normals of all walkers first; the Bernoulli steps
        // are drawn per group.
        L xi[NG][6], xlo[NG][6];
        if (NOISE == 0) {
            uint32_t words[WPT][6];
            move_words_all<WPT>(pre, step, k0, k1, words);
#pragma unroll
            for (int g = 0; g < NG; ++g) normals6_lanes<L>(&words[g * LW], xi[g], r2_fix, s_cs);
        }
        advance(s, xi, xlo);
        after(s);
    }
    // walkers alive now store their state (the ones killed during the launch
    // were stored when they died; dead ones are unchanged in memory)
#pragma unroll
    for (int k = 0; k < WPT; ++k) {
        if (!valid[k] || sg[k] == 0) continue;
        float xk[6];
#pragma unroll
        for (int d = 0; d < 6; ++d) xk[d] = lane_at(x[k / LW][d], k % LW);
        store_mixed(st, slot[k], xk, Lw[k], sg[k]);
    }
    flush_counters(counters, inst, n_nonfinite, n_node, n_coal);
}

// Dynamic shared memory of the walk kernel for `threads` threads per block.
static size_t walk_smem_bytes(int threads, int noise) {
    const size_t nwarps = (size_t)threads / 32;
    return 4 * (2 * kRing * 5 * nwarps + nwarps * 4 * kStageMove) +
           (noise == 0 ? sizeof(float2) * kAngleGrid : 0);
}

// run = false only prepares the kernel (the shared-memory opt-in), so that it
// can happen before a stream capture rather than inside it.
template <int NOISE, typename K>
static void launch_walk(K kernel, int nblk, int blk0, int grid, int threads, cudaStream_t stream,
                        const InstDev* insts, const BlockMap& bm, const StateMixed& st,
                        uint32_t step0, int nsteps, PartialRec* part,
                        unsigned long long* counters, const TrialDev<float>& tk, bool run) {
    const size_t smem = walk_smem_bytes(threads, NOISE);
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
            launch_walk<NOISE>(walk_mixed_kernel<KIND, 1, NOISE, PARAM, CKPT>, nblk, blk0, grid, threads, stream,
                        insts, bm, st, step0, nsteps, part, counters, tk, run);
            break;
        case 2:
            launch_walk<NOISE>(walk_mixed_kernel<KIND, 2, NOISE, PARAM, CKPT>, nblk, blk0, grid, threads, stream,
                        insts, bm, st, step0, nsteps, part, counters, tk, run);
            break;
        default:
            launch_walk<NOISE>(walk_mixed_kernel<KIND, 4, NOISE, PARAM, CKPT>, nblk, blk0, grid, threads, stream,
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
    if (st.ckpt != nullptr || st.traj != nullptr) {
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
    if (one_trial && kind == 0 && NOISE == 0)
        launch_walk_mixed_k<0, NOISE, true>(wpt, threads, nblk, blk0, grid, insts, bm, st, step0, nsteps,
                                            part, counters, tk, stream, run);
    else if (one_trial && kind == 1) {
        // a two-term trial (the P_z pair) takes the kernel whose term loops are
        // fixed at two; preparing (run = false) readies both kernels
        if (one_trial->nterms == 2 || !run)
            launch_walk_mixed_k<4, NOISE, true>(wpt, threads, nblk, blk0, grid, insts, bm, st, step0,
                                                nsteps, part, counters, tk, stream, run);
        if (one_trial->nterms != 2 || !run)
            launch_walk_mixed_k<1, NOISE, true>(wpt, threads, nblk, blk0, grid, insts, bm, st, step0,
                                                nsteps, part, counters, tk, stream, run);
    }
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
