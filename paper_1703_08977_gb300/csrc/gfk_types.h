// Plain structs shared by the host launch code and the kernels of the GFK
// library (device memory layouts and kernel arguments).
#pragma once

#include <cstdint>

#include <vector_types.h>

#include "gfk.h"   // include/ is on the include path
#include "gfk_debug.h"

namespace gfk {

// Trial function in FP64 as given by the caller (see gfk_set_trial).
struct TrialHost {
    int32_t kind;       // gfk_trial_kind
    int32_t nterms;     // kind 1: number of orbital-pair terms
    double Z;           // kind 0: orbital exponent
    double a, beta;     // Jastrow a rho + sum c_k rho^{k+1}, rho = r/(1+beta r)
    double ck[4];
    double s[GFK_MAX_TERMS];                 // kind 1: term signs / weights
    double alpha[GFK_MAX_TERMS][2];          // [term][electron]
    double c0[GFK_MAX_TERMS][2];
    double c1[GFK_MAX_TERMS][2];
    double cz[GFK_MAX_TERMS][2];
};

// One instance as the kernels see it.
struct InstDev {
    int64_t n;          // walkers
    int64_t off;        // first slot of this instance in the state planes
    double dt, sqrt_dt, e_trial, sigma;
    uint32_t k0, k1;    // Philox key = seed
    uint32_t stream;    // third Philox counter word
    uint32_t id0;       // Philox id of the instance's first walker
    int32_t ee_on;
    int32_t noise;      // gfk_noise: Gaussian (Philox normals) or Bernoulli (Superduper)
    float dt_f32;       // mixed path: the drift's time step,
    float sdt_f32;      //   the noise scale sqrt(dt),
    float sdt_lo;       //   Bernoulli: the step length's sub-ulp part,
    float r2_fix;       //   the Box-Muller radius constant (gfk_mixed_consts.h),
    float et_f32;       //   E_T in FP32,
    float dt_log2e;     //   dt log2(e) in FP32,
    double et_fix;      //   and et_f32 - E_T in FP64
    const float2* angle_cs;   // mixed path, Gaussian noise: the Box-Muller angle table
    TrialHost trial;
};

// Block ranges per instance for one launch shape (passed by value).
struct BlockMap {
    int32_t n_inst;
    int32_t wpt;                        // walkers per thread
    int32_t begin[GFK_MAX_INSTANCES + 1];
};

// Population sums of one block for one step, relative to the block's shift c:
// W = sum e^{logw - c}, P = sum w E_L, Q = sum w^2, R = sum w E_L^2, n = alive.
struct PartialRec {
    double c, W, P, Q, R, n;
};

// Per-step population sums of one instance (same fields, merged over blocks).
typedef PartialRec SeriesRow;

// FP64 walker state, structure of arrays over slots.
struct StateF64 {
    double* x;          // 6 planes of `stride` doubles: x1, y1, z1, x2, y2, z2
    double* logw;       // -inf for dead walkers
    int8_t* sgn;        // sign of psi at the start; 0 = dead
    int64_t stride;
};

// Mixed-precision walker state: two float4 planes per slot,
// p0 = (x1, y1, z1, x2), p1 = (y2, z2, logw bits low, logw bits high).
struct StateMixed {
    float4* p0;
    float4* p1;
    int8_t* sgn;
    // Optional position checkpoints written by the walk kernel (gfk_grad's
    // forward): after a move that completes global move j * ckpt_every, for
    // 1 <= j < ckpt_count, each slot's positions go to the planes at
    // ckpt + j * 2 * ckpt_slots: (x1, y1, z1, x2) at [slot], (y2, z2, 0, 0) at
    // [ckpt_slots + slot].  Written at the kernel's 64-move folds, so
    // ckpt_every must be a multiple of kRing and launches must start on a
    // multiple of it.  NULL: none.
    float4* ckpt;
    int64_t ckpt_slots;
    int32_t ckpt_every, ckpt_count;
    // Optional whole trajectory written by the walk kernel (gfk_grad's forward
    // when it keeps every position): the positions after global move m (m = 0:
    // the initial ones, written by a launch that starts at move 0) of walker i
    // (slot - off) go to traj + m * 6 * traj_stride as (x1, y1, z1, x2) at
    // float4 [i] and (y2, z2) at float2 [2 * traj_stride + i] -- the adjoint's
    // segment layout (traj_stride even).  NULL: none.
    float* traj;
    int64_t traj_stride;
};

// Steps between flushes of the per-step block sums; also the mixed path's
// fold period of the FP32 log-weight increments into the FP64 base.
constexpr int kRing = 64;
constexpr int kMaxThreads = 512;
constexpr int kMaxWarps = kMaxThreads / 32;
// The mixed walk with 4 walkers per thread (two packed pairs, two independent
// dependency chains per thread) is compiled for blocks of at most 128 threads,
// which lets it hold its state in up to 255 registers per thread.
constexpr int kMaxThreadsWpt4 = 128;
// The mixed walk's per-warp staging area: for each of four moves, two
// half-planes of 16 lanes x 4 sums (64 floats) padded to kStageHalf, so a move
// takes kStageMove floats; both are multiples of 4 (16-byte float4 stores) and
// kStageMove = 8 mod 32 (conflict-free column reads).
constexpr int kStageHalf = 68;
constexpr int kStageMove = 2 * kStageHalf;

// Points of the Box-Muller angle grid (the 10-bit angle fields of a move's
// Philox block), and so entries of the mixed path's angle table.
constexpr int kAngleGrid = 1024;

// Counters per instance: [0] non-finite kills, [1] node kills, [2] coalescences.
constexpr int kNumCounters = 3;

}  // namespace gfk
