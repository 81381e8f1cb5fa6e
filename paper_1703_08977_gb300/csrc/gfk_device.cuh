// Device-side building blocks of the GFK walk: counter-based normals, trial
// functions with their drift and local energy, and warp-level sums.
//
// Method: importance-sampled generalized Feynman-Kac for helium (Datta,
// Rejcek, Fry, arXiv:1703.08977).  The walk is the drifted diffusion written
// under Eq. 4, dY = grad(psi)/psi dt + dX, and the weight is exp(-int V_P)
// with V_P = E_L - E_T, E_L = -Delta(psi)/(2 psi) + V (the GFK split H = H0 +
// V_P of the "Path Integral Theory" section, with the 1/2 that H0 psi =
// lambda0 psi requires).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "gfk_lanes.cuh"
#include "gfk_types.h"

namespace gfk {

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11).  Counter
// (walker id, step, rng stream, tag), key (seed low word, seed high word).
// ---------------------------------------------------------------------------
struct Words4 { uint32_t w[4]; };

__device__ __forceinline__ Words4 philox10(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                           uint32_t k0, uint32_t k1) {
    constexpr uint32_t kMulA = 0xD2511F53u, kMulB = 0xCD9E8D57u;
    constexpr uint32_t kBumpA = 0x9E3779B9u, kBumpB = 0xBB67AE85u;
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        uint32_t hiA = __umulhi(kMulA, c0), loA = kMulA * c0;
        uint32_t hiB = __umulhi(kMulB, c2), loB = kMulB * c2;
        uint32_t n0 = hiB ^ c1 ^ k0;
        uint32_t n2 = hiA ^ c3 ^ k1;
        c0 = n0; c1 = loB; c2 = n2; c3 = loA;
        k0 += kBumpA; k1 += kBumpB;
    }
    Words4 o;
    o.w[0] = c0; o.w[1] = c1; o.w[2] = c2; o.w[3] = c3;
    return o;
}

// Counter layout: move n of a walker (from global step n to n + 1) takes the
// one block (walker, n, stream, 0), the initial position the block
// (walker, 0, stream, 1).  A block's four words give the six words the
// Box-Muller transforms read, as (radius word, angle index) pairs: the radius
// words are the block's words 0, 1, 2 and the angle indices the three 10-bit
// fields (bits 0-9, 10-19, 20-29) of its word 3.
__device__ __forceinline__ void block_words(const Words4& b, uint32_t w[6]) {
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        w[2 * j] = b.w[j];
        w[2 * j + 1] = (b.w[3] >> (10 * j)) & 1023u;
    }
}
__device__ __forceinline__ void move_words(uint32_t walker, uint32_t step, uint32_t stream,
                                           uint32_t k0, uint32_t k1, uint32_t w[6]) {
    block_words(philox10(walker, step, stream, 0u, k0, k1), w);
}

__device__ __forceinline__ void init_words(uint32_t walker, uint32_t stream, uint32_t k0,
                                           uint32_t k1, uint32_t w[6]) {
    block_words(philox10(walker, 0u, stream, 1u, k0, k1), w);
}

// Six N(0,1) variates from the six words of block_words: Box-Muller on
// (w0, k0), (w2, k1), (w4, k2), xi_a = sqrt(-2 ln u_a) cos(2 pi u_b),
// xi_b = sqrt(-2 ln u_a) sin(2 pi u_b), with the radius uniform u_a from the
// radius word and the angle uniform u_b = (k + 1/2) / 1024 on an equally
// spaced grid of 1024 angles (on such a grid cos^p and sin^p average to their
// continuous values for every p below 1024).
// FP64: u_a = (w + 1/2) 2^-32 and library log/sqrt/sin/cos.
__device__ __forceinline__ void normals6_f64(const uint32_t w[6], double xi[6]) {
    constexpr double kTwoPi = 6.283185307179586476925286766559;
    constexpr double kInv32 = 1.0 / 4294967296.0;
    constexpr double kInv10 = 1.0 / 1024.0;
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        double ua = ((double)w[2 * j] + 0.5) * kInv32;
        double ub = ((double)w[2 * j + 1] + 0.5) * kInv10;
        double rho = sqrt(-2.0 * log(ua));
        double ang = kTwoPi * ub;
        xi[2 * j] = rho * cos(ang);
        xi[2 * j + 1] = rho * sin(ang);
    }
}

// The Philox blocks of one walker share walker id and stream, so their first
// round depends only on the move index and the tag: PhiloxPre holds the
// first-round products of the walker id and the stream (with the key words
// folded in), formed once per launch, and philox10_tag runs the other nine
// rounds; it equals philox10 word for word.
struct PhiloxPre {
    uint32_t hiB_k0;    // umulhi(M_B, stream) ^ k0
    uint32_t loB;       // M_B * stream
    uint32_t hiA_k1;    // umulhi(M_A, walker) ^ k1
    uint32_t loA;       // M_A * walker
};

__device__ __forceinline__ PhiloxPre philox_pre(uint32_t walker, uint32_t stream, uint32_t k0,
                                                uint32_t k1) {
    constexpr uint32_t kMulA = 0xD2511F53u, kMulB = 0xCD9E8D57u;
    PhiloxPre p;
    p.hiB_k0 = __umulhi(kMulB, stream) ^ k0;
    p.loB = kMulB * stream;
    p.hiA_k1 = __umulhi(kMulA, walker) ^ k1;
    p.loA = kMulA * walker;
    return p;
}

__device__ __forceinline__ Words4 philox10_tag(const PhiloxPre& p, uint32_t m, uint32_t tag,
                                               uint32_t k0, uint32_t k1) {
    constexpr uint32_t kMulA = 0xD2511F53u, kMulB = 0xCD9E8D57u;
    constexpr uint32_t kBumpA = 0x9E3779B9u, kBumpB = 0xBB67AE85u;
    // round 1 from the precomputed products: counters (walker, m, stream, tag)
    uint32_t c0 = p.hiB_k0 ^ m, c1 = p.loB, c2 = p.hiA_k1 ^ tag, c3 = p.loA;
#pragma unroll
    for (int r = 1; r < 10; ++r) {
        k0 += kBumpA; k1 += kBumpB;
        const uint32_t hA = __umulhi(kMulA, c0), lA = kMulA * c0;
        const uint32_t hB = __umulhi(kMulB, c2), lB = kMulB * c2;
        const uint32_t n0 = hB ^ c1 ^ k0, n2 = hA ^ c3 ^ k1;
        c0 = n0; c1 = lB; c2 = n2; c3 = lA;
    }
    Words4 o;
    o.w[0] = c0; o.w[1] = c1; o.w[2] = c2; o.w[3] = c3;
    return o;
}

// The words of move `step` for all WPT walkers of a thread (block_words of
// the block (walker, step, stream, 0)).
template <int WPT>
__device__ __forceinline__ void move_words_all(const PhiloxPre (&pre)[WPT], uint32_t step,
                                               uint32_t k0, uint32_t k1,
                                               uint32_t (&words)[WPT][6]) {
#pragma unroll
    for (int k = 0; k < WPT; ++k) block_words(philox10_tag(pre[k], step, 0u, k0, k1), words[k]);
}

// FP32: the same words.  The radius uniform keeps the full 32-bit resolution,
// u_a = fl(fl(w) 2^-32 + 2^-33) (exact for w < 2^23, where the Gaussian tail
// lives; elsewhere within an FP32 ulp of (w + 1/2) 2^-32).  A coarser grid
// would bias the walk: with N equal bins at their midpoints, the mean of
// -ln u falls short of 1 by (1 - ln 2)/N (the first bin, next to the log
// singularity), so the normals' variance -- the diffusion constant -- would be
// low by that fraction and E(t) high by about that fraction of the kinetic
// energy.  u_a is at least 2^-33 > 0; values that round to 1 give radius 0
// (the square root of 0 is 0).  The angle is the grid point
// 2 pi (u_b - 1/2), u_b = (k + 1/2)/1024, of the 10-bit index k; its cosine
// and sine come from a table of their correctly rounded FP32 values
// (angle_cs_entry), and the signs are flipped back:
// cos(2 pi u) = -cos(2 pi (u - 1/2)).  On the equally spaced grid cos^2 and
// sin^2 average to 1/2 exactly, and the FP32 values keep the grid's
// symmetries (the quarter-turn maps the grid onto itself), so their mean
// squares are equal.  The radius takes the hardware log2 with its mean error
// over the 2^32 words removed (radius2_f32 below), then the hardware square
// root.
// The squared Box-Muller radius -2 ln u_a of the FP32 path from its word w,
// u_a = fl(fl(w) 2^-32 + 2^-33).  The logarithm is the hardware base-2 one
// (a single MUFU operation) scaled by -2 ln 2, plus r2_fix.  The walk sees the
// radius only through the normals' variance, and r2_fix (set per instance on
// the host, gfk_mixed_consts.h) cancels the mean errors of this logarithm, of
// the hardware square root and of the angle table's rounding, measured
// exhaustively over all radius words and angles, and matches the variance to
// the drift's FP32 time step.
// The lane forms (one walker, or two in float2 lanes: the same rounded
// operations, paired where they are plain arithmetic) and the one-walker
// functions built on them.
template <typename L>
__device__ __forceinline__ L radius2_lanes(L wf, float r2_fix) {   // wf = (float)w per lane
    constexpr float kInv32 = 1.0f / 4294967296.0f;                        // 2^-32
    constexpr float kHalfInv32 = 0.5f / 4294967296.0f;                    // 2^-33
    constexpr float kMinus2Ln2 = -1.3862943611198906f;
    const L ua = lfma(wf, splat<L>(kInv32), splat<L>(kHalfInv32));
    L l2;
#pragma unroll
    for (int k = 0; k < LaneCount<L>::value; ++k) {
        float v;
        asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(v) : "f"(lane_at(ua, k)));
        set_lane(l2, k, v);
    }
    return lmax(lfma(splat<L>(kMinus2Ln2), l2, splat<L>(r2_fix)), splat<L>(0.0f));  // -2 ln u >= 0
}
__device__ __forceinline__ float radius2_f32(uint32_t w, float r2_fix) {
    return radius2_lanes<float>((float)w, r2_fix);
}

// The Box-Muller radius from its square (hardware square root; 0 gives 0).
__device__ __forceinline__ float radius_f32(float r2) {
    float rho;
    asm("sqrt.approx.f32 %0, %1;" : "=f"(rho) : "f"(r2));
    return rho;
}

// The angle of grid point k, theta_k = 2 pi ((k + 1/2)/1024 - 1/2) =
// pi ((2k + 1)/1024 - 1), as the pair (cos theta_k, sin theta_k) rounded to
// FP32.  The argument of sincospi is exact in FP64 (a dyadic rational), and
// the FP64 library values round to the correctly rounded FP32 values for all
// but ties closer than the FP64 error, so the FP32 angle carries no error of
// its own beyond the final rounding.  The walk kernels gather these pairs from
// a 1024-entry table (filled once per context by fill_angle_table)
// instead of evaluating the hardware sine and cosine per normal.
__device__ __forceinline__ float2 angle_cs_entry(uint32_t k) {
    double s, c;
    sincospi((double)(2u * k + 1u) * (1.0 / (double)kAngleGrid) - 1.0, &s, &c);
    return make_float2((float)c, (float)s);
}

// Six N(0,1) variates per walker from its six words (block_words: Box-Muller
// on (w0,k0), (w2,k1), (w4,k2)) for the walkers of a lane group (w[k]: lane
// k's words); cs is the angle table (kAngleGrid pairs, shared memory in the
// kernels).
template <typename L>
__device__ __forceinline__ void normals6_lanes(const uint32_t (*w)[6], L xi[6], float r2_fix,
                                               const float2* __restrict__ cs) {
    constexpr int W = LaneCount<L>::value;
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        L wf;
#pragma unroll
        for (int k = 0; k < W; ++k) set_lane(wf, k, (float)w[k][2 * j]);
        const L r2 = radius2_lanes<L>(wf, r2_fix);
        L rho, sn, cn;
#pragma unroll
        for (int k = 0; k < W; ++k) {
            const float2 t = cs[w[k][2 * j + 1]];
            set_lane(rho, k, radius_f32(lane_at(r2, k)));
            set_lane(cn, k, t.x);
            set_lane(sn, k, t.y);
        }
        const L nrho = lneg(rho);
        xi[2 * j] = lmul(nrho, cn);
        xi[2 * j + 1] = lmul(nrho, sn);
    }
}
__device__ __forceinline__ void normals6_f32(const uint32_t w[6], float xi[6], float r2_fix,
                                             const float2* __restrict__ cs) {
    normals6_lanes<float>(reinterpret_cast<const uint32_t(*)[6]>(w), xi, r2_fix, cs);
}

// ---------------------------------------------------------------------------
// Bernoulli increments: the paper's own random walk (each coordinate moves by
// +-1/sqrt(n) per time step 1/n, the construction of W(l) before the
// invariance principle), with eps drawn from the "Superduper" congruential
// generator S_i = (69069 S_{i-1} + 1) mod 2^32, eps_i = +1 if S_i > 2^31 and
// -1 otherwise.  Every walker runs its own generator: S_0 is word 0 of the
// Philox block (walker, 0, stream, 5), and move `step` takes the outputs
// 6 step + 1 .. 6 step + 6 for x1, y1, z1, x2, y2, z2.
// ---------------------------------------------------------------------------
constexpr uint32_t kSuperduperMult = 69069u;

__device__ __forceinline__ uint32_t superduper_seed(uint32_t walker, uint32_t stream,
                                                    uint32_t k0, uint32_t k1) {
    return philox10(walker, 0u, stream, 5u, k0, k1).w[0];
}

__device__ __forceinline__ uint32_t superduper_next(uint32_t s) {
    return kSuperduperMult * s + 1u;              // unsigned arithmetic wraps mod 2^32
}

// The state n outputs later: the affine map x -> a x + 1 composed n times by
// binary powering.  The generator's period is 2^32 (c odd, a = 1 mod 4), so the
// count is taken mod 2^32.
__device__ __forceinline__ uint32_t superduper_skip(uint32_t s, uint32_t n) {
    uint32_t A = 1u, C = 0u;                      // the accumulated map
    uint32_t a = kSuperduperMult, c = 1u;         // the map composed 2^j times
    while (n != 0u) {
        if (n & 1u) {
            A = a * A;
            C = a * C + c;
        }
        c = a * c + c;
        a = a * a;
        n >>= 1;
    }
    return A * s + C;
}

// Generator state at the start of move `step` (before its six outputs).
__device__ __forceinline__ uint32_t superduper_at(uint32_t walker, uint32_t stream, uint32_t k0,
                                                  uint32_t k1, uint32_t step) {
    return superduper_skip(superduper_seed(walker, stream, k0, k1), 6u * step);
}

// The six increments of one move; advances the state by six outputs.
template <typename R>
__device__ __forceinline__ void bernoulli6(uint32_t& s, R eps[6]) {
#pragma unroll
    for (int d = 0; d < 6; ++d) {
        s = superduper_next(s);
        eps[d] = s > 0x80000000u ? R(1) : R(-1);
    }
}

// The same six increments already scaled, as a two-part step length:
// +-sdt and +-sdt_lo with the same sign.
__device__ __forceinline__ void bernoulli6_steps(uint32_t& s, float sdt, float sdt_lo,
                                                 float step[6], float step_lo[6]) {
#pragma unroll
    for (int d = 0; d < 6; ++d) {
        s = superduper_next(s);
        const bool up = s > 0x80000000u;
        step[d] = up ? sdt : -sdt;
        step_lo[d] = up ? sdt_lo : -sdt_lo;
    }
}

// The FP32 move of the mixed path (the forward walk and the adjoint's segment
// recompute both use these, so their positions agree bit for bit).  In both
// the increment is formed first and meets X in a single rounding:
// Gaussian: X + (b dt + sdt xi).  Rounding twice at X's scale,
//   fl(fl(X + b dt) + sdt xi), shifted the mixed estimator by up to -4e-8
//   hartree (measured against FP64 positions, dt 0.0025); the increment-first
//   form is within 2e-9 of them.
// Bernoulli: X + ((b dt +- sdt_lo) +- sdt).  Adding the fixed step sdt
//   straight to X would round it to the grid of X's binade each time, a
//   binade-dependent step length (a systematic diffusion error of up to
//   ulp(X)/sdt).  The sub-ulp part sdt_lo rides on the drift's multiply-add.
template <typename L>
__device__ __forceinline__ L move_gauss_lanes(L x, L b, L xi, L dt, L sdt) {
    return ladd(x, lfma(sdt, xi, lmul(b, dt)));
}
template <typename L>
__device__ __forceinline__ L move_bern_lanes(L x, L b, L step, L step_lo, L dt) {
    return ladd(x, ladd(lfma(b, dt, step_lo), step));
}
__device__ __forceinline__ float move_gauss_f32(float x, float b, float xi, float dt, float sdt) {
    return move_gauss_lanes<float>(x, b, xi, dt, sdt);
}
__device__ __forceinline__ float move_bern_f32(float x, float b, float step, float step_lo,
                                               float dt) {
    return move_bern_lanes<float>(x, b, step, step_lo, dt);
}

// ---------------------------------------------------------------------------
// Precision helpers
// ---------------------------------------------------------------------------
// Distance and inverse distance from a squared distance.  FP32: one hardware
// reciprocal square root.  FP64: the correctly rounded square root first (the
// plain definition r = sqrt(x^2 + y^2 + z^2)), then its reciprocal.
__device__ __forceinline__ void radius(float s, float& r, float& i) {
    i = rsqrtf(s);
    r = s * i;
}
__device__ __forceinline__ void radius(double s, double& r, double& i) {
    r = sqrt(s);
    i = 1.0 / r;
}
__device__ __forceinline__ float rcp(float x) {   // hardware reciprocal (<= 1 ulp)
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ double rcp(double x) { return 1.0 / x; }
__device__ __forceinline__ float expn(float x) { return __expf(x); }
__device__ __forceinline__ double expn(double x) { return exp(x); }
__device__ __forceinline__ bool finite_(float x) { return isfinite(x); }
__device__ __forceinline__ bool finite_(double x) { return isfinite(x); }

// ---------------------------------------------------------------------------
// Trial parameters in the working precision (derived from TrialHost).
// ---------------------------------------------------------------------------
template <typename R>
struct TrialDev {
    int kind, nterms;
    int poly;                      // any c_k != 0 (else the Jastrow polynomial is skipped)
    int plain;                     // kind 1 whose orbitals all lack r and z prefactor terms
    R Z, Zm2, Z2;                  // kind 0: Z, Z - 2, Z^2
    R a, beta, ee, eem2a, eebeta;  // Jastrow: a, beta, ee (0/1), ee - 2a, ee*beta
    R c2, c3, c4, c5;              // 2c1, 3c2, 4c3, 5c4 (du/drho coefficients)
    R d2, d6, d12, d20;            // 2c1, 6c2, 12c3, 20c4 (d2u/drho2 coefficients)
    R s[GFK_MAX_TERMS];
    R al[GFK_MAX_TERMS][2], c0[GFK_MAX_TERMS][2], c1[GFK_MAX_TERMS][2], cz[GFK_MAX_TERMS][2];
    R km2[GFK_MAX_TERMS][2];       // alpha - 2
    R hal2[GFK_MAX_TERMS][2];      // alpha^2 / 2
    // FP32 lane evaluation (gfk_lanes.cuh): parameter products formed here
    R mZ, m2beta;                  // -Z, -2 beta
    R mal[GFK_MAX_TERMS][2];       // -alpha
    R sc[GFK_MAX_TERMS];           // s c0A c0B (orbitals without prefactor terms)
};

template <typename R>
__host__ __device__ __forceinline__ void load_trial(const TrialHost& h, int ee_on, TrialDev<R>& t) {
    t.kind = h.kind;
    t.nterms = h.nterms;
    t.poly = (h.ck[0] != 0.0 || h.ck[1] != 0.0 || h.ck[2] != 0.0 || h.ck[3] != 0.0) ? 1 : 0;
    t.plain = h.kind == GFK_TRIAL_ORBITAL_PAIRS ? 1 : 0;
    for (int i = 0; i < h.nterms && i < GFK_MAX_TERMS; ++i)
        for (int e = 0; e < 2; ++e)
            if (h.c1[i][e] != 0.0 || h.cz[i][e] != 0.0) t.plain = 0;
    t.Z = (R)h.Z;
    t.Zm2 = (R)(h.Z - 2.0);
    t.Z2 = (R)(h.Z * h.Z);
    t.a = (R)h.a;
    t.beta = (R)h.beta;
    t.ee = ee_on ? R(1) : R(0);
    t.eem2a = (R)((ee_on ? 1.0 : 0.0) - 2.0 * h.a);
    t.eebeta = ee_on ? (R)h.beta : R(0);
    t.c2 = (R)(2.0 * h.ck[0]);
    t.c3 = (R)(3.0 * h.ck[1]);
    t.c4 = (R)(4.0 * h.ck[2]);
    t.c5 = (R)(5.0 * h.ck[3]);
    t.d2 = (R)(2.0 * h.ck[0]);
    t.d6 = (R)(6.0 * h.ck[1]);
    t.d12 = (R)(12.0 * h.ck[2]);
    t.d20 = (R)(20.0 * h.ck[3]);
    for (int i = 0; i < GFK_MAX_TERMS; ++i) {
        t.s[i] = (R)h.s[i];
        for (int e = 0; e < 2; ++e) {
            t.al[i][e] = (R)h.alpha[i][e];
            t.c0[i][e] = (R)h.c0[i][e];
            t.c1[i][e] = (R)h.c1[i][e];
            t.cz[i][e] = (R)h.cz[i][e];
            t.km2[i][e] = (R)(h.alpha[i][e] - 2.0);
            t.hal2[i][e] = (R)(0.5 * h.alpha[i][e] * h.alpha[i][e]);
            t.mal[i][e] = (R)(-h.alpha[i][e]);
        }
        t.sc[i] = (R)(h.s[i] * h.c0[i][0] * h.c0[i][1]);
    }
    t.mZ = (R)(-h.Z);
    t.m2beta = (R)(-2.0 * h.beta);
}

// Result of one trial evaluation.
template <typename R>
struct EvalOut {
    R b[6];        // drift grad ln|psi|
    R el;          // local energy
    int sign;      // sign of psi (0: exactly zero)
    R rmin;        // min(r1, r2, r12), for the coalescence diagnostic
};

// Jastrow factor u(r12) = a rho + sum c_k rho^{k+1}, rho = r/(1+beta r): returns
// u', u'' and the combination (ee - 2u')/r12 written without the 1/r12
// cancellation:  (ee - 2 a rho')/r = [(ee - 2a)/r + ee beta (2 + beta r)] rho',
// and 2 rho h rho'/r = 2 h rho' / (1 + beta r) with h = (du/drho - a)/rho.
template <typename R>
struct JastrowOut { R up, upp, jee; };

// Whether the Jastrow polynomial terms are present (a block-uniform branch).
// The evaluators below are
// compiled for POLY = 0 (no polynomial terms) or 1 (with them); POLY = -1
// selects one of the two at run time with a single branch at the top, so every
// kernel evaluates a given trial function with the same arithmetic.  The
// specialised mixed walk kernels pass POLY = 0 (their launcher gives them
// polynomial-free trial functions only): the branch then disappears from the
// move loop, which lets the compiler interleave a thread's walkers across it.
template <typename R>
__device__ __forceinline__ bool has_poly(const TrialDev<R>& t) { return t.poly != 0; }

template <typename R, typename TD, int POLY>
__device__ __forceinline__ JastrowOut<R> jastrow(const TD& t, R r12, R i12) {
    R q = R(1) + t.beta * r12;
    R iq = rcp(q);
    R rho = r12 * iq;
    R drho = iq * iq;                          // d rho / dr
    R d2rho = R(-2) * t.beta * drho * iq;      // d2 rho / dr2
    JastrowOut<R> o;
    const R jee0 = (t.eem2a * i12 + t.eebeta * (R(2) + t.beta * r12)) * drho;
    if (POLY != 0) {
        R h = t.c2 + rho * (t.c3 + rho * (t.c4 + rho * t.c5));   // (du/drho - a) / rho
        R du = t.a + rho * h;                                   // du / drho
        R d2u = t.d2 + rho * (t.d6 + rho * (t.d12 + rho * t.d20));
        o.up = du * drho;
        o.upp = d2u * drho * drho + du * d2rho;
        o.jee = jee0 - R(2) * h * drho * iq;
    } else {                                   // u = a rho: du/drho = a, d2u/drho2 = 0
        o.up = t.a * drho;
        o.upp = t.a * d2rho;
        o.jee = jee0;
    }
    return o;
}

}  // namespace gfk

#include "gfk_eval_f32.cuh"   // the FP32 evaluation (one walker, or two in float2 lanes)

namespace gfk {

// The FP32 evaluation in EvalOut<float> form (one walker: the lane code with
// L = float, so that it equals either lane of the paired evaluation bit for bit).
template <int KIND, bool UNROLL, int POLY>
__device__ __forceinline__ void eval_f32(const TrialDev<float>& t, const float x[6],
                                         EvalOut<float>& o) {
    EvalLanes<float> e;
    eval_lanes<KIND, float, UNROLL, POLY>(t, x, e);
#pragma unroll
    for (int d = 0; d < 6; ++d) o.b[d] = e.b[d];
    o.el = e.el;
    o.sign = e.sign[0];
    o.rmin = e.rmin;
}

// Kind 0: psi = exp(-Z r1 - Z r2 + u(r12)).
//   b_1 = -Z r1_hat + u' e12,  b_2 = -Z r2_hat - u' e12   (e12 = (r1 - r2)/r12)
//   E_L = (Z - 2)(1/r1 + 1/r2) - Z^2 + (ee - 2u')/r12 - u'' - u'^2
//         + Z u' (r1_hat - r2_hat) . e12
// (the nuclear 1/r terms cancel exactly for Z = 2).
template <typename R, typename TD, int POLY = -1>
__device__ __forceinline__ void eval_kind0(const TD& t, const R x[6], EvalOut<R>& o) {
    if constexpr (sizeof(R) == 4) {           // FP32: the lane evaluation
        eval_f32<0, false, POLY>(t, x, o);
        return;
    } else if constexpr (POLY < 0) {
        if (has_poly(t)) eval_kind0<R, TD, 1>(t, x, o);
        else eval_kind0<R, TD, 0>(t, x, o);
        return;
    }
    R s1 = x[0] * x[0] + x[1] * x[1] + x[2] * x[2];
    R s2 = x[3] * x[3] + x[4] * x[4] + x[5] * x[5];
    R dx = x[0] - x[3], dy = x[1] - x[4], dz = x[2] - x[5];
    R s12 = dx * dx + dy * dy + dz * dz;
    R r1, r2, r12, i1, i2, i12;
    radius(s1, r1, i1);
    radius(s2, r2, i2);
    radius(s12, r12, i12);
    R ex = dx * i12, ey = dy * i12, ez = dz * i12;
    JastrowOut<R> j = jastrow<R, TD, POLY>(t, r12, i12);
    R h1x = x[0] * i1, h1y = x[1] * i1, h1z = x[2] * i1;
    R h2x = x[3] * i2, h2y = x[4] * i2, h2z = x[5] * i2;
    o.b[0] = -t.Z * h1x + j.up * ex;
    o.b[1] = -t.Z * h1y + j.up * ey;
    o.b[2] = -t.Z * h1z + j.up * ez;
    o.b[3] = -t.Z * h2x - j.up * ex;
    o.b[4] = -t.Z * h2y - j.up * ey;
    o.b[5] = -t.Z * h2z - j.up * ez;
    R proj = (h1x - h2x) * ex + (h1y - h2y) * ey + (h1z - h2z) * ez;
    o.el = t.Zm2 * (i1 + i2) - t.Z2 + j.jee - j.upp - j.up * j.up + t.Z * j.up * proj;
    o.sign = finite_(s1 + s2) ? 1 : 0;   // psi > 0 wherever X is finite
    o.rmin = fmin(fmin(r1, r2), r12);
}

// Kind 1: psi = Phi exp(u(r12)), Phi = sum_t s_t f_A(r1) f_B(r2), orbitals
// f = p e^{-alpha r}, p = c0 + c1 r + cz z.  Each term is evaluated with the
// largest exponent factored out (ratios are unchanged; no underflow).
// Per orbital, with g = e^{-alpha r}:
//   grad f / g          = c1 r_hat + cz z_hat - alpha p r_hat
//   (-lap f / 2 - 2 f / r) / g
//                       = -c1/r + alpha (c1 + cz z / r) - alpha^2 p / 2 + (alpha - 2) p / r
// (the second line folds the nuclear attraction into the kinetic term so the
// 1/r singularities cancel exactly when the orbital meets the cusp).  Then
//   b_1 = grad_1 Phi / Phi + u' e12,  b_2 = grad_2 Phi / Phi - u' e12
//   E_L = T / Phi - u' (grad_1 Phi - grad_2 Phi) . e12 / Phi - u'' - u'^2
//         + (ee - 2u')/r12,
//   T = sum_t s_t [K_A p_B + p_A K_B] g_A g_B.
// One term s_t f_A f_B of the orbital-pair trial function: its contribution
// to Phi, to the kinetic sum T and to the gradients G1, G2 (see eval_kind1).
template <typename R>
struct Kind1Acc {
    R Phi = R(0), T = R(0);
    R G1[3] = {R(0), R(0), R(0)}, G2[3] = {R(0), R(0), R(0)};
};

// PLAIN: every orbital is c0 e^{-alpha r} (no r or z prefactor terms), so the
// prefactor terms, which would be exact zeros, are left out.
template <typename R, bool PLAIN = false>
__device__ __forceinline__ void kind1_term(const TrialDev<R>& t, int k, R r1, R r2, const R rr[2],
                                           const R ir[2], const R zz[2], const R h1[3],
                                           const R h2[3], R emax, Kind1Acc<R>& acc) {
    constexpr bool kF64 = sizeof(R) == 8;
    R gA = R(1), gB = R(1), g;
    if (kF64) {
        gA = expn(-t.al[k][0] * r1);
        gB = expn(-t.al[k][1] * r2);
        g = gA * gB;
    } else {
        g = expn(-(t.al[k][0] * r1 + t.al[k][1] * r2) - emax);
    }
    R p[2], K[2], gr[2][3];
#pragma unroll
    for (int e = 0; e < 2; ++e) {
        const R* hh = e == 0 ? h1 : h2;
        if (PLAIN) {
            const R c0 = t.c0[k][e];
            const R radial = -t.al[k][e] * c0;
            gr[e][0] = radial * hh[0];
            gr[e][1] = radial * hh[1];
            gr[e][2] = radial * hh[2];
            K[e] = c0 * (t.km2[k][e] * ir[e] - t.hal2[k][e]);
            p[e] = c0;
            continue;
        }
        R al = t.al[k][e], c1 = t.c1[k][e], cz = t.cz[k][e];
        R pe = t.c0[k][e] + c1 * rr[e] + cz * zz[e];
        R radial = c1 - al * pe;                      // coefficient of r_hat
        gr[e][0] = radial * hh[0];
        gr[e][1] = radial * hh[1];
        gr[e][2] = radial * hh[2] + cz;
        K[e] = -c1 * ir[e] + al * (c1 + cz * zz[e] * ir[e]) - t.hal2[k][e] * pe +
               t.km2[k][e] * pe * ir[e];
        p[e] = pe;
    }
    R sg = t.s[k] * g;
    if (kF64) acc.Phi += t.s[k] * (p[0] * gA) * (p[1] * gB);
    else acc.Phi += sg * p[0] * p[1];
    acc.T += sg * (K[0] * p[1] + p[0] * K[1]);
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        acc.G1[d] += sg * gr[0][d] * p[1];
        acc.G2[d] += sg * p[0] * gr[1][d];
    }
}

// UNROLL: the term loops run to GFK_MAX_TERMS with a uniform early exit, so
// every parameter index is a compile-time constant (for a trial held in the
// kernel's parameter bank); otherwise they run to t.nterms (fewer registers).
template <typename R, bool UNROLL = false, bool PLAIN = false, int POLY = -1>
__device__ __forceinline__ void eval_kind1(const TrialDev<R>& t, const R x[6], EvalOut<R>& o) {
    if constexpr (sizeof(R) == 4) {           // FP32: the lane evaluation
        eval_f32<PLAIN ? 3 : 1, UNROLL, POLY>(t, x, o);
        return;
    } else if constexpr (POLY < 0) {
        if (has_poly(t)) eval_kind1<R, UNROLL, PLAIN, 1>(t, x, o);
        else eval_kind1<R, UNROLL, PLAIN, 0>(t, x, o);
        return;
    }
    R s1 = x[0] * x[0] + x[1] * x[1] + x[2] * x[2];
    R s2 = x[3] * x[3] + x[4] * x[4] + x[5] * x[5];
    R dx = x[0] - x[3], dy = x[1] - x[4], dz = x[2] - x[5];
    R s12 = dx * dx + dy * dy + dz * dz;
    R r1, r2, r12, i1, i2, i12;
    radius(s1, r1, i1);
    radius(s2, r2, i2);
    radius(s12, r12, i12);
    R ex = dx * i12, ey = dy * i12, ez = dz * i12;
    R h1[3] = {x[0] * i1, x[1] * i1, x[2] * i1};
    R h2[3] = {x[3] * i2, x[4] * i2, x[5] * i2};
    const R rr[2] = {r1, r2};
    const R ir[2] = {i1, i2};
    const R zz[2] = {x[2], x[5]};

    // FP32: the largest exponent -(alphaA r1 + alphaB r2) over the terms is
    // factored out so no term underflows.  FP64 has the range to evaluate each
    // orbital's exponential as it stands, which keeps the sign of Phi (the node
    // test) computed exactly as the plain sum of products s f_A f_B.
    constexpr bool kF64 = sizeof(R) == 8;
    R emax = R(0);
    if (!kF64) {
        emax = -(t.al[0][0] * r1 + t.al[0][1] * r2);
        if constexpr (UNROLL) {
#pragma unroll
            for (int k = 1; k < GFK_MAX_TERMS; ++k) {
                if (k >= t.nterms) break;
                emax = fmax(emax, -(t.al[k][0] * r1 + t.al[k][1] * r2));
            }
        } else {
            for (int k = 1; k < t.nterms; ++k)
                emax = fmax(emax, -(t.al[k][0] * r1 + t.al[k][1] * r2));
        }
    }

    Kind1Acc<R> acc;
    if constexpr (UNROLL) {
#pragma unroll
        for (int k = 0; k < GFK_MAX_TERMS; ++k) {
            if (k >= t.nterms) break;
            kind1_term<R, PLAIN>(t, k, r1, r2, rr, ir, zz, h1, h2, emax, acc);
        }
    } else {
        for (int k = 0; k < t.nterms; ++k)
            kind1_term<R, PLAIN>(t, k, r1, r2, rr, ir, zz, h1, h2, emax, acc);
    }
    const R Phi = acc.Phi, T = acc.T;
    const R* G1 = acc.G1;
    const R* G2 = acc.G2;
    JastrowOut<R> j = jastrow<R, TrialDev<R>, POLY>(t, r12, i12);
    R iP = rcp(Phi);
    o.b[0] = G1[0] * iP + j.up * ex;
    o.b[1] = G1[1] * iP + j.up * ey;
    o.b[2] = G1[2] * iP + j.up * ez;
    o.b[3] = G2[0] * iP - j.up * ex;
    o.b[4] = G2[1] * iP - j.up * ey;
    o.b[5] = G2[2] * iP - j.up * ez;
    R cross = (G1[0] - G2[0]) * ex + (G1[1] - G2[1]) * ey + (G1[2] - G2[2]) * ez;
    o.el = (T - j.up * cross) * iP - j.upp - j.up * j.up + j.jee;
    o.sign = Phi > R(0) ? 1 : (Phi < R(0) ? -1 : 0);
    o.rmin = fmin(fmin(r1, r2), r12);
}

// KIND 0 / 1 select the family at compile time; KIND 2 dispatches on t.kind
// (used when one launch covers instances of both families); KIND 3 is the
// orbital-pair family whose orbitals all lack the r and z prefactor terms
// (the mixed walk's launcher picks it when every instance qualifies).  POLY as
// for jastrow (KIND 2 always decides at run time).
template <int KIND, typename R, bool UNROLL = false, int POLY = -1>
__device__ __forceinline__ void eval_trial(const TrialDev<R>& t, const R x[6], EvalOut<R>& o) {
    if (KIND == 0) eval_kind0<R, TrialDev<R>, POLY>(t, x, o);
    else if (KIND == 1) eval_kind1<R, UNROLL, false, POLY>(t, x, o);
    else if (KIND == 3) eval_kind1<R, UNROLL, true, POLY>(t, x, o);
    else if (t.kind == 0) eval_kind0<R>(t, x, o);
    else eval_kind1<R>(t, x, o);
}

// A sum is finite only if every term is (an infinity or NaN in any term makes
// it infinite or NaN), so one test covers the drift and the local energy.
template <typename R>
__device__ __forceinline__ bool eval_finite(const EvalOut<R>& o) {
    return finite_(((o.b[0] + o.b[1]) + (o.b[2] + o.b[3])) + ((o.b[4] + o.b[5]) + o.el));
}

// ---------------------------------------------------------------------------
// Warp sums
// ---------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// Error-free sum (Knuth's TwoSum): s + e == a + b exactly.
__device__ __forceinline__ void two_sum(double a, double b, double& s, double& e) {
    s = __dadd_rn(a, b);
    double bb = __dsub_rn(s, a);
    e = __dadd_rn(__dsub_rn(a, __dsub_rn(s, bb)), __dsub_rn(b, bb));
}

}  // namespace gfk
