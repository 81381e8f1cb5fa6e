// Adjoint (reverse) sweep of the GFK walk: the gradient of the space-averaged
// final energy, or of the weighted variance of E_L, with respect to the trial
// function's parameters, through the Euler-Maruyama trajectories.
//
// Method.  The forward walk (the drifted diffusion under Eq. 4 with the
// right-point log-weights of Eq. 4) gives per walker X_0..X_S, the final
// weight w = e^{logw} and e = E_L(X_S).  With W = sum w, L = sum w e / W and
// Var = sum w e^2 / W - L^2, a change of the parameters theta moves every
// walker by
//   dL_i = alpha_i de_i(X_S) - gamma_i dt sum_{n=1..S} dE_L(X_n)
// (loss E: alpha = w/W, gamma = (w/W)(e - L); loss Var: alpha = 2 (w/W)(e - L),
// gamma = (w/W)((e - L)^2 - Var)), and X_{n+1} = X_n + b(X_n) dt + sqrt(dt) xi_n
// with the noise held fixed (X_0 does not depend on theta).  The adjoint of
// this recursion, with phi_n = dt lambda_{n+1} . b(X_n) [n < S]
// - gamma dt E_L(X_n) [n >= 1] + alpha E_L(X_n) [n = S], is
//   lambda_n = lambda_{n+1} + grad_X phi_n,   theta_bar += grad_theta phi_n,
// for n = S down to 0.  phi_n is one scalar, w . b(X_n) + w_E E_L(X_n), so a
// reverse-mode pass through the trial evaluation (adj_grad_kind0: the
// evaluation's statements, then their adjoints in reverse order) gives both
// gradients, 6 + 7 numbers, at a few times the cost of the evaluation.
//
// Positions: the forward keeps them every K moves (checkpoints), and the
// backward recomputes each K-move segment from its checkpoint with the same
// noise (Philox words, or the walker's Superduper generator skipped ahead to
// the segment's first move) and the same arithmetic as the forward kernel of
// its precision, then sweeps it in reverse.  Where device memory allows, the
// mixed path's forward instead keeps the whole trajectory (24 bytes per walker
// and move) and the backward sweeps the same K-move segments straight from it
// with nothing recomputed: the same positions, so the same gradient bit for
// bit.
#pragma once

#include <cuda_runtime.h>

#include <type_traits>

#include "gfk_device.cuh"
#include "gfk_types.h"

namespace gfk {

constexpr int kAdjThreads = 128;
constexpr int kNumTheta = 7;                  // kind 0: Z, a, beta, c1..c4

// Terminal quantities shared by every walker: {c, W, L, Var, loss}.
struct AdjTerminal {
    double c, W, L, Var, loss;
};

// Positions of a walker in the precision's state layout.
template <typename T> struct PosIO;
template <> struct PosIO<double> {
    // checkpoint / segment planes: [6][n] doubles
    __device__ __forceinline__ static bool ok(const double* base, int64_t n, int64_t i) {
        return GFK_DBG_OK(base + i, sizeof(double), kDbgPositions) &&
               GFK_DBG_OK(base + 5 * n + i, sizeof(double), kDbgPositions);
    }
    __device__ __forceinline__ static void load(const double* base, int64_t n, int64_t i, double x[6]) {
        const bool in = ok(base, n, i);
#pragma unroll
        for (int d = 0; d < 6; ++d) x[d] = in ? base[d * n + i] : 0.0;
    }
    __device__ __forceinline__ static void store(double* base, int64_t n, int64_t i, const double x[6]) {
        if (!ok(base, n, i)) return;
#pragma unroll
        for (int d = 0; d < 6; ++d) base[d * n + i] = x[d];
    }
    static constexpr int kWords = 6;          // doubles per walker per plane set
};
template <> struct PosIO<float> {
    // planes: two float4 per walker (x1,y1,z1,x2), (y2,z2,-,-) -- the state layout
    __device__ __forceinline__ static bool ok(const float* base, int64_t n, int64_t i) {
        return GFK_DBG_OK(reinterpret_cast<const float4*>(base) + i, sizeof(float4), kDbgPositions) &&
               GFK_DBG_OK(reinterpret_cast<const float4*>(base) + n + i, sizeof(float4),
                          kDbgPositions);
    }
    __device__ __forceinline__ static void load(const float* base, int64_t n, int64_t i, float x[6]) {
        if (!ok(base, n, i)) {
            for (int d = 0; d < 6; ++d) x[d] = 0.f;
            return;
        }
        const float4 a = reinterpret_cast<const float4*>(base)[i];
        const float4 b = reinterpret_cast<const float4*>(base)[n + i];
        x[0] = a.x; x[1] = a.y; x[2] = a.z; x[3] = a.w; x[4] = b.x; x[5] = b.y;
    }
    __device__ __forceinline__ static void store(float* base, int64_t n, int64_t i, const float x[6]) {
        if (!ok(base, n, i)) return;
        reinterpret_cast<float4*>(base)[i] = make_float4(x[0], x[1], x[2], x[3]);
        reinterpret_cast<float4*>(base)[n + i] = make_float4(x[4], x[5], 0.f, 0.f);
    }
    static constexpr int kWords = 8;          // floats per walker per plane set
};

// The recomputed positions of one segment, with a plane stride ns (walkers,
// even).  FP64: six planes of ns doubles per move (PosIO).  FP32: per move a
// float4 plane (x1, y1, z1, x2) and a float2 plane (y2, z2), 24 bytes a walker
// (two loads, like the state's two float4 planes, but a quarter less
// traffic); with ns even every float4 plane starts a multiple of 48 bytes
// from the (256-byte aligned) segment buffer, as 16-byte vector loads need.
template <typename T> struct SegIO : PosIO<T> {};
template <> struct SegIO<float> {
    __device__ __forceinline__ static bool ok(const float* base, int64_t ns, int64_t i) {
        return GFK_DBG_OK(reinterpret_cast<const float4*>(base) + i, sizeof(float4), kDbgPositions) &&
               GFK_DBG_OK(reinterpret_cast<const float2*>(base + 4 * ns) + i, sizeof(float2),
                          kDbgPositions);
    }
    __device__ __forceinline__ static void load(const float* base, int64_t ns, int64_t i, float x[6]) {
        if (!ok(base, ns, i)) {
            for (int d = 0; d < 6; ++d) x[d] = 0.f;
            return;
        }
        const float4 a = reinterpret_cast<const float4*>(base)[i];
        const float2 b = reinterpret_cast<const float2*>(base + 4 * ns)[i];
        x[0] = a.x; x[1] = a.y; x[2] = a.z; x[3] = a.w; x[4] = b.x; x[5] = b.y;
    }
    __device__ __forceinline__ static void store(float* base, int64_t ns, int64_t i, const float x[6]) {
        if (!ok(base, ns, i)) return;
        reinterpret_cast<float4*>(base)[i] = make_float4(x[0], x[1], x[2], x[3]);
        reinterpret_cast<float2*>(base + 4 * ns)[i] = make_float2(x[4], x[5]);
    }
    static constexpr int kWords = 6;          // floats per walker per move
};

// The forward move of the precision, written exactly as the walk kernel of
// that precision writes it (so the recomputed positions are the forward's).
// FP64: X + b dt + sdt xi for both noise modes (xi = +-1 for Bernoulli).
// FP32: the mixed kernel's helpers; for Bernoulli xi already holds +-sdt and
// xlo +-sdt_lo.
__device__ __forceinline__ void adj_move(double x[6], const double b[6], const double xi[6],
                                         const double*, double dt, double sdt, bool) {
#pragma unroll
    for (int d = 0; d < 6; ++d) x[d] = x[d] + b[d] * dt + sdt * xi[d];
}
__device__ __forceinline__ void adj_move(float x[6], const float b[6], const float xi[6],
                                         const float xlo[6], float dt, float sdt, bool bern) {
#pragma unroll
    for (int d = 0; d < 6; ++d)
        x[d] = bern ? move_bern_f32(x[d], b[d], xi[d], xlo[d], dt)
                    : move_gauss_f32(x[d], b[d], xi[d], dt, sdt);
}
__device__ __forceinline__ void adj_normals(const uint32_t w[6], double xi[6], const InstDev*,
                                            const float2*) {
    normals6_f64(w, xi);
}
__device__ __forceinline__ void adj_normals(const uint32_t w[6], float xi[6], const InstDev* inst,
                                            const float2* cs) {
    normals6_f32(w, xi, inst->r2_fix, cs);
}
__device__ __forceinline__ void adj_bernoulli(uint32_t& s, double, const InstDev*, double xi[6],
                                              double*) {
    bernoulli6<double>(s, xi);
}
__device__ __forceinline__ void adj_bernoulli(uint32_t& s, float sdt, const InstDev* inst,
                                              float xi[6], float xlo[6]) {
    bernoulli6_steps(s, sdt, inst->sdt_lo, xi, xlo);
}
// The time step and noise scale the forward walk of the precision uses.
__device__ __forceinline__ void adj_steps(const InstDev* inst, double& dt, double& sdt) {
    dt = inst->dt;
    sdt = inst->sqrt_dt;
}
__device__ __forceinline__ void adj_steps(const InstDev* inst, float& dt, float& sdt) {
    dt = inst->dt_f32;
    sdt = inst->sdt_f32;
}

// Recomputes the positions of moves n_lo + 1 .. n_hi of walker i from its
// position x at move n_lo and stores them (with x itself) in the segment
// planes: the forward walk's noise (the same Philox block of each move, or the
// walker's Superduper generator skipped ahead to move n_lo) and arithmetic.
// NOISE and POLY are fixed for the whole segment, so the loop has no branch.
template <int NOISE, int POLY, typename T>
__device__ __forceinline__ void adj_recompute(const TrialDev<T>& tp, const InstDev* inst,
                                              int64_t ns, int64_t i, int n_lo, int n_hi, T dt,
                                              T sdt, T x[6], T* seg, const float2* cs) {
    SegIO<T>::store(seg, ns, i, x);
    const uint32_t id = inst->id0 + (uint32_t)i;
    uint32_t lcg = 0u;
    PhiloxPre pre[1];
    if (NOISE == 1) lcg = superduper_at(id, inst->stream, inst->k0, inst->k1, (uint32_t)n_lo);
    else pre[0] = philox_pre(id, inst->stream, inst->k0, inst->k1);
    for (int m = n_lo; m < n_hi; ++m) {
        T xi[6], xlo[6] = {T(0), T(0), T(0), T(0), T(0), T(0)};
        if (NOISE == 1) {
            adj_bernoulli(lcg, sdt, inst, xi, xlo);
        } else {
            uint32_t words[1][6];
            move_words_all<1>(pre, (uint32_t)m, inst->k0, inst->k1, words);
            adj_normals(words[0], xi, inst, cs);
        }
        EvalOut<T> ev;
        eval_kind0<T, TrialDev<T>, POLY>(tp, x, ev);
        adj_move(x, ev.b, xi, xlo, dt, sdt, NOISE == 1);
        SegIO<T>::store(seg + (int64_t)(m - n_lo + 1) * SegIO<T>::kWords * ns, ns, i, x);
    }
}

// Reverse-mode gradient of phi = w . b(X) + wE E_L(X) for the kind-0 trial
// psi = exp(-Z r1 - Z r2 + u(r12)), u = a rho + sum_k c_k rho^{k+1} (the
// evaluation of eval_kind0 with the polynomial terms, whose derivatives are
// wanted even where the c_k vanish): xbar = d phi / dX and
// thbar = d phi / d(Z, a, beta, c1, c2, c3, c4).  The forward statements come
// first, as eval_kind0 and jastrow write them:
//   d = r1_vec - r2_vec, (r, 1/r) of |x1|^2, |x2|^2, |d|^2, e = d / r12,
//   h1 = x1 / r1, h2 = x2 / r2, q = 1 + beta r12, iq = 1/q, rho = r12 iq,
//   drho = iq^2, d2rho = -2 beta drho iq,
//   A = (ee - 2a) / r12 + ee beta (2 + beta r12), jee = A drho - 2 hh drho iq,
//   hh = 2c1 + 3c2 rho + 4c3 rho^2 + 5c4 rho^3, du = a + rho hh,
//   d2u = 2c1 + 6c2 rho + 12c3 rho^2 + 20c4 rho^3,
//   up = du drho, upp = d2u drho^2 + du d2rho,
//   b1 = -Z h1 + up e, b2 = -Z h2 - up e, proj = (h1 - h2) . e,
//   E_L = (Z - 2)(1/r1 + 1/r2) - Z^2 + jee - upp - up^2 + Z up proj;
// then the adjoint of each statement, last to first (a suffix b marks the
// derivative of phi with respect to that quantity).
template <typename T>
__device__ __forceinline__ void adj_grad_kind0(const TrialDev<T>& t, const T x[6], const T w[6],
                                               T wE, T xbar[6], T thbar[kNumTheta]) {
    // forward
    const T s1 = x[0] * x[0] + x[1] * x[1] + x[2] * x[2];
    const T s2 = x[3] * x[3] + x[4] * x[4] + x[5] * x[5];
    const T d[3] = {x[0] - x[3], x[1] - x[4], x[2] - x[5]};
    const T s12 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
    T r1, r2, r12, i1, i2, i12;
    radius(s1, r1, i1);
    radius(s2, r2, i2);
    radius(s12, r12, i12);
    const T e[3] = {d[0] * i12, d[1] * i12, d[2] * i12};
    const T h1[3] = {x[0] * i1, x[1] * i1, x[2] * i1};
    const T h2[3] = {x[3] * i2, x[4] * i2, x[5] * i2};
    const T q = T(1) + t.beta * r12;
    const T iq = rcp(q);
    const T rho = r12 * iq;
    const T drho = iq * iq;
    const T d2rho = T(-2) * t.beta * drho * iq;
    const T A = t.eem2a * i12 + t.eebeta * (T(2) + t.beta * r12);
    const T hh = t.c2 + rho * (t.c3 + rho * (t.c4 + rho * t.c5));
    const T du = t.a + rho * hh;
    const T d2u = t.d2 + rho * (t.d6 + rho * (t.d12 + rho * t.d20));
    const T up = du * drho;
    const T proj = (h1[0] - h2[0]) * e[0] + (h1[1] - h2[1]) * e[1] + (h1[2] - h2[2]) * e[2];

    // E_L
    T i1b = wE * t.Zm2, i2b = wE * t.Zm2;
    T Zb = wE * up * proj;
    const T Zm2b = wE * (i1 + i2);
    const T Z2b = -wE;
    const T jeeb = wE, uppb = -wE;
    T upb = wE * (t.Z * proj - T(2) * up);
    const T projb = wE * t.Z * up;
    // b1, b2 and proj
    T eb[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const T wd = w[c] - w[3 + c];
        const T h1b = projb * e[c] - t.Z * w[c];
        const T h2b = -projb * e[c] - t.Z * w[3 + c];
        eb[c] = projb * (h1[c] - h2[c]) + up * wd;
        upb += e[c] * wd;
        Zb -= w[c] * h1[c] + w[3 + c] * h2[c];
        // h1 = x1 i1, h2 = x2 i2
        xbar[c] = h1b * i1;
        xbar[3 + c] = h2b * i2;
        i1b += h1b * x[c];
        i2b += h2b * x[3 + c];
    }
    // jee, upp, up
    const T Ab = jeeb * drho;
    T drhob = jeeb * (A - T(2) * hh * iq) + uppb * T(2) * d2u * drho + upb * du;
    T iqb = T(-2) * jeeb * hh * drho;
    T hhb = T(-2) * jeeb * drho * iq;
    const T d2ub = uppb * drho * drho;
    const T dub = uppb * d2rho + upb * drho;
    const T d2rhob = uppb * du;
    // d2u, du, hh
    const T rho2 = rho * rho, rho3 = rho2 * rho;
    T rhob = d2ub * (t.d6 + rho * (T(2) * t.d12 + T(3) * rho * t.d20)) + dub * hh;
    hhb += dub * rho;
    rhob += hhb * (t.c3 + rho * (T(2) * t.c4 + T(3) * rho * t.c5));
    // A
    T i12b = Ab * t.eem2a;
    const T eem2ab = Ab * i12;
    const T eebetab = Ab * (T(2) + t.beta * r12);
    T betab = Ab * t.eebeta * r12;
    T r12b = Ab * t.eebeta * t.beta;
    // d2rho, drho, rho, iq, q
    betab += T(-2) * d2rhob * drho * iq;
    drhob += T(-2) * d2rhob * t.beta * iq;
    iqb += T(-2) * d2rhob * t.beta * drho;
    iqb += T(2) * drhob * iq;
    r12b += rhob * iq;
    iqb += rhob * r12;
    const T qb = -iqb * iq * iq;
    betab += qb * r12;
    r12b += qb * t.beta;
    // e, the three radii (d r / d s = 1/(2r), d (1/r) / d s = -1/(2 r^3)), d
#pragma unroll
    for (int c = 0; c < 3; ++c) i12b += eb[c] * d[c];
    const T s12b = r12b * T(0.5) * i12 - i12b * T(0.5) * i12 * i12 * i12;
    const T s1b = -i1b * T(0.5) * i1 * i1 * i1;
    const T s2b = -i2b * T(0.5) * i2 * i2 * i2;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const T db = eb[c] * i12 + T(2) * d[c] * s12b;
        xbar[c] += T(2) * x[c] * s1b + db;
        xbar[3 + c] += T(2) * x[3 + c] * s2b - db;
    }
    // the parameters behind Z - 2, Z^2, ee - 2a, ee beta and the polynomial
    // coefficients (2, 3, 4, 5) c_k and (2, 6, 12, 20) c_k
    thbar[0] = Zb + Zm2b + T(2) * t.Z * Z2b;
    thbar[1] = dub - T(2) * eem2ab;
    thbar[2] = betab + t.ee * eebetab;
    thbar[3] = T(2) * (hhb + d2ub);
    thbar[4] = T(3) * hhb * rho + T(6) * d2ub * rho;
    thbar[5] = T(4) * hhb * rho2 + T(12) * d2ub * rho2;
    thbar[6] = T(5) * hhb * rho3 + T(20) * d2ub * rho3;
}

// Terminal pass 1: per block, the largest final log-weight of live walkers.
template <typename T>
__global__ void __launch_bounds__(kAdjThreads)
adj_terminal_max_kernel(const double* __restrict__ logw, int64_t n, double* __restrict__ part_max) {
    __shared__ double s[kAdjThreads / 32];
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    double m = (i < n) ? logw[i] : -INFINITY;
    m = warp_max(m);
    if ((threadIdx.x & 31) == 0) s[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
        double r = s[0];
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w) r = fmax(r, s[w]);
        part_max[blockIdx.x] = r;
    }
}

// Terminal pass 2: per walker e = E_L(X_S) and w = e^{logw - c}; per block the
// sums of w, w e, w e^2 (FP64).
template <typename T>
__global__ void __launch_bounds__(kAdjThreads)
adj_terminal_sums_kernel(const InstDev* __restrict__ inst, const T* __restrict__ pos,
                         const double* __restrict__ logw, int64_t n,
                         const double* __restrict__ part_max, int nblk,
                         double* __restrict__ ew, double* __restrict__ part_sums) {
    __shared__ TrialDev<T> s_trial;
    __shared__ double s_c;
    __shared__ double s_red[3][kAdjThreads / 32];
    if (threadIdx.x == 0) load_trial<T>(inst->trial, inst->ee_on, s_trial);
    // the shift c: the largest block maximum, scanned by the whole block
    {
        double c = -INFINITY;
        for (int b = threadIdx.x; b < nblk; b += blockDim.x) c = fmax(c, part_max[b]);
        c = warp_max(c);
        if ((threadIdx.x & 31) == 0) s_red[0][threadIdx.x >> 5] = c;
        __syncthreads();
        if (threadIdx.x == 0) {
            double m = s_red[0][0];
            for (int w = 1; w < (int)(blockDim.x >> 5); ++w) m = fmax(m, s_red[0][w]);
            s_c = isfinite(m) ? floor(m) : 0.0;
        }
        __syncthreads();
    }
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    double q[3] = {0.0, 0.0, 0.0};
    if (i < n) {
        double e = 0.0, w = 0.0;
        if (logw[i] > -INFINITY) {
            T x[6];
            PosIO<T>::load(pos, n, i, x);
            EvalOut<T> ev;
            eval_kind0<T>(s_trial, x, ev);
            e = (double)ev.el;
            w = exp(logw[i] - s_c);
        }
        ew[2 * i] = e;
        ew[2 * i + 1] = w;
        q[0] = w;
        q[1] = w * e;
        q[2] = w * e * e;
    }
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const double v = warp_sum(q[k]);
        if ((threadIdx.x & 31) == 0) s_red[k][threadIdx.x >> 5] = v;
    }
    __syncthreads();
    if (threadIdx.x < 3) {
        double r = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) r += s_red[threadIdx.x][w];
        part_sums[3 * blockIdx.x + threadIdx.x] = r;
    }
}

// Threads of the final-sum kernels, and a Neumaier-compensated running sum.
constexpr int kFinalThreads = 256;
struct NeumaierSum {
    double s = 0.0, c = 0.0;
    __device__ __forceinline__ void add(double v) {
        const double t = s + v;
        c += fabs(s) >= fabs(v) ? (s - t) + v : (v - t) + s;
        s = t;
    }
};

// Adds the compensated sums (s[u], c[u]) of the kFinalThreads threads in a
// fixed pairwise tree (u + stride into u, stride 128, 64, ..., 1), each step
// error-free (TwoSum) on the sums; the total is s[0] + c[0].  All threads of
// the block call it.
__device__ __forceinline__ void tree_sum(double* s, double* c) {
    const int u = threadIdx.x;
#pragma unroll
    for (int stride = kFinalThreads / 2; stride > 0; stride >>= 1) {
        __syncthreads();
        if (u < stride) {
            double t, e;
            two_sum(s[u], s[u + stride], t, e);
            c[u] = c[u] + c[u + stride] + e;
            s[u] = t;
        }
    }
    __syncthreads();
}

// Terminal pass 3 (one block): W, L, Var and the loss.  Thread u sums blocks
// u, u + 256, ... (Neumaier); the threads' sums are then added in a fixed
// tree (tree_sum), so the result does not change from run to run.
static __global__ void __launch_bounds__(kFinalThreads)
adj_terminal_final_kernel(const double* __restrict__ part_max,
                          const double* __restrict__ part_sums, int nblk, int loss_kind,
                          AdjTerminal* __restrict__ out) {
    __shared__ double s_max[kFinalThreads / 32];
    __shared__ double s_part[3][2][kFinalThreads];
    const int u = threadIdx.x;
    double c = -INFINITY;
    NeumaierSum acc[3];
    for (int b = u; b < nblk; b += kFinalThreads) {
        c = fmax(c, part_max[b]);
#pragma unroll
        for (int k = 0; k < 3; ++k) acc[k].add(part_sums[3 * b + k]);
    }
    c = warp_max(c);
    if ((u & 31) == 0) s_max[u >> 5] = c;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        s_part[k][0][u] = acc[k].s;
        s_part[k][1][u] = acc[k].c;
    }
#pragma unroll
    for (int k = 0; k < 3; ++k) tree_sum(s_part[k][0], s_part[k][1]);
    if (u != 0) return;
    double cm = s_max[0];
    for (int v = 1; v < kFinalThreads / 32; ++v) cm = fmax(cm, s_max[v]);
    const double W = s_part[0][0][0] + s_part[0][1][0];
    const double P = s_part[1][0][0] + s_part[1][1][0];
    const double R = s_part[2][0][0] + s_part[2][1][0];
    AdjTerminal r;
    r.c = isfinite(cm) ? floor(cm) : 0.0;
    r.W = W;
    r.L = P / W;
    r.Var = R / W - r.L * r.L;
    r.loss = loss_kind == 0 ? r.L : r.Var;
    *out = r;
}

// The reverse sweep: one thread per walker, all segments from the last to the
// first; per block the summed parameter adjoint theta_bar.  traj: the whole
// trajectory in the segment layout (plane m = the positions after move m), or
// NULL to recompute each segment from its checkpoint into seg.
// Blocks per SM the reverse sweep is compiled for, and the moves between a
// position's load and its use: the FP32 sweep runs 5 blocks (96 registers, no
// spills) loading 3 moves ahead.  Measured on 2^18 walkers x 2000 moves (ms
// per gradient call, checkpointed / stored trajectory): 1 move ahead at 6
// blocks 13.82 / 10.90, at 5 blocks 13.79 / 10.68; 2 ahead at 6 blocks (spills)
// 13.98 / 10.77, at 5 blocks 13.80 / 10.58; 3 ahead at 5 blocks 13.66 / 10.41;
// 4 ahead at 5 blocks 13.91 / 10.54, at 4 blocks 13.72 / 10.32; 6 ahead at 5
// blocks 14.14 / 10.67; 8 ahead at 4 blocks 14.25 / 10.72.  The FP64 sweep
// keeps the default bound.
template <typename T>
constexpr int adj_min_blocks() { return sizeof(T) == 4 ? 5 : 1; }
constexpr int kAdjAhead = 3;

template <typename T>
__global__ void __launch_bounds__(kAdjThreads, adj_min_blocks<T>())
adj_backward_kernel(const InstDev* __restrict__ inst, int64_t n, int S, int K, int J,
                    int loss_kind, const T* __restrict__ ckpt, T* __restrict__ seg,
                    const T* __restrict__ traj, const double* __restrict__ ew, const AdjTerminal* __restrict__ term,
                    double* __restrict__ part_theta) {
    __shared__ TrialDev<T> s_trial;
    __shared__ double s_red[kNumTheta][kAdjThreads / 32];
    // Per-thread FP64 parameter adjoints, updated once per segment from the
    // segment's sums in T (kept here rather than in registers).
    __shared__ double s_theta[kNumTheta][kAdjThreads];
    // the FP32 recompute's Box-Muller angle table (the forward walk's)
    __shared__ float2 s_cs[std::is_same<T, float>::value ? kAngleGrid : 1];
    if (threadIdx.x == 0) load_trial<T>(inst->trial, inst->ee_on, s_trial);
    if (std::is_same<T, float>::value && inst->noise != GFK_NOISE_BERNOULLI)
        for (int k = threadIdx.x; k < kAngleGrid; k += blockDim.x) s_cs[k] = inst->angle_cs[k];
    __syncthreads();
    const TrialDev<T>& tp = s_trial;
    T dt, sdt;
    adj_steps(inst, dt, sdt);
    const bool bern = inst->noise == GFK_NOISE_BERNOULLI;
    const bool poly = has_poly(tp);
    const int64_t ns = (n + 1) & ~(int64_t)1;   // segment plane stride (SegIO): even
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    double* theta = &s_theta[0][threadIdx.x];   // theta[k * kAdjThreads]
#pragma unroll
    for (int k = 0; k < kNumTheta; ++k) theta[k * kAdjThreads] = 0.0;

    if (i < n) {
        const AdjTerminal tr = *term;
        const double e = ew[2 * i], w = ew[2 * i + 1];
        const double om = w / tr.W;
        double alpha, gamma;
        if (loss_kind == 0) {
            alpha = om;
            gamma = om * (e - tr.L);
        } else {
            alpha = 2.0 * om * (e - tr.L);
            gamma = om * ((e - tr.L) * (e - tr.L) - tr.Var);
        }
        if (w > 0.0) {
            const T a_t = (T)alpha, g_dt = (T)(gamma * inst->dt);
            T lambda[6] = {T(0), T(0), T(0), T(0), T(0), T(0)};
            for (int j = J - 1; j >= 0; --j) {
                const int n_lo = j * K;
                const int n_hi = (n_lo + K < S) ? n_lo + K : S;
                // the segment's positions n_lo .. n_hi: planes m - p0 of pos
                const T* pos = traj;
                int p0 = 0;
                if (traj == nullptr) {
                    // recomputed from the checkpoint
                    T x[6];
                    PosIO<T>::load(ckpt + (int64_t)j * PosIO<T>::kWords * n, n, i, x);
                    if (bern) {
                        if (poly) adj_recompute<1, 1, T>(tp, inst, ns, i, n_lo, n_hi, dt, sdt, x, seg, s_cs);
                        else adj_recompute<1, 0, T>(tp, inst, ns, i, n_lo, n_hi, dt, sdt, x, seg, s_cs);
                    } else {
                        if (poly) adj_recompute<0, 1, T>(tp, inst, ns, i, n_lo, n_hi, dt, sdt, x, seg, s_cs);
                        else adj_recompute<0, 0, T>(tp, inst, ns, i, n_lo, n_hi, dt, sdt, x, seg, s_cs);
                    }
                    pos = seg;
                    p0 = n_lo;
                }
                // sweep it backwards
                const int n_top = (j == J - 1) ? n_hi : n_hi - 1;
                T tseg[kNumTheta];
#pragma unroll
                for (int k = 0; k < kNumTheta; ++k) tseg[k] = T(0);
                // each move loads the position kAdjAhead moves on, so the load's
                // latency hides behind kAdjAhead gradient evaluations
                T xq[kAdjAhead][6];
#pragma unroll
                for (int a = 0; a < kAdjAhead; ++a) {
                    const int ma = n_top - a >= n_lo ? n_top - a : n_lo;
                    SegIO<T>::load(pos + (int64_t)(ma - p0) * SegIO<T>::kWords * ns, ns, i, xq[a]);
                }
#pragma unroll kAdjAhead
                for (int m = n_top; m >= n_lo; --m) {
                    T xv[6], xnext[6];
#pragma unroll
                    for (int d = 0; d < 6; ++d) xv[d] = xq[0][d];
#pragma unroll
                    for (int a = 0; a + 1 < kAdjAhead; ++a)
#pragma unroll
                        for (int d = 0; d < 6; ++d) xq[a][d] = xq[a + 1][d];
                    const int mp = m - kAdjAhead >= n_lo ? m - kAdjAhead : n_lo;
                    SegIO<T>::load(pos + (int64_t)(mp - p0) * SegIO<T>::kWords * ns, ns, i, xnext);
#pragma unroll
                    for (int d = 0; d < 6; ++d) xq[kAdjAhead - 1][d] = xnext[d];
                    // phi = w . b + wE E_L at X_m
                    T wv[6];
#pragma unroll
                    for (int d = 0; d < 6; ++d) wv[d] = m < S ? dt * lambda[d] : T(0);
                    const T wE = (m >= 1 ? -g_dt : T(0)) + (m == S ? a_t : T(0));
                    T xb[6], thb[kNumTheta];
                    adj_grad_kind0<T>(tp, xv, wv, wE, xb, thb);
#pragma unroll
                    for (int d = 0; d < 6; ++d) lambda[d] += xb[d];
#pragma unroll
                    for (int k = 0; k < kNumTheta; ++k) tseg[k] += thb[k];
                }
#pragma unroll
                for (int k = 0; k < kNumTheta; ++k) theta[k * kAdjThreads] += (double)tseg[k];
            }
        }
    }
#pragma unroll
    for (int k = 0; k < kNumTheta; ++k) {
        const double v = warp_sum(theta[k * kAdjThreads]);
        if ((threadIdx.x & 31) == 0) s_red[k][threadIdx.x >> 5] = v;
    }
    __syncthreads();
    if (threadIdx.x < kNumTheta) {
        double r = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) r += s_red[threadIdx.x][w];
        part_theta[(int64_t)kNumTheta * blockIdx.x + threadIdx.x] = r;
    }
}

// Sum of the blocks' theta_bar (one block): thread u sums blocks u, u + 256,
// ... per parameter (Neumaier); the threads' sums are then added in a fixed
// tree (tree_sum).
static __global__ void __launch_bounds__(kFinalThreads)
adj_grad_final_kernel(const double* __restrict__ part_theta, int nblk, double* __restrict__ grad) {
    __shared__ double s_part[kNumTheta][2][kFinalThreads];
    const int u = threadIdx.x;
    NeumaierSum acc[kNumTheta];
    for (int b = u; b < nblk; b += kFinalThreads) {
#pragma unroll
        for (int k = 0; k < kNumTheta; ++k) acc[k].add(part_theta[(int64_t)kNumTheta * b + k]);
    }
#pragma unroll
    for (int k = 0; k < kNumTheta; ++k) {
        s_part[k][0][u] = acc[k].s;
        s_part[k][1][u] = acc[k].c;
    }
#pragma unroll
    for (int k = 0; k < kNumTheta; ++k) tree_sum(s_part[k][0], s_part[k][1]);
    if (u < kNumTheta) grad[u] = s_part[u][0][0] + s_part[u][1][0];
}

// Host side of one precision: terminal passes, reverse sweep, final sum.
template <typename T>
cudaError_t adj_run(const InstDev* inst, int64_t n, int S, int K, int loss_kind, const T* ckpt,
                    T* seg, const T* traj, const T* pos_final, const double* logw_final, double* ew,
                    double* part_max, double* part_sums, double* part_theta, AdjTerminal* term,
                    double* grad, cudaStream_t stream) {
    const int nblk = (int)((n + kAdjThreads - 1) / kAdjThreads);
    const int J = (S + K - 1) / K;
    adj_terminal_max_kernel<T><<<nblk, kAdjThreads, 0, stream>>>(logw_final, n, part_max);
    adj_terminal_sums_kernel<T><<<nblk, kAdjThreads, 0, stream>>>(inst, pos_final, logw_final, n,
                                                                   part_max, nblk, ew, part_sums);
    adj_terminal_final_kernel<<<1, kFinalThreads, 0, stream>>>(part_max, part_sums, nblk, loss_kind,
                                                            term);
    adj_backward_kernel<T><<<nblk, kAdjThreads, 0, stream>>>(inst, n, S, K, J, loss_kind, ckpt, seg,
                                                              traj, ew, term, part_theta);
    adj_grad_final_kernel<<<1, kFinalThreads, 0, stream>>>(part_theta, nblk, grad);
    return cudaGetLastError();
}

}  // namespace gfk
