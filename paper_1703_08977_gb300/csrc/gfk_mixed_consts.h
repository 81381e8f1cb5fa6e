// Per-instance FP32 constants of the mixed-precision walk, chosen on the host
// so that the walk's diffusion matches its drift in FP32.
//
// The drifted diffusion (the SDE under Eq. 4) discretised as
//   X <- X + b dt + sqrt(dt) xi
// samples psi^2 only if the drift's time step and the noise's variance agree:
// a relative mismatch kappa between the two shifts the mixed estimator by
// about 0.7 kappa hartree for the ground-state workloads (measured), so
// FP32-rounded dt and sqrt(dt), each off by up to 2^-24, would bias E by
// ~1e-7.
//
// Gaussian noise: the FP32 Box-Muller normals' variance is exactly
//   Var = (2 + e_r2 + e_sqrt) (1/2 + e_angle)
// where e_r2 is the mean error of the squared radius r2 over the 2^32 radius
// words, e_sqrt the mean change of r2 by the hardware square root, and
// e_angle the mean error of cos^2 (and sin^2) over the 1024-point angle grid,
// whose FP32 values come from a table (angle_cs_entry).  The first two were
// measured exhaustively on sm_103a (gfk_normal_moments re-measures them):
//   the hardware log2 scaled by -2 ln 2 has mean error  -1.630718e-7,
//   the square root changes the mean of r2 by           -4.860740e-8;
// the table holds the correctly rounded FP32 cosines and sines of the grid
// angles, whose squares average 1/2 - 2.798833e-9 (cos^2 and sin^2 alike: the
// quarter turn maps the grid onto itself), computed from the correctly
// rounded values and re-measured from the table by gfk_normal_moments.
// The additive constant of the r2 multiply-add (r2_fix) is set so that
// dt_f32 = fl(dt) and Var * sdt_f32^2 = dt_f32 exactly (to first order in the
// small terms): the noise then diffuses by exactly the drift's time step.
//
// Bernoulli noise: the steps are +-(sdt + sdt_lo) with sdt = fl(sqrt(dt)) and
// sdt_lo chosen so that their mean square is the drift's time step
// dt_f32 = fl(dt) exactly (to first order); sdt_lo lies below the ulp of the
// step, so it enters the increment through the drift's multiply-add, where
// the exact product's low bits make its rounding unbiased.
//
// Measured sensitivities of the ground-state mixed estimator: about 0.7
// hartree per unit relative mismatch between the drift's time step and the
// noise's variance, and about 0.05 hartree per unit relative rescaling of the
// walk's time (drift and noise together) against the weights' dt.  With both
// mismatches removed and the rescaling at most 2^-24, the paired
// mixed-minus-FP64 energy is a few 1e-9 hartree.
#pragma once

#include <cmath>

namespace gfk {

constexpr double kLog2MeanError = -1.630718e-7;   // mean of -2 ln2 lg2.approx(u) + 2 ln u
constexpr double kSqrtMeanShift = -4.860740e-8;   // mean of sqrt.approx(r2)^2 - r2
constexpr double kAngleMeanError = -2.798833e-9;  // mean of cos^2 - 1/2 (= of sin^2 - 1/2), table

struct MixedConsts {
    float dt, sdt, r2_fix;
    float sdt_lo;        // Bernoulli: sub-ulp part of the step length (0 for Gaussian)
    float et;            // E_T rounded to FP32 (the per-move increments use it)
    float dt_log2e;      // dt log2(e), the in-window weight's exponent scale
    double et_fix;       // et - E_T, restored in FP64 when increments are folded
};

// r2_fix for a relative variance target 1 + eta.
inline double gaussian_r2_fix(double eta) {
    const double target_rho2 = (1.0 + eta) / (0.5 + kAngleMeanError);   // E[rho^2] wanted
    return -kLog2MeanError + (target_rho2 - 2.0) - kSqrtMeanShift;
}

// Every derived constant is formed here, once, on the host: the kernels only
// load plain values (a conversion from FP64 inside the walk kernel may be
// re-evaluated in its inner loop, where FP64 arithmetic is slow).
inline MixedConsts mixed_consts(double dt, double e_trial, int noise) {
    MixedConsts c;
    c.et = (float)e_trial;
    c.et_fix = (double)c.et - e_trial;
    c.dt_log2e = (float)(dt * 1.4426950408889634);
    c.sdt = (float)std::sqrt(dt);
    const double s2 = (double)c.sdt * (double)c.sdt;       // exact in FP64
    c.dt = (float)dt;
    c.sdt_lo = 0.0f;
    if (noise == GFK_NOISE_BERNOULLI) {
        // (sdt + sdt_lo)^2 = dt_f32 to first order in sdt_lo
        c.sdt_lo = (float)(((double)c.dt - s2) / (2.0 * (double)c.sdt));
        c.r2_fix = 0.0f;
    } else {
        c.r2_fix = (float)gaussian_r2_fix((double)c.dt / s2 - 1.0);
    }
    return c;
}

}  // namespace gfk
