"""Host-side constants of the mixed walk (csrc/gfk_mixed_consts.h), on the CPU.

The header is compiled with g++ into a small probe that prints the constants
for a range of time steps; the checks restate what the constants must
satisfy:
  Bernoulli: the steps +-(sdt + sdt_lo) have mean square (sdt + sdt_lo)^2 equal
             to the drift's time step fl(dt) (relative 1e-14), and sdt_lo is
             within one ulp of sdt (fl(dt) and fl(sqrt(dt))^2 differ by up to
             1.5 2^-24 relative);
  Gaussian:  with the measured mean errors of the generator, the normals'
             variance (2 + e_r2 + r2_fix + e_sqrt)(1/2 + e_angle) times sdt^2
             equals the drift's time step fl(dt) (relative 1e-12);
  both:      E_T, dt log2(e) rounded once from FP64, and et_fix = fl(E_T) - E_T.
"""
import math
import os
import shutil
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1703_08977_gb300", "csrc")
INCLUDE = os.path.join(ROOT, "include")

PROBE = r'''
#include <cstdio>
#include <cstdint>
#include "gfk.h"
#include "gfk_mixed_consts.h"
int main() {
    const double dts[] = {0.01, 0.005, 0.0025, 0.00125, 1.0 / 900.0, 3e-4, 0.0173};
    for (double dt : dts)
        for (int noise = 0; noise < 2; ++noise) {
            const gfk::MixedConsts c = gfk::mixed_consts(dt, -2.9037, noise);
            std::printf("%d %.17g %.17g %.17g %.17g %.17g %.17g %.17g %.17g\n", noise, dt,
                        (double)c.dt, (double)c.sdt,
                        (double)c.sdt_lo, (double)c.r2_fix, (double)c.et, (double)c.dt_log2e,
                        c.et_fix);
        }
    std::printf("K %.17g %.17g %.17g\n", gfk::kLog2MeanError, gfk::kSqrtMeanShift,
                gfk::kAngleMeanError);
    return 0;
}
'''


@pytest.fixture(scope="module")
def consts(tmp_path_factory):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("g++ not available")
    d = tmp_path_factory.mktemp("consts")
    src = d / "probe.cpp"
    src.write_text(PROBE)
    exe = d / "probe"
    subprocess.run([gxx, "-std=c++17", "-O1", "-I", CSRC, "-I", INCLUDE, str(src), "-o", str(exe)],
                   check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    rows, k = [], None
    for line in out:
        if not line:
            continue
        f = line.split()
        if f[0] == "K":
            k = tuple(float(x) for x in f[1:])
        else:
            rows.append((int(f[0]), *(float(x) for x in f[1:])))
    return rows, k


def test_bernoulli_steps_mean_square_is_the_drift_time_step(consts):
    rows, _ = consts
    for noise, dt, dt32, sdt, sdt_lo, r2_fix, et, dtl, etfix in rows:
        if noise != 1:
            continue
        assert dt32 == float(np.float32(dt))
        assert sdt == float(np.float32(math.sqrt(dt)))
        ms = (sdt + sdt_lo) ** 2
        assert abs(ms / dt32 - 1.0) < 1e-14, (dt, ms, dt32)
        assert abs(sdt_lo) <= np.spacing(np.float32(sdt)), (dt, sdt_lo)
        assert r2_fix == 0.0


def test_gaussian_variance_times_sdt_squared_is_the_drift_time_step(consts):
    rows, (e_log2, e_sqrt, e_angle) = consts
    for noise, dt, dt32, sdt, sdt_lo, r2_fix, et, dtl, etfix in rows:
        if noise != 0:
            continue
        assert dt32 == float(np.float32(dt)) and sdt_lo == 0.0
        var = (2.0 + e_log2 + r2_fix + e_sqrt) * (0.5 + e_angle)
        # r2_fix is stored in FP32: ~3e-14 absolute, far below the 1e-9 the walk resolves
        assert abs(var * sdt * sdt / dt32 - 1.0) < 1e-12, (dt, var)


def test_energy_and_weight_constants(consts):
    rows, _ = consts
    for noise, dt, dt32, sdt, sdt_lo, r2_fix, et, dtl, etfix in rows:
        assert et == float(np.float32(-2.9037))
        assert etfix == et - (-2.9037)
        assert dtl == float(np.float32(dt * 1.4426950408889634))


def test_angle_constant_is_the_mean_over_the_rounded_table(consts):
    """kAngleMeanError is the mean of c^2 - 1/2 over the walk's angle table: the
    correctly rounded FP32 cosines of the grid angles pi ((2k + 1)/1024 - 1),
    k = 0..1023 (computed here in 120-bit arithmetic).  The sines give the same
    mean, and the cosines and sines both sum to exactly 0."""
    mpmath = pytest.importorskip("mpmath")
    _, (_, _, e_angle) = consts
    mpmath.mp.prec = 120
    ang = [mpmath.mpf(2 * k + 1) / 1024 - 1 for k in range(1024)]
    c = [float(np.float32(float(mpmath.cospi(a)))) for a in ang]
    s = [float(np.float32(float(mpmath.sinpi(a)))) for a in ang]
    # x * x of an FP32 value is exact in FP64; fsum adds exactly
    mc = (math.fsum(x * x for x in c) - 512.0) / 1024.0
    ms = (math.fsum(x * x for x in s) - 512.0) / 1024.0
    assert mc == ms
    assert math.fsum(c) == 0.0 and math.fsum(s) == 0.0
    assert abs(mc - e_angle) < 1e-15, (mc, e_angle)
