"""Statistical checks of the GPU walk against what the physics fixes (GPU).

- The mixed-precision path's energy on the same walkers and noise as the FP64
  path differs from it by less than 1e-7 hartree (the stated bound; measured
  2.5e-8 at dt = 0.005).
- The GFK energy of the nodeless 1^1S state and of the 2^3S state (whose node
  r1 = r2 is exact) extrapolated to dt -> 0 reproduces the exact variational
  energies printed in the paper's summary table (-2.9037243770 and
  -2.1752293782) within the statistical error.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def test_mixed_minus_fp64_bias_below_1e7(gfk_lib):
    from paper_1703_08977_gb300 import experiments as ex
    r = ex.paired_difference(0, 0.005, 20.0, 1 << 14, 16)
    assert abs(r["bias"]) < 1e-7, r
    assert abs(r["bias"]) < 5e-8 + 5 * r["bias_err"], r


def test_ground_state_energy_extrapolates_to_exact(gfk_lib):
    from paper_1703_08977_gb300 import experiments as ex
    r = ex.dt_study(0, [0.01, 0.005, 0.0025], 20.0, 1 << 16, 16)
    assert abs(r["E_dt0"] - ex.EXACT[0]) < 4 * r["E_dt0_err"] + 1e-4, r


def test_triplet_energy_extrapolates_to_exact(gfk_lib):
    from paper_1703_08977_gb300 import experiments as ex
    r = ex.dt_study(1, [0.005, 0.0025, 0.00125], 60.0, 1 << 16, 16)
    assert abs(r["E_dt0"] - ex.EXACT[1]) < 4 * r["E_dt0_err"] + 1e-4, r


def test_fp32_box_muller_radius_mean_is_exact(gfk_lib):
    """Exhaustive over the 2^32 radius words: the mixed path's squared radius r2 has a
    mean error below 5e-9 against -2 ln((w + 1/2) 2^-32) in FP64, so the normals'
    variance (the diffusion constant, E[r2]/2) is right to 2.5e-9 relative.  The
    uncorrected hardware log2 is short by the constant the kernels add back, and the
    library logarithm is shown beside it."""
    gfk = gfk_lib
    m_kernel = gfk.gfk_radius_mean_error("kernel")
    m_hw = gfk.gfk_radius_mean_error("hw_log2")
    m_lib = gfk.gfk_radius_mean_error("logf")
    assert abs(m_kernel) < 5e-9, m_kernel
    assert abs(m_hw + 1.630718e-7) < 2e-9, m_hw
    assert abs(m_lib) < 2e-8, m_lib
