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
