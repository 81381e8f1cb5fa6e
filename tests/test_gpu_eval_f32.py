"""The mixed walk's FP32 trial evaluation at fixed positions (gfk_eval_f32), GPU.

The walk kernels evaluate one walker in a float or two in the lanes of a float2
(packed FP32 instructions); both forms must give the same drift, local energy and
sign bit for bit.  Against the oracle's FP64 evaluation at the same (FP32)
positions the FP32 forms -- the cusp-cancelled local energies -- must agree to
FP32 accuracy wherever the point is not ill-conditioned: away from the nuclei,
from electron coalescence and from the node, where the local energy's terms
grow like the inverse distance."""
import numpy as np
import pytest

import oracle
from paper_1703_08977_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

FAMILIES = {
    "ground": (0, wl.ground()),
    "ground_poly": (0, wl.ground(Z=1.85, a=0.5, beta=0.37, c=(0.11, -0.07, 0.05, 0.02))),
    "triplet_2s3": (1, wl.triplet_2s3()),
    "pz_plus": (1, wl.pz_state(+1.0)),
    "fn3": (1, wl.fn3()),
    "fn7": (1, wl.fn7(1.1, 1.9, a=0.5, beta=0.6)),
}


@pytest.mark.parametrize("name", sorted(FAMILIES))
@pytest.mark.parametrize("ee_on", [1, 0])
def test_fp32_evaluation(gfk_lib, name, ee_on):
    gfk = gfk_lib
    kind, p = FAMILIES[name]
    rng = np.random.default_rng(11)
    X = rng.normal(0.0, 0.9, (20001, 6)).astype(np.float32)       # odd: the last walker pairs with itself
    b1, e1, s1 = gfk.gfk_eval_f32(kind, p, X, lanes=1, ee_on=ee_on)
    b2, e2, s2 = gfk.gfk_eval_f32(kind, p, X, lanes=2, ee_on=ee_on)
    np.testing.assert_array_equal(b1, b2)
    np.testing.assert_array_equal(e1, e2)
    np.testing.assert_array_equal(s1, s2)

    X64 = X.astype(np.float64)
    so, bo, eo, _ = oracle.trial_eval_many(kind, p, X64, ee_on=bool(ee_on))
    r1 = np.linalg.norm(X64[:, :3], axis=1)
    r2 = np.linalg.norm(X64[:, 3:], axis=1)
    r12 = np.linalg.norm(X64[:, :3] - X64[:, 3:], axis=1)
    dn = oracle.node_distance(kind, p, X64)
    ok = (np.minimum(np.minimum(r1, r2), r12) > 0.05) & (dn > 0.01)
    assert ok.sum() > 10000
    np.testing.assert_array_equal(s1[ok], so[ok])
    tol_e = 1e-4 * (1.0 + np.abs(eo[ok]))
    assert np.all(np.abs(e1[ok] - eo[ok]) <= tol_e), np.max(np.abs(e1[ok] - eo[ok]) / tol_e)
    tol_b = 1e-4 * (1.0 + np.abs(bo[ok]))
    assert np.all(np.abs(b1[ok] - bo[ok]) <= tol_b), np.max(np.abs(b1[ok] - bo[ok]) / tol_b)
    # the bulk is far more accurate than the bound
    assert np.median(np.abs(e1[ok] - eo[ok]) / (1.0 + np.abs(eo[ok]))) < 1e-6


def test_fp32_evaluation_rejects_bad_arguments(gfk_lib):
    gfk = gfk_lib
    X = np.zeros((4, 6), dtype=np.float32) + 0.3
    with pytest.raises(gfk.GfkError):
        gfk.gfk_eval_f32(0, wl.ground()[:2], X)
    with pytest.raises(gfk.GfkError):
        gfk.gfk_eval_f32(0, wl.ground(), X, lanes=3)


def test_fp32_evaluation_far_from_the_nucleus(gfk_lib):
    """The FP32 orbital-pair evaluation factors the largest exponential out of psi,
    so hundreds of bohr out, where the unscaled psi of the FP64 path and of the
    oracle underflows to exactly 0 (a node kill), the sign stays defined and the
    drift and local energy finite: the mixed path keeps such a walker alive."""
    gfk = gfk_lib
    rng = np.random.default_rng(4)
    u = rng.normal(0.0, 1.0, (64, 6))
    u[:, :3] /= np.linalg.norm(u[:, :3], axis=1)[:, None]
    u[:, 3:] /= np.linalg.norm(u[:, 3:], axis=1)[:, None]
    X = u.copy()
    X[:, :3] *= 400.0
    X[:, 3:] *= 390.0
    p = wl.triplet_2s3()
    so = oracle.trial_eval_many(1, p, X)[0]
    assert np.all(so == 0)
    b, el, s = gfk.gfk_eval_f32(1, p, X.astype(np.float32))
    assert np.all(s != 0)
    assert np.all(np.isfinite(el)) and np.all(np.isfinite(b))
