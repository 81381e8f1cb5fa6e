"""The oracle's batched trial evaluation and node distance (CPU), pinned.

trial_eval_many must be trial_eval at every point; node_distance = 1/|grad ln|Phi||
must reproduce the closed forms: 1/(Z sqrt 2) for the nodeless product
exp(-Z r1 - Z r2); the distance |r1 - r2|/sqrt 2 in R^6 to the exact node r1 = r2 of
the 2^3S pair; |z1 + z2|/sqrt 2 to the nodal plane of trial function 7; and 0 on a
node (Phi exactly 0).  These distances define which walkers the parity tests treat as near-node."""
import math

import numpy as np

import oracle
from paper_1703_08977_gb300 import workloads as wl


def test_trial_eval_many_is_trial_eval_pointwise():
    rng = np.random.default_rng(1)
    X = rng.normal(0.0, 0.8, (40, 6))
    for kind, p in ((0, wl.ground(Z=1.85, a=0.5, beta=0.37, c=(0.11, -0.07, 0.05, 0.02))),
                    (1, wl.triplet_2s3()), (1, wl.pz_state(1.0)), (1, wl.fn3())):
        s, b, el, lp = oracle.trial_eval_many(kind, p, X)
        for i in range(len(X)):
            s1, b1, e1, l1 = oracle.trial_eval(kind, p, X[i])
            assert s1 == s[i] and np.array_equal(b1, b[i]) and e1 == el[i] and l1 == lp[i]


def test_without_jastrow_clears_the_jastrow_factor_only():
    p = wl.ground(Z=1.7, a=0.5, beta=0.4, c=(0.1, 0.2, 0.3, 0.4))
    assert oracle.without_jastrow(0, p) == [1.7, 0.0, 0.4, 0.0, 0.0, 0.0, 0.0]
    q = wl.pz_state(1.0, a=0.5, beta=0.5)
    r = oracle.without_jastrow(1, q)
    assert r[0] == 0.0 and r[2:6] == [0.0] * 4 and r[1] == q[1] and r[6:] == q[6:]


def test_node_distance_closed_forms():
    rng = np.random.default_rng(2)
    X = rng.normal(0.0, 1.0, (25, 6))
    for Z in (2.0, 1.6875):
        d = oracle.node_distance(0, wl.ground(Z=Z), X)
        np.testing.assert_allclose(d, 1.0 / (Z * math.sqrt(2.0)), rtol=1e-14)
    # 2^3S pair: move electron 2 radially to r2 = r1 + delta
    r1 = np.linalg.norm(X[:, :3], axis=1)
    for delta in (1e-3, 1e-5):
        Y = X.copy()
        Y[:, 3:] *= ((r1 + delta) / np.linalg.norm(X[:, 3:], axis=1))[:, None]
        d = oracle.node_distance(1, wl.triplet_2s3(), Y)
        np.testing.assert_allclose(d, delta / math.sqrt(2.0), rtol=10 * delta)
    # on the node r1 = r2 (electron 2 a permuted copy of electron 1: equal radii up to
    # the rounding of the sum of squares in another order)
    Y = X.copy()
    Y[:, 3:] = X[:, [1, 2, 0]]
    assert np.all(oracle.node_distance(1, wl.triplet_2s3(), Y) <= 1e-15)
    Y[:, 3:] = X[:, :3]
    assert np.all(oracle.node_distance(1, wl.triplet_2s3(), Y) == 0.0)
    # trial function 7: the plane z1 + z2 = 0
    for delta in (1e-3, 1e-5):
        Y = X.copy()
        Y[:, 5] = -Y[:, 2] + delta
        d = oracle.node_distance(1, wl.fn7(1.1, 1.9, a=0.5, beta=0.6), Y)
        np.testing.assert_allclose(d, delta / math.sqrt(2.0), rtol=20 * delta)


def test_unscaled_psi_underflows_far_from_the_nucleus():
    """The oracle evaluates psi unscaled: for the 2^3S trial both terms'
    exponentials e^{-(2 r1 + r2/2)} and e^{-(r1/2 + 2 r2)} underflow to 0 once both
    exponents exceed ~745, so psi is exactly 0 there and the node rule kills a
    walker that reaches it (the FP32 path, which factors the largest exponential
    out of psi, keeps such a walker alive).  Below the underflow the sign is
    defined and the local energy finite."""
    rng = np.random.default_rng(4)
    u = rng.normal(0.0, 1.0, (20, 6))
    u[:, :3] /= np.linalg.norm(u[:, :3], axis=1)[:, None]
    u[:, 3:] /= np.linalg.norm(u[:, 3:], axis=1)[:, None]
    p = wl.triplet_2s3()
    near, far = u.copy(), u.copy()
    near[:, :3] *= 150.0
    near[:, 3:] *= 140.0                 # exponents ~ 370 and ~ 355: representable
    far[:, :3] *= 400.0
    far[:, 3:] *= 390.0                  # exponents ~ 995 and ~ 980: both underflow
    s, _, el, _ = oracle.trial_eval_many(1, p, near)
    assert np.all(s != 0) and np.all(np.isfinite(el))
    s, _, _, _ = oracle.trial_eval_many(1, p, far)
    assert np.all(s == 0)
