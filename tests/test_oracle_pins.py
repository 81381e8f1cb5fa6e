"""Pins of the oracle against things other than itself (CPU only).

Each test ties one oracle function to a fact the paper, the mathematics or an
independent implementation fixes, chosen so that a plausible slip (a dropped
term, a wrong sign, swapped electrons, a wrong step counter) fails one of them.
"""
import math
import os
import subprocess
import sys
import textwrap

import numpy as np
import pytest

import oracle
from paper_1703_08977_gb300 import workloads as wl

mp = pytest.importorskip("mpmath")


# --------------------------------------------------------------------------
# Philox4x32-10 against an independent implementation
# --------------------------------------------------------------------------

_TRITON_PHILOX = textwrap.dedent(r'''
    import os, sys
    os.environ["TRITON_INTERPRET"] = "1"
    import numpy as np, torch, triton, triton.language as tl

    @triton.jit
    def k(cp, kp, op, N: tl.constexpr):
        i = tl.arange(0, N)
        c0 = tl.load(cp + 4 * i + 0).to(tl.uint32, bitcast=True)
        c1 = tl.load(cp + 4 * i + 1).to(tl.uint32, bitcast=True)
        c2 = tl.load(cp + 4 * i + 2).to(tl.uint32, bitcast=True)
        c3 = tl.load(cp + 4 * i + 3).to(tl.uint32, bitcast=True)
        k0 = tl.load(kp + 2 * i + 0).to(tl.uint32, bitcast=True)
        k1 = tl.load(kp + 2 * i + 1).to(tl.uint32, bitcast=True)
        r0, r1, r2, r3 = tl.philox_impl(c0, c1, c2, c3, k0, k1, 10)
        tl.store(op + 4 * i + 0, r0.to(tl.int32, bitcast=True))
        tl.store(op + 4 * i + 1, r1.to(tl.int32, bitcast=True))
        tl.store(op + 4 * i + 2, r2.to(tl.int32, bitcast=True))
        tl.store(op + 4 * i + 3, r3.to(tl.int32, bitcast=True))

    d = np.load(sys.argv[1])
    N = d["ctr"].shape[0]
    c = torch.from_numpy(d["ctr"].view(np.int32).copy())
    kk = torch.from_numpy(d["key"].view(np.int32).copy())
    o = torch.zeros(4 * N, dtype=torch.int32)
    k[(1,)](c, kk, o, N=N)
    np.save(sys.argv[2], o.numpy().view(np.uint32).reshape(N, 4))
''')


def test_philox_matches_triton_interpreter(tmp_path):
    """The oracle's Philox4x32-10 equals triton's (a third-party implementation of
    Salmon et al. 2011), run on the CPU by triton's interpreter, bit for bit."""
    pytest.importorskip("triton")
    rng = np.random.default_rng(12345)
    N = 64
    ctr = rng.integers(0, 2**32, size=(N, 4), dtype=np.uint64).astype(np.uint32)
    key = rng.integers(0, 2**32, size=(N, 2), dtype=np.uint64).astype(np.uint32)
    ctr[0] = 0
    key[0] = 0
    ctr[1] = [2**32 - 1] * 4
    key[1] = [2**32 - 1] * 2
    ctr[2] = [7, 11, 0, 1]          # a walker/step/inst/tag style counter
    inp = tmp_path / "in.npz"
    out = tmp_path / "out.npy"
    np.savez(inp, ctr=ctr, key=key)
    script = tmp_path / "tp.py"
    script.write_text(_TRITON_PHILOX)
    r = subprocess.run([sys.executable, str(script), str(inp), str(out)],
                       capture_output=True, text=True, timeout=600)
    if r.returncode != 0:
        pytest.skip("triton interpreter unavailable: " + r.stderr[-300:])
    ref = np.load(out)
    mine = np.array([oracle.philox4x32_10(ctr[i], key[i]) for i in range(N)])
    np.testing.assert_array_equal(mine, ref)


def test_uniform_map_endpoints():
    # u = (w + 1/2) 2^-32: strictly inside (0, 1), symmetric about 1/2
    assert oracle.uniform(0) == 2.0 ** -33
    assert oracle.uniform(2**32 - 1) == 1.0 - 2.0 ** -33
    assert oracle.uniform(2**31) == 0.5 + 2.0 ** -33


def test_angle_uniform_grid():
    # (k + 1/2) / 1024 for a 10-bit index: the midpoints of 1024 equal cells
    assert oracle.angle_uniform(0) == 0.5 / 1024
    assert oracle.angle_uniform(1023) == 1.0 - 0.5 / 1024
    assert oracle.angle_uniform(512) == 0.5 + 0.5 / 1024


def test_normals_are_standard_normal():
    """Box-Muller output: Kolmogorov-Smirnov against N(0,1) per component, unit
    variance, no correlation between the six components of a move, between
    consecutive moves, or in the initial positions."""
    stats = pytest.importorskip("scipy.stats")
    even = np.array([oracle.move_normals(99, i, 6, 1) for i in range(20000)])
    odd = np.array([oracle.move_normals(99, i, 7, 1) for i in range(20000)])
    init = np.array([oracle.init_normals(99, i, 1) for i in range(20000)])
    for xs in (even, odd, init):
        for d in range(6):
            p = stats.kstest(xs[:, d], "norm").pvalue
            assert p > 1e-4, (d, p)
        assert abs(xs.mean()) < 0.01
        assert abs(xs.var() - 1.0) < 0.01
    cc = np.corrcoef(np.hstack([even, odd, init]).T)
    assert np.max(np.abs(cc - np.eye(18))) < 0.03
    # distinct counters give distinct streams
    a = oracle.move_normals(0, 5, 0, 0)
    for other in (oracle.move_normals(0, 5, 1, 0), oracle.move_normals(0, 5, 2, 0),
                  oracle.move_normals(0, 5, 0, 1), oracle.move_normals(0, 6, 0, 0),
                  oracle.move_normals(1, 5, 0, 0), oracle.move_normals(1 << 32, 5, 0, 0),
                  oracle.init_normals(0, 5, 0)):
        assert not np.allclose(a, other)


def test_normals_layout_and_angle_grid():
    """Move n of a walker is the one Philox block (walker, n, instance, 0) and the
    initial position the block (walker, 0, instance, 1): the radii of its three
    Box-Muller pairs come from words 0, 1, 2 (rho^2 = -2 ln u, u = (w + 1/2) 2^-32)
    and every pair's angle lies on the 1024-point grid 2 pi (k + 1/2) / 1024, with
    k the 10-bit fields of word 3 in order.  The angular moments of such a grid are
    the continuous ones: the mean of cos^2 over it is 1/2 and of cos^4 3/8."""
    for seed, walker, step, inst in ((99, 7, 6, 1), (3, 1 << 20, 12345, 0), (1 << 40, 0, 0, 9)):
        for tag, xi in ((0, oracle.move_normals(seed, walker, step, inst)),
                        (1, oracle.init_normals(seed, walker, inst))):
            n = step if tag == 0 else 0
            w = oracle.philox4x32_10([walker, n, inst, tag],
                                     [seed & 0xffffffff, seed >> 32]).astype(np.uint64)
            for j in range(3):
                a, b = xi[2 * j], xi[2 * j + 1]
                u = (float(w[j]) + 0.5) * 2.0 ** -32
                assert abs((a * a + b * b) - (-2.0 * math.log(u))) <= 1e-12 * max(1.0, a * a + b * b)
                k = (int(w[3]) >> (10 * j)) & 1023
                ang = math.atan2(b, a) % (2 * math.pi)
                want = 2 * math.pi * (k + 0.5) / 1024
                assert abs(math.remainder(ang - want, 2 * math.pi)) <= 1e-12
    grid = 2 * np.pi * (np.arange(1024) + 0.5) / 1024
    assert abs(np.mean(np.cos(grid) ** 2) - 0.5) < 1e-15
    assert abs(np.mean(np.cos(grid) ** 4) - 0.375) < 1e-15


# --------------------------------------------------------------------------
# Trial functions: closed forms, finite differences, symmetry
# --------------------------------------------------------------------------

def _rand_points(n, seed, scale=1.0):
    rng = np.random.default_rng(seed)
    return rng.normal(0.0, scale, size=(n, 6))


def _mp_lnpsi(kind, params, X):
    """ln|psi| written from the definition, in 50-digit arithmetic."""
    x1 = [X[0], X[1], X[2]]
    x2 = [X[3], X[4], X[5]]
    r1 = mp.sqrt(sum(v * v for v in x1))
    r2 = mp.sqrt(sum(v * v for v in x2))
    r12 = mp.sqrt(sum((x1[d] - x2[d]) ** 2 for d in range(3)))
    if kind == 0:
        Z, a, beta = (mp.mpf(params[0]), mp.mpf(params[1]), mp.mpf(params[2]))
        ck = [mp.mpf(c) for c in params[3:]] + [mp.mpf(0)] * (7 - len(params))
        rho = r12 / (1 + beta * r12)
        u = a * rho + sum(ck[k] * rho ** (k + 2) for k in range(4))
        return -Z * r1 - Z * r2 + u
    a, beta = mp.mpf(params[0]), mp.mpf(params[1])
    ck = [mp.mpf(c) for c in params[2:6]]
    nt = int(params[6])
    phi = mp.mpf(0)
    for t in range(nt):
        q = [mp.mpf(v) for v in params[7 + 9 * t: 16 + 9 * t]]
        s = q[0]
        fa = (q[2] + q[3] * r1 + q[4] * x1[2]) * mp.exp(-q[1] * r1)
        fb = (q[6] + q[7] * r2 + q[8] * x2[2]) * mp.exp(-q[5] * r2)
        phi += s * fa * fb
    rho = r12 / (1 + beta * r12) if beta != 0 else r12
    u = a * rho + sum(ck[k] * rho ** (k + 2) for k in range(4))
    return mp.log(abs(phi)) + u


def _mp_drift_el(kind, params, X, ee_on=True):
    """b = grad ln|psi| and E_L = -(Lap ln|psi| + |grad ln|psi||^2)/2 + V by central
    differences at 50 digits (h = 1e-12: truncation ~1e-24, rounding ~1e-26)."""
    mp.mp.dps = 50
    Xm = [mp.mpf(float(v)) for v in X]
    h = mp.mpf("1e-12")
    f0 = _mp_lnpsi(kind, params, Xm)
    grad, lap = [], mp.mpf(0)
    for d in range(6):
        xp = list(Xm); xp[d] += h
        xm = list(Xm); xm[d] -= h
        fp, fm = _mp_lnpsi(kind, params, xp), _mp_lnpsi(kind, params, xm)
        grad.append((fp - fm) / (2 * h))
        lap += (fp - 2 * f0 + fm) / (h * h)
    r1 = mp.sqrt(sum(v * v for v in Xm[:3]))
    r2 = mp.sqrt(sum(v * v for v in Xm[3:]))
    r12 = mp.sqrt(sum((Xm[d] - Xm[3 + d]) ** 2 for d in range(3)))
    V = -2 / r1 - 2 / r2 + (1 / r12 if ee_on else 0)
    el = -(lap + sum(g * g for g in grad)) / 2 + V
    return np.array([float(g) for g in grad]), float(el), float(f0)


TRIALS = {
    "ground": (0, wl.ground()),
    "ground_jastrow_poly": (0, wl.ground(Z=1.85, a=0.5, beta=0.37, c=(0.11, -0.07, 0.05, 0.02))),
    "triplet_2s3": (1, wl.triplet_2s3()),
    "pz_plus": (1, wl.pz_state(+1.0)),
    "pz_minus": (1, wl.pz_state(-1.0)),
    "fn3": (1, wl.fn3()),
    "fn5": (1, wl.fn3(0.73351723, 0.636748, 2.002777)),
    "fn7": (1, wl.fn7(1.1, 1.9, a=0.5, beta=0.6)),
    "pairs_poly_jastrow": (1, wl.pairs([wl.term(1.0, wl.orb(1.7, 0.3, 0.4, 0.2), wl.orb(0.8)),
                                        wl.term(-0.6, wl.orb(0.8, 1.0, -0.3), wl.orb(1.7, 0.0, 0.0, 1.0))],
                                       a=0.3, beta=0.45, c=(0.02, 0.01, -0.03, 0.04))),
}


@pytest.mark.parametrize("name", sorted(TRIALS))
def test_drift_and_local_energy_match_50_digit_finite_differences(name):
    kind, p = TRIALS[name]
    for X in _rand_points(6, seed=hash(name) % 1000, scale=0.9):
        s, b, el, lp = oracle.trial_eval(kind, p, X)
        gb, gel, glp = _mp_drift_el(kind, p, X)
        assert s in (1, -1)
        np.testing.assert_allclose(lp, glp, rtol=1e-13, atol=1e-13)
        np.testing.assert_allclose(b, gb, rtol=1e-10, atol=1e-10 * max(1.0, np.abs(gb).max()))
        assert abs(el - gel) <= 1e-10 * max(1.0, abs(gel)), (el, gel)


def test_hydrogenic_product_has_constant_local_energy():
    """exp(-2 r1 - 2 r2) is an exact eigenfunction of H without e-e repulsion:
    E_L = -4 everywhere and the drift is -2 r_hat per electron."""
    p = wl.ground(Z=2.0, a=0.0)
    for X in _rand_points(200, 1, 1.5):
        s, b, el, _ = oracle.trial_eval(0, p, X, ee_on=False)
        r1, r2 = np.linalg.norm(X[:3]), np.linalg.norm(X[3:])
        assert s == 1
        assert abs(el + 4.0) <= 4e-15 * (1 + 2 / r1 + 2 / r2)
        np.testing.assert_allclose(b[:3], -2.0 * X[:3] / r1, rtol=1e-14, atol=1e-15)
        np.testing.assert_allclose(b[3:], -2.0 * X[3:] / r2, rtol=1e-14, atol=1e-15)


@pytest.mark.parametrize("trial", ["1s2s", "1s2pz+", "1s2pz-"])
def test_excited_hydrogenic_products_have_constant_local_energy(trial):
    """1s(Z=2)2s(Z=2) antisymmetrised (= trial function 3 with r0=1, alpha=(1,2)) and
    1s 2p_z (anti)symmetrised are exact without e-e repulsion: E = -Z^2/2 - Z^2/8 = -2.5."""
    p = {"1s2s": wl.hydrogenic_1s2s_triplet(), "1s2pz+": wl.hydrogenic_1s2pz(+1.0),
         "1s2pz-": wl.hydrogenic_1s2pz(-1.0)}[trial]
    for X in _rand_points(200, 2, 1.5):
        s, b, el, _ = oracle.trial_eval(1, p, X, ee_on=False)
        if s == 0:
            continue
        r1, r2 = np.linalg.norm(X[:3]), np.linalg.norm(X[3:])
        assert abs(el + 2.5) <= 1e-12 * (1 + 2 / r1 + 2 / r2), el


def _swap(X):
    return np.concatenate([X[3:], X[:3]])


@pytest.mark.parametrize("name,parity", [("ground", 1), ("ground_jastrow_poly", 1),
                                         ("triplet_2s3", -1), ("fn3", -1), ("fn5", -1),
                                         ("pz_plus", 1), ("pz_minus", -1), ("fn7", 1)])
def test_exchange_symmetry(name, parity):
    """psi(P12 X) = +-psi(X); hence b(P12 X) = P12 b(X) and E_L(P12 X) = E_L(X)."""
    kind, p = TRIALS[name]
    for X in _rand_points(50, 3, 1.2):
        s, b, el, lp = oracle.trial_eval(kind, p, X)
        s2, b2, el2, lp2 = oracle.trial_eval(kind, p, _swap(X))
        assert s2 == parity * s
        assert abs(lp2 - lp) <= 1e-13 * max(1, abs(lp))
        np.testing.assert_allclose(b2, _swap(b), rtol=1e-12, atol=1e-12)
        assert abs(el2 - el) <= 1e-11 * max(1, abs(el))


def test_triplet_node_is_r1_equals_r2():
    """The 2^3S trial changes sign exactly where r1 = r2 (the exact node)."""
    kind, p = TRIALS["triplet_2s3"]
    for X in _rand_points(500, 4, 1.3):
        s, *_ = oracle.trial_eval(kind, p, X)
        r1, r2 = np.linalg.norm(X[:3]), np.linalg.norm(X[3:])
        assert s == (1 if r2 > r1 else -1)


def test_fn7_node_is_z1_plus_z2_plane():
    """Trial function 7 vanishes on z1 = -z2 (the necessary nodal condition for P_z)."""
    kind, p = TRIALS["fn7"]
    for X in _rand_points(500, 5, 1.3):
        s, *_ = oracle.trial_eval(kind, p, X)
        assert s == (1 if X[2] + X[5] > 0 else -1)


def test_bad_parameter_vectors_rejected():
    with pytest.raises(ValueError):
        oracle.trial_eval(0, [2.0, 0.5], np.ones(6))
    with pytest.raises(ValueError):
        oracle.trial_eval(1, wl.triplet_2s3()[:-1], np.ones(6))
    with pytest.raises(ValueError):
        oracle.trial_eval(7, wl.ground(), np.ones(6))


# --------------------------------------------------------------------------
# The walk
# --------------------------------------------------------------------------

def test_exact_eigenfunction_gives_exact_weights():
    """With an exact eigenfunction (E_L = -4) the Feynman-Kac weight of Eq. 4 is
    exp(-(E_L - E_T) t) for every walker: E(t) = -4 and ln z(t) = -(-4 - E_T) t."""
    p = wl.ground(Z=2.0, a=0.0)
    dt = 0.01
    for e_t in (-4.0, -3.5):
        w = oracle.Walk(0, p, n_walkers=64, dt=dt, e_trial=e_t, seed=3, ee_on=False)
        w.advance(100)
        s = w.series()
        t = np.arange(101) * dt
        np.testing.assert_allclose(s["E"], -4.0, rtol=0, atol=1e-11)
        np.testing.assert_allclose(s["ln_z"], (4.0 + e_t) * t, rtol=0, atol=1e-11)
        np.testing.assert_allclose(s["ess"], 64.0, rtol=1e-12)
        assert w.alive.all()


def test_single_step_by_hand():
    """One walker, two steps, each recomputed from its definition: X0 = sigma xi(initial),
    X1 = X0 + b(X0) dt + sqrt(dt) xi(move 0), logw1 = -(E_L(X1) - E_T) dt, with b and
    E_L from 50-digit finite differences of ln psi (right-point rule)."""
    kind, p = TRIALS["ground_jastrow_poly"]
    dt, et, seed, sigma, wid, inst = 0.01, -2.9, 77, 0.5, 5, 2
    w = oracle.Walk(kind, p, ids=[wid], dt=dt, e_trial=et, seed=seed, inst=inst, sigma=sigma)
    X = sigma * oracle.init_normals(seed, wid, inst)
    np.testing.assert_array_equal(w.x[0], X)
    logw = 0.0
    for step in range(2):
        b, _, _ = _mp_drift_el(kind, p, X)
        X = X + b * dt + math.sqrt(dt) * oracle.move_normals(seed, wid, step, inst)
        _, el, _ = _mp_drift_el(kind, p, X)
        logw -= (el - et) * dt
        w.advance(1)
        np.testing.assert_allclose(w.x[0], X, rtol=1e-12, atol=1e-12)
        assert abs(w.logw[0] - logw) <= 1e-12
        assert abs(w.el[0] - el) <= 1e-10 * abs(el)


def test_population_sums_against_fsum():
    """E = sum w E_L / sum w, ESS = (sum w)^2 / sum w^2, z = sum w / N, recomputed with
    math.fsum from the oracle's per-walker state."""
    kind, p = TRIALS["triplet_2s3"]
    w = oracle.Walk(kind, p, n_walkers=300, dt=0.02, e_trial=-2.17, seed=5)
    w.advance(150)
    s = w.series()
    a = w.alive.astype(bool)
    wt = np.exp(w.logw[a])
    el = w.el[a]
    W = math.fsum(wt)
    assert abs(s["E"][-1] - math.fsum(wt * el) / W) <= 1e-14 * 3
    assert abs(s["ess"][-1] - W * W / math.fsum(wt * wt)) <= 1e-12 * s["ess"][-1]
    assert abs(s["ln_z"][-1] - math.log(W / 300)) <= 1e-13
    assert s["n_alive"][-1] == a.sum()


def _neumaier_bound(x, exact):
    # |error| <= 2 eps |sum| + 2 n eps^2 sum|x_i|  (Neumaier 1974)
    eps = 2.0 ** -53
    return 2 * eps * abs(exact) + 2 * len(x) * eps * eps * float(np.abs(x).sum())


def test_neumaier_sum_against_exact():
    """Compensated sums meet Neumaier's bound against math.fsum (exactly rounded),
    on inputs where a plain sum loses every digit."""
    v = np.array([1.0, 1e100, 1.0, -1e100, 3.0, 1e-3, -2.5e15, 2.5e15, 7e-17])
    exact = math.fsum(v)
    assert abs(oracle.neumaier_sum(v) - exact) <= _neumaier_bound(v, exact)
    plain = 0.0
    for e in v:
        plain += e
    assert abs(plain - exact) > 1.0          # a plain running sum loses the 1s here
    rng = np.random.default_rng(1)
    x = rng.normal(size=10000) * 10.0 ** rng.integers(-8, 8, size=10000)
    exact = math.fsum(x)
    assert abs(oracle.neumaier_sum(x) - exact) <= _neumaier_bound(x, exact)


def test_growth_identity():
    """ln z(t+dt) - ln z(t) = -(E(t+dt) - E_T) dt + O(dt^2 var(E_L)) (continuous-time
    link between Eq. 4's growth estimator and the space-averaged energy)."""
    kind, p = TRIALS["ground"]
    dt = 0.002
    w = oracle.Walk(kind, p, n_walkers=500, dt=dt, e_trial=-2.9, seed=11)
    w.advance(200)
    s = w.series()
    dlnz = np.diff(s["ln_z"])
    pred = -(s["E"][1:] - (-2.9)) * dt
    bound = 2.0 * dt * dt * (np.abs(s["var"][1:]) + np.abs(s["var"][:-1]) + 1.0)
    assert np.all(np.abs(dlnz - pred) <= bound)


def test_node_kill_invariants():
    """Fixed-node rule: alive walkers never leave the nodal pocket they started in
    (sign(r2 - r1) constant); a killed walker's frozen position lies on the other side."""
    kind, p = TRIALS["triplet_2s3"]
    w = oracle.Walk(kind, p, n_walkers=400, dt=0.02, e_trial=-2.17, seed=9)
    start = np.sign(np.linalg.norm(w.x[:, 3:], axis=1) - np.linalg.norm(w.x[:, :3], axis=1))
    for _ in range(10):
        w.advance(20)
        side = np.sign(np.linalg.norm(w.x[:, 3:], axis=1) - np.linalg.norm(w.x[:, :3], axis=1))
        a = w.alive.astype(bool)
        assert np.all(side[a] == start[a])
        assert np.all(side[~a] != start[~a])
        assert np.all(np.isneginf(w.logw[~a]))
    assert (~w.alive.astype(bool)).sum() > 0
    assert w.counters[1] == (~w.alive.astype(bool)).sum()


def test_shard_merge_equals_single_population():
    """Walkers are independent and the random stream is keyed by walker id, so two
    shards' per-step sums, merged with their shifts, equal the full population's."""
    kind, p = TRIALS["ground"]
    kw = dict(dt=0.01, e_trial=-2.9, seed=4)
    full = oracle.Walk(kind, p, n_walkers=200, **kw).advance(50)
    a = oracle.Walk(kind, p, ids=np.arange(0, 120), **kw).advance(50)
    b = oracle.Walk(kind, p, ids=np.arange(120, 200), **kw).advance(50)
    np.testing.assert_array_equal(np.vstack([a.x, b.x]), full.x)
    np.testing.assert_array_equal(np.concatenate([a.logw, b.logw]), full.logw)
    ra, rb, rf = np.array(a.rows), np.array(b.rows), np.array(full.rows)
    c = np.maximum(ra[:, 0], rb[:, 0])
    for col, pw in ((1, 1), (2, 1), (3, 2), (4, 1)):
        merged = ra[:, col] * np.exp(pw * (ra[:, 0] - c)) + rb[:, col] * np.exp(pw * (rb[:, 0] - c))
        np.testing.assert_allclose(merged, rf[:, col] * np.exp(pw * (rf[:, 0] - c)), rtol=1e-14)


def test_resume_is_bitwise():
    kind, p = TRIALS["pz_plus"]
    kw = dict(dt=0.01, e_trial=-2.12, seed=8, inst=3)
    one = oracle.Walk(kind, p, n_walkers=50, **kw).advance(40)
    two = oracle.Walk(kind, p, n_walkers=50, **kw).advance(15).advance(25)
    np.testing.assert_array_equal(one.x, two.x)
    np.testing.assert_array_equal(one.logw, two.logw)
    np.testing.assert_array_equal(np.array(one.rows), np.array(two.rows))


def _stationary_mean_el(kind, p, n, steps, burn, dt, seed, ee_on=True, sigma=0.5, noise=0):
    """Unweighted time-and-space average of E_L after burn-in, and its standard error
    from the spread of per-walker time averages (walkers are independent)."""
    w = oracle.Walk(kind, p, n_walkers=n, dt=dt, e_trial=0.0, seed=seed, ee_on=ee_on,
                    sigma=sigma, noise=noise)
    w.advance(burn)
    acc = np.zeros(n)
    cnt = np.zeros(n)
    for _ in range(steps):
        w.advance(1)
        a = w.alive.astype(bool)
        acc[a] += w.el[a]
        cnt[a] += 1
    m = acc[cnt > 0] / cnt[cnt > 0]
    return m.mean(), m.std(ddof=1) / math.sqrt(len(m))


@pytest.mark.parametrize("Z,exact", [(2.0, 4.0 - 27.0 / 4.0), (27.0 / 16.0, -(27.0 / 16.0) ** 2)])
def test_stationary_density_is_psi_squared(Z, exact):
    """The drifted walk samples psi^2 (the stationary law quoted under Eq. 4): for
    psi = exp(-Z (r1 + r2)) with e-e repulsion, <E_L>_{psi^2} = Z^2 - 27 Z / 8 (textbook
    variational closed form).  Checked within 5 standard errors plus an O(dt) allowance."""
    mean, se = _stationary_mean_el(0, wl.ground(Z=Z, a=0.0), n=1000, steps=600, burn=200,
                                   dt=0.002, seed=21)
    assert abs(mean - exact) < 5 * se + 0.01, (mean, exact, se)


def _slater_1s2s_triplet_energy(Z=2.0):
    """-Z^2/2 - Z^2/8 + J(1s,2s) - K(1s,2s) for hydrogenic orbitals of charge Z, with the
    Coulomb and exchange integrals done by 2-D radial quadrature (only the k = 0
    multipole survives for s orbitals)."""
    integrate = pytest.importorskip("scipy.integrate")
    P1 = lambda r: r * 2.0 * Z ** 1.5 * math.exp(-Z * r)
    P2 = lambda r: r * 2.0 * (Z / 2) ** 1.5 * (1 - Z * r / 2) * math.exp(-Z * r / 2)
    inner = lambda f, g: integrate.dblquad(lambda r2, r1: f(r1) * g(r2) / max(r1, r2),
                                           0, 40, 0, 40, epsabs=1e-11, epsrel=1e-11)[0]
    J = inner(lambda r: P1(r) ** 2, lambda r: P2(r) ** 2)
    K = inner(lambda r: P1(r) * P2(r), lambda r: P1(r) * P2(r))
    return -Z * Z / 2 - Z * Z / 8 + J - K, J, K


def test_fn3_variational_energy_matches_table1_lambda0():
    """Trial function 3 with r0 = 1, alpha = (1, 2) is the antisymmetrised hydrogenic
    1s2s product, so its variational energy is -2.5 + J - K.  The paper prints
    lambda0 = -2.12412661 for it (Table 1).  The walk's stationary <E_L> must
    reproduce that energy within its statistical error (the diffuse 2s electron
    needs ~10 a.u. of burn-in, so the population starts wide and walks 10 a.u.)."""
    e_var, J, K = _slater_1s2s_triplet_energy()
    assert abs(J - 17 * 2 / 81) < 1e-8 and abs(K - 16 * 2 / 729) < 1e-8   # textbook values
    assert abs(e_var - (-2.12412661)) < 5e-5                               # Table 1 lambda0
    mean, se = _stationary_mean_el(1, wl.fn3(), n=1000, steps=1000, burn=1000, dt=0.01,
                                   seed=31, sigma=1.5)
    assert abs(mean - e_var) < 5 * se + 0.01, (mean, e_var, se)


# --------------------------------------------------------------------------
# Gradient oracle (PyTorch CPU FP64 autograd)
# --------------------------------------------------------------------------

def test_grad_oracle_drift_and_energy_match_c_oracle():
    """The autograd drift and Laplacian of ln psi reproduce the C oracle's closed forms."""
    torch = pytest.importorskip("torch")
    from oracle import grad as og
    theta = [1.85, 0.5, 0.37, 0.11, -0.07, 0.05, 0.02]
    X = _rand_points(16, 8, 0.9)
    b, el = og.drift_and_local_energy(torch.tensor(X), torch.tensor(theta, dtype=torch.float64))
    for i in range(16):
        _, bc, elc, _ = oracle.trial_eval(0, theta, X[i])
        np.testing.assert_allclose(b[i].detach().numpy(), bc, rtol=1e-12, atol=1e-12)
        assert abs(float(el[i]) - elc) <= 1e-11 * max(1, abs(elc))


@pytest.mark.parametrize("noise", [0, 1])
def test_grad_oracle_loss_matches_c_oracle_walk(noise):
    """Its walk is the C oracle's walk (either noise mode): same final E(t) and weighted
    variance."""
    torch = pytest.importorskip("torch")
    from oracle import grad as og
    theta = [2.0, 0.5, 0.5, 0.0, 0.0, 0.0, 0.0]
    kw = dict(n_walkers=24, n_steps=12, dt=0.01, e_trial=-2.9, seed=4, inst=1, noise=noise)
    L = og.walk_loss(torch.tensor(theta, dtype=torch.float64), **kw)
    V = og.walk_loss(torch.tensor(theta, dtype=torch.float64), loss_kind=1, **kw)
    w = oracle.Walk(0, theta, n_walkers=24, dt=0.01, e_trial=-2.9, seed=4, inst=1,
                    noise=noise).advance(12)
    s = w.series()
    assert abs(float(L) - s["E"][-1]) <= 1e-11
    assert abs(float(V) - s["var"][-1]) <= 1e-10


def test_grad_oracle_gradient_matches_finite_differences():
    """autograd's d(loss)/d(theta) equals central differences of the same loss
    (common random numbers, h = 1e-5), for both losses."""
    torch = pytest.importorskip("torch")
    from oracle import grad as og
    theta = np.array([1.9, 0.5, 0.45, 0.05, -0.02, 0.01, 0.003])
    kw = dict(n_walkers=12, n_steps=8, dt=0.01, e_trial=-2.9, seed=7)
    for loss_kind in (0, 1):
        _, g = og.gradient(theta, loss_kind=loss_kind, **kw)
        h = 1e-5
        for k in range(7):
            tp, tm = theta.copy(), theta.copy()
            tp[k] += h
            tm[k] -= h
            fd = (float(og.walk_loss(torch.tensor(tp), loss_kind=loss_kind, **kw)) -
                  float(og.walk_loss(torch.tensor(tm), loss_kind=loss_kind, **kw))) / (2 * h)
            assert abs(fd - g[k]) <= 1e-6 * max(1.0, np.abs(g).max()), (loss_kind, k, fd, g[k])


# --------------------------------------------------------------------------
# Bernoulli steps from the "Superduper" congruential generator
# --------------------------------------------------------------------------

_SD_A, _SD_M = 69069, 1 << 32


def _sd_closed_form(s0, k):
    """S_k of S_i = (a S_{i-1} + 1) mod 2^32 in closed form: a^k S_0 + (a^k - 1)/(a - 1),
    the geometric series summed exactly in Python integers before the reduction."""
    ak = _SD_A ** k
    return (ak * s0 + (ak - 1) // (_SD_A - 1)) % _SD_M


def _affine_pow_mod(k):
    """(A, C) with S_k = A S_0 + C mod 2^32, by binary powering of the affine map
    S -> a S + 1 (an independent route to the same numbers, usable at k = 2^32)."""
    A, C = 1, 0                   # identity
    a, c = _SD_A, 1               # the map applied 2^j times
    while k:
        if k & 1:
            A, C = (a * A) % _SD_M, (a * C + c) % _SD_M
        a, c = (a * a) % _SD_M, (a * c + c) % _SD_M
        k >>= 1
    return A, C


def test_superduper_recurrence_matches_closed_form():
    """Outputs of the oracle's generator equal the closed form of the congruential
    recurrence (a dropped increment, a wrong multiplier or a lost wrap-around fails)."""
    rng = np.random.default_rng(12)
    for s0 in [0, 1, 2 ** 31, 2 ** 32 - 1, *rng.integers(0, 2 ** 32, 4).tolist()]:
        s = int(s0)
        for k in range(1, 2001):
            s = oracle.superduper_next(s)
            if k in (1, 2, 3, 17, 640, 2000):
                assert s == _sd_closed_form(int(s0), k), (s0, k)
    assert oracle.superduper_next(1) == 69070


def test_superduper_has_the_full_period():
    """The generator's cycle is 2^32 (the paper chooses a cycle of 2^32): the affine map
    composed 2^32 times is the identity and 2^31 times is not (Hull-Dobell: c odd,
    a = 1 mod 4); and the binary powering agrees with the closed form at small k."""
    for k in (1, 5, 100, 999):
        A, C = _affine_pow_mod(k)
        assert (A * 12345 + C) % _SD_M == _sd_closed_form(12345, k)
    assert _affine_pow_mod(1 << 32) == (1, 0)
    assert _affine_pow_mod(1 << 31) != (1, 0)
    assert _SD_A % 4 == 1


def test_bernoulli_threshold_is_the_papers():
    """eps = +1 if S > 2^31, else -1 (so S = 2^31 itself gives -1)."""
    cases = {0: -1, 1: -1, 2 ** 31 - 1: -1, 2 ** 31: -1, 2 ** 31 + 1: 1, 2 ** 32 - 1: 1}
    for st, e in cases.items():
        assert oracle.bernoulli_eps(st) == e, st


def test_bernoulli_move_consumes_six_outputs_per_move():
    """Move `step` of a walker uses outputs 6 step + 1 .. 6 step + 6 of its generator,
    which starts at word 0 of the Philox block (walker, 0, stream, 5)."""
    for seed, walker, step, inst in [(0, 0, 0, 0), (5, 17, 3, 2), (2 ** 40 + 7, 999, 250, 7)]:
        key = [seed & 0xFFFFFFFF, seed >> 32]
        s0 = int(oracle.philox4x32_10([walker, 0, inst, 5], key)[0])
        assert oracle.superduper_seed(seed, walker, inst) == s0
        want = [1.0 if _sd_closed_form(s0, 6 * step + d + 1) > 2 ** 31 else -1.0
                for d in range(6)]
        np.testing.assert_array_equal(oracle.move_bernoulli(seed, walker, step, inst), want)


def test_bernoulli_increments_are_balanced_and_independent():
    """+1 and -1 equally likely, no correlation between coordinates, between the
    consecutive moves of a walker, or between neighbouring walkers (4 standard errors)."""
    n = 3000
    e = np.array([[oracle.move_bernoulli(3, i, st, 1) for st in (0, 1)] for i in range(n)])
    tol = 4.0 / math.sqrt(n)
    assert abs(e.mean()) < 4.0 / math.sqrt(e.size)
    c = np.corrcoef(e[:, 0, :].T)
    assert np.abs(c - np.eye(6)).max() < tol
    for d in range(6):
        assert abs(np.corrcoef(e[:, 0, d], e[:, 1, d])[0, 1]) < tol
        assert abs(np.corrcoef(e[:-1, 0, d], e[1:, 0, d])[0, 1]) < tol


def test_bernoulli_single_step_by_hand():
    """X1 = X0 + b(X0) dt + sqrt(dt) eps, logw1 = -(E_L(X1) - E_T) dt, with b and E_L from
    50-digit finite differences of ln psi and eps from the pinned generator."""
    kind, p = TRIALS["ground_jastrow_poly"]
    dt, et, seed, sigma, wid, inst = 1.0 / 900.0, -2.9, 41, 0.5, 9, 1
    w = oracle.Walk(kind, p, ids=[wid], dt=dt, e_trial=et, seed=seed, inst=inst, sigma=sigma,
                    noise=oracle.NOISE_BERNOULLI)
    X = sigma * oracle.init_normals(seed, wid, inst)
    np.testing.assert_array_equal(w.x[0], X)
    logw = 0.0
    for step in range(3):
        b, _, _ = _mp_drift_el(kind, p, X)
        X = X + b * dt + math.sqrt(dt) * oracle.move_bernoulli(seed, wid, step, inst)
        _, el, _ = _mp_drift_el(kind, p, X)
        logw -= (el - et) * dt
        w.advance(1)
        np.testing.assert_allclose(w.x[0], X, rtol=1e-12, atol=1e-12)
        assert abs(w.logw[0] - logw) <= 1e-12
        assert abs(w.el[0] - el) <= 1e-10 * abs(el)


def test_bernoulli_exact_eigenfunction_gives_exact_weights():
    p = wl.ground(Z=2.0, a=0.0)
    dt = 1.0 / 900.0
    w = oracle.Walk(0, p, n_walkers=64, dt=dt, e_trial=-3.5, seed=3, ee_on=False,
                    noise=oracle.NOISE_BERNOULLI)
    w.advance(200)
    s = w.series()
    np.testing.assert_allclose(s["E"], -4.0, rtol=0, atol=1e-11)
    np.testing.assert_allclose(s["ln_z"], (4.0 - 3.5) * np.arange(201) * dt, rtol=0, atol=1e-11)
    assert w.alive.all()


def test_bernoulli_walk_resume_is_bitwise():
    kind, p = TRIALS["triplet_2s3"]
    kw = dict(dt=0.0025, e_trial=-2.17, seed=8, inst=3, noise=oracle.NOISE_BERNOULLI)
    one = oracle.Walk(kind, p, n_walkers=50, **kw).advance(40)
    two = oracle.Walk(kind, p, n_walkers=50, **kw).advance(15).advance(25)
    np.testing.assert_array_equal(one.x, two.x)
    np.testing.assert_array_equal(one.lcg, two.lcg)
    np.testing.assert_array_equal(np.array(one.rows), np.array(two.rows))


def test_bernoulli_walk_samples_psi_squared():
    """By the invariance principle the +-1 walk converges to the drifted diffusion, whose
    stationary law is psi^2: for psi = exp(-2 (r1 + r2)) with e-e repulsion,
    <E_L> = 4 - 27/4 = -2.75 (textbook closed form), within 5 standard errors plus an
    O(dt) allowance."""
    mean, se = _stationary_mean_el(0, wl.ground(Z=2.0, a=0.0), n=1000, steps=600, burn=200,
                                   dt=0.002, seed=23, noise=oracle.NOISE_BERNOULLI)
    assert abs(mean - (4.0 - 27.0 / 4.0)) < 5 * se + 0.01, (mean, se)
