"""The Bernoulli walk (the paper's +-1 steps from the "Superduper" generator) on
the GPU, through the C ABI, against the FP64 oracle's serial generators.

The kernels do not store the generator state: each launch skips every walker's
generator ahead to its first move, so runs split into chunks of odd lengths
exercise that skip at many starting steps.
"""
import numpy as np
import pytest

import oracle
from paper_1703_08977_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

REL_WALKER = 1e-12
DT = 1.0 / 900.0            # the paper's scale 30: step length 1/30 = sqrt(dt)


def _gpu(gfk, kind, params, n, chunks, dt, et, seed, prec, stream_id=0, launch=None,
         walker_id0=0):
    d = gfk.InstanceDesc(n_walkers=n, dt=dt, e_trial=et, seed=seed, prec=prec,
                         rng_stream=stream_id, noise=gfk.GFK_NOISE_BERNOULLI,
                         walker_id0=walker_id0)
    with gfk.Context([d], trials=[(kind, params)], launch=launch) as ctx:
        for c in chunks:
            ctx.propagate(c)
        x, lw, al = ctx.walkers(0)
        return dict(x=x, logw=lw, alive=al, energy=ctx.energy(0), sums=ctx.sums(0),
                    counters=ctx.counters(0))


def _oracle(kind, params, n, steps, dt, et, seed, stream_id=0):
    w = oracle.Walk(kind, params, n_walkers=n, dt=dt, e_trial=et, seed=seed, inst=stream_id,
                    noise=oracle.NOISE_BERNOULLI)
    return w.advance(steps)


def _errors(g, w):
    a = w.alive.astype(bool)
    np.testing.assert_array_equal(g["alive"].astype(bool), a)
    dx = np.abs(g["x"] - w.x).max(axis=1) / np.maximum(1.0, np.abs(w.x).max(axis=1))
    dl = np.zeros_like(dx)
    dl[a] = np.abs(g["logw"][a] - w.logw[a]) / np.maximum(1.0, np.abs(w.logw[a]))
    return dx, dl


def test_fp64_bernoulli_ground_matches_oracle_across_chunks(gfk_lib):
    """Ground state, 2061 walkers (ragged), 500 moves at dt = 1/900 in chunks of 37, 200
    and 263 moves: every walker to 1e-12 and every step of E(t) to 1e-13."""
    gfk = gfk_lib
    p = wl.ground()
    n, chunks, et, seed = 2048 + 13, [37, 200, 263], -2.9037, 5
    g = _gpu(gfk, 0, p, n, chunks, DT, et, seed, gfk.GFK_PREC_FP64, stream_id=2)
    w = _oracle(0, p, n, sum(chunks), DT, et, seed, stream_id=2)
    dx, dl = _errors(g, w)
    assert dx.max() <= REL_WALKER and dl.max() <= REL_WALKER, (dx.max(), dl.max())
    s = w.series()
    np.testing.assert_allclose(g["energy"]["E"], s["E"], rtol=1e-13, atol=0)
    np.testing.assert_allclose(g["energy"]["ln_z"], s["ln_z"], rtol=0, atol=1e-12)
    np.testing.assert_array_equal(g["sums"][:, 5], s["n_alive"])


@pytest.mark.parametrize("name", ["triplet_2s3", "pz_plus"])
def test_fp64_bernoulli_node_kills_match_oracle(gfk_lib, name):
    """Excited states: the +-1 steps cross the node; kill decisions and counts agree
    exactly with the oracle, walkers to 1e-12 (a few near-node walkers to 1e-8)."""
    gfk = gfk_lib
    kind, p, et = {"triplet_2s3": (1, wl.triplet_2s3(), -2.1752),
                   "pz_plus": (1, wl.pz_state(+1.0), -2.1238)}[name]
    n, chunks, seed = 1000 + 37, [100, 101, 99], 9
    g = _gpu(gfk, kind, p, n, chunks, 0.0025, et, seed, gfk.GFK_PREC_FP64, stream_id=1)
    w = _oracle(kind, p, n, sum(chunks), 0.0025, et, seed, stream_id=1)
    dx, dl = _errors(g, w)
    bad = (dx > REL_WALKER) | (dl > REL_WALKER)
    assert bad.sum() <= max(2, n // 200), (bad.sum(), dx.max(), dl.max())
    assert dx.max() <= 1e-8 and dl.max() <= 1e-8
    if name == "triplet_2s3":
        assert w.counters[1] > 0                 # the +-1 steps do cross the node r1 = r2
    np.testing.assert_array_equal(g["counters"][:2], w.counters[:2])
    np.testing.assert_allclose(g["energy"]["E"], w.series()["E"], rtol=1e-11, atol=0)


def test_mixed_bernoulli_tracks_oracle(gfk_lib):
    """FP32 physics with the same +-1 steps: walkers within FP32-level distance of the
    oracle's FP64 trajectories after 130 moves (chunks 30 + 100), E(t) within 1e-4."""
    gfk = gfk_lib
    p = wl.ground()
    n, chunks = 2048 + 11, [30, 100]
    g = _gpu(gfk, 0, p, n, chunks, 0.005, -2.9, 3, gfk.GFK_PREC_MIXED, launch=(256, 2))
    w = _oracle(0, p, n, sum(chunks), 0.005, -2.9, 3)
    np.testing.assert_array_equal(g["alive"], w.alive)
    dx = np.abs(g["x"] - w.x).max(axis=1)
    assert np.median(dx) < 1e-5 and np.quantile(dx, 0.99) < 1e-3, (np.median(dx), dx.max())
    assert np.median(np.abs(g["logw"] - w.logw)) < 1e-5
    assert np.max(np.abs(g["energy"]["E"] - w.series()["E"])) < 1e-4


@pytest.mark.parametrize("prec", [0, 1])
def test_bernoulli_launch_shape_resume_and_shards(gfk_lib, prec):
    """Walkers do not depend on the launch shape, on 64-move chunking with a checkpoint
    restored into a fresh context, or on sharding by walker id."""
    gfk = gfk_lib
    p = wl.triplet_2s3()
    kw = dict(dt=0.0025, e_trial=-2.1752, seed=6, prec=prec, noise=gfk.GFK_NOISE_BERNOULLI)
    d = gfk.InstanceDesc(n_walkers=1500, **kw)
    one = gfk.Context([d], trials=[(1, p)], launch=(128, 1 if prec == 0 else 2)).propagate(256)
    other = gfk.Context([d], trials=[(1, p)], launch=(512, 1) if prec == 0 else (64, 4)).propagate(256)
    two = gfk.Context([d], trials=[(1, p)]).propagate(64)
    blob = two.checkpoint()
    three = gfk.Context([d], trials=[(1, p)])
    three.restore(blob)
    three.propagate(192)
    ref = one.walkers()
    for c in (other, three):
        for u, v in zip(ref, c.walkers()):
            np.testing.assert_array_equal(u, v)
    np.testing.assert_array_equal(one.sums()[:, 5], three.sums()[:, 5])
    parts = [gfk.Context([gfk.InstanceDesc(n_walkers=k, walker_id0=i0, **kw)],
                         trials=[(1, p)]).propagate(256) for i0, k in ((0, 700), (700, 800))]
    xs = [c.walkers() for c in parts]
    np.testing.assert_array_equal(np.vstack([xs[0][0], xs[1][0]]), ref[0])
    np.testing.assert_array_equal(np.concatenate([xs[0][2], xs[1][2]]), ref[2])
    for c in [one, other, two, three] + parts:
        c.close()


def test_bernoulli_differs_from_gaussian_and_moves_by_sqrt_dt(gfk_lib):
    """The noise mode is honoured: with psi's drift removed from the displacement, every
    coordinate of a one-move Bernoulli step is exactly +-sqrt(dt) (FP64 path), whereas
    the Gaussian step is not."""
    gfk = gfk_lib
    p = wl.ground()
    n, dt = 512, 0.0025
    res = {}
    for noise in (0, 1):
        d = gfk.InstanceDesc(n_walkers=n, dt=dt, e_trial=-2.9, seed=4, prec=0, noise=noise)
        with gfk.Context([d], trials=[(0, p)]) as ctx:
            ctx.propagate(0)
            x0 = ctx.walkers(0)[0]
            ctx.propagate(1)
            res[noise] = (x0, ctx.walkers(0)[0])
    for noise, (x0, x1) in res.items():
        b = np.array([oracle.trial_eval(0, p, x)[1] for x in x0])
        step = (x1 - (x0 + b * dt)) / np.sqrt(dt)
        if noise == 1:
            np.testing.assert_allclose(np.abs(step), 1.0, rtol=0, atol=1e-9)
        else:
            assert np.abs(np.abs(step) - 1.0).max() > 0.5


def test_fp64_bernoulli_gradient_matches_autograd_oracle(gfk_lib):
    """gfk_grad with Bernoulli noise: the adjoint's segment recompute skips each
    walker's generator to the segment start; the gradient equals autograd through the
    oracle's Bernoulli walk."""
    pytest.importorskip("torch")
    from oracle import grad as og
    gfk = gfk_lib
    theta = [1.9, 0.5, 0.45, 0.05, -0.02, 0.01, 0.003]
    n, S, K = 40, 30, 8
    d = gfk.InstanceDesc(n_walkers=n, dt=0.01, e_trial=-2.9, seed=7, prec=0, rng_stream=1,
                         noise=gfk.GFK_NOISE_BERNOULLI)
    for loss_kind in (0, 1):
        with gfk.Context([d], trials=[(0, theta)]) as c:
            loss, g = gfk.gfk_grad(c.handle, 0, loss_kind, S, K)
        ref_loss, ref_g = og.gradient(theta, n_walkers=n, n_steps=S, dt=0.01, e_trial=-2.9,
                                      seed=7, inst=1, loss_kind=loss_kind, noise=1)
        assert abs(loss - ref_loss) <= 1e-12 * max(1.0, abs(ref_loss))
        np.testing.assert_allclose(g, ref_g, rtol=0, atol=1e-9 * max(1.0, np.abs(ref_g).max()))
