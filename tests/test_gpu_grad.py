"""The adjoint gradient gfk_grad (GPU) against the autograd oracle and against
common-random-number central finite differences."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

THETA = [1.9, 0.5, 0.45, 0.05, -0.02, 0.01, 0.003]


def _ctx(gfk, n, dt, prec, theta=THETA, seed=7, stream=1):
    d = gfk.InstanceDesc(n_walkers=n, dt=dt, e_trial=-2.9, seed=seed, prec=prec, rng_stream=stream)
    return gfk.Context([d], trials=[(0, theta)])


@pytest.mark.parametrize("loss_kind", [0, 1])
@pytest.mark.parametrize("S,K", [(24, 8), (30, 8), (17, 64)])
@pytest.mark.parametrize("n", [40, 41])
def test_fp64_grad_matches_autograd_oracle(gfk_lib, loss_kind, S, K, n):
    """FP64 adjoint (checkpointed every K moves, ragged last segment; an odd walker count
    pads the segment planes' stride) = autograd through the oracle's walk with the same
    Philox noise."""
    torch = pytest.importorskip("torch")
    from oracle import grad as og
    gfk = gfk_lib
    with _ctx(gfk, n, 0.01, gfk.GFK_PREC_FP64) as c:
        loss, g = gfk.gfk_grad(c.handle, 0, loss_kind, S, K)
    ref_loss, ref_g = og.gradient(THETA, n_walkers=n, n_steps=S, dt=0.01, e_trial=-2.9, seed=7,
                                  inst=1, loss_kind=loss_kind)
    assert abs(loss - ref_loss) <= 1e-12 * max(1.0, abs(ref_loss))
    np.testing.assert_allclose(g, ref_g, rtol=0, atol=1e-9 * max(1.0, np.abs(ref_g).max()))


@pytest.mark.parametrize("loss_kind", [0, 1])
def test_fp64_grad_matches_central_differences(gfk_lib, loss_kind):
    """The FP64 adjoint on 4096 walkers x 200 moves against CRN central differences of
    the same loss.  Plain central differences at h = 1e-4 carry a truncation error
    (h^2/6 times the third derivative) that reaches 1e-5 here, as halving h shows, so
    the 1e-6 comparison is made against the Richardson combination
    (4 D(h/2) - D(h)) / 3, whose error is O(h^4); the plain h = 1e-4 difference must
    still agree to 3e-5."""
    gfk = gfk_lib
    n, S, dt, h = 4096, 200, 0.005, 1e-4
    with _ctx(gfk, n, dt, gfk.GFK_PREC_FP64) as c:
        _, g = gfk.gfk_grad(c.handle, 0, loss_kind, S, 64)

        def central(step):
            fd = np.zeros(7)
            for k in range(7):
                vals = []
                for sgn in (+1, -1):
                    th = list(THETA)
                    th[k] += sgn * step
                    c.reset()
                    c.set_trial(0, 0, th)
                    vals.append(gfk.gfk_grad(c.handle, 0, loss_kind, S, 64)[0])
                fd[k] = (vals[0] - vals[1]) / (2 * step)
            return fd

        d1 = central(h)
        d2 = central(h / 2)
    rich = (4 * d2 - d1) / 3
    scale = np.abs(rich).max()
    err_rich = np.abs(g - rich).max() / scale
    err_plain = np.abs(g - d1).max() / scale
    assert err_rich <= 1e-6, (err_rich, err_plain, g, rich)
    assert err_plain <= 3e-5, (err_plain, g, d1)


@pytest.mark.parametrize("n", [8192, 8191])
def test_mixed_grad_close_to_fp64(gfk_lib, n):
    """The mixed path's gradient (FP32 positions and trial arithmetic, FP64 weights and
    adjoint sums) stays within 1e-3 of the FP64 gradient on the same seeds; also for an
    odd walker count (the segment planes' padded stride)."""
    gfk = gfk_lib
    S = 200
    with _ctx(gfk, n, 0.005, gfk.GFK_PREC_FP64) as c:
        l64, g64 = gfk.gfk_grad(c.handle, 0, 0, S, 64)
    with _ctx(gfk, n, 0.005, gfk.GFK_PREC_MIXED) as c:
        l32, g32 = gfk.gfk_grad(c.handle, 0, 0, S, 64)
    assert abs(l32 - l64) < 1e-5
    assert np.abs(g32 - g64).max() <= 1e-3 * np.abs(g64).max(), (g32, g64)


def test_grad_leaves_population_and_rejects_bad_calls(gfk_lib):
    gfk = gfk_lib
    with _ctx(gfk, 300, 0.01, gfk.GFK_PREC_FP64) as a, _ctx(gfk, 300, 0.01, gfk.GFK_PREC_FP64) as b:
        a.propagate(40)
        b.propagate(40)
        gfk.gfk_grad(b.handle, 0, 0, 20, 8)
        a.propagate(10)
        b.propagate(10)
        for u, v in zip(a.walkers(), b.walkers()):
            np.testing.assert_array_equal(u, v)
        with pytest.raises(gfk.GfkError):
            gfk.gfk_grad(a.handle, 0, 2, 10, 8)         # unknown loss
        with pytest.raises(gfk.GfkError):
            gfk.gfk_grad(a.handle, 0, 0, 0, 8)          # no moves
        with pytest.raises(gfk.GfkError):
            gfk.gfk_grad(a.handle, 0, 0, 10, -1)        # no such checkpoint interval
    from paper_1703_08977_gb300 import workloads as wl
    d = gfk.InstanceDesc(n_walkers=64, dt=0.01, e_trial=-2.17)
    with gfk.Context([d], trials=[(1, wl.triplet_2s3())]) as c:
        with pytest.raises(gfk.GfkError):
            gfk.gfk_grad(c.handle, 0, 0, 10, 8)         # only the Jastrow-product family


def test_autograd_function_and_adam_reduce_variance(gfk_lib):
    """GFKLoss as a torch.autograd.Function; a few Adam steps of variance minimisation
    from a deliberately poor start lower the weighted variance of E_L."""
    torch = pytest.importorskip("torch")
    from paper_1703_08977_gb300 import tuning
    gfk = gfk_lib
    theta0 = [1.8, 0.5, 0.8, 0.0, 0.0, 0.0, 0.0]
    with _ctx(gfk, 1 << 14, 0.005, gfk.GFK_PREC_MIXED, theta=theta0) as c:
        th = torch.tensor(theta0, dtype=torch.float64, requires_grad=True)
        loss = tuning.GFKLoss.apply(th, c.handle, 0, 1, 200, 64)
        loss.backward()
        _, g = gfk.gfk_grad(c.handle, 0, 1, 200, 64)
        np.testing.assert_allclose(th.grad.numpy(), g, rtol=1e-12)
        hist, theta = tuning.tune(c.handle, 0, theta0, steps=12, lr=0.03, loss_kind=1, n_steps=200)
    assert hist[-1][0] < 0.9 * hist[0][0], [h[0] for h in hist]


def test_mixed_grad_does_not_depend_on_checkpoint_interval(gfk_lib):
    """Checkpoints every 64 moves are written by the walk kernel at its folds; other
    intervals are copied between launches.  The recomputed trajectories are the
    forward's either way, so the gradient agrees across intervals (to the rounding of
    the per-segment FP32 partial sums), on an odd walker count and a ragged last
    segment."""
    gfk = gfk_lib
    n, S = 4099, 300
    out = {}
    for K in (64, 128, 32, 100):
        with _ctx(gfk, n, 0.005, gfk.GFK_PREC_MIXED) as c:
            out[K] = gfk.gfk_grad(c.handle, 0, 1, S, K)
    l64, g64 = out[64]
    for K, (l, g) in out.items():
        # intervals that are not multiples of 64 fold the FP32 log-weight sums at
        # other moves (launch ends), so the loss agrees to rounding, not bitwise
        if K % 64 == 0:
            assert l == l64, (K, l, l64)
        assert abs(l - l64) <= 1e-7 * abs(l64), (K, l, l64)
        np.testing.assert_allclose(g, g64, rtol=2e-5, atol=2e-5 * np.abs(g64).max())


@pytest.mark.parametrize("noise", [0, 1])
@pytest.mark.parametrize("theta", [THETA, [2.0, 0.5, 0.5, 0.0, 0.0, 0.0, 0.0]])
@pytest.mark.parametrize("wpt", [1, 2, 4])
def test_mixed_grad_from_the_stored_trajectory_is_the_checkpointed_one(gfk_lib, noise, theta,
                                                                      wpt):
    """ckpt_every = 0 keeps the forward's whole trajectory and sweeps it with nothing
    recomputed.  The positions the walk kernel stores are the ones the checkpointed
    path recomputes (same noise, same arithmetic in every launch shape), and the sweep
    flushes its FP32 partial sums at the same 64-move boundaries, so loss and gradient
    are bitwise those of ckpt_every = 64: both losses, Gaussian and Bernoulli noise,
    with and without Jastrow polynomial terms, 1, 2 and 4 walkers per thread, an odd
    walker count and a ragged last segment.  The FP64 path runs 64 for 0."""
    gfk = gfk_lib
    n, S = 4099, 300
    for loss_kind in (0, 1):
        d = gfk.InstanceDesc(n_walkers=n, dt=0.005, e_trial=-2.9, seed=7, rng_stream=1,
                             noise=noise, prec=gfk.GFK_PREC_MIXED)
        with gfk.Context([d], trials=[(0, theta)]) as c:
            c.set_launch(128, wpt)
            l64, g64 = gfk.gfk_grad(c.handle, 0, loss_kind, S, 64)
            l0, g0 = gfk.gfk_grad(c.handle, 0, loss_kind, S, 0)
        assert l0 == l64, (l0, l64)
        np.testing.assert_array_equal(g0, g64)
    d = gfk.InstanceDesc(n_walkers=300, dt=0.005, e_trial=-2.9, seed=7, noise=noise,
                         prec=gfk.GFK_PREC_FP64)
    with gfk.Context([d], trials=[(0, theta)]) as c:
        assert gfk.gfk_grad(c.handle, 0, 0, 100, 0)[0] == gfk.gfk_grad(c.handle, 0, 0, 100, 64)[0]


def test_grad_at_the_gradient_workload_size(gfk_lib):
    """The gradient workload at full size (2^18 walkers, 2000 moves at dt 0.005,
    checkpoints every 64 moves, the start theta = [2, 0.5, 0.5, 0, 0, 0, 0]): the
    FP64 adjoint against Richardson-extrapolated common-random-number central
    differences of the same loss (the final space-averaged energy, from gfk_energy
    of the FP64 walk), to 1e-6 of the gradient's largest component; and the mixed
    gradient (FP32 forward with FP64 weights) against the FP64 one, whose relative
    difference is stated here: below 1e-5."""
    gfk = gfk_lib
    n, S, dt, K, h = 1 << 18, 2000, 0.005, 64, 1e-4
    theta = [2.0, 0.5, 0.5, 0.0, 0.0, 0.0, 0.0]

    def ctx(prec, th):
        d = gfk.InstanceDesc(n_walkers=n, dt=dt, e_trial=-2.9037, seed=0, prec=prec)
        return gfk.Context([d], trials=[(0, th)])

    with ctx(gfk.GFK_PREC_FP64, theta) as c:
        l64, g64 = gfk.gfk_grad(c.handle, 0, 0, S, K)
        # the same loss through the forward walk and the per-step sums
        c.propagate(S)
        assert abs(c.energy(0)["E"][-1] - l64) <= 1e-12 * abs(l64)

        def central(step):
            fd = np.zeros(7)
            for k in range(7):
                vals = []
                for sgn in (+1, -1):
                    th = list(theta)
                    th[k] += sgn * step
                    c.reset()
                    c.set_trial(0, 0, th)
                    c.propagate(S)
                    vals.append(c.energy(0)["E"][-1])
                fd[k] = (vals[0] - vals[1]) / (2 * step)
            return fd

        d1 = central(h)
        d2 = central(h / 2)
    rich = (4 * d2 - d1) / 3
    scale = np.abs(rich).max()
    assert np.abs(g64 - rich).max() <= 1e-6 * scale, (np.abs(g64 - rich).max() / scale, g64, rich)
    with ctx(gfk.GFK_PREC_MIXED, theta) as c:
        l32, g32 = gfk.gfk_grad(c.handle, 0, 0, S, K)
        # the whole trajectory kept (12.6 GB): bitwise the checkpointed gradient
        l0, g0 = gfk.gfk_grad(c.handle, 0, 0, S, 0)
    assert l0 == l32
    np.testing.assert_array_equal(g0, g32)
    assert abs(l32 - l64) < 1e-6, (l32, l64)
    assert np.abs(g32 - g64).max() <= 1e-5 * np.abs(g64).max(), (g32, g64)


def test_stored_trajectory_that_does_not_fit_reports_enomem(gfk_lib):
    """ckpt_every = 0 asks for n_walkers x (n_steps + 1) x 24 bytes of trajectory; when
    that cannot be allocated (here 2^12 walkers x 2^30 moves, 1e14 bytes) gfk_grad
    returns GFK_ENOMEM before walking, and the context stays usable: the same call
    with checkpoints then succeeds."""
    gfk = gfk_lib
    d = gfk.InstanceDesc(n_walkers=1 << 12, dt=0.005, e_trial=-2.9, seed=7,
                         prec=gfk.GFK_PREC_MIXED)
    with gfk.Context([d], trials=[(0, THETA)]) as c:
        with pytest.raises(gfk.GfkError) as err:
            gfk.gfk_grad(c.handle, 0, 0, 1 << 30, 0)
        assert err.value.status == gfk.GFK_ENOMEM
        loss, g = gfk.gfk_grad(c.handle, 0, 0, 64, 64)
        assert np.isfinite(loss) and np.all(np.isfinite(g))
