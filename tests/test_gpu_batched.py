"""Batched instances, CUDA-graph replay and the autotuner (GPU)."""
import numpy as np
import pytest

from paper_1703_08977_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


def _descs(gfk, insts, prec):
    return [gfk.InstanceDesc(n_walkers=d["n_walkers"], dt=d["dt"], e_trial=d["e_trial"],
                             seed=d["seed"], state=d["state"], prec=prec,
                             rng_stream=d["rng_stream"]) for d in insts]


@pytest.mark.parametrize("prec", [0, 1])
def test_graph_replay_matches_direct_launches(gfk_lib, prec):
    """gfk_set_graph: the captured sequence (init + chunks), and its replay after a reset,
    give bitwise the walkers and sums of the direct launches."""
    gfk = gfk_lib
    insts, _ = wl.batched(scale=1 / 64)
    descs = _descs(gfk, insts[:5], prec)
    trials = [(d["kind"], d["params"]) for d in insts[:5]]
    a = gfk.Context(descs, trials=trials).propagate(100)
    b = gfk.Context(descs, trials=trials)
    b.set_graph(True)
    b.propagate(100)
    for i in range(5):
        for u, v in zip(a.walkers(i), b.walkers(i)):
            np.testing.assert_array_equal(u, v)
        np.testing.assert_array_equal(a.sums(i), b.sums(i))
    b.reset()
    b.propagate(100)          # replays the cached graph
    for i in range(5):
        np.testing.assert_array_equal(a.sums(i), b.sums(i))
    b.propagate(64)           # continues with a new graph
    a.propagate(64)
    for i in range(5):
        np.testing.assert_array_equal(a.sums(i), b.sums(i))
    a.close()
    b.close()


@pytest.mark.parametrize("kind,p1,p2", [
    (1, wl.triplet_2s3(), wl.fn3()),
    (0, wl.ground(), wl.ground(Z=1.85, a=0.5, beta=0.37, c=(0.11, -0.07, 0.05, 0.02)))])
def test_graph_replay_follows_a_new_trial_function(gfk_lib, kind, p1, p2):
    """A single-instance walk takes its trial function as a launch argument, which a
    captured graph holds: after a reset and gfk_set_trial with other parameters, the
    replay must walk the new trial (bitwise equal to direct launches with it)."""
    gfk = gfk_lib
    d = gfk.InstanceDesc(n_walkers=3000, dt=0.01, e_trial=-2.5, seed=4, prec=1)
    g = gfk.Context([d], trials=[(kind, p1)])
    g.set_graph(True)
    g.propagate(96)
    g.reset()
    g.set_trial(0, kind, p2)
    g.propagate(96)
    ref = gfk.Context([d], trials=[(kind, p2)]).propagate(96)
    for u, v in zip(ref.walkers(0), g.walkers(0)):
        np.testing.assert_array_equal(u, v)
    np.testing.assert_array_equal(ref.sums(0), g.sums(0))
    g.reset()
    g.set_trial(0, kind, p1)
    g.propagate(96)                 # back to the first trial's cached graph
    first = gfk.Context([d], trials=[(kind, p1)]).propagate(96)
    np.testing.assert_array_equal(first.sums(0), g.sums(0))
    for c in (g, ref, first):
        c.close()


@pytest.mark.parametrize("noise", [0, 1])
def test_graph_capture_at_512_threads(gfk_lib, noise):
    """512-thread blocks need more than the default 48 KB of dynamic shared memory; the
    opt-in is made before the capture starts, so a graph captured at that launch shape
    (in a fresh process this may be the first launch of the kernel) reproduces direct
    launches bitwise, on its first capture and on replay."""
    gfk = gfk_lib
    d = gfk.InstanceDesc(n_walkers=20000, dt=0.005, e_trial=-2.9, seed=6, prec=1, noise=noise)
    direct = gfk.Context([d], trials=[(0, wl.ground())], launch=(512, 2)).propagate(200)
    g = gfk.Context([d], trials=[(0, wl.ground())], launch=(512, 2))
    g.set_graph(True)
    g.propagate(200)
    for u, v in zip(direct.walkers(0), g.walkers(0)):
        np.testing.assert_array_equal(u, v)
    np.testing.assert_array_equal(direct.sums(0), g.sums(0))
    g.reset()
    g.propagate(200)                  # replay
    np.testing.assert_array_equal(direct.sums(0), g.sums(0))
    direct.close()
    g.close()


def test_batched_mixed_instances_match_single(gfk_lib):
    """The twelve-instance mix in one context (mixed path, one launch per chunk with the
    trial family dispatched per block) reproduces each instance run alone, walker by
    walker (positions and log-weights do not depend on the batch or launch shape)."""
    gfk = gfk_lib
    insts, _ = wl.batched(scale=1 / 256)
    descs = _descs(gfk, insts, 1)
    ctx = gfk.Context(descs, trials=[(d["kind"], d["params"]) for d in insts])
    ctx.set_graph(True)
    ctx.propagate(96)
    for i in (0, 5, 11):
        d = insts[i]
        with gfk.Context([descs[i]], trials=[(d["kind"], d["params"])]) as one:
            one.propagate(96)
            for u, v in zip(ctx.walkers(i), one.walkers(0)):
                np.testing.assert_array_equal(u, v)
            np.testing.assert_allclose(ctx.energy(i)["E"], one.energy(0)["E"], rtol=2e-6)
    ctx.close()


def test_kind_segments_match_single_instances_and_count_kernels(gfk_lib):
    """Three instances of three kernel kinds (ground product; 2^3S, whose orbitals
    have no prefactor terms; P_z), each above the segmentation threshold: the walk
    runs one specialised launch per instance run, and every instance's walkers and
    sums equal those of the instance walked alone, bitwise.  gfk_kernel_count counts
    the kernels exactly: init and its merge, then per chunk three walks and a merge;
    a CUDA-graph capture counts when it runs."""
    gfk = gfk_lib
    specs = [(0, wl.ground(), -2.9037), (1, wl.triplet_2s3(), -2.1752), (1, wl.pz_state(1.0), -2.1238)]
    descs = [gfk.InstanceDesc(n_walkers=300000, dt=0.005, e_trial=et, seed=2, rng_stream=i, prec=1)
             for i, (_, _, et) in enumerate(specs)]
    trials = [(k, p) for (k, p, _) in specs]
    ctx = gfk.Context(descs, trials=trials, launch=(128, 2))
    gfk.gfk_kernel_count(ctx.handle, reset=True)
    ctx.propagate(64)
    assert gfk.gfk_kernel_count(ctx.handle) == 2 + 3 + 1
    for i, (k, p, _) in enumerate(specs):
        with gfk.Context([descs[i]], trials=[(k, p)], launch=(128, 2)) as one:
            one.propagate(64)
            for u, v in zip(ctx.walkers(i), one.walkers(0)):
                np.testing.assert_array_equal(u, v)
            np.testing.assert_array_equal(ctx.sums(i), one.sums(0))
    ctx.close()
    # runs of two instances that share a trial function (different dt): the run's
    # launch takes that function as its argument; still equal to single instances
    descs2, trials2 = [], []
    for i, (k, p, et) in enumerate(specs):
        for j, dt in enumerate((0.005, 0.01)):
            descs2.append(gfk.InstanceDesc(n_walkers=150000, dt=dt, e_trial=et, seed=4,
                                           rng_stream=10 * i + j, prec=1))
            trials2.append((k, p))
    ctx2 = gfk.Context(descs2, trials=trials2, launch=(128, 2)).propagate(64)
    for i in (1, 2, 5):
        with gfk.Context([descs2[i]], trials=[trials2[i]], launch=(128, 2)) as one:
            one.propagate(64)
            for u, v in zip(ctx2.walkers(i), one.walkers(0)):
                np.testing.assert_array_equal(u, v)
            np.testing.assert_array_equal(ctx2.sums(i), one.sums(0))
    ctx2.close()
    g = gfk.Context(descs[:1], trials=trials[:1], launch=(128, 2))
    g.set_graph(True)
    g.propagate(64)                      # captured and run: init + merge + walk + merge
    assert gfk.gfk_kernel_count(g.handle, reset=True) == 4
    g.reset()
    g.propagate(64)                      # replay
    assert gfk.gfk_kernel_count(g.handle) == 4
    g.close()


def test_autotune_restores_population(gfk_lib):
    """gfk_autotune times every launch shape on the live population and restores it:
    the walk continued after tuning equals an untuned walk."""
    gfk = gfk_lib
    insts, _ = wl.batched(scale=1 / 128)
    descs = _descs(gfk, insts[:4], 1)
    trials = [(d["kind"], d["params"]) for d in insts[:4]]
    a = gfk.Context(descs, trials=trials).propagate(64)
    b = gfk.Context(descs, trials=trials).propagate(64)
    t, w, rate = gfk.gfk_autotune(b.handle, 64)
    assert t in (64, 128, 256, 512) and w in (1, 2, 4) and rate > 0
    a.propagate(64)
    b.propagate(64)
    for i in range(4):
        for u, v in zip(a.walkers(i), b.walkers(i)):
            np.testing.assert_array_equal(u, v)
        np.testing.assert_array_equal(a.counters(i), b.counters(i))
        np.testing.assert_allclose(a.energy(i)["E"], b.energy(i)["E"], rtol=2e-6)
    a.close()
    b.close()


def test_maximum_instance_count(gfk_lib):
    """GFK_MAX_INSTANCES (64) instances of both trial families, uneven sizes (1 to 900
    walkers, so the launch dispatches per block), 70 moves: every instance equals the
    same instance walked alone."""
    gfk = gfk_lib
    rng = np.random.default_rng(8)
    sizes = rng.integers(1, 900, 64)
    fams = [(0, wl.ground(), -2.9), (1, wl.triplet_2s3(), -2.17), (1, wl.pz_state(1.0), -2.12)]
    descs, trials = [], []
    for i, n in enumerate(sizes):
        k, p, et = fams[i % 3]
        descs.append(gfk.InstanceDesc(n_walkers=int(n), dt=0.01, e_trial=et, seed=3, rng_stream=i,
                                      prec=1))
        trials.append((k, p))
    with gfk.Context(descs, trials=trials) as ctx:
        ctx.propagate(70)
        for i in (0, 1, 2, 31, 62, 63):
            with gfk.Context([descs[i]], trials=[trials[i]]) as one:
                one.propagate(70)
                for u, v in zip(ctx.walkers(i), one.walkers(0)):
                    np.testing.assert_array_equal(u, v)
