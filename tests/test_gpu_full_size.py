"""Parity at the benchmark's full sizes, in the launch configurations bench.py times (GPU).

The 2^3S workload (2^20 walkers, dt 0.0025; the mixed walk at 128 threads x 2
walkers per thread) over one full 1024-move launch, and the twelve-instance
batch at its full walker counts (7.75e6 walkers; the autotuned launch shape,
replayed as a CUDA graph) over 256 moves.  Sampled walkers -- block edges, the
first and last walker of each instance and random ids -- are recomputed one by
one by the oracle (each instance alone, on its own Philox stream), with the
node criterion of the smaller parity tests: on the FP64 path every walker whose
oracle trajectory stays at least NODE_DISTANCE bohr from the node agrees to
1e-12 and the others to 1e-8, and kills agree for all; on the mixed path kills
agree for walkers at least NODE_DISTANCE_FP32 bohr from the node and positions
stay at FP32 distance."""
import numpy as np
import pytest

import oracle
from oracle_tracks import NODE_DISTANCE, walk_tracking_node
from paper_1703_08977_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

NODE_DISTANCE_FP32 = 1e-2


def _planes(ctx, inst):
    x, lw, al = ctx.walkers(inst)
    return x, lw, al.astype(bool)


def _check_fp64(x, lw, al, w, d_min, tag):
    a = w.alive.astype(bool)
    np.testing.assert_array_equal(al, a, err_msg=tag)
    dx = np.abs(x - w.x).max(axis=1) / np.maximum(1.0, np.abs(w.x).max(axis=1))
    dl = np.zeros_like(dx)
    dl[a] = np.abs(lw[a] - w.logw[a]) / np.maximum(1.0, np.abs(w.logw[a]))
    dev = np.maximum(dx, dl)
    near = d_min < NODE_DISTANCE
    assert dev[~near].max(initial=0.0) <= 1e-12, (tag, dev[~near].max())
    assert dev[near].max(initial=0.0) <= 1e-8, (tag, dev[near].max())
    return int(near.sum())


def _check_mixed(x, al, w, d_min, tag):
    a = w.alive.astype(bool)
    far = d_min >= NODE_DISTANCE_FP32
    np.testing.assert_array_equal(al[far], a[far], err_msg=tag)
    both = a & al & far
    if both.any():
        dx = np.abs(x[both] - w.x[both]).max(axis=1)
        assert np.median(dx) < 1e-4 and dx.max() < 1e-2, (tag, np.median(dx), dx.max())


def test_triplet_workload_full_size(gfk_lib):
    """2^3S at 2^20 walkers, one 1024-move launch on both paths: sampled walkers
    against the oracle; and the final E of the mixed path against the FP64 path's
    on the same walkers, within 1e-6 hartree for the FP32 rounding of the walk
    (the ground state's difference stays below 1e-8 over 2000 moves) plus the
    whole contribution w_i (|E_L,i| + |E|) / W of each walker alive on one path
    and not the other.  Such walkers come from the node: one that straddles it
    within FP32 rounding, or one that a near-node drift kick (|b| dt >> 1)
    threw hundreds of bohr out, where the unscaled FP64 psi of the FP64 path
    and of the oracle underflows to exactly 0 (a kill) while the mixed path,
    which factors the largest exponential out of psi, keeps it alive."""
    gfk = gfk_lib
    n, moves, dt, et, seed = 1 << 20, 1024, 0.0025, wl.E_T[1], 0
    p = wl.triplet_2s3()
    rng = np.random.default_rng(9)
    ids = np.unique(np.concatenate([[0, 1, 127, 128, 255, 256, 511, 512, n - 256, n - 1],
                                    rng.integers(0, n, 54)])).astype(np.uint32)
    out = {}
    for prec in (gfk.GFK_PREC_FP64, gfk.GFK_PREC_MIXED):
        d = gfk.InstanceDesc(n_walkers=n, dt=dt, e_trial=et, seed=seed, prec=prec, state=1)
        launch = (128, 2) if prec == gfk.GFK_PREC_MIXED else None
        with gfk.Context([d], trials=[(1, p)], launch=launch) as ctx:
            ctx.propagate(moves)
            out[prec] = _planes(ctx, 0) + (ctx.energy(0)["E"],)
    w, d_min, _ = walk_tracking_node(1, p, ids=ids, steps=moves, dt=dt, e_trial=et, seed=seed)
    x64, lw64, al64, e64 = out[gfk.GFK_PREC_FP64]
    x32, lw32, al32, e32 = out[gfk.GFK_PREC_MIXED]
    n_near = _check_fp64(x64[ids], lw64[ids], al64[ids], w, d_min, "fp64")
    _check_mixed(x32[ids], al32[ids], w, d_min, "mixed")

    # the whole population: mixed vs FP64 at the last move.  A walker alive on
    # one path and dead on the other enters with its whole contribution, its
    # local energy from the path on which it is alive (the oracle's FP64
    # evaluation, or the mixed walk's own FP32 one).
    mis = np.flatnonzero(al32 != al64)
    c = max(lw64[al64].max(), lw32[al32].max())
    W = np.exp(lw64[al64] - c).sum()
    budget = 1e-6
    n_far = 0
    if mis.size:
        in64 = al64[mis]
        lw = np.where(in64, lw64[mis], lw32[mis])
        el = np.empty(mis.size)
        if in64.any():
            el[in64] = oracle.trial_eval_many(1, p, x64[mis[in64]])[2]
        if (~in64).any():
            el[~in64] = gfk.gfk_eval_f32(1, p, x32[mis[~in64]].astype(np.float32))[1]
        budget += float((2.0 * np.exp(lw - c) * (np.abs(el) + abs(e64[-1]))).sum() / W)
        r = np.linalg.norm(np.where(in64[:, None], x64[mis], x32[mis]).reshape(-1, 2, 3), axis=2)
        n_far = int((r.min(axis=1) > 300.0).sum())
    print(f"near-node sampled walkers {n_near}, alive mismatches {mis.size} "
          f"({n_far} beyond 300 bohr), final dE {abs(e32[-1] - e64[-1]):.3e}, budget {budget:.3e}")
    assert mis.size <= 1e-4 * n, mis.size
    assert abs(e32[-1] - e64[-1]) <= budget, (abs(e32[-1] - e64[-1]), budget)


def test_batch_workload_full_size(gfk_lib):
    """The twelve-instance batch at its full walker counts, 256 moves: the mixed
    path at the autotuned launch shape with CUDA-graph replay (as bench.py times
    it), the FP64 path at its own launch; nine sampled walkers per instance
    against the oracle."""
    gfk = gfk_lib
    insts, _ = wl.batched()
    moves = 256
    trials = [(q["kind"], q["params"]) for q in insts]
    rng = np.random.default_rng(13)
    sample = [np.unique(np.concatenate([[0, 1, 255, 256, q["n_walkers"] - 1],
                                        rng.integers(0, q["n_walkers"], 4)])).astype(np.uint32)
              for q in insts]
    out = {}
    for prec in (gfk.GFK_PREC_FP64, gfk.GFK_PREC_MIXED):
        descs = [gfk.InstanceDesc(n_walkers=q["n_walkers"], dt=q["dt"], e_trial=q["e_trial"],
                                  seed=q["seed"], state=q["state"], prec=prec,
                                  rng_stream=q["rng_stream"]) for q in insts]
        ctx = gfk.Context(descs, trials=trials)
        if prec == gfk.GFK_PREC_MIXED:
            gfk.autotune_cached(ctx.handle, descs, trials, probe_steps=256)
            ctx.set_graph(True)
            ctx.reset()
        ctx.propagate(moves)
        out[prec] = []
        for i, ids in enumerate(sample):
            x, lw, al = _planes(ctx, i)
            out[prec].append((ids, x[ids].copy(), lw[ids].copy(), al[ids].copy()))
            del x, lw, al
        ctx.close()
    n_near = 0
    for i, q in enumerate(insts):
        ids, x64, lw64, al64 = out[gfk.GFK_PREC_FP64][i]
        _, x32, _, al32 = out[gfk.GFK_PREC_MIXED][i]
        w, d_min, _ = walk_tracking_node(q["kind"], q["params"], ids=ids, steps=moves,
                                         dt=q["dt"], e_trial=q["e_trial"], seed=q["seed"],
                                         inst=q["rng_stream"])
        tag = f"state {q['state']} dt {q['dt']} n {q['n_walkers']}"
        n_near += _check_fp64(x64, lw64, al64, w, d_min, tag)
        _check_mixed(x32, al32, w, d_min, tag)
    print(f"near-node sampled walkers {n_near}")
