"""The allocation-free entry point gfk_propagate_noalloc (GPU).

It exists for callers that cannot let a library call cudaMalloc (frameworks
that own all device memory through their own allocator or a fixed arena, and
processes with a fixed memory budget).  Here the test plays that caller: it
allocates every buffer itself with torch, calls the entry point twice in a row
through the C ABI (an initialising call, then a continuing one), and checks
walkers, per-step sums and counters against the ordinary gfk_propagate on the
same workload.  This file is collected last so that a first failure here
comes after every other test has run.
"""
import numpy as np
import pytest

import oracle
from paper_1703_08977_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("kind,params,et,noise", [(0, wl.ground(), -2.9, 0),
                                                  (1, wl.triplet_2s3(), -2.175, 0),
                                                  (0, wl.ground(), -2.9, 1)])
def test_noalloc_matches_propagate_on_two_calls(gfk_lib, kind, params, et, noise):
    import torch
    gfk = gfk_lib
    n, m1, m2 = 5000 + 7, 48, 80
    desc = gfk.InstanceDesc(n_walkers=n, dt=0.01, e_trial=et, seed=3, prec=gfk.GFK_PREC_MIXED,
                            rng_stream=2, noise=noise)

    # the ordinary path: the library allocates
    with gfk.Context([desc], trials=[(kind, params)], launch=(256, 2)) as ctx:
        ctx.propagate(m1)
        ctx.propagate(m2)
        ref_rows = ctx.sums(0)
        ref_x, ref_lw, ref_al = ctx.walkers(0)
        ref_cnt = ctx.counters(0)

    # the allocation-free path: the caller owns every buffer
    dev = torch.device("cuda")
    p0 = torch.empty((n, 4), dtype=torch.float32, device=dev)
    p1 = torch.empty((n, 4), dtype=torch.float32, device=dev)
    sgn = torch.empty(n, dtype=torch.int8, device=dev)
    rows1 = torch.empty((m1 + 1, 6), dtype=torch.float64, device=dev)
    rows2 = torch.empty((m2, 6), dtype=torch.float64, device=dev)
    cnt = torch.empty(3, dtype=torch.int64, device=dev)
    st = gfk.gfk_propagate_noalloc(desc, kind, params, p0, p1, sgn, 1, 0, m1, rows1, cnt)
    assert st == gfk.GFK_OK, gfk.status_string(st)
    st = gfk.gfk_propagate_noalloc(desc, kind, params, p0, p1, sgn, 0, m1, m2, rows2, cnt)
    assert st == gfk.GFK_OK, gfk.status_string(st)
    torch.cuda.synchronize()

    rows = np.vstack([rows1.cpu().numpy(), rows2.cpu().numpy()])
    np.testing.assert_allclose(rows, ref_rows, rtol=1e-15, atol=0)
    a = p0.cpu().numpy()
    b = p1.cpu().numpy()
    x = np.concatenate([a, b[:, :2]], axis=1).astype(np.float64)
    lw = b[:, 2:].copy().view(np.float64)[:, 0]
    al = sgn.cpu().numpy() != 0
    np.testing.assert_array_equal(al, ref_al.astype(bool))
    np.testing.assert_array_equal(x, ref_x)
    np.testing.assert_array_equal(lw[al], ref_lw[al])
    np.testing.assert_array_equal(cnt.cpu().numpy(), ref_cnt)


def _planes_to_walkers(p0, p1, sgn):
    a = p0.cpu().numpy()
    b = p1.cpu().numpy()
    x = np.concatenate([a, b[:, :2]], axis=1).astype(np.float64)
    lw = b[:, 2:].copy().view(np.float64)[:, 0]
    al = sgn.cpu().numpy() != 0
    return x, lw, al


def test_noalloc_multichunk_at_capacity(gfk_lib):
    """At the largest population the call accepts (GFK_NOALLOC_MAX_WALKERS, 8192
    blocks) the scratch holds the block records of 64 moves, so each call walks
    several 64-move chunks (100 moves: 64 + 36; then 164 moves: 64 + 64 + 36).
    Chunks of whole 64-move fold windows fold the FP32 log-weight increments after
    the same moves as gfk_propagate's single launches, so walkers, per-step sums and
    counters equal gfk_propagate's bit for bit; sampled walkers (block edges, the
    last one, random ids) are alive exactly when the FP64 oracle's are and at FP32
    distance from them."""
    import torch
    gfk = gfk_lib
    n, m1, m2 = gfk.GFK_NOALLOC_MAX_WALKERS, 100, 164
    et, dt, seed = -2.9037, 0.005, 4
    p = wl.ground()
    desc = gfk.InstanceDesc(n_walkers=n, dt=dt, e_trial=et, seed=seed, prec=gfk.GFK_PREC_MIXED,
                            rng_stream=1)
    with gfk.Context([desc], trials=[(0, p)], launch=(256, 2)) as ctx:
        ctx.propagate(m1)
        ctx.propagate(m2)
        ref_rows = ctx.sums(0)
        ref_x, ref_lw, ref_al = ctx.walkers(0)
        ref_cnt = ctx.counters(0)
    torch.cuda.empty_cache()

    dev = torch.device("cuda")
    p0 = torch.empty((n, 4), dtype=torch.float32, device=dev)
    p1 = torch.empty((n, 4), dtype=torch.float32, device=dev)
    sgn = torch.empty(n, dtype=torch.int8, device=dev)
    rows1 = torch.empty((m1 + 1, 6), dtype=torch.float64, device=dev)
    rows2 = torch.empty((m2, 6), dtype=torch.float64, device=dev)
    cnt = torch.empty(3, dtype=torch.int64, device=dev)
    st = gfk.gfk_propagate_noalloc(desc, 0, p, p0, p1, sgn, 1, 0, m1, rows1, cnt)
    assert st == gfk.GFK_OK, gfk.status_string(st)
    st = gfk.gfk_propagate_noalloc(desc, 0, p, p0, p1, sgn, 0, m1, m2, rows2, cnt)
    assert st == gfk.GFK_OK, gfk.status_string(st)
    torch.cuda.synchronize()

    rows = np.vstack([rows1.cpu().numpy(), rows2.cpu().numpy()])
    np.testing.assert_array_equal(rows, ref_rows)
    x, lw, al = _planes_to_walkers(p0, p1, sgn)
    np.testing.assert_array_equal(al, ref_al.astype(bool))
    np.testing.assert_array_equal(x, ref_x)
    np.testing.assert_array_equal(lw[al], ref_lw[al])
    np.testing.assert_array_equal(cnt.cpu().numpy(), ref_cnt)

    rng = np.random.default_rng(8)
    ids = np.unique(np.concatenate([[0, 1, 255, 256, 511, 512, n - 512, n - 1],
                                    rng.integers(0, n, 24)])).astype(np.uint32)
    w = oracle.Walk(0, p, ids=ids, dt=dt, e_trial=et, seed=seed, inst=1).advance(m1 + m2)
    np.testing.assert_array_equal(al[ids], w.alive.astype(bool))
    dx = np.abs(x[ids] - w.x).max(axis=1)
    assert np.median(dx) < 1e-4 and dx.max() < 1e-2, (np.median(dx), dx.max())


def test_noalloc_rejects_oversize_and_bad_arguments(gfk_lib):
    import torch
    gfk = gfk_lib
    dev = torch.device("cuda")
    p0 = torch.empty((64, 4), dtype=torch.float32, device=dev)
    p1 = torch.empty((64, 4), dtype=torch.float32, device=dev)
    sgn = torch.empty(64, dtype=torch.int8, device=dev)
    rows = torch.empty((2, 6), dtype=torch.float64, device=dev)
    cnt = torch.empty(3, dtype=torch.int64, device=dev)
    big = gfk.InstanceDesc(n_walkers=gfk.GFK_NOALLOC_MAX_WALKERS + 1, dt=0.01, e_trial=-2.9,
                           prec=gfk.GFK_PREC_MIXED)
    assert gfk.gfk_propagate_noalloc(big, 0, wl.ground(), p0, p1, sgn, 1, 0, 1, rows,
                                     cnt) == gfk.GFK_EINVAL
    fp64 = gfk.InstanceDesc(n_walkers=64, dt=0.01, e_trial=-2.9, prec=gfk.GFK_PREC_FP64)
    assert gfk.gfk_propagate_noalloc(fp64, 0, wl.ground(), p0, p1, sgn, 1, 0, 1, rows,
                                     cnt) == gfk.GFK_EINVAL
    ok = gfk.InstanceDesc(n_walkers=64, dt=0.01, e_trial=-2.9, prec=gfk.GFK_PREC_MIXED)
    assert gfk.gfk_propagate_noalloc(ok, 0, wl.ground()[:2], p0, p1, sgn, 1, 0, 1, rows,
                                     cnt) == gfk.GFK_EINVAL
    assert gfk.gfk_propagate_noalloc(ok, 0, wl.ground(), p0, p1, sgn, 1, 5, 1, rows,
                                     cnt) == gfk.GFK_EINVAL
