"""The multi-rank path on CPU: two gloo ranks shard one population by walker id,
run it with the oracle, merge their per-step sums, and must reproduce the
single-population sums."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_1703_08977_gb300 import distributed as gd
from paper_1703_08977_gb300 import workloads as wl


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank_main(rank, world, port, n, steps, kind, params, out_path):
    import torch.distributed as dist
    import oracle
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    id0, n_loc = gd.shard(n, world, rank)
    w = oracle.Walk(kind, params, ids=np.arange(id0, id0 + n_loc), dt=0.01, e_trial=-2.17,
                    seed=3, inst=2).advance(steps)
    merged = gd.merge_sums(np.array(w.rows), device="cpu")
    if rank == 0:
        np.save(out_path, merged)
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("kind,params", [(0, wl.ground()), (1, wl.triplet_2s3())])
def test_two_rank_shards_merge_to_single_population(tmp_path, kind, params):
    n, steps, world = 301, 40, 2
    out = str(tmp_path / "merged.npy")
    mp.start_processes(_rank_main, args=(world, _free_port(), n, steps, kind, params, out),
                       nprocs=world, join=True, start_method="spawn")
    merged = np.load(out)
    import oracle
    full = oracle.Walk(kind, params, n_walkers=n, dt=0.01, e_trial=-2.17, seed=3, inst=2)
    full.advance(steps)
    ref = np.array(full.rows)
    # same shift convention after rescaling: compare shift-free quantities
    for col, pw in ((1, 1), (2, 1), (3, 2), (4, 1)):
        np.testing.assert_allclose(merged[:, col] * np.exp(pw * (merged[:, 0] - ref[:, 0])),
                                   ref[:, col], rtol=1e-14)
    np.testing.assert_array_equal(merged[:, 5], ref[:, 5])
    e_m = gd.estimators(merged, n)
    e_r = full.series()
    np.testing.assert_allclose(e_m["E"], e_r["E"], rtol=1e-14)
    np.testing.assert_allclose(e_m["ln_z"], e_r["ln_z"], rtol=0, atol=1e-13)


def test_shard_ranges_cover_the_population():
    for n, world in ((10, 3), (7, 7), (1 << 20, 8), (5, 8)):
        seen = []
        for r in range(world):
            id0, k = gd.shard(n, world, r)
            seen.extend(range(id0, id0 + k))
        assert seen == list(range(n))
