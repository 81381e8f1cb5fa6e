"""The bounds-checked debug library (GPU, in-range case).

A child process loads libgfk_debug.so (GFK_DEBUG=1; built in-tree on first
use) and drives every path whose accesses the debug build checks: the FP64
and mixed walks (chunked, graph-replayed, batched with several instances),
walker export, checkpoint and restore, the gradient with checkpoints and with
the stored trajectory, and the allocation-free entry point on caller-owned
buffers.  All of them stay inside their buffers, so the status word must read
zero; and the checks only guard accesses, so the results must be the release
library's (run the same way in a second child)."""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r"""
import json, sys
import numpy as np
import torch
sys.path.insert(0, sys.argv[1])
from paper_1703_08977_gb300 import gfk, workloads as wl
out = {}
G, B = gfk.GFK_NOISE_GAUSSIAN, gfk.GFK_NOISE_BERNOULLI
for prec in (gfk.GFK_PREC_FP64, gfk.GFK_PREC_MIXED):
    descs = [gfk.InstanceDesc(n_walkers=n, dt=0.01, e_trial=-2.9, seed=5, prec=prec, rng_stream=s)
             for n, s in ((3001, 0), (517, 1))]
    with gfk.Context(descs, trials=[(0, wl.ground()), (1, wl.triplet_2s3())]) as c:
        c.propagate(70)
        blob = c.checkpoint()
        c.propagate(60)
        e1 = c.energy(0)["E"].tolist()
        c.restore(blob)
        c.set_graph(True)
        c.propagate(60)
        out[f"E_{prec}"] = [e1, c.energy(0)["E"].tolist(), c.energy(1)["E"].tolist()]
        x, lw, al = c.walkers(1)
        out[f"x_{prec}"] = x[:50].tolist()
    d = gfk.InstanceDesc(n_walkers=1025, dt=0.005, e_trial=-2.9, seed=2, prec=prec, noise=B)
    with gfk.Context([d], trials=[(0, [1.9, 0.5, 0.45, 0.05, -0.02, 0.01, 0.003])]) as c:
        out[f"grad_{prec}"] = [gfk.gfk_grad(c.handle, 0, 1, 150, K)[1].tolist() for K in (64, 0, 40)]
n = 4099
desc = gfk.InstanceDesc(n_walkers=n, dt=0.01, e_trial=-2.9, seed=3, prec=gfk.GFK_PREC_MIXED)
dev = torch.device("cuda")
p0 = torch.empty((n, 4), dtype=torch.float32, device=dev)
p1 = torch.empty((n, 4), dtype=torch.float32, device=dev)
sgn = torch.empty(n, dtype=torch.int8, device=dev)
rows = torch.empty((101, 6), dtype=torch.float64, device=dev)
cnt = torch.empty(3, dtype=torch.int64, device=dev)
assert gfk.gfk_propagate_noalloc(desc, 0, wl.ground(), p0, p1, sgn, 1, 0, 100, rows, cnt) == 0
torch.cuda.synchronize()
out["noalloc"] = rows.cpu().numpy().tolist()
out["debug"] = list(gfk.gfk_debug_status(clear=True))
print("RESULT " + json.dumps(out))
"""


def _child(debug):
    env = dict(os.environ)
    env["GFK_DEBUG"] = "1" if debug else "0"
    r = subprocess.run([sys.executable, "-c", CHILD, ROOT], env=env, capture_output=True,
                       text=True, timeout=1500)
    assert r.returncode == 0, r.stdout[-3000:] + r.stderr[-3000:]
    line = [l for l in r.stdout.splitlines() if l.startswith("RESULT ")][-1]
    return json.loads(line[len("RESULT "):])


def test_debug_build_in_range_paths_are_clean_and_match_release():
    dbg = _child(True)
    rel = _child(False)
    assert dbg["debug"] == [1, 0, 0], dbg["debug"]
    assert rel["debug"] == [0, 0, 0]
    for key in sorted(rel):
        if key == "debug":
            continue
        a, b = np.asarray(dbg[key], dtype=float), np.asarray(rel[key], dtype=float)
        assert a.shape == b.shape, key
        # the checks only guard accesses: the same arithmetic, the same results
        np.testing.assert_array_equal(a, b, err_msg=key)
