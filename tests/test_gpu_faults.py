"""Failure handling without any device fault (GPU).

Failures are made on the host: an allocation the library is told to fail, a
non-finite walker planted in a checkpoint blob, a blob from another context.
Every call reports a status; nothing traps, and the context stays usable.
"""
import os
import struct
import subprocess
import sys

import numpy as np
import pytest

from paper_1703_08977_gb300 import workloads as wl

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = 56          # bytes of the checkpoint blob header before the state planes

_CHILD = r'''
import sys
sys.path.insert(0, sys.argv[1])
from paper_1703_08977_gb300 import gfk, workloads as wl
d = gfk.InstanceDesc(n_walkers=1000, dt=0.01, e_trial=-2.9)
try:
    gfk.Context([d], trials=[(0, wl.ground())])
    print("created")
except gfk.GfkError as e:
    print("status", e.status)
c = gfk.Context([d], trials=[(0, wl.ground())]).propagate(10)    # later allocations work
print("ok", c.steps)
'''


@pytest.mark.parametrize("nth", [1, 3, 4])
def test_injected_allocation_failure_reports_enomem(nth):
    """GFK_FAULT_ALLOC=n: the n-th device allocation of the process fails on the host;
    gfk_create returns GFK_ENOMEM, frees what it took, and later contexts work."""
    env = dict(os.environ, GFK_FAULT_ALLOC=str(nth))
    r = subprocess.run([sys.executable, "-c", _CHILD, ROOT], capture_output=True, text=True,
                       env=env, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = r.stdout.split()
    assert "status" in lines and lines[lines.index("status") + 1] == "2", r.stdout
    assert "ok" in lines and lines[lines.index("ok") + 1] == "10", r.stdout


@pytest.mark.parametrize("planted", [0.0, float("nan"), float("inf")])
@pytest.mark.parametrize("prec", [0, 1])
def test_planted_nonfinite_walker_is_counted_not_trapped(gfk_lib, prec, planted):
    """A walker placed on the nucleus (r1 = 0: infinite drift), or given a NaN or an
    infinite position, through a checkpoint blob is killed and counted as non-finite;
    gfk_energy reports GFK_ENONFINITE with finite outputs; the other walkers continue
    unchanged."""
    gfk = gfk_lib
    n = 256
    d = gfk.InstanceDesc(n_walkers=n, dt=0.01, e_trial=-2.9, seed=2, prec=prec)
    a = gfk.Context([d], trials=[(0, wl.ground())]).propagate(32)
    blob = bytearray(a.checkpoint())
    victim = 17
    n_slots = struct.unpack_from("<q", blob, 24)[0]
    if prec == 0:        # six double planes of n_slots: x1 of the victim to 0, y1, z1 too
        for dim in range(3):
            struct.pack_into("<d", blob, HEADER + 8 * (dim * n_slots + victim), planted)
    else:                # float4 plane p0 = (x1, y1, z1, x2)
        struct.pack_into("<fff", blob, HEADER + 16 * victim, planted, planted, planted)
    b = gfk.Context([d], trials=[(0, wl.ground())])
    b.restore(bytes(blob))
    b.propagate(8)
    a.propagate(8)
    cb, ca = b.counters(), a.counters()
    assert cb[0] == ca[0] + 1 and cb[1] == ca[1]
    e = b.energy()
    assert e["status"] == gfk.GFK_ENONFINITE
    assert np.isfinite(e["E"]).all()
    xa, la, aa = a.walkers()
    xb, lb, ab = b.walkers()
    keep = np.arange(n) != victim
    np.testing.assert_array_equal(xa[keep], xb[keep])
    assert ab[victim] == 0 and aa[victim] == 1
    a.close()
    b.close()


def test_blob_from_another_context_is_rejected(gfk_lib):
    gfk = gfk_lib
    d1 = gfk.InstanceDesc(n_walkers=100, dt=0.01, e_trial=-2.9, seed=1)
    d2 = gfk.InstanceDesc(n_walkers=100, dt=0.01, e_trial=-2.9, seed=2)
    a = gfk.Context([d1], trials=[(0, wl.ground())]).propagate(4)
    b = gfk.Context([d2], trials=[(0, wl.ground())])
    with pytest.raises(gfk.GfkError) as e:
        b.restore(a.checkpoint())
    assert e.value.status == gfk.GFK_EINVAL
    with pytest.raises(gfk.GfkError):
        b.restore(a.checkpoint()[:100])
    b.propagate(4)                      # still usable
    assert b.steps == 4
    a.close()
    b.close()
