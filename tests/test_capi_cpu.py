"""The C-ABI library on a machine without a GPU: it builds, loads, exports every
entry point include/gfk.h declares, and rejects malformed descriptors before
touching CUDA.  No compute call is made here."""
import ctypes
import os
import re

import pytest

from paper_1703_08977_gb300 import gfk

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_symbols():
    src = open(os.path.join(ROOT, "include", "gfk.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(gfk_[a-z_0-9]+)\s*\(", src)))


def test_library_exports_every_declared_symbol():
    lib = gfk.load()
    declared = _declared_symbols()
    assert len(declared) >= 15
    for name in declared:
        assert hasattr(lib, name), name
    assert set(declared) == set(gfk.EXPORTS)


def test_status_strings():
    for s in range(8):
        assert gfk.status_string(s)
    assert gfk.status_string(999) == "unknown status"


def _desc(**kw):
    d = dict(n_walkers=64, dt=0.01, e_trial=-2.9, seed=0)
    d.update(kw)
    return gfk.InstanceDesc(**d).c()


@pytest.mark.parametrize("bad", [
    dict(n_walkers=0), dict(n_walkers=-5), dict(n_walkers=2**31), dict(dt=0.0), dict(dt=-1e-3),
    dict(dt=float("nan")), dict(e_trial=float("inf")), dict(init_sigma=0.0), dict(state=7),
    dict(prec=3), dict(ee_on=2), dict(noise=2), dict(noise=-1)])
def test_create_rejects_bad_descriptors(bad):
    lib = gfk.load()
    arr = (gfk.gfk_instance_desc * 1)(_desc(**bad))
    out = ctypes.c_void_p(1)
    assert lib.gfk_create(arr, 1, None, ctypes.byref(out)) == gfk.GFK_EINVAL
    assert out.value is None


def test_create_rejects_bad_counts_and_mixed_precisions_or_noise():
    lib = gfk.load()
    out = ctypes.c_void_p()
    arr = (gfk.gfk_instance_desc * 2)(_desc(prec=0), _desc(prec=1))
    assert lib.gfk_create(arr, 2, None, ctypes.byref(out)) == gfk.GFK_EINVAL
    mixed_noise = (gfk.gfk_instance_desc * 2)(_desc(noise=gfk.GFK_NOISE_GAUSSIAN),
                                              _desc(noise=gfk.GFK_NOISE_BERNOULLI))
    assert lib.gfk_create(mixed_noise, 2, None, ctypes.byref(out)) == gfk.GFK_EINVAL
    assert lib.gfk_create(arr, 0, None, ctypes.byref(out)) == gfk.GFK_EINVAL
    assert lib.gfk_create(None, 1, None, ctypes.byref(out)) == gfk.GFK_EINVAL
    assert lib.gfk_create(arr, 1, None, None) == gfk.GFK_EINVAL


def test_null_context_calls_are_rejected():
    lib = gfk.load()
    v = ctypes.c_int64()
    assert lib.gfk_propagate(None, 10) == gfk.GFK_EINVAL
    assert lib.gfk_steps(None, ctypes.byref(v)) == gfk.GFK_EINVAL
    assert lib.gfk_energy(None, 0, None, None, None, 0, None) == gfk.GFK_EINVAL
    assert lib.gfk_reset(None) == gfk.GFK_EINVAL
    assert lib.gfk_set_launch(None, 128, 1) == gfk.GFK_EINVAL
    lib.gfk_destroy(None)
    assert lib.gfk_last_error(None) == b""
