"""Oracle for the GFK helium walk: plain FP64 C on the CPU, loaded with ctypes.

TEST INFRASTRUCTURE ONLY.  The test suite, the smoke check and the benchmark's
CPU-baseline leg are the only callers.  The oracle shares no code with the CUDA
library (``paper_1703_08977_gb300``) and imports nothing from it.

The C source (``gfk_oracle.c``) cites the paper passage each part follows.  This
module only compiles it (gcc, ``-ffp-contract=off``) and marshals arrays.

Parity status per function (what pins it is in ``tests/test_oracle_pins.py``):
  philox4x32_10     pinned: an independent implementation (triton's Philox,
                    run by its CPU interpreter) agrees bitwise.
  move_normals,
  init_normals      pinned: Kolmogorov-Smirnov and moment tests against N(0,1), no
                    correlation between components or between consecutive
                    moves; every angle on the 1024-point grid; the counter
                    layout against philox4x32_10 (pinned above).
  trial_eval        pinned: closed-form eigenfunctions (E_L constant), 50-digit
                    finite differences of ln|psi|, exchange (anti)symmetry.
  run               pinned: exact weights for an exact eigenfunction, a
                    hand-computed single step, the variational closed form
                    <E_L> = Z^2 - 27 Z / 8 at stationarity, node invariants,
                    the growth identity d ln z / dt = -(E - E_T) + O(dt).
  neumaier_sum      pinned: math.fsum (exactly rounded) on cancelling inputs.
  superduper_next,
  bernoulli_eps,
  move_bernoulli    pinned: the closed form S_k = a^k S_0 + (a^k - 1)/(a - 1) mod 2^32
                    of the congruential recurrence (exact integers), the paper's
                    threshold at 2^31, balance and independence of the +-1 steps.
  run (noise 1)     pinned: a hand-computed Bernoulli step, exact weights for an
                    exact eigenfunction, and the stationary <E_L> closed form.
  trial_eval_many   pinned: equal to trial_eval point by point (a loop over it).
  node_distance     pinned: the closed forms 1/(Z sqrt 2) (nodeless product),
                    |r1 - r2|/sqrt 2 (2^3S pair), |z1 + z2|/sqrt 2 (function 7), 0 on
                    a node.
  opcount (module)  pinned: its restatement of a walker-step equals the C walk bit
                    for bit; its counts follow hand counts of the noise.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gfk_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

KIND_JASTROW_PRODUCT = 0
KIND_ORBITAL_PAIRS = 1


def build(force: bool = False) -> str:
    """Compile the oracle into oracle/_build/liboracle.so (plain gcc, no FMA contraction)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math",
           "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build())
        c = ctypes
        dp = c.POINTER(c.c_double)
        lib.orc_philox4x32_10.argtypes = [c.POINTER(c.c_uint32), c.POINTER(c.c_uint32),
                                          c.POINTER(c.c_uint32)]
        lib.orc_philox4x32_10.restype = None
        lib.orc_uniform.argtypes = [c.c_uint32]
        lib.orc_uniform.restype = c.c_double
        lib.orc_angle_uniform.argtypes = [c.c_uint32]
        lib.orc_angle_uniform.restype = c.c_double
        lib.orc_move_normals.argtypes = [c.c_uint64, c.c_uint32, c.c_uint32, c.c_uint32, dp]
        lib.orc_move_normals.restype = None
        lib.orc_init_normals.argtypes = [c.c_uint64, c.c_uint32, c.c_uint32, dp]
        lib.orc_init_normals.restype = None
        lib.orc_trial_eval.argtypes = [c.c_int, dp, c.c_int, c.c_int, dp,
                                       c.POINTER(c.c_int), dp, dp, dp]
        lib.orc_trial_eval.restype = c.c_int
        lib.orc_trial_eval_many.argtypes = [c.c_int, dp, c.c_int, c.c_int, c.c_int64, dp,
                                            c.POINTER(c.c_int), dp, dp, dp]
        lib.orc_trial_eval_many.restype = c.c_int
        lib.orc_neumaier_sum.argtypes = [dp, c.c_int64]
        lib.orc_neumaier_sum.restype = c.c_double
        lib.orc_run.argtypes = [c.c_int, dp, c.c_int, c.c_int,
                                c.c_double, c.c_double, c.c_uint64, c.c_uint32, c.c_double,
                                c.c_int64, c.POINTER(c.c_uint32),
                                dp, dp, dp, c.POINTER(c.c_uint8), c.POINTER(c.c_int8),
                                c.c_uint32, c.c_int64, c.c_int,
                                dp, c.POINTER(c.c_int64), c.c_int, c.POINTER(c.c_uint32)]
        lib.orc_run.restype = c.c_int
        lib.orc_superduper_next.argtypes = [c.c_uint32]
        lib.orc_superduper_next.restype = c.c_uint32
        lib.orc_bernoulli_eps.argtypes = [c.c_uint32]
        lib.orc_bernoulli_eps.restype = c.c_int
        lib.orc_superduper_seed.argtypes = [c.c_uint64, c.c_uint32, c.c_uint32]
        lib.orc_superduper_seed.restype = c.c_uint32
        lib.orc_move_bernoulli.argtypes = [c.c_uint64, c.c_uint32, c.c_uint32, c.c_uint32, dp]
        lib.orc_move_bernoulli.restype = None
        _lib = lib
        return lib


def _ptr(a: np.ndarray, ctype):
    return a.ctypes.data_as(ctypes.POINTER(ctype))


def philox4x32_10(ctr, key) -> np.ndarray:
    """One Philox4x32-10 block: 4 counter words, 2 key words -> 4 output words."""
    lib = _load()
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    lib.orc_philox4x32_10(_ptr(c, ctypes.c_uint32), _ptr(k, ctypes.c_uint32),
                          _ptr(out, ctypes.c_uint32))
    return out


def uniform(word: int) -> float:
    return _load().orc_uniform(int(word))


def angle_uniform(k: int) -> float:
    """The Box-Muller angle uniform (k + 1/2) / 1024 of a 10-bit grid index."""
    return _load().orc_angle_uniform(int(k))


def move_normals(seed: int, walker: int, step: int, inst: int) -> np.ndarray:
    """The six normals of move `step` of walker `walker` (instance stream `inst`)."""
    out = np.zeros(6)
    _load().orc_move_normals(int(seed), int(walker), int(step), int(inst),
                             _ptr(out, ctypes.c_double))
    return out


def init_normals(seed: int, walker: int, inst: int) -> np.ndarray:
    """The six normals that place walker `walker` initially (X0 = sigma * xi)."""
    out = np.zeros(6)
    _load().orc_init_normals(int(seed), int(walker), int(inst), _ptr(out, ctypes.c_double))
    return out


NOISE_GAUSSIAN = 0
NOISE_BERNOULLI = 1


def superduper_next(state: int) -> int:
    """One step of the "Superduper" generator: (69069 S + 1) mod 2^32."""
    return int(_load().orc_superduper_next(int(state)))


def bernoulli_eps(state: int) -> int:
    """The +-1 increment a generator output gives (+1 iff S > 2^31)."""
    return int(_load().orc_bernoulli_eps(int(state)))


def superduper_seed(seed: int, walker: int, inst: int) -> int:
    """Initial generator state S_0 of walker `walker` (instance stream `inst`)."""
    return int(_load().orc_superduper_seed(int(seed), int(walker), int(inst)))


def move_bernoulli(seed: int, walker: int, step: int, inst: int) -> np.ndarray:
    """The six +-1 increments of move `step` of walker `walker` (serial replay)."""
    out = np.zeros(6)
    _load().orc_move_bernoulli(int(seed), int(walker), int(step), int(inst),
                               _ptr(out, ctypes.c_double))
    return out


def trial_eval(kind: int, params, x, ee_on: bool = True):
    """(sign, drift b (6,), E_L, ln|psi|) of the trial function at X (6,)."""
    lib = _load()
    p = np.ascontiguousarray(params, dtype=np.float64)
    xv = np.ascontiguousarray(x, dtype=np.float64)
    assert xv.shape == (6,)
    s = ctypes.c_int(0)
    b = np.zeros(6)
    el = ctypes.c_double(0.0)
    lp = ctypes.c_double(0.0)
    rc = lib.orc_trial_eval(int(kind), _ptr(p, ctypes.c_double), len(p), int(bool(ee_on)),
                            _ptr(xv, ctypes.c_double), ctypes.byref(s),
                            _ptr(b, ctypes.c_double), ctypes.byref(el), ctypes.byref(lp))
    if rc != 0:
        raise ValueError("oracle: malformed trial parameter vector")
    return s.value, b, el.value, lp.value


def trial_eval_many(kind: int, params, x, ee_on: bool = True):
    """trial_eval at every row of x (n, 6): (sign (n,), b (n, 6), E_L (n,), ln|psi| (n,))."""
    lib = _load()
    p = np.ascontiguousarray(params, dtype=np.float64)
    xv = np.ascontiguousarray(x, dtype=np.float64).reshape(-1, 6)
    n = xv.shape[0]
    s = np.zeros(n, dtype=np.intc)
    b = np.zeros((n, 6))
    el = np.zeros(n)
    lp = np.zeros(n)
    rc = lib.orc_trial_eval_many(int(kind), _ptr(p, ctypes.c_double), len(p), int(bool(ee_on)),
                                 n, _ptr(xv, ctypes.c_double), _ptr(s, ctypes.c_int),
                                 _ptr(b, ctypes.c_double), _ptr(el, ctypes.c_double),
                                 _ptr(lp, ctypes.c_double))
    if rc != 0:
        raise ValueError("oracle: malformed trial parameter vector")
    return s, b, el, lp


def without_jastrow(kind: int, params):
    """The parameter vector with the Jastrow factor removed (a = 0, c_k = 0), so that
    psi = Phi: the orbital part alone, which carries every node."""
    p = [float(v) for v in params]
    if int(kind) == KIND_JASTROW_PRODUCT:
        p = p[:1] + [0.0] + p[2:3] + [0.0] * max(0, len(p) - 3)
    else:
        p[0] = 0.0
        p[2:6] = [0.0, 0.0, 0.0, 0.0]
    return p


def node_distance(kind: int, params, x) -> np.ndarray:
    """First-order distance (bohr, in R^6) from each row of x (n, 6) to the nodal
    surface Phi = 0 of the trial function: |Phi| / |grad Phi| = 1 / |grad ln|Phi||,
    from the oracle's drift of the trial function without its Jastrow factor (which
    has no zeros).  Exact for a planar node; 0 on the node; for a nodeless Phi it is
    the inverse of the orbital drift, e.g. 1 / (Z sqrt 2) for exp(-Z r1 - Z r2)."""
    s, b, _, _ = trial_eval_many(kind, without_jastrow(kind, params), x, ee_on=True)
    g = np.sqrt((b * b).sum(axis=1))
    with np.errstate(divide="ignore", invalid="ignore"):
        d = np.where(s == 0, 0.0, 1.0 / g)
    return d


def neumaier_sum(v) -> float:
    a = np.ascontiguousarray(v, dtype=np.float64)
    return _load().orc_neumaier_sum(_ptr(a, ctypes.c_double), len(a))


class Walk:
    """Oracle walker population for one instance.

    Holds (X, logw, E_L, alive, sign) for the walker ids given (default 0..n-1)
    and advances them with the global step counter, so a subset of walker ids
    replays exactly the trajectories those ids have in a full population.
    """

    def __init__(self, kind, params, *, n_walkers=None, ids=None, dt, e_trial, seed,
                 inst=0, sigma=0.5, ee_on=True, noise=NOISE_GAUSSIAN):
        if ids is None:
            ids = np.arange(int(n_walkers), dtype=np.uint32)
        self.ids = np.ascontiguousarray(ids, dtype=np.uint32)
        n = len(self.ids)
        self.kind = int(kind)
        self.params = np.ascontiguousarray(params, dtype=np.float64)
        self.dt, self.e_trial, self.seed = float(dt), float(e_trial), int(seed)
        self.inst, self.sigma, self.ee_on = int(inst), float(sigma), bool(ee_on)
        self.noise = int(noise)
        self.lcg = np.zeros(n, dtype=np.uint32)     # Superduper states (noise 1)
        self.x = np.zeros((n, 6))
        self.logw = np.zeros(n)
        self.el = np.zeros(n)
        self.alive = np.zeros(n, dtype=np.uint8)
        self.sgn = np.zeros(n, dtype=np.int8)
        self.step = 0
        self.counters = np.zeros(3, dtype=np.int64)
        self.rows = []          # per-step population sums {c, W, P, Q, R, n_alive}
        self._call(0, do_init=True)

    def _call(self, n_steps, do_init=False):
        lib = _load()
        n = len(self.ids)
        nrows = n_steps + (1 if do_init else 0)
        stats = np.zeros((max(nrows, 1), 6))
        rc = lib.orc_run(self.kind, _ptr(self.params, ctypes.c_double), len(self.params),
                         int(self.ee_on), self.dt, self.e_trial, self.seed, self.inst,
                         self.sigma, n, _ptr(self.ids, ctypes.c_uint32),
                         _ptr(self.x, ctypes.c_double), _ptr(self.logw, ctypes.c_double),
                         _ptr(self.el, ctypes.c_double), _ptr(self.alive, ctypes.c_uint8),
                         _ptr(self.sgn, ctypes.c_int8), self.step, int(n_steps), int(do_init),
                         _ptr(stats, ctypes.c_double), _ptr(self.counters, ctypes.c_int64),
                         self.noise, _ptr(self.lcg, ctypes.c_uint32))
        if rc != 0:
            raise ValueError("oracle: bad walk parameters")
        self.rows.extend(stats[:nrows])
        self.step += int(n_steps)

    def advance(self, n_steps: int):
        self._call(int(n_steps))
        return self

    # --- space-averaged estimators from the per-step sums -------------------
    def series(self):
        """dict of per-step arrays: E (=P/W), ln_z (=ln(W e^c / N0)), ess (=W^2/Q),
        var (=R/W - E^2), n_alive; index k = after k steps."""
        r = np.array(self.rows)
        c, W, P, Q, R, na = r.T
        n0 = len(self.ids)
        with np.errstate(divide="ignore", invalid="ignore"):
            E = P / W
            return {"E": E, "ln_z": c + np.log(W) - np.log(n0), "ess": W * W / Q,
                    "var": R / W - E * E, "n_alive": na, "W": W, "P": P, "Q": Q,
                    "R": R, "c": c}
