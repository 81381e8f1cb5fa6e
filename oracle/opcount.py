"""Operation counts of one walker-step of the GFK walk, taken from the oracle's procedure.

TEST INFRASTRUCTURE ONLY.  This module restates, operation for operation, what
``gfk_oracle.c`` does for one move of one walker -- the Philox4x32-10 words, the
Box-Muller normals (or the paper's +-1 Bernoulli increments), the Euler-Maruyama
move, the trial evaluation (drift and local energy through the orbitals' values,
gradients and Laplacians and the Jastrow factor), the fixed-node test, the
right-point weight update of Eq. 4 and one walker's share of the population sums
-- on a counting value type, and counts the operations the step's outputs need.
Its values equal the C oracle's bit for bit (``tests/test_op_counts.py``), which is
what ties the counts to the oracle.  The counts are the numerator of the
benchmark's ALU roofline (the algorithmic work per walker-step).

How an operation is counted:
  * Every arithmetic operation on a walker-dependent value is a node of an
    expression graph.  Identical operations on identical operands are one node
    (the oracle recomputes r1, r2 and the Philox blocks it already had; the work
    is needed once), and only nodes that the outputs of the step depend on count.
  * Operations whose operands are all trial or instance parameters are folded
    (done once per launch, not per walker-step), as are the identities x * 0,
    x * 1, x + 0, x - 0 and x / 1 (a parameter that is exactly 0 or 1, such as
    the absent prefactor terms of an orbital, costs nothing).
  * Negation and absolute value are free (sign modifiers of the operation that
    consumes them).
  * A step is counted as two consecutive moves of one walker divided by two.
    Each move draws one Philox block; the two blocks share the first-round
    products of the walker and instance words.  Each move evaluates the trial function once, at the new position; its
    drift serves the next move (the oracle re-evaluates the drift at the old
    position, a convenience of its loop that the walk does not need).
  * The population sums are the four plain accumulations of w, w E_L, w^2 and
    w E_L^2 with w = exp(logw - c); the oracle's Neumaier compensation of them is
    an accuracy device of the reduction and is not counted.

Categories: fp_add (additions and subtractions), fp_mul, fp_div, fp_sqrt, fp_exp,
fp_log, fp_sin, fp_cos, fp_pow, cmp (comparisons and finiteness tests), cvt (integer to
floating-point conversions), int_mulwide (32 x 32 -> 64-bit products), int_xor, int_add,
int_mul (32-bit products), int_bit (bit-field extractions). "flops" = fp_add + fp_mul +
fp_div (a fused multiply-add is a multiply and an add, two flops); "special" = the
transcendental and root operations (one special-function-unit operation each on a GPU);
"int" = the integer operations.

    python -m oracle.opcount            # prints the table as JSON
"""
from __future__ import annotations

import json
import math

__all__ = ["count_step", "COUNT_CASES", "table"]

M32 = 0xFFFFFFFF


class Tape:
    """The expression graph of one counting run."""

    def __init__(self):
        self.nodes = []           # (op, (arg ids ...)); id = index
        self.index = {}           # (op, args, extra) -> id

    def node(self, op, args, extra=None):
        key = (op, args, extra)
        i = self.index.get(key)
        if i is None:
            i = len(self.nodes)
            self.nodes.append((op, args))
            self.index[key] = i
        return i

    def count(self, outputs):
        """Category counts of the nodes the outputs depend on."""
        seen, stack = set(), [v.id for v in outputs if isinstance(v, (V, I)) and v.id is not None]
        while stack:
            i = stack.pop()
            if i in seen:
                continue
            seen.add(i)
            stack.extend(a for a in self.nodes[i][1] if a is not None)
        out = {}
        for i in seen:
            op = self.nodes[i][0]
            if op in ("input", "neg", "abs", "hi", "lo"):
                continue
            out[op] = out.get(op, 0) + 1
        return out


class V:
    """A value with its node in the tape (id None: a parameter or constant)."""

    __slots__ = ("t", "v", "id")

    def __init__(self, t, v, i=None):
        self.t, self.v, self.id = t, v, i

    # -- helpers -----------------------------------------------------------
    @staticmethod
    def _w(t, x):
        return x if isinstance(x, V) else V(t, x)

    def _bin(self, other, op, f, rev=False):
        a, b = (V._w(self.t, other), self) if rev else (self, V._w(self.t, other))
        val = f(a.v, b.v)
        if a.id is None and b.id is None:
            return V(self.t, val)
        # identities with an exact parameter 0 or 1
        if op == "fp_mul":
            for p, q in ((a, b), (b, a)):
                if p.id is None and p.v == 0.0:
                    return V(self.t, 0.0 * q.v)
                if p.id is None and p.v == 1.0:
                    return q
                if p.id is None and p.v == -1.0:
                    return -q
        if op == "fp_add":
            if a.id is None and a.v == 0.0:
                return b
            if b.id is None and b.v == 0.0:
                return a
        if op == "fp_sub":
            if b.id is None and b.v == 0.0:
                return a
            if a.id is None and a.v == 0.0:
                return -b
        if op == "fp_div" and b.id is None and b.v == 1.0:
            return a
        if op == "fp_div" and a.id is None and a.v == 0.0:
            return V(self.t, 0.0 * b.v)
        kind = "fp_add" if op == "fp_sub" else op
        # a parameter operand enters the key by its value (x + 0.5 and x + 0.25 differ)
        consts = (None if a.id is not None else a.v, None if b.id is not None else b.v)
        return V(self.t, val, self.t.node(kind, (a.id, b.id), (op, consts)))

    def __add__(self, o): return self._bin(o, "fp_add", lambda x, y: x + y)
    def __radd__(self, o): return self._bin(o, "fp_add", lambda x, y: x + y, rev=True)
    def __sub__(self, o): return self._bin(o, "fp_sub", lambda x, y: x - y)
    def __rsub__(self, o): return self._bin(o, "fp_sub", lambda x, y: x - y, rev=True)
    def __mul__(self, o): return self._bin(o, "fp_mul", lambda x, y: x * y)
    def __rmul__(self, o): return self._bin(o, "fp_mul", lambda x, y: x * y, rev=True)
    def __truediv__(self, o): return self._bin(o, "fp_div", lambda x, y: x / y)
    def __rtruediv__(self, o): return self._bin(o, "fp_div", lambda x, y: x / y, rev=True)

    def __neg__(self):
        if self.id is None:
            return V(self.t, -self.v)
        return V(self.t, -self.v, self.t.node("neg", (self.id,)))

    # comparisons give plain booleans (the branch the oracle takes) and count
    def _cmp(self, other, f):
        o = V._w(self.t, other)
        if self.id is not None or o.id is not None:
            consts = (None if self.id is not None else self.v, None if o.id is not None else o.v)
            self.t.cmp_ids.append(self.t.node("cmp", (self.id, o.id), (f.__name__, consts)))
        return f(self.v, o.v)

    def __gt__(self, o): return self._cmp(o, _gt)
    def __lt__(self, o): return self._cmp(o, _lt)
    def __ge__(self, o): return self._cmp(o, _ge)


def _gt(a, b): return a > b
def _lt(a, b): return a < b
def _ge(a, b): return a >= b


def _un(op, f, x):
    if not isinstance(x, V) or x.id is None:
        xv = x.v if isinstance(x, V) else x
        return V(x.t, f(xv)) if isinstance(x, V) else f(xv)
    return V(x.t, f(x.v), x.t.node(op, (x.id,)))


def sqrt(x): return _un("fp_sqrt", math.sqrt, x)
def exp(x): return _un("fp_exp", math.exp, x)
def log(x): return _un("fp_log", math.log, x)
def sin(x): return _un("fp_sin", math.sin, x)
def cos(x): return _un("fp_cos", math.cos, x)
def fabs(x): return _un("abs", abs, x)


def pw(x, k):
    if not isinstance(x, V) or x.id is None:
        return V(x.t, math.pow(x.v, k)) if isinstance(x, V) else math.pow(x, k)
    return V(x.t, math.pow(x.v, k), x.t.node("fp_pow", (x.id,), k))


def isfinite(x):
    if isinstance(x, V) and x.id is not None:
        x.t.cmp_ids.append(x.t.node("cmp", (x.id,), "isfinite"))
        return math.isfinite(x.v)
    return math.isfinite(x.v if isinstance(x, V) else x)


# -- integers (Philox, Superduper) --------------------------------------------
class I:
    """A 32-bit (or 64-bit product) integer value with its node."""

    __slots__ = ("t", "v", "id")

    def __init__(self, t, v, i=None):
        self.t, self.v, self.id = t, v, i


def _iw(t, x):
    return x if isinstance(x, I) else I(t, x)


def imulwide(a, b):
    """32 x 32 -> 64-bit product (one operation giving both halves)."""
    a, b = _iw(a.t if isinstance(a, I) else b.t, a), _iw(a.t if isinstance(a, I) else b.t, b)
    v = (a.v & M32) * (b.v & M32)
    if a.id is None and b.id is None:
        return I(a.t, v)
    return I(a.t, v, a.t.node("int_mulwide", (a.id, b.id)))


def ihi(p):
    return I(p.t, p.v >> 32, None if p.id is None else p.t.node("hi", (p.id,)))


def ilo(p):
    return I(p.t, p.v & M32, None if p.id is None else p.t.node("lo", (p.id,)))


def ixor(a, b):
    t = a.t if isinstance(a, I) else b.t
    a, b = _iw(t, a), _iw(t, b)
    v = a.v ^ b.v
    if a.id is None and b.id is None:
        return I(t, v)
    if a.id is None and a.v == 0:
        return b
    if b.id is None and b.v == 0:
        return a
    ids = tuple(sorted(i for i in (a.id, b.id) if i is not None))   # xor commutes
    const = None if (a.id is not None and b.id is not None) else (a.v if a.id is None else b.v)
    return I(t, v, t.node("int_xor", ids, const))


def iadd(a, b):
    t = a.t if isinstance(a, I) else b.t
    a, b = _iw(t, a), _iw(t, b)
    v = (a.v + b.v) & M32
    if a.id is None and b.id is None:
        return I(t, v)
    return I(t, v, t.node("int_add", (a.id, b.id), (a.v if a.id is None else None,
                                                      b.v if b.id is None else None)))


def imul(a, b):
    t = a.t if isinstance(a, I) else b.t
    a, b = _iw(t, a), _iw(t, b)
    v = (a.v * b.v) & M32
    if a.id is None and b.id is None:
        return I(t, v)
    return I(t, v, t.node("int_mul", (a.id, b.id), (a.v if a.id is None else None,
                                                      b.v if b.id is None else None)))


def ifield(a, shift, bits):
    """(a >> shift) & (2^bits - 1): one bit-field extraction."""
    t = a.t
    v = (a.v >> shift) & ((1 << bits) - 1)
    if a.id is None:
        return I(t, v)
    return I(t, v, t.node("int_bit", (a.id,), (shift, bits)))


def i2f(w):
    """Integer word to double (the uniform map's conversion)."""
    if w.id is None:
        return V(w.t, float(w.v))
    return V(w.t, float(w.v), w.t.node("cvt", (w.id,)))


def f_input(t, v, name):
    return V(t, float(v), t.node("input", (), name))


def i_input(t, v, name):
    return I(t, int(v) & M32, t.node("input", (), name))


# -- the oracle's procedure, restated ------------------------------------------
PHILOX_M0, PHILOX_M1 = 0xD2511F53, 0xCD9E8D57
PHILOX_W0, PHILOX_W1 = 0x9E3779B9, 0xBB67AE85


def philox4x32_10(ctr, key):
    """orc_philox4x32_10 on counting integers."""
    c0, c1, c2, c3 = ctr
    k0, k1 = key
    for rnd in range(10):
        if rnd > 0:
            k0 = iadd(k0, PHILOX_W0)
            k1 = iadd(k1, PHILOX_W1)
        p0 = imulwide(I(c0.t if isinstance(c0, I) else k0.t, PHILOX_M0), c0)
        p1 = imulwide(I(p0.t, PHILOX_M1), c2)
        hi0, lo0, hi1, lo1 = ihi(p0), ilo(p0), ihi(p1), ilo(p1)
        n0 = ixor(ixor(hi1, c1), k0)
        n2 = ixor(ixor(hi0, c3), k1)
        c0, c1, c2, c3 = n0, lo1, n2, lo0
    return [c0, c1, c2, c3]


def uniform(w):
    """orc_uniform: (w + 1/2) 2^-32."""
    return (i2f(w) + 0.5) * (1.0 / 4294967296.0)


def angle_uniform(k):
    """orc_angle_uniform: (k + 1/2) / 1024."""
    return (i2f(k) + 0.5) * (1.0 / 1024.0)


def box_muller(wa, kb):
    two_pi = 6.283185307179586476925286766559
    ua, ub = uniform(wa), angle_uniform(kb)
    rho = sqrt(-2.0 * log(ua))
    ang = two_pi * ub
    return rho * cos(ang), rho * sin(ang)


def move_normals(t, key, walker, n_word, inst):
    """orc_move_normals: the one block (walker, n, inst, 0); radius words 0-2, the
    10-bit angle fields of word 3."""
    w = philox4x32_10([walker, n_word, inst, I(t, 0)], key)
    xi = []
    for j in range(3):
        xi += list(box_muller(w[j], ifield(w[3], 10 * j, 10)))
    return xi


def superduper_step(s):
    """Six outputs of the congruential generator and their +-1 increments."""
    eps = []
    for _ in range(6):
        s = iadd(imul(s, 69069), 1)
        # the threshold test of orc_bernoulli_eps
        s.t.cmp_ids.append(s.t.node("cmp", (s.id,), "gt2^31"))
        eps.append(1.0 if s.v > 2147483648 else -1.0)
    return s, eps


def trial_parse(kind, p):
    """orc_trial_parse: (a, beta, ck, terms [(s, alpha[2], c0[2], c1[2], cz[2])])."""
    if kind == 0:
        Z = p[0]
        ck = [p[3 + k] if 3 + k < len(p) else 0.0 for k in range(4)]
        return p[1], p[2], ck, [(1.0, [Z, Z], [1.0, 1.0], [0.0, 0.0], [0.0, 0.0])]
    nt = int(p[6])
    terms = []
    for i in range(nt):
        q = p[7 + 9 * i: 16 + 9 * i]
        terms.append((q[0], [q[1], q[5]], [q[2], q[6]], [q[3], q[7]], [q[4], q[8]]))
    return p[0], p[1], list(p[2:6]), terms


def orbital(alpha, c0, c1, cz, rv):
    """orc_orbital: value, gradient and Laplacian of (c0 + c1 r + cz z) e^{-alpha r}."""
    r = sqrt(rv[0] * rv[0] + rv[1] * rv[1] + rv[2] * rv[2])
    ex = exp(-alpha * r)
    p = c0 + c1 * r + cz * rv[2]
    gp = [c1 * rv[0] / r, c1 * rv[1] / r, c1 * rv[2] / r + cz]
    g = [(gp[d] - alpha * p * rv[d] / r) * ex for d in range(3)]
    lap_p = 2.0 * c1 / r
    gp_dot_rhat = c1 + cz * rv[2] / r
    lap = (lap_p - 2.0 * alpha * gp_dot_rhat + p * (alpha * alpha - 2.0 * alpha / r)) * ex
    return p * ex, g, lap


def jastrow(a, beta, ck, r):
    """orc_jastrow: u, u', u''."""
    q = 1.0 + beta * r
    rho = r / q
    drho = 1.0 / (q * q)
    d2rho = -2.0 * beta / (q * q * q)
    val = a * rho
    d1 = a
    d2 = 0.0
    for k in range(1, 5):
        c = ck[k - 1]
        if c == 0.0:
            continue          # the term is c * (...) with c = 0: folded away
        val = val + c * pw(rho, k + 1)
        d1 = d1 + c * (k + 1) * pw(rho, k)
        d2 = d2 + c * (k + 1) * k * pw(rho, k - 1)
    return val, d1 * drho, d2 * drho * drho + d1 * d2rho


def evaluate(trial, ee_on, x):
    """orc_eval: (sign, drift (6), E_L)."""
    a, beta, ck, terms = trial
    r1v, r2v = x[0:3], x[3:6]
    Phi, lapPhi = 0.0, 0.0
    g1, g2 = [0.0] * 3, [0.0] * 3
    for (s, al, c0, c1, cz) in terms:
        fa, ga, la = orbital(al[0], c0[0], c1[0], cz[0], r1v)
        fb, gb, lb = orbital(al[1], c0[1], c1[1], cz[1], r2v)
        Phi = Phi + s * fa * fb
        lapPhi = lapPhi + s * (la * fb + fa * lb)
        for d in range(3):
            g1[d] = g1[d] + s * ga[d] * fb
            g2[d] = g2[d] + s * fa * gb[d]
    r1 = sqrt(r1v[0] * r1v[0] + r1v[1] * r1v[1] + r1v[2] * r1v[2])
    r2 = sqrt(r2v[0] * r2v[0] + r2v[1] * r2v[1] + r2v[2] * r2v[2])
    d12 = [r1v[d] - r2v[d] for d in range(3)]
    r12 = sqrt(d12[0] * d12[0] + d12[1] * d12[1] + d12[2] * d12[2])
    u, up, upp = jastrow(a, beta, ck, r12)
    if not (Phi > 0.0 or Phi < 0.0):
        return 0, None, None, (r1, r2, r12)
    sign = 1 if Phi > 0.0 else -1
    gu1 = [up * d12[d] / r12 for d in range(3)]
    gu2 = [-v for v in gu1]
    cross = 0.0
    b = [None] * 6
    for d in range(3):
        b[d] = g1[d] / Phi + gu1[d]
        b[3 + d] = g2[d] / Phi + gu2[d]
        cross = cross + (g1[d] * gu1[d] + g2[d] * gu2[d])   # C's "+=" adds the sum
    lap_u = 2.0 * (upp + 2.0 * up / r12)
    grad_u_sq = 2.0 * up * up
    lap_over_psi = lapPhi / Phi + 2.0 * cross / Phi + lap_u + grad_u_sq
    V_ = -2.0 / r1 - 2.0 / r2 + (1.0 / r12 if ee_on else 0.0)
    return sign, b, -0.5 * lap_over_psi + V_, (r1, r2, r12)


def count_step(kind, params, noise=0, ee_on=True, x0=None, seed=7, walker=12345, inst=3,
               dt=0.005, e_trial=-2.9037, lcg0=0x1234567, return_values=False):
    """Counts of one walker-step (two consecutive moves, divided by two) of the walk of
    trial function (kind, params) with Gaussian (noise 0) or Bernoulli (1) increments.
    With return_values, also the positions, drifts, local energies and log-weights
    after each of the two moves (for the comparison with the C oracle)."""
    t = Tape()
    t.cmp_ids = []
    trial = trial_parse(int(kind), [float(v) for v in params])
    if x0 is None:
        x0 = [0.31, -0.52, 0.17, -0.44, 0.58, 0.26]
    x = [f_input(t, v, f"x{d}") for d, v in enumerate(x0)]
    # drift at the starting position: an input (the previous move's evaluation)
    s0, b0, _, _ = evaluate(trial, ee_on, [float(v) for v in x0])
    b = [f_input(t, v, f"b{d}") for d, v in enumerate(b0)]
    logw = f_input(t, 0.0, "logw")
    c_shift = f_input(t, 0.0, "c")
    key = [i_input(t, seed & M32, "k0"), i_input(t, seed >> 32, "k1")]
    wid = i_input(t, walker, "walker")
    ist = i_input(t, inst, "inst")
    n_word = i_input(t, 0, "n")
    lcg = i_input(t, lcg0, "lcg")
    sqrt_dt = math.sqrt(dt)
    outs = []
    values = []
    sgn = s0
    for odd in (0, 1):
        if noise == 0:
            # moves n and n + 1 (the step counter advanced by one)
            xi = move_normals(t, key, wid, iadd(n_word, 1) if odd else n_word, ist)
        else:
            lcg, xi = superduper_step(lcg)
        x = [x[d] + b[d] * dt + sqrt_dt * xi[d] for d in range(6)]
        s1, b1, e1, (r1, r2, r12) = evaluate(trial, ee_on, x)
        # the coalescence diagnostic, the node test and the finiteness tests
        _ = (r1 < 1e-10, r2 < 1e-10, r12 < 1e-10)
        xfinite = all(isfinite(v) for v in x)
        assert xfinite and s1 == sgn, "the counting position must stay alive"
        _ = isfinite(e1) and all(isfinite(v) for v in b1)
        logw = logw - (e1 - e_trial) * dt
        # this walker's share of the population sums of the step
        w = exp(logw - c_shift)
        sums = [w, w * e1, w * w, w * e1 * e1]
        outs += x + b1 + [e1, logw] + sums + ([lcg] if noise == 1 else [])
        values.append(([v.v for v in x], [v.v for v in b1], e1.v, logw.v))
        b = b1
    c = t.count(outs)
    c["cmp"] = len(set(t.cmp_ids))
    # four accumulations per move: add into the running sums
    c["fp_add"] = c.get("fp_add", 0) + 4 * 2
    half = {k: v / 2.0 for k, v in c.items()}
    for k in ("fp_add", "fp_mul", "fp_div", "fp_sqrt", "fp_exp", "fp_log", "fp_sin", "fp_cos",
              "fp_pow", "cmp", "cvt", "int_mulwide", "int_xor", "int_add", "int_mul",
              "int_bit"):
        half.setdefault(k, 0.0)
    half["flops"] = half["fp_add"] + half["fp_mul"] + half["fp_div"]
    half["special"] = sum(half[k] for k in ("fp_sqrt", "fp_exp", "fp_log", "fp_sin", "fp_cos",
                                            "fp_pow"))
    half["int"] = (half["int_mulwide"] + half["int_xor"] + half["int_add"] + half["int_mul"] +
                   half["int_bit"])
    if return_values:
        return half, values
    return half


def _cases():
    # the benchmark workloads' trial functions (same vectors as the seeded workloads):
    # ground 1^1S product with the Pade-Jastrow factor; the 2^3S pair; the P_z pair
    ground = [2.0, 0.5, 0.5, 0.0, 0.0, 0.0, 0.0]
    t2 = [0.25, 0.3, 0, 0, 0, 0, 2,
          1.0, 2.0, 1.0, 0.0, 0.0, 0.5, 1.0, 0.0, 0.0,
          -1.0, 0.5, 1.0, 0.0, 0.0, 2.0, 1.0, 0.0, 0.0]
    pz = [0.5, 0.5, 0, 0, 0, 0, 2,
          1.0, 2.0, 1.0, 0.0, 0.0, 0.5, 0.0, 0.0, 1.0,
          1.0, 0.5, 0.0, 0.0, 1.0, 2.0, 1.0, 0.0, 0.0]
    return {"ground": (0, ground), "triplet_2s3": (1, t2), "pz": (1, pz)}


COUNT_CASES = _cases()


def table():
    """{noise: {case: counts}} for the benchmark workloads' trial functions."""
    out = {}
    for noise in (0, 1):
        out[str(noise)] = {name: count_step(k, p, noise=noise)
                           for name, (k, p) in COUNT_CASES.items()}
    return out


if __name__ == "__main__":
    print(json.dumps(table(), indent=1, sort_keys=True))
