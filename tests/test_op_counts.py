"""The op-counting restatement of the oracle's walker-step (oracle/opcount.py) and the
operation counts the benchmark's roofline uses (CPU).

The restatement runs the oracle's procedure on a counting value type; that it is the
oracle's procedure is pinned by its values, which must equal the C oracle's bit for
bit (positions, drift, local energy and log-weight after each of two moves), so a
dropped or reordered operation in it would show.  The counts committed in bench.py
must equal the ones it produces."""
import importlib.util
import os

import numpy as np
import pytest

import oracle
from oracle import opcount

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.mark.parametrize("noise", [0, 1])
@pytest.mark.parametrize("case", sorted(opcount.COUNT_CASES))
def test_restatement_equals_the_c_oracle(case, noise):
    kind, p = opcount.COUNT_CASES[case]
    seed, walker, inst, dt, et = 7, 12345, 3, 0.005, -2.9037
    w = oracle.Walk(kind, p, ids=np.array([walker], dtype=np.uint32), dt=dt, e_trial=et,
                    seed=seed, inst=inst, noise=noise)
    x0 = w.x[0].copy()
    counts, vals = opcount.count_step(kind, p, noise=noise, x0=list(x0), seed=seed,
                                      walker=walker, inst=inst, dt=dt, e_trial=et,
                                      lcg0=int(w.lcg[0]), return_values=True)
    for k in range(2):
        w.advance(1)
        x, b, el, logw = vals[k]
        assert np.array_equal(np.array(x), w.x[0]), (k, np.array(x) - w.x[0])
        assert el == w.el[0] and logw == w.logw[0]
        _, bo, elo, _ = oracle.trial_eval(kind, p, w.x[0])
        assert np.array_equal(np.array(b), bo) and el == elo
    assert counts["flops"] > 0


def test_counts_follow_the_definitions():
    """What the counts must contain for the ground-state product (hand count): Gaussian
    noise needs three logarithms, three square roots of the Box-Muller radius, three
    cosines and three sines per move, the three distances three more roots, the two
    orbital exponentials one each, and the weight one exponential; six conversions of
    words to uniforms.  Philox4x32-10 at one block per move: at most 20 32x32->64
    products and 40 exclusive-ors per move (fewer where the two moves' blocks share
    a product), the key schedule's 18 additions once per two moves and the move
    counter's increment, and the three 10-bit angle fields of the block's last word.
    The Bernoulli walk replaces all of the noise by six congruential steps (a 32-bit
    product and an addition each) and six threshold tests."""
    g = opcount.count_step(*opcount.COUNT_CASES["ground"], noise=0)
    assert g["fp_log"] == 3 and g["fp_sin"] == 3 and g["fp_cos"] == 3
    assert g["fp_sqrt"] == 6 and g["fp_exp"] == 3 and g["cvt"] == 6
    assert 16 <= g["int_mulwide"] <= 20 and 30 <= g["int_xor"] <= 40
    assert g["int_add"] == 9.5 and g["int_bit"] == 3
    bern = opcount.count_step(*opcount.COUNT_CASES["ground"], noise=1)
    assert bern["int_mul"] == 6 and bern["int_add"] == 6 and bern["int_mulwide"] == 0
    assert bern["fp_log"] == 0 and bern["fp_sin"] == 0 and bern["fp_sqrt"] == 3
    # the noise is the only difference: Box-Muller's and the Gaussian move's flops
    # (uniform map 2 x 6, radius 3, angle 3, products 6, and one more multiply per
    # coordinate in the move: sqrt(dt) xi against the folded sqrt(dt) eps)
    assert g["flops"] - bern["flops"] == 12 + 3 + 3 + 6 + 6
    # a two-term orbital pair costs more than the single product
    t = opcount.count_step(*opcount.COUNT_CASES["triplet_2s3"], noise=0)
    assert t["flops"] > g["flops"] and t["fp_exp"] == 5


def _bench_module():
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    m = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(m)
    return m


def test_bench_counts_equal_the_restatement():
    bench = _bench_module()
    tab = opcount.table()
    assert len(bench.OP_COUNTS) == sum(len(c) for c in tab.values())
    for noise, cases in tab.items():
        for case, c in cases.items():
            committed = bench.OP_COUNTS[(int(noise), case)]
            for k, v in committed.items():
                assert v == c[k], (noise, case, k, v, c[k])


def test_count_cases_are_the_workloads_trial_functions():
    """The counted trial functions are the ones the benchmark workloads walk, per state."""
    from paper_1703_08977_gb300 import workloads as wl
    bench = _bench_module()
    for state, case in bench.STATE_CASE.items():
        kind, params = wl.trial_for_state(state)
        ck, cp = opcount.COUNT_CASES[case]
        assert ck == kind and np.array_equal(np.asarray(cp, float), np.asarray(params, float))
