"""Seeded, synthetic inputs shared by the tests, the benchmark and the oracle runs.

This module holds parameter vectors and workload shapes only: none of the
method's arithmetic lives here, so both the CUDA path and the oracle can be fed
from it without sharing code.

Layouts (both sides read the same vectors):
  kind 0, Jastrow product:  [Z, a, beta, c1, c2, c3, c4]
  kind 1, orbital pairs:    [a, beta, c1, c2, c3, c4, nterms,
                             (s, alphaA, c0A, c1A, czA, alphaB, c0B, c1B, czB) * nterms]
Each orbital is (c0 + c1 r + cz z) exp(-alpha r); the Jastrow factor is
exp(a rho + sum c_k rho^(k+1)) with rho = r12 / (1 + beta r12).
"""

KIND0 = 0
KIND1 = 1


def ground(Z=2.0, a=0.5, beta=0.5, c=(0.0, 0.0, 0.0, 0.0)):
    """exp(-Z r1 - Z r2) exp(a r12/(1+beta r12) + ...): the 1^1S trial of the benchmarks."""
    return [Z, a, beta, *c]


def pairs(terms, a=0.0, beta=0.0, c=(0.0, 0.0, 0.0, 0.0)):
    v = [a, beta, *c, float(len(terms))]
    for t in terms:
        assert len(t) == 9
        v.extend(float(q) for q in t)
    return v


def orb(alpha, c0=1.0, c1=0.0, cz=0.0):
    return (alpha, c0, c1, cz)


def term(s, A, B):
    return (s, *A, *B)


def triplet_2s3(a=0.25, beta=0.3):
    """(e^{-2 r1 - 0.5 r2} - e^{-0.5 r1 - 2 r2}) exp(r12/(4(1+0.3 r12))): the 2^3S benchmark trial."""
    return pairs([term(1.0, orb(2.0), orb(0.5)), term(-1.0, orb(0.5), orb(2.0))], a=a, beta=beta)


def pz_state(sign=1.0, a=0.5, beta=0.5):
    """z2 e^{-2 r1 - 0.5 r2} + sign * exchange, times the ground-state Jastrow factor."""
    return pairs([term(1.0, orb(2.0), orb(0.5, c0=0.0, cz=1.0)),
                  term(sign, orb(0.5, c0=0.0, cz=1.0), orb(2.0))], a=a, beta=beta)


def fn3(r0=1.0, a1=1.0, a2=2.0, a=0.0, beta=0.0):
    """Trial function 3 of the paper: (r0 - r1) e^{-a1 r1 - a2 r2} - (r0 - r2) e^{-a2 r1 - a1 r2}.
    Functions 4 and 5 are the same form with other (r0, a1, a2)."""
    return pairs([term(1.0, orb(a1, c0=r0, c1=-1.0), orb(a2)),
                  term(-1.0, orb(a2), orb(a1, c0=r0, c1=-1.0))], a=a, beta=beta)


def fn7(a1, a2, a=0.0, beta=0.0):
    """Trial function 7 (P_z): (z1 + z2)(e^{-a1 r1 - a2 r2} + e^{-a2 r1 - a1 r2})."""
    z = dict(c0=0.0, cz=1.0)
    return pairs([term(1.0, orb(a1, **z), orb(a2)), term(1.0, orb(a2, **z), orb(a1)),
                  term(1.0, orb(a1), orb(a2, **z)), term(1.0, orb(a2), orb(a1, **z))],
                 a=a, beta=beta)


def hydrogenic_1s2s_triplet():
    """Antisymmetrised 1s(Z=2) 2s(Z=2) product = function 3 with r0=1, a1=1, a2=2."""
    return fn3(1.0, 1.0, 2.0)


def hydrogenic_1s2pz(sign=1.0):
    """1s(Z=2) 2p_z(Z=2) product, (anti)symmetrised: exact eigenfunction without e-e repulsion."""
    return pairs([term(1.0, orb(2.0), orb(1.0, c0=0.0, cz=1.0)),
                  term(sign, orb(1.0, c0=0.0, cz=1.0), orb(2.0))])


# ---------------------------------------------------------------------------
# Benchmark workloads (synthetic, seeded).  Each instance is a plain dict:
# state (0 = 1^1S, 1 = 2^3S, 2 = P_z), n_walkers, dt, e_trial, seed,
# rng_stream, kind and params of the trial function.
# ---------------------------------------------------------------------------
# Trial energies: the variational energies of the paper's summary table,
# rounded (they shift every log-weight equally and leave E(t) unchanged).
E_T = {0: -2.9037, 1: -2.1752, 2: -2.1238}


def trial_for_state(state):
    """The workloads' trial function per state: ground product with Jastrow a=1/2,
    beta=0.5; the 2^3S antisymmetric 2s-like pair with a=1/4, beta=0.3; the P_z
    pair with + exchange and the ground Jastrow factor."""
    return {0: (KIND0, ground()), 1: (KIND1, triplet_2s3()), 2: (KIND1, pz_state(+1.0))}[state]


def instance(state, n_walkers, dt, seed=0, rng_stream=0, noise=0):
    kind, params = trial_for_state(state)
    return dict(state=state, n_walkers=int(n_walkers), dt=float(dt), e_trial=E_T[state],
                seed=int(seed), rng_stream=int(rng_stream), kind=kind, params=params,
                noise=int(noise))


def ground_fp64_correctness():
    """He 1^1S in FP64: 4096 walkers, dt 0.01, E_T -2.9, 2000 moves, seed 0."""
    d = instance(0, 4096, 0.01)
    d["e_trial"] = -2.9
    return [d], 2000


def ground_at_scale(dt=0.005):
    """He 1^1S: 2^20 walkers, 20000 moves at dt in {0.005, 0.0025, 0.00125}."""
    return [instance(0, 1 << 20, dt)], 20000


def triplet_at_scale():
    """He 2^3S with the exact node: 2^20 walkers, dt 0.0025, 20000 moves."""
    return [instance(1, 1 << 20, 0.0025)], 20000


def bernoulli_at_scale():
    """He 1^1S walked with the paper's +-1 steps (Superduper generators): 2^20 walkers,
    20000 moves at dt = 1/900, i.e. the paper's scale 30 (step length 1/30), t = 22.2."""
    return [instance(0, 1 << 20, 1.0 / 900.0, noise=1)], 20000


def batched(seed=1, n_moves=10000, scale=1.0):
    """Twelve instances: {1^1S, 2^3S, P_z} x dt {0.01, 0.005, 0.0025, 0.00125}, walker
    counts round(2^U) with U ~ U[16, 21] from numpy's default_rng(seed), one Philox
    stream each.  `scale` shrinks the walker counts for tests."""
    import numpy as np
    rng = np.random.default_rng(seed)
    out = []
    i = 0
    for state in (0, 1, 2):
        for dt in (0.01, 0.005, 0.0025, 0.00125):
            n = int(round(2.0 ** rng.uniform(16.0, 21.0) * scale))
            out.append(instance(state, max(n, 1), dt, seed=0, rng_stream=i))
            i += 1
    return out, n_moves
