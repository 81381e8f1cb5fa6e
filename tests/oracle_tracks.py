"""Oracle trajectories with per-walker node proximity, for the parity tests.

A walker that passes close to the nodal surface of its trial function is
ill-conditioned: there the drift grad ln|psi| ~ 1/d grows like the inverse
distance d to the node, and Phi = sum of terms of nearly equal size and
opposite sign, so a one-ulp difference between two exponential functions (the
CUDA library's and the host C library's) is amplified by ~1/d in the drift and
the position error grows along the rest of the path.  Walkers whose oracle
trajectory stays at least NODE_DISTANCE bohr from the node are held to the
strict per-walker tolerance; the others are counted and held to a looser one.
"""
import numpy as np

import oracle

# Walkers whose oracle trajectory comes closer than this (first-order distance in
# R^6, bohr) to the node of their trial function are the near-node walkers.
NODE_DISTANCE = 1e-3


def walk_tracking_node(kind, params, *, ids=None, n_walkers=None, steps, dt, e_trial, seed,
                       inst=0, sigma=0.5, ee_on=True, noise=0, keep_series=False,
                       near=NODE_DISTANCE):
    """Advance an oracle.Walk one move at a time.  Returns (walk, d_min, k_near):
    d_min[i] is the smallest first-order node distance (oracle.node_distance) of
    walker i over its positions while alive (the initial one, each one after a move,
    and the one that killed it); k_near[i] the first step (0 = initial position) at
    which that distance fell below `near` (steps + 1 if it never did).  With
    keep_series, walk.history holds per step (logw, E_L, alive) copies of every
    walker."""
    w = oracle.Walk(kind, params, ids=ids, n_walkers=n_walkers, dt=dt, e_trial=e_trial,
                    seed=seed, inst=inst, sigma=sigma, ee_on=ee_on, noise=noise)
    d_min = np.where(w.alive.astype(bool), oracle.node_distance(kind, params, w.x), np.inf)
    k_near = np.where(d_min < near, 0, int(steps) + 1)
    hist = [(w.logw.copy(), w.el.copy(), w.alive.copy())] if keep_series else None
    for k in range(1, int(steps) + 1):
        before = w.alive.astype(bool)
        w.advance(1)
        d = oracle.node_distance(kind, params, w.x)
        d_min = np.where(before, np.minimum(d_min, d), d_min)
        k_near = np.where((k_near > k) & (d_min < near), k, k_near)
        if keep_series:
            hist.append((w.logw.copy(), w.el.copy(), w.alive.copy()))
    w.history = hist
    return w, d_min, k_near


def energy_error_budget(w, k_near, rel_far=1e-13, rel_near=1e-8):
    """Per-step bound on |E_gpu(t) - E_oracle(t)| from the walkers' own tolerances.

    E(t) = sum_i w_i E_L,i / sum_i w_i.  A walker held to a relative tolerance r
    changes it by at most about 2 r (|E_L,i| + |E|) w_i / W (one r from its weight,
    one from its local energy).  Walkers away from the node give rel_far |E| in
    all (their sums agree to rounding); a near-node walker contributes with
    rel_near from the step k_near[i] at which it first came near the node (before
    that it is an ordinary walker).  Needs the history that
    walk_tracking_node(keep_series=True) keeps."""
    E = w.series()["E"]
    rel_far = np.broadcast_to(np.asarray(rel_far, dtype=float), E.shape)
    out = np.zeros(len(w.history))
    for k, (logw, el, alive) in enumerate(w.history):
        a = alive.astype(bool)
        out[k] = rel_far[k] * abs(E[k]) if np.isfinite(E[k]) else 0.0
        sel = a & (k_near <= k)
        if not sel.any():
            continue
        c = logw[a].max()
        wt = np.exp(logw[sel] - c)
        W = np.exp(logw[a] - c).sum()
        out[k] += rel_near * (2.0 * wt * (np.abs(el[sel]) + abs(E[k]))).sum() / W
    return out
