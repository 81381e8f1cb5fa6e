"""Statistical runs of the GFK walk on the GPU (energies with error bars).

replica_energies: R independent replicas of one instance (distinct Philox
streams) in one batched context; per replica the space-averaged energy E(t)
averaged over the second half of the run, and the growth estimate
lambda_1 = E_T - A from ln z(t)/t = A + B/t (Eq. 4).  Mean and standard error
over the replicas.

dt_study: the same at several time steps, and the linear dt -> 0 extrapolation
of the mixed estimator.

Run:  python -m paper_1703_08977_gb300.experiments --state 0 --walkers 65536 \
          --replicas 16 --t 20 --dts 0.01 0.005 0.0025
"""
from __future__ import annotations

import argparse
import json

import numpy as np

from . import analysis, gfk, workloads

EXACT = {0: -2.9037243770341195, 1: -2.17522937823679130, 2: -2.123843086498093}


def replica_energies(state, dt, t_total, n_walkers, replicas, seed=0, prec=gfk.GFK_PREC_MIXED,
                     growth_times=None, noise=gfk.GFK_NOISE_GAUSSIAN):
    kind, params = workloads.trial_for_state(state)
    et = workloads.E_T[state]
    descs = [gfk.InstanceDesc(n_walkers=n_walkers, dt=dt, e_trial=et, seed=seed, state=state,
                              prec=prec, rng_stream=100 + r, noise=noise)
             for r in range(replicas)]
    n_moves = int(round(t_total / dt))
    with gfk.Context(descs, trials=[(kind, params)] * replicas) as ctx:
        ctx.propagate(n_moves)
        e_mean, lam, ess_end = [], [], []
        for r in range(replicas):
            en = ctx.energy(r)
            e = en["E"]
            e_mean.append(float(np.mean(e[len(e) // 2:])))
            ess_end.append(float(en["ess"][-1]))
            if growth_times is not None:
                lam.append(analysis.growth_from_series(et, dt, en["ln_z"], growth_times)[0])
    e_mean = np.array(e_mean)
    out = {"state": state, "dt": dt, "t": t_total, "walkers": n_walkers, "replicas": replicas,
           "noise": noise,
           "E": float(e_mean.mean()), "E_err": float(e_mean.std(ddof=1) / np.sqrt(replicas)),
           "ess_final_over_N": float(np.mean(ess_end)) / n_walkers}
    if lam:
        lam = np.array(lam)
        out["lambda_growth"] = float(lam.mean())
        out["lambda_growth_err"] = float(lam.std(ddof=1) / np.sqrt(replicas))
    return out


def dt_study(state, dts, t_total, n_walkers, replicas, seed=0, prec=gfk.GFK_PREC_MIXED,
             noise=gfk.GFK_NOISE_GAUSSIAN):
    rows = [replica_energies(state, dt, t_total, n_walkers, replicas, seed, prec, noise=noise)
            for dt in dts]
    e0, err, slope = analysis.dt_extrapolate([r["dt"] for r in rows], [r["E"] for r in rows],
                                             [r["E_err"] for r in rows])
    return {"rows": rows, "E_dt0": e0, "E_dt0_err": err, "slope": slope, "exact": EXACT[state]}


def paired_bias(state, dt, t_total, n_walkers, replicas, seed=0):
    """Mixed minus FP64 energy on the same walkers and noise: per replica the
    difference of the second-half time averages of E(t); mean and standard error."""
    a = replica_energies(state, dt, t_total, n_walkers, replicas, seed, gfk.GFK_PREC_MIXED)
    b = replica_energies(state, dt, t_total, n_walkers, replicas, seed, gfk.GFK_PREC_FP64)
    return {"mixed": a, "fp64": b}


def replica_series(state, dt, t_total, n_walkers, replicas, seed, prec,
                   noise=gfk.GFK_NOISE_GAUSSIAN):
    kind, params = workloads.trial_for_state(state)
    descs = [gfk.InstanceDesc(n_walkers=n_walkers, dt=dt, e_trial=workloads.E_T[state],
                              seed=seed, state=state, prec=prec, rng_stream=100 + r, noise=noise)
             for r in range(replicas)]
    with gfk.Context(descs, trials=[(kind, params)] * replicas) as ctx:
        ctx.propagate(int(round(t_total / dt)))
        return np.array([ctx.energy(r)["E"] for r in range(replicas)])


def paired_difference(state, dt, t_total, n_walkers, replicas, seed=0,
                      noise=gfk.GFK_NOISE_GAUSSIAN):
    """Per replica the second-half time average of E_mixed(t) - E_fp64(t) on the same
    walkers and noise; mean and standard error over replicas."""
    em = replica_series(state, dt, t_total, n_walkers, replicas, seed, gfk.GFK_PREC_MIXED, noise)
    ef = replica_series(state, dt, t_total, n_walkers, replicas, seed, gfk.GFK_PREC_FP64, noise)
    d = em - ef
    per = d[:, d.shape[1] // 2:].mean(axis=1)
    return {"state": state, "dt": dt, "t": t_total, "walkers": n_walkers, "replicas": replicas,
            "noise": noise, "bias": float(per.mean()), "bias_err": float(per.std(ddof=1) / np.sqrt(replicas)),
            "max_abs_step_difference": float(np.abs(d).max())}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--state", type=int, default=0)
    ap.add_argument("--walkers", type=int, default=1 << 16)
    ap.add_argument("--replicas", type=int, default=16)
    ap.add_argument("--t", type=float, default=20.0)
    ap.add_argument("--dts", type=float, nargs="+", default=[0.01, 0.005, 0.0025])
    ap.add_argument("--prec", type=int, default=1)
    ap.add_argument("--noise", type=int, default=0, help="0 Gaussian, 1 Bernoulli (+-1)")
    a = ap.parse_args()
    print(json.dumps(dt_study(a.state, a.dts, a.t, a.walkers, a.replicas, prec=a.prec,
                              noise=a.noise)))


if __name__ == "__main__":
    main()
