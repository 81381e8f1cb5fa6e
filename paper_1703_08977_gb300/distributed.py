"""Several GPUs: one population sharded by walker id, merged per step.

The walk has no interaction between walkers, so ranks advance disjoint id
ranges of one population (InstanceDesc.walker_id0 = first id of the shard)
with no communication.  The only exchange is the space average itself: each
rank's per-step sums {c, W, P, Q, R, n} (W = sum e^{logw - c}, ...) are merged
with one all-reduce of the shifts (max) and one of the rescaled sums (sum).
The merged rows equal the single-population rows up to rounding order.
"""
from __future__ import annotations

import numpy as np
import torch
import torch.distributed as dist


def shard(n_walkers: int, world: int, rank: int):
    """(walker_id0, n_local) of rank's contiguous share of n_walkers ids."""
    base, extra = divmod(int(n_walkers), int(world))
    n_local = base + (1 if rank < extra else 0)
    id0 = rank * base + min(rank, extra)
    return id0, n_local


def merge_sums(rows, group=None, device=None):
    """Merge every rank's per-step sums (array (S+1, 6): c, W, P, Q, R, n) over the
    process group; returns the merged (S+1, 6) float64 numpy array on every rank."""
    dev = device or ("cuda" if dist.get_backend(group) == "nccl" else "cpu")
    t = torch.as_tensor(np.asarray(rows, dtype=np.float64), device=dev)
    c, W, P, Q, R, n = t.unbind(1)
    live = n > 0
    cmax = torch.where(live, c, torch.full_like(c, -float("inf")))
    dist.all_reduce(cmax, op=dist.ReduceOp.MAX, group=group)
    C = torch.where(torch.isfinite(cmax), cmax, torch.zeros_like(cmax))
    f = torch.where(live, torch.exp(c - C), torch.zeros_like(c))
    q = torch.stack([W * f, P * f, Q * f * f, R * f, n], dim=1)
    dist.all_reduce(q, op=dist.ReduceOp.SUM, group=group)
    return torch.cat([C[:, None], q], dim=1).cpu().numpy()


def estimators(rows, n_walkers_total):
    """E(t) = P/W, ln z(t) = c + ln W - ln N, ESS = W^2/Q from (merged) sums."""
    r = np.asarray(rows)
    c, W, P, Q, R, n = r.T
    with np.errstate(divide="ignore", invalid="ignore"):
        return {"E": P / W, "ln_z": c + np.log(W) - np.log(n_walkers_total), "ess": W * W / Q,
                "var": R / W - (P / W) ** 2, "n_alive": n}
