"""Host-side statistics of LRDMC energy traces and replica combination.

These read the per-interval trace that lrdmc_get_energy_trace returns
(e_k = weighted mean local energy, wbar_k = mean weight) and do no GPU work.

* ``energy_estimate``: the population-control-corrected estimator of the
  fixed-population (reconfiguration) method: e_k weighted by the product of
  the last L mean weights.
* ``reblock``: error of the mean of a correlated series by the blocking
  method of Flyvbjerg and Petersen, J. Chem. Phys. 91, 461 (1989).
* ``efficiency``: DMC efficiency 1 / (sigma^2 t) from the error of the mean
  and the wall time that produced it.
* ``combine_replicas`` / ``gather_and_combine``: independent replicas (one
  population per GPU, no data-path collective) are combined on the host by
  weighting each replica's estimate with its inverse variance;
  ``gather_and_combine`` exchanges the per-replica estimates through
  torch.distributed (any backend).
"""
from __future__ import annotations

import math

import numpy as np


def energy_estimate(e, wbar, L=0):
    """Mixed estimator sum_k G_k e_k / sum_k G_k, G_k = prod_{l<L} wbar_{k-l}
    (L = 0: the plain mean of e_k)."""
    e = np.asarray(e, dtype=np.float64)
    if L <= 0:
        return float(np.mean(e))
    lw = np.log(np.asarray(wbar, dtype=np.float64))
    c = np.concatenate([[0.0], np.cumsum(lw)])
    k = np.arange(len(e))
    lo = np.maximum(k - L + 1, 0)
    G = np.exp(c[k + 1] - c[lo])
    return float(np.sum(G * e) / np.sum(G))


def reblock(e, min_blocks=16):
    """(error of the mean, block levels) by repeated pairwise blocking; the
    error is the largest one over levels with at least ``min_blocks`` blocks
    (the plateau for a well-converged run)."""
    x = np.asarray(e, dtype=np.float64).copy()
    if len(x) < 2:
        return 0.0, []
    levels = []
    while len(x) >= min_blocks:
        err = float(np.std(x, ddof=1) / math.sqrt(len(x)))
        levels.append(err)
        n = len(x) // 2 * 2
        x = 0.5 * (x[0:n:2] + x[1:n:2])
    return (max(levels) if levels else float(np.std(x, ddof=1) / math.sqrt(len(x)))), levels


def efficiency(e, seconds):
    """1 / (sigma^2 t): sigma the reblocked error of the mean of e, t the
    time that produced the series."""
    err, _ = reblock(e)
    if err <= 0.0 or seconds <= 0.0:
        return float("inf")
    return 1.0 / (err * err * seconds)


def combine_replicas(estimates, errors):
    """Inverse-variance weighted mean of independent replica estimates and
    its error."""
    est = np.asarray(estimates, dtype=np.float64)
    err = np.asarray(errors, dtype=np.float64)
    if np.any(err <= 0):
        return float(np.mean(est)), float(np.std(est, ddof=1) / math.sqrt(len(est))) if len(est) > 1 else 0.0
    w = 1.0 / (err * err)
    return float(np.sum(w * est) / np.sum(w)), float(1.0 / math.sqrt(np.sum(w)))


def gather_and_combine(e, wbar, L=0, group=None):
    """Every rank passes its own trace; all ranks return the combined
    (estimate, error) over the replicas, exchanged with torch.distributed."""
    import torch
    import torch.distributed as dist

    est = energy_estimate(e, wbar, L)
    err, _ = reblock(e)
    mine = torch.tensor([est, err], dtype=torch.float64)
    world = dist.get_world_size(group)
    parts = [torch.zeros(2, dtype=torch.float64) for _ in range(world)]
    dist.all_gather(parts, mine, group=group)
    allv = torch.stack(parts).numpy()
    return combine_replicas(allv[:, 0], allv[:, 1])


def reduce_throughput(local_ms, local_moves, group=None):
    """Whole-job throughput of replicas: total moves of all ranks over the
    slowest rank's time (max over ranks), exchanged with torch.distributed."""
    import torch
    import torch.distributed as dist

    t = torch.tensor([float(local_ms), float(local_moves)], dtype=torch.float64)
    world = dist.get_world_size(group)
    parts = [torch.zeros(2, dtype=torch.float64) for _ in range(world)]
    dist.all_gather(parts, t, group=group)
    allv = torch.stack(parts).numpy()
    total_ms = float(allv[:, 0].max())
    moves = float(allv[:, 1].sum())
    return moves / (total_ms * 1e-3), total_ms, moves
