"""Batched projection of several systems and the autotuner of their grids.

A batch (``LrdmcBatch``, lrdmc_batch_create) runs one CUDA graph per step
whose parallel branches are every system's interval and reconfiguration
kernels. Each interval kernel is a persistent grid whose warps fetch
walkers through an atomic counter, so the grid size decides how much of
the GPU a system holds while the branches run together; it never changes
results. ``tune`` chooses the grid sizes by measurement:

1. every system alone at its occupancy-default grid gives its GPU time per
   step, w_i;
2. candidate plans: every system concurrent with its default grid, or
   with grids proportional to w_i (so that the branches finish together)
   at several oversubscription factors; every system in turn on the whole
   GPU; the same order pipelined (programmatic dependent launches: each
   system's kernel starts on the SMs the previous one frees in its tail);
   the heaviest system alone, then the rest concurrently;
3. each plan is timed over a few batched steps with CUDA events on the
   batch stream, and the fastest is kept.

The tuning steps are real projection steps of the populations (they count
as equilibration).
"""
from __future__ import annotations

import math

import numpy as np

WARPS_PER_BLOCK = 4


def candidate_grids(defaults, work, need, factors=(1.0, 1.5, 2.0)):
    """Candidate persistent-grid sizes for systems sharing one GPU at once.

    defaults[i]: occupancy-default blocks of system i (the whole GPU);
    work[i]: GPU time per step of system i alone on its default grid;
    need[i]: blocks that give every walker its own warp.
    Returns [(name, [blocks_i])] with 1 <= blocks_i <= min(defaults_i, need_i):
    the defaults, then shares proportional to work (so that concurrent
    branches finish together) at several oversubscription factors."""
    n = len(defaults)
    cap = [max(1, min(int(d), int(m))) for d, m in zip(defaults, need)]
    total = float(sum(work))
    out = [("default", list(cap))]
    if n == 1 or total <= 0.0:
        return out
    share = [w / total for w in work]
    for f in factors:
        out.append((f"proportional x{f:g}",
                    [max(1, min(c, int(math.ceil(f * s * d)))) for c, s, d in zip(cap, share, defaults)]))
    seen, uniq = set(), []
    for name, b in out:
        key = tuple(b)
        if key not in seen:
            seen.add(key)
            uniq.append((name, b))
    return uniq


def candidate_plans(defaults, work, need):
    """Execution plans [(name, groups, blocks, carveout, pipelined)]: every
    system concurrent (with each candidate grid, under the default and
    under the maximal shared-memory carveout), every system in turn on the
    whole GPU (heaviest first), the same order pipelined (each system's
    interval kernel starting while the previous one drains, heaviest first
    and lightest first), and the heaviest alone followed by the rest
    concurrently (grids proportional to the rest's work)."""
    n = len(defaults)
    cap = [max(1, min(int(d), int(m))) for d, m in zip(defaults, need)]
    grids = candidate_grids(defaults, work, need)
    plans = [("concurrent " + name, [0] * n, b, -1, 0) for name, b in grids]
    plans += [("concurrent " + name + ", max shared carveout", [0] * n, b, 100, 0) for name, b in grids]
    if n == 1:
        return plans
    by_work = sorted(range(n), key=lambda i: -work[i])
    serial = [0] * n
    for rank, i in enumerate(by_work):
        serial[i] = rank
    plans.append(("serial", serial, list(cap), -1, 0))
    plans.append(("pipelined, heaviest first", serial, list(cap), -1, 1))
    plans.append(("pipelined, heaviest first, max shared carveout", serial, list(cap), 100, 1))
    plans.append(("pipelined, lightest first", [n - 1 - r for r in serial], list(cap), -1, 1))
    heavy = by_work[0]
    rest = [i for i in range(n) if i != heavy]
    rest_grids = candidate_grids([defaults[i] for i in rest], [work[i] for i in rest], [need[i] for i in rest],
                                 factors=(1.5,))
    for name, b in rest_grids:
        blocks = list(cap)
        for i, bi in zip(rest, b):
            blocks[i] = bi
        split = [0 if i == heavy else 1 for i in range(n)]
        plans.append((f"heaviest alone, rest concurrent {name}", split, blocks, -1, 0))
        plans.append((f"heaviest alone, rest concurrent {name}, max shared carveout", split, blocks, 100, 0))
    return plans


def choose(timings):
    """The fastest plan; timings = [(name, groups, blocks, carveout, pipelined, ms)]."""
    return min(timings, key=lambda t: t[-1])


def _time_system_steps(torch, g, n, a, spacing):
    stream = g.stream
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    g.step(n, a, spacing)
    e1.record(stream)
    g.sync()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / n


def _time_batch_steps(torch, batch, n):
    stream = torch.cuda.ExternalStream(batch.stream_ptr)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    batch.step(n)
    e1.record(stream)
    batch.sync()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / n


def tune(batch, a, spacing, trial_steps=3):
    """Measure, pick and set the grid sizes of a batch's systems. Returns a
    report: per-system alone times, every candidate's time per batched step,
    and the choice."""
    import torch

    systems = batch.systems
    defaults, need, work = [], [], []
    for g, ai, sp in zip(systems, a, spacing):
        g.set_interval_blocks(0)
        _, d = g.interval_blocks()
        defaults.append(d)
        need.append(int(math.ceil(g.W / WARPS_PER_BLOCK)))
        g.step(1, ai, sp)  # first evaluation outside the timing
        work.append(_time_system_steps(torch, g, trial_steps, ai, sp))
    timings = []
    for name, groups, blocks, carve, pipe in candidate_plans(defaults, work, need):
        batch.set_groups(groups)
        batch.set_carveout(carve)
        batch.set_pipelined(pipe)
        for g, b in zip(systems, blocks):
            g.set_interval_blocks(b)
        batch.step(1)  # capture the graphs of this plan
        batch.step(1)
        batch.sync()
        timings.append((name, groups, blocks, carve, pipe, _time_batch_steps(torch, batch, trial_steps)))
    name, groups, blocks, carve, pipe, ms = choose(timings)
    batch.set_groups(groups)
    batch.set_carveout(carve)
    batch.set_pipelined(pipe)
    for g, b in zip(systems, blocks):
        g.set_interval_blocks(b)
    return {"alone_ms_per_step": work, "sum_alone_ms": float(np.sum(work)), "defaults": defaults,
            "candidates": [{"name": n, "groups": gr, "blocks": b, "carveout": c, "pipelined": pp, "ms_per_step": t}
                           for n, gr, b, c, pp, t in timings],
            "choice": {"name": name, "groups": groups, "blocks": blocks, "carveout": carve, "pipelined": pipe,
                       "ms_per_step": ms}}


def tau_for(pkg, system, a, spacing, jumps, x, rot):
    """Interval length giving about ``jumps`` jumps per walker: jumps / <b>
    with <b> the mean total rate of the configurations x (rotations rot),
    from one stateless evaluation."""
    import torch

    g = pkg.LrdmcSystem(system)
    _, _, b, _ = g.evaluate(torch.as_tensor(x, device="cuda"), torch.as_tensor(rot, device="cuda"), a, spacing)
    return float(jumps / torch.mean(b).item())
