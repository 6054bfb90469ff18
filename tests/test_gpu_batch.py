"""Batches of heterogeneous systems (one CUDA graph per step) against the
same systems stepped one by one: the walkers, traces and move counts agree
bit for bit, across graph re-captures (precision change, grid sizes) and
after the autotuner has chosen the grids."""
import numpy as np
import pytest

import lrdmc_synth as S

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1909_01589_gb300 import build

    build.build()
    import paper_1909_01589_gb300 as p

    p.load_library()
    return p


CASES = [  # name, walkers, a, spacing, tau, e_trial
    ("He", 300, 0.2, "single", 0.05, -2.9),
    ("Ne", 512, 0.2, "this_work", 0.02, -128.9),
    ("H2O", 384, 0.1, "previous", 0.01, -76.0),
    ("Ar", 130, 1 / 63, "this_work", 2e-4, -527.0),
]


def _spacing(pkg, kind):
    return pkg.Spacing({"single": pkg.SINGLE, "this_work": pkg.THIS_WORK, "previous": pkg.PREVIOUS}[kind])


def _make(pkg, seed0):
    out = []
    for q, (name, W, a, kind, tau, et) in enumerate(CASES):
        system = S.make_system(name)
        g = pkg.LrdmcSystem(system)
        g.init_walkers(torch.tensor(S.initial_positions(system, W, seed0 + q), device="cuda"), seed=seed0 + 10 * q,
                       tau=tau, e_trial=et, recompute_every=3, trace_capacity=128)
        out.append(g)
    return out


def _state(g):
    w = g.walkers()
    e, wb, j = g.energy_trace()
    return w["x"], w["EL"], w["parent"], e, wb, g.moves()


def _equal(s1, s2):
    return all(np.array_equal(a, b) for a, b in zip(s1[:5], s2[:5])) and s1[5] == s2[5]


def test_batched_steps_equal_single_steps(pkg):
    a = [c[2] for c in CASES]
    sp = [_spacing(pkg, c[3]) for c in CASES]
    solo = _make(pkg, 100)
    for g, ai, s in zip(solo, a, sp):
        g.step(7, ai, s)
        g.sync()
    batched = _make(pkg, 100)
    batch = pkg.LrdmcBatch(batched, a, sp)
    batch.step(3)   # odd: the next call starts from the other buffer parity
    batch.set_groups([2, 0, 1, 0])  # grouping changes the schedule, not the results
    batch.step(4)
    batch.sync()
    for g1, g2 in zip(solo, batched):
        assert _equal(_state(g1), _state(g2))
    # a precision change and new grid sizes force re-captures; a single step
    # of one system in between is ordered with the batch
    for g in solo + batched:
        g.set_precision(pkg.PRECISION_FP64)
    for g, b in zip(batched, (7, 3, 11, 2)):
        g.set_interval_blocks(b)
    for g, ai, s in zip(solo, a, sp):
        g.step(2, ai, s)
    batched[1].step(1, a[1], sp[1])
    batch.step(1)
    for q, g in enumerate(batched):
        if q != 1:
            g.step(1, a[q], sp[q])
    batch.sync()
    for g1, g2 in zip(solo, batched):
        assert _equal(_state(g1), _state(g2))


def test_tuned_batch_keeps_results(pkg):
    from paper_1909_01589_gb300 import batch as B

    a = [c[2] for c in CASES]
    sp = [_spacing(pkg, c[3]) for c in CASES]
    batched = _make(pkg, 200)
    batch = pkg.LrdmcBatch(batched, a, sp)
    report = B.tune(batch, a, sp, trial_steps=2)
    assert report["choice"]["ms_per_step"] > 0 and len(report["candidates"]) >= 2
    steps_done = [g.energy_trace()[0].shape[0] for g in batched]
    batch.step(3)
    batch.sync()
    solo = _make(pkg, 200)
    for g, ai, s, n in zip(solo, a, sp, steps_done):
        g.step(n + 3, ai, s)
        g.sync()
    for g1, g2 in zip(solo, batched):
        assert _equal(_state(g1), _state(g2))


def test_batch_errors(pkg):
    a = [c[2] for c in CASES[:2]]
    sp = [_spacing(pkg, c[3]) for c in CASES[:2]]
    gs = _make(pkg, 300)[:2]
    batch = pkg.LrdmcBatch(gs, a, sp)
    with pytest.raises(pkg.LrdmcError) as e:
        batch.step(129)  # beyond the trace capacity of 128
    assert e.value.status == pkg.ERR_ARG
    with pytest.raises(pkg.LrdmcError):
        pkg.LrdmcBatch([gs[0], gs[0]], a, sp)  # a system twice


def test_full_size_batch_equals_single_steps(pkg):
    """The batched workload at full size: 8192 walkers each of He, Ne, Ar, Kr
    and H2O at a = 1/(3.5 Z_max) on this work's double grid, tau for about
    10 jumps per walker, two steps in one CUDA graph each. Walkers, traces
    and move counts equal those of the same systems stepped one by one."""
    from paper_1909_01589_gb300 import batch as B

    names = ("He", "Ne", "Ar", "Kr", "H2O")
    e_trial = (-2.90, -128.9, -527.5, -2753.0, -76.0)
    sp = pkg.Spacing(pkg.THIS_WORK)
    systems = [S.make_system(nm) for nm in names]
    a = [1.0 / (3.5 * float(np.max(s.Z))) for s in systems]
    taus = [B.tau_for(pkg, s, ai, sp, 10.0, S.initial_positions(s, 256, 500 + q), S.random_rotations(256, 600 + q))
            for q, (s, ai) in enumerate(zip(systems, a))]

    def make():
        gs = []
        for q, (s, tau) in enumerate(zip(systems, taus)):
            g = pkg.LrdmcSystem(s)
            g.init_walkers(torch.tensor(S.initial_positions(s, 8192, 700 + q), device="cuda"), seed=800 + q,
                           tau=tau, e_trial=e_trial[q], recompute_every=5, trace_capacity=8)
            gs.append(g)
        return gs

    solo = make()
    for g, ai in zip(solo, a):
        g.step(2, ai, sp)
        g.sync()
    batched = make()
    batch = pkg.LrdmcBatch(batched, a, [sp] * len(batched))
    batch.step(2)
    batch.sync()
    for g1, g2 in zip(solo, batched):
        assert _equal(_state(g1), _state(g2))


@pytest.mark.parametrize("pipelined", [False, True])
def test_batch_matches_oracle(pkg, oracle_mod, pipelined):
    """A batch of four systems of uneven size (He, Ne, H2O, Ar: N = 2 to 18;
    single grid, this work's and the previous double grid), stepped one
    interval per CUDA graph, against each system's own oracle population
    walker by walker after every interval: jump counts, log-weights, comb
    parents, positions and local energies at the parity tolerance, then the
    traces. A parting is accepted only on a near-edge decision of the walker
    or slot that parted."""
    import os

    import _parity_util as U

    cases = [("He", 48, 0.2, "single", 0.05, -2.9), ("Ne", 24, 0.2, "this_work", 0.02, -128.9),
             ("H2O", 16, 0.1, "previous", 0.01, -76.0), ("Ar", 8, 1 / 63, "this_work", 2e-4, -527.0)]
    okind = {"single": oracle_mod.SINGLE, "this_work": oracle_mod.THIS_WORK, "previous": oracle_mod.PREVIOUS}
    threads = max(1, min(16, os.cpu_count() or 1))
    gs, pops, lats, systems = [], [], [], []
    for q, (name, W, a, kind, tau, et) in enumerate(cases):
        system = S.make_system(name)
        x0 = S.initial_positions(system, W, 900 + q)
        g = pkg.LrdmcSystem(system)
        g.init_walkers(torch.tensor(x0, device="cuda"), seed=950 + q, tau=tau, e_trial=et, recompute_every=3,
                       trace_capacity=8)
        o = oracle_mod.OracleSystem(system)
        pops.append(oracle_mod.OraclePopulation(o, x0, seed=950 + q, tau=tau, e_trial=et, recompute_every=3))
        lats.append(oracle_mod.lattice_for(system, a, okind[kind]))
        gs.append(g)
        systems.append((system, o))
    batch = pkg.LrdmcBatch(gs, [c[2] for c in cases], [_spacing(pkg, c[3]) for c in cases])
    if pipelined:
        batch.set_groups([3, 2, 1, 0])
        batch.set_pipelined(True)
    tag = "pipelined " if pipelined else ""
    entries = [{"test": f"{tag}batch vs oracle: {c[0]} {c[3]} (W={c[1]})", "kind": "projection (batched)",
                "walkers": c[1], "intervals_requested": 4, "intervals_compared": 0, "parted": False} for c in cases]
    live = [True] * len(cases)
    try:
        for k in range(4):
            batch.step(1)
            batch.sync()
            for q in range(len(cases)):
                pops[q].step(lats[q], 1, threads)
                if not live[q]:
                    continue
                info = U.compare_interval(systems[q][0], gs[q].walkers(), pops[q].walkers(lats[q].G),
                                          pops[q].margins(teeth=True))
                U.merge_worst(entries[q], info)
                if not info["ok"]:
                    entries[q].update(parted=True, parted_at=k, excused=info["excused"])
                    assert info["excused"], (cases[q][0], k, info["parted_walkers"][:8], info["parted_teeth"][:8])
                    live[q] = False
                    continue
                entries[q]["intervals_compared"] = k + 1
        for q in range(len(cases)):
            if live[q]:
                ge = gs[q].energy_trace()[0]
                oe = pops[q].trace()[0]
                assert np.all(np.abs(ge - oe) <= U.RTOL * np.abs(oe)), cases[q][0]
                assert gs[q].moves() == pops[q].moves
        assert sum(live) >= 3
    finally:
        for e in entries:
            U.record(e)


def test_pipelined_batch_equals_single_steps(pkg):
    """The pipelined schedule (interval kernels chained with programmatic
    dependent launches, each starting in the previous one's tail) gives the
    single steps' results bit for bit, heaviest first and lightest first,
    across a switch from and back to the fork/join schedule."""
    a = [c[2] for c in CASES]
    sp = [_spacing(pkg, c[3]) for c in CASES]
    solo = _make(pkg, 400)
    for g, ai, s in zip(solo, a, sp):
        g.step(6, ai, s)
        g.sync()
    batched = _make(pkg, 400)
    batch = pkg.LrdmcBatch(batched, a, sp)
    batch.set_groups([3, 2, 1, 0])
    batch.set_pipelined(True)
    batch.step(2)
    batch.set_groups([0, 1, 2, 3])
    batch.step(1)
    batch.set_pipelined(False)
    batch.step(1)
    batch.set_pipelined(True)
    batch.step(2)
    batch.sync()
    for g1, g2 in zip(solo, batched):
        assert _equal(_state(g1), _state(g2))
