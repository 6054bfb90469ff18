"""Pins of the oracle's projection (continuous-time lattice Green's function
Monte Carlo with fixed node and reconfiguration)."""
import numpy as np
import pytest

import lrdmc_synth as S


def _run(oracle_mod, system, lat_kw, W=64, steps=30, tau=0.02, seed=3, threads=4, e_trial=0.0):
    o = oracle_mod.OracleSystem(system)
    x = S.initial_positions(system, W, seed)
    pop = oracle_mod.OraclePopulation(o, x, seed=seed, tau=tau, e_trial=e_trial, recompute_every=4)
    lat = oracle_mod.lattice_for(system, **lat_kw)
    pop.step(lat, steps, threads)
    return pop, lat


ZERO_VAR = [
    ("H", dict(a=0.3, kind=0), -0.5),
    ("H", dict(a=0.3, kind=3, rc=0.5, aprime_over_a=1.5), -0.5),
    ("H", dict(a=0.3, kind=2), -0.5),
    ("Be_bare", dict(a=0.2, kind=0), -20.0),
    ("Be_bare", dict(a=0.1, kind=3, rc=0.3, aprime_over_a=2.0), -20.0),
]


@pytest.mark.parametrize("name,lat,E", ZERO_VAR)
def test_zero_variance_exact_trial(oracle_mod, name, lat, E):
    """With the exact ground state (H 1s) or an exact fixed-node state
    (four free electrons in 1s/2s of Z = 4, with nodes) the regularized
    local energy is constant, so every interval's energy equals E exactly and
    the population weights never change (zero variance at every a, single or
    double grid, Pade or Gaussian p)."""
    pop, _ = _run(oracle_mod, S.make_system(name), lat, tau=0.05)
    e, wbar, jumps = pop.trace()
    assert len(e) == 30
    assert np.max(np.abs(e - E)) < 1e-11 * abs(E)
    assert np.mean(jumps) > 0.5
    assert pop.moves > 0


def test_hydrogen_fixed_node_energy(oracle_mod):
    """Nodeless H with a non-exact trial function exp(-0.8 r) (cusp completed
    by the e-n factor) projects to the exact -0.5 Ha up to the O(a^2) lattice
    error; its variational energy is far higher."""
    s = S.hydrogen(0.8)
    s.en_b1 = np.array([0.2])
    pop, _ = _run(oracle_mod, s, dict(a=0.2, kind=0), W=256, steps=1200, tau=0.05, e_trial=-0.5, threads=8)
    e, wbar, _ = pop.trace()
    e = e[200:]
    # plain mean of the interval energies; its standard error from the
    # spread of 20 consecutive batch means (batches much longer than the
    # correlation time of the trace)
    E = float(np.mean(e))
    batches = np.array([np.mean(b) for b in np.array_split(e, 20)])
    err = float(np.std(batches, ddof=1) / np.sqrt(len(batches)))
    assert abs(E + 0.5) < 4 * err + 2e-3
    # the trial function alone: mean local energy at the start is much higher
    o = oracle_mod.OracleSystem(s)
    x = S.initial_positions(s, 2000, 1)
    evmc = np.mean([o.local_energy(x[w]) for w in range(2000)])
    assert evmc > -0.49


def test_determinism_and_split_steps(oracle_mod):
    """Counter-based randomness: 3 + 2 steps equal 5 steps bit for bit, and
    the thread count does not change any result."""
    s = S.neon()
    lat = dict(a=0.2, kind=1)
    p1, _ = _run(oracle_mod, s, lat, W=16, steps=5, threads=1)
    o = oracle_mod.OracleSystem(s)
    x = S.initial_positions(s, 16, 3)
    p2 = oracle_mod.OraclePopulation(o, x, seed=3, tau=0.02, e_trial=0.0, recompute_every=4)
    L = oracle_mod.lattice_for(s, **lat)
    p2.step(L, 3, 4)
    p2.step(L, 2, 2)
    a, b = p1.walkers(2), p2.walkers(2)
    assert np.array_equal(a["x"], b["x"]) and np.array_equal(a["EL"], b["EL"])
    assert np.array_equal(p1.trace()[0], p2.trace()[0])


def test_jump_rate_matches_total_rate(oracle_mod):
    """The waiting time at x is exponential with rate b_x, so the mean
    number of jumps per interval is about tau times the mean of b."""
    s = S.helium()
    pop, lat = _run(oracle_mod, s, dict(a=0.2, kind=0), W=256, steps=200, tau=0.02)
    e, w, jumps = pop.trace()
    wk = pop.walkers(1)
    assert abs(np.mean(jumps[50:]) / (0.02 * np.mean(wk["b"])) - 1) < 0.1


def test_reconfiguration_resets_and_copies(oracle_mod):
    """After an interval every slot holds a copy of a parent chosen by the
    comb from the end-of-interval weights; the trace's e_k is the weighted
    mean of the parents' local energies."""
    s = S.helium()
    o = oracle_mod.OracleSystem(s)
    W = 32
    x = S.initial_positions(s, W, 4)
    pop = oracle_mod.OraclePopulation(o, x, seed=4, tau=0.02, e_trial=-2.9, recompute_every=0)
    L = oracle_mod.lattice_for(s, a=0.2, kind=0)
    pop.step(L, 1, 1)
    before = pop.walkers(1)
    pop.step(L, 1, 1)
    after = pop.walkers(1)
    parent = after["parent"]
    assert np.all(np.diff(parent) >= 0)
    w = np.exp(after["logw_pre"])
    counts = np.bincount(parent, minlength=W)
    assert np.all(np.abs(counts - W * w / w.sum()) < 1.0 + 1e-12)
    e, wbar, _ = pop.trace()
    assert abs(wbar[-1] - w.mean()) < 1e-14 * w.mean()
    del before


def test_decision_margins_per_walker_and_tooth(oracle_mod):
    """The margins the GPU parity tests use to excuse a parting: every
    walker's margin is finite and positive after an interval with jumps, and
    the comb's per-tooth margins have the comb's overall margin as their
    minimum; each tooth's margin is the distance of its target from the
    nearer edge of its parent's bin (checked by recomputing the comb from
    the logged weights)."""
    s = S.helium()
    pop, _ = _run(oracle_mod, s, dict(a=0.2, kind=1), W=64, steps=1, tau=0.05, e_trial=-2.9)
    mw, mc, mt = pop.margins(teeth=True)
    assert np.all(np.isfinite(mw)) and np.all(mw > 0)
    assert mt.min() == mc
    wt = np.exp(pop.walkers(2)["logw_pre"])
    parent = pop.walkers(2)["parent"]
    C = np.cumsum(wt)
    u = oracle_mod.uniform(int(oracle_mod.philox4x64([2 ** 64 - 1, 0, 0, 2], [3, 0])[0]))
    for t in range(64):
        target = (t + u) * C[-1] / 64
        q = parent[t]
        lo = C[q - 1] if q > 0 else -np.inf
        assert lo <= target < C[q] or q == 63
        edge = min(abs(target - C[q]), abs(target - lo) if q > 0 else np.inf) / C[-1]
        assert abs(edge - mt[t]) <= 1e-12
