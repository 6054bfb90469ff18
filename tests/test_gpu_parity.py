"""GPU-vs-oracle parity of the CUDA path, through the C ABI.

Bar (FP64): lattice-move ratios, rates, total rates and local energies
within 1e-10 relative (ratios: relative to the magnitude of the terms of
their determinant dot product, at least max(1, |ratio|); see
_parity_util.ratio_scale; the local energies of projected walkers, which
can sit close to a heavy nucleus: relative to the magnitude of their
kinetic and Coulomb terms, see _parity_util.el_scale); positions,
log-weights and trace energies within 1e-10; rates element by element
within 1e-10 of their own scale (weight and spacing factor times the scale
of their ratio); jump counts, comb parents and move choices identical,
except where the oracle reports that the decision of the walker or comb
slot that parted lay within 1e-10 of a bin edge (then the trajectories may
part and the comparison stops). Every run's intervals compared, decisions,
near-edge decisions, partings and worst errors - plainly relative to
|value| as well as against the term scale - go to the parity report
(conftest.py writes it at the end of the session).
"""
import os

import numpy as np
import pytest

import lrdmc_synth as S
import _parity_util as U
from _parity_util import EDGE, RTOL, el_scale, rate_tolerance, ratio_scale

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
THREADS = max(1, min(16, os.cpu_count() or 1))


@pytest.fixture(scope="module")
def pkg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1909_01589_gb300 import build

    build.build()
    import paper_1909_01589_gb300 as p

    p.load_library()
    return p


def spacing_pair(pkg, oracle_mod, system, a, kind, rc=0.5, ratio=1.5):
    if kind == "single":
        return pkg.Spacing(pkg.SINGLE), oracle_mod.lattice_for(system, a, oracle_mod.SINGLE)
    if kind == "this_work":
        return pkg.Spacing(pkg.THIS_WORK), oracle_mod.lattice_for(system, a, oracle_mod.THIS_WORK)
    if kind == "previous":
        return pkg.Spacing(pkg.PREVIOUS), oracle_mod.lattice_for(system, a, oracle_mod.PREVIOUS)
    return (pkg.Spacing(pkg.EXPLICIT, rc=rc, aprime_over_a=ratio),
            oracle_mod.lattice_for(system, a, oracle_mod.EXPLICIT, rc=rc, aprime_over_a=ratio))


EVAL_CASES = [
    ("He", "single", 0.2), ("He", "this_work", 0.2), ("Ne", "single", 0.1), ("Ne", "this_work", 0.2),
    ("Ne", "previous", 0.4), ("tiny_mixed", "explicit", 0.3), ("Be_bare", "explicit", 0.25),
    ("H", "this_work", 0.3), ("Ar", "this_work", 1 / 63), ("Kr", "this_work", 1 / 126),
    ("Kr", "single", 0.05), ("H2O", "this_work", 0.1),
]


PRECISIONS = ["fp64", "df64"]


def _check_rates(c, T, ref, tsc, scale):
    """Every rate of configuration c within its tolerance (rate_tolerance);
    on failure, the worst move with its weight, ratio and scales."""
    err = np.abs(T - ref["T"])
    bad = err > tsc
    if np.any(bad):
        j = int(np.argmax(np.where(bad, err / np.maximum(tsc, 1e-300), 0.0)))
        raise AssertionError(f"config {c} move {j} (grid {(j // 6) % 2}): T {T[j]!r} vs {ref['T'][j]!r}, "
                             f"w {ref['w'][j]!r}, ratio {ref['ratio'][j]!r}, ratio scale {scale[j]!r}, "
                             f"rate tolerance {tsc[j]!r}, {int(np.sum(bad))} moves off")


def _w_abs(prec):
    return U.W_ABS if prec != "fp64" else 0.0


class _EvalWorst:
    """Worst errors of an evaluation case: plainly relative to |value| (the
    plain 1e-10 relative bar, shown as measured) and against the floating-point
    scale the assertions use; with the count of elements whose plain
    relative error exceeds 1e-10."""

    def __init__(self):
        self.d = {"worst_ratio_rel": 0.0, "worst_ratio_scaled": 0.0, "worst_T_rel": 0.0, "worst_T_scaled": 0.0,
                  "worst_b_rel": 0.0, "worst_EL_rel": 0.0, "ratios_above_1e-10_rel": 0, "ratios": 0}

    def add(self, r, rr, rs, t, tr, ts, b, br, e, er):
        d = self.d
        rel = np.abs(r - rr) / np.maximum(np.abs(rr), 1e-300)
        nz = rr != 0
        d["worst_ratio_rel"] = max(d["worst_ratio_rel"], float(np.max(rel[nz])) if np.any(nz) else 0.0)
        d["ratios_above_1e-10_rel"] += int(np.sum(rel[nz] > 1e-10))
        d["ratios"] += int(np.sum(nz))
        d["worst_ratio_scaled"] = max(d["worst_ratio_scaled"], float(np.max(np.abs(r - rr) / rs)))
        pos = tr > 0
        if np.any(pos):
            d["worst_T_rel"] = max(d["worst_T_rel"], float(np.max(np.abs(t[pos] - tr[pos]) / tr[pos])))
        d["worst_T_scaled"] = max(d["worst_T_scaled"], RTOL * float(np.max(np.abs(t - tr) / np.maximum(ts, 1e-300))))
        d["worst_b_rel"] = max(d["worst_b_rel"], abs(b - br) / br)
        d["worst_EL_rel"] = max(d["worst_EL_rel"], abs(e - er) / abs(er))

    def entry(self, label, n):
        return {"test": label, "kind": "evaluation", "configurations": n, **self.d}


def _prec(pkg, name):
    return pkg.PRECISION_FP64 if name == "fp64" else pkg.PRECISION_DF64


@pytest.mark.parametrize("prec", PRECISIONS)
@pytest.mark.parametrize("name,kind,a", EVAL_CASES)
def test_evaluate_matches_oracle(pkg, oracle_mod, name, kind, a, prec):
    """All 6N / 12N ratios, rates, total rate and local energy of 37
    configurations (nine warps of four, a ragged last block), in IEEE double
    and in double-float arithmetic."""
    system = S.make_system(name)
    if name == "H" and kind == "this_work":
        system = S.hydrogen(0.8)
    g = pkg.LrdmcSystem(system).set_precision(_prec(pkg, prec))
    o = oracle_mod.OracleSystem(system)
    n = 37
    x = S.initial_positions(system, n, 101)
    R = S.random_rotations(n, 102)
    sp, lat = spacing_pair(pkg, oracle_mod, system, a, kind)
    ratio, T, b, el = g.evaluate(torch.tensor(x, device="cuda"), torch.tensor(R, device="cuda"), a, sp)
    ratio, T, b, el = (t.cpu().numpy() for t in (ratio, T, b, el))
    worst = _EvalWorst()
    for c in range(n):
        ref = o.lattice_eval(lat, x[c], R[c])
        scale = ratio_scale(o, system, lat, x[c], R[c], ref["ratio"])
        err = np.abs(ratio[c] - ref["ratio"])
        assert np.all(err <= RTOL * scale), (c, np.max(err / scale))
        tsc = rate_tolerance(lat, ref["w"], scale, w_abs=_w_abs(prec))
        _check_rates(c, T[c], ref, tsc, scale)
        assert abs(b[c] - ref["b"]) <= RTOL * ref["b"]
        assert abs(el[c] - ref["EL"]) <= RTOL * max(1.0, abs(ref["EL"]))
        worst.add(ratio[c], ref["ratio"], scale, T[c], ref["T"], tsc, b[c], ref["b"], el[c], ref["EL"])
    U.record(worst.entry(f"evaluate {name} {kind} a={a:.6g} {prec}", n))


@pytest.mark.parametrize("prec", PRECISIONS)
def test_evaluate_full_size_sampled(pkg, oracle_mod, prec):
    """The Ne workload at full size (4096 configurations, double grid with
    the paper's parameters, a = 0.2): 64 sampled configurations against the
    oracle one by one, every total rate positive and finite."""
    system = S.neon()
    g = pkg.LrdmcSystem(system).set_precision(_prec(pkg, prec))
    o = oracle_mod.OracleSystem(system)
    n = 4096
    x = S.initial_positions(system, n, 201)
    R = S.random_rotations(n, 202)
    sp, lat = spacing_pair(pkg, oracle_mod, system, 0.2, "this_work")
    ratio, T, b, el = g.evaluate(torch.tensor(x, device="cuda"), torch.tensor(R, device="cuda"), 0.2, sp)
    ratio, b, el = ratio.cpu().numpy(), b.cpu().numpy(), el.cpu().numpy()
    assert np.all(np.isfinite(el)) and np.all(b > 0)
    T = T.cpu().numpy()
    worst = _EvalWorst()
    for c in np.random.default_rng(3).choice(n, 64, replace=False):
        ref = o.lattice_eval(lat, x[c], R[c])
        scale = ratio_scale(o, system, lat, x[c], R[c], ref["ratio"])
        assert np.all(np.abs(ratio[c] - ref["ratio"]) <= RTOL * scale)
        tsc = rate_tolerance(lat, ref["w"], scale, w_abs=_w_abs(prec))
        _check_rates(c, T[c], ref, tsc, scale)
        assert abs(el[c] - ref["EL"]) <= RTOL * abs(ref["EL"])
        worst.add(ratio[c], ref["ratio"], scale, T[c], ref["T"], tsc, b[c], ref["b"], el[c], ref["EL"])
    U.record(worst.entry(f"evaluate Ne full size (4096, 64 sampled) {prec}", 64))


def _compare_runs(pkg, oracle_mod, system, kind, a, W, n_steps, tau, seed, e_trial, rc_every=3,
                  prec="df64", label=None):
    """Project the same population on the GPU and in the oracle, interval by
    interval, comparing every walker after each one (U.compare_interval).
    A parting is accepted only when every walker or comb slot that parted
    had a decision within EDGE of a bin edge in the oracle; the comparison
    then stops (the trajectories are no longer the same). Returns
    (intervals compared, parted) and records the run in the parity report."""
    g = pkg.LrdmcSystem(system).set_precision(_prec(pkg, prec))
    o = oracle_mod.OracleSystem(system)
    x0 = S.initial_positions(system, W, seed)
    sp, lat = spacing_pair(pkg, oracle_mod, system, a, kind)
    g.init_walkers(torch.tensor(x0, device="cuda"), seed=seed, tau=tau, e_trial=e_trial,
                   recompute_every=rc_every, trace_capacity=n_steps)
    pop = oracle_mod.OraclePopulation(o, x0, seed=seed, tau=tau, e_trial=e_trial, recompute_every=rc_every)
    entry = {"test": label or f"projection {kind} a={a:.6g} W={W} {prec}", "kind": "projection",
             "walkers": W, "intervals_requested": n_steps, "intervals_compared": 0, "parted": False}
    compared = 0
    try:
        for k in range(n_steps):
            g.step(1, a, sp)
            pop.step(lat, 1, THREADS)
            gw, ow = g.walkers(), pop.walkers(lat.G)
            info = U.compare_interval(system, gw, ow, pop.margins(teeth=True))
            U.merge_worst(entry, info)
            if not info["ok"]:
                entry.update(parted=True, parted_at=k, parted_walkers=info["parted_walkers"][:16],
                             parted_teeth=info["parted_teeth"][:16], excused=info["excused"])
                assert info["excused"], (f"interval {k}: walkers {info['parted_walkers'][:8]} / teeth "
                                         f"{info['parted_teeth'][:8]} parted without a near-edge decision")
                return compared, True
            compared += 1
            entry["intervals_compared"] = compared
        ge, gwb, gj = g.energy_trace()
        oe, owb, oj = pop.trace()
        entry["worst_trace_e_rel"] = float(np.max(np.abs(ge - oe) / np.abs(oe)))
        assert np.all(np.abs(ge - oe) <= RTOL * np.abs(oe))
        assert np.all(np.abs(gwb - owb) <= RTOL * owb)
        assert np.array_equal(gj, oj)
        assert g.moves() == pop.moves
        return compared, False
    finally:
        U.record(entry)


@pytest.mark.parametrize("prec", PRECISIONS)
@pytest.mark.parametrize("name,kind,a,W,steps,tau,et", [
    ("He", "single", 0.2, 64, 25, 0.02, -2.9),
    ("He", "this_work", 0.2, 61, 25, 0.02, -2.9),
    ("Ne", "this_work", 0.2, 32, 8, 0.02, -128.9),
    ("Ne", "previous", 0.3, 9, 6, 0.01, -128.9),
    ("Be_bare", "explicit", 0.2, 16, 10, 0.02, -20.0),
    ("H", "single", 0.3, 5, 10, 0.05, -0.5),
    ("Ar", "this_work", 1 / 63, 12, 3, 2e-4, -527.5),
    ("Kr", "this_work", 1 / 126, 6, 2, 3e-5, -2752.0),
    ("H2O", "this_work", 0.1, 20, 4, 0.005, -76.0),
])
def test_projection_matches_oracle(pkg, oracle_mod, name, kind, a, W, steps, tau, et, prec):
    """Whole intervals: waiting times, heat-bath choices, Sherman-Morrison
    updates, inverse recomputation, weights and comb reconfiguration."""
    compared, parted = _compare_runs(pkg, oracle_mod, S.make_system(name), kind, a, W, steps, tau, 11, et,
                                     prec=prec, label=f"projection {name} {kind} a={a:.6g} W={W} {prec}")
    assert compared >= (1 if parted else steps)


@pytest.mark.parametrize("prec", PRECISIONS)
def test_projection_full_size(pkg, oracle_mod, prec):
    """The Ne workload at full size (4096 walkers, a = 0.2, the paper's
    double grid, tau = 0.025) for two intervals, walker by walker."""
    compared, parted = _compare_runs(pkg, oracle_mod, S.neon(), "this_work", 0.2, 4096, 2, 0.025, 5, -128.9,
                                     prec=prec, label=f"projection Ne full size (4096) {prec}")
    assert compared >= 1


@pytest.mark.parametrize("W", [1, 63, 255, 256, 257, 4097, 8193, 16384, 16385, 20000])
def test_reconfiguration_blocks(pkg, oracle_mod, W):
    """The reconfiguration over its grid of blocks (at least 256 slots a
    block): one walker, one block, the boundary from one block to two (255,
    256, 257), ragged last blocks (4097, 8193), the last population whose
    running sums fit in shared memory and the first that does not (16384,
    16385) and one beyond (20000: sums read from global memory). He, three
    intervals, every parent, weight and trace entry against the oracle's
    sequential comb."""
    compared, parted = _compare_runs(pkg, oracle_mod, S.helium(), "this_work", 0.2, W, 3, 0.05, 41, -2.9,
                                     label=f"projection He reconfiguration blocks W={W} df64")
    assert compared >= (1 if parted else 3)


def test_reconfiguration_at_the_largest_population(pkg, oracle_mod):
    """LRDMC_MAX_WALKERS He walkers (128 blocks of 32768 slots, the running
    sums in global memory, a float per slot in shared memory), two
    intervals. Too large for the oracle's projection; instead the comb is
    recomputed on the host from the GPU's own log-weights with a sequential
    running sum and the comb uniform from the oracle's Philox: every parent
    agrees except where the target lies within 1e-10 (relative) of a bin
    edge, and the parents are non-decreasing."""
    W = 4194304
    system = S.helium()
    seed = 43
    g = pkg.LrdmcSystem(system)
    g.init_walkers(torch.tensor(S.initial_positions(system, W, seed), device="cuda"), seed=seed, tau=0.05,
                   e_trial=-2.9, recompute_every=3, trace_capacity=2)
    g.step(2, 0.2, pkg.Spacing(pkg.THIS_WORK))
    e, wbar, jumps = g.energy_trace()
    assert np.all(np.isfinite(e)) and np.all(np.isfinite(wbar)) and np.all(jumps > 0)
    w = g.walkers()
    parent, logw = w["parent"].astype(np.int64), w["logw_pre"]
    del w
    assert np.all(np.diff(parent) >= 0) and parent[0] >= 0 and parent[-1] < W
    wt = np.exp(logw)
    C = np.cumsum(wt)
    total = C[-1]
    xi = oracle_mod.uniform(int(oracle_mod.philox4x64([2 ** 64 - 1, 1, 0, 2], [seed, 0])[0]))
    target = (np.arange(W, dtype=np.float64) + xi) * total / W
    ref = np.minimum(np.searchsorted(C, target, side="right"), W - 1)
    differ = np.flatnonzero(ref != parent)
    lo = np.where(ref > 0, C[np.maximum(ref - 1, 0)], -np.inf)
    margin = np.minimum(np.abs(target - C[ref]), np.abs(target - lo)) / total
    assert np.all(margin[differ] < EDGE), (len(differ), differ[:8])
    assert abs(wbar[-1] - total / W) <= 1e-9 * wbar[-1]


@pytest.mark.parametrize("name,E", [("H", -0.5), ("Be_bare", -20.0)])
def test_zero_variance_on_gpu(pkg, name, E):
    system = S.make_system(name)
    g = pkg.LrdmcSystem(system)
    g.init_walkers(torch.tensor(S.initial_positions(system, 1000, 4), device="cuda"), seed=4, tau=0.05,
                   e_trial=E, recompute_every=5, trace_capacity=50)
    g.step(50, 0.2, pkg.Spacing(pkg.EXPLICIT, rc=0.4, aprime_over_a=1.8))
    e, w, j = g.energy_trace()
    assert np.max(np.abs(e - E)) < 1e-10 * abs(E)
    assert np.max(np.abs(w - 1.0)) < 1e-10 and np.mean(j) > 0.5


def test_energy_trace_async_matches_sync_read(pkg):
    """Per-step asynchronous trace reads into pinned memory hold, after
    sync(), the same bits as the synchronous read of the whole trace; an
    entry beyond the intervals stepped is LRDMC_ERR_ARG."""
    system = S.neon()
    g = pkg.LrdmcSystem(system)
    g.init_walkers(torch.tensor(S.initial_positions(system, 512, 6), device="cuda"), seed=6, tau=0.02,
                   e_trial=-128.9, recompute_every=3, trace_capacity=8)
    out = torch.zeros((3, 8), dtype=torch.float64).pin_memory()
    sp = pkg.Spacing(pkg.THIS_WORK)
    for k in range(6):
        g.step(1, 0.2, sp)
        g.energy_trace_async(k, 1, out)
    with pytest.raises(pkg.LrdmcError) as e:
        g.energy_trace_async(5, 2, out)
    assert e.value.status == pkg.ERR_ARG
    g.sync()
    e_, w_, j_ = g.energy_trace()
    assert np.array_equal(out[0, :6].numpy(), e_) and np.array_equal(out[1, :6].numpy(), w_)
    assert np.array_equal(out[2, :6].numpy(), j_)


def test_checkpoint_resume_bitwise(pkg, tmp_path):
    """save after 3 intervals, run 4 more; load and run the same 4: identical."""
    system = S.helium()
    sp = pkg.Spacing(pkg.THIS_WORK)
    g = pkg.LrdmcSystem(system)
    g.init_walkers(torch.tensor(S.initial_positions(system, 100, 8), device="cuda"), seed=8, tau=0.02,
                   e_trial=-2.9, recompute_every=2, trace_capacity=10)
    g.step(3, 0.2, sp)
    path = str(tmp_path / "ckpt.bin")
    g.save(path)
    g.step(4, 0.2, sp)
    e1 = g.energy_trace()[0]
    x1 = g.walkers()["x"]
    g.load(path)
    g.step(4, 0.2, sp)
    assert np.array_equal(g.energy_trace()[0], e1)
    assert np.array_equal(g.walkers()["x"], x1)


def test_deterministic_repeat(pkg):
    system = S.neon()
    sp = pkg.Spacing(pkg.THIS_WORK)
    out = []
    for _ in range(2):
        g = pkg.LrdmcSystem(system)
        g.init_walkers(torch.tensor(S.initial_positions(system, 300, 9), device="cuda"), seed=9, tau=0.02,
                       e_trial=-128.9, recompute_every=3, trace_capacity=5)
        g.step(5, 0.2, sp)
        out.append((g.energy_trace()[0], g.walkers()["x"]))
    assert np.array_equal(out[0][0], out[1][0]) and np.array_equal(out[0][1], out[1][1])


def test_errors_are_reported_not_faulted(pkg):
    system = S.neon()
    g = pkg.LrdmcSystem(system)
    x0 = S.initial_positions(system, 8, 10)
    x0[3, 1] = x0[3, 0]  # two spin-up electrons on one point: singular Slater matrix
    with pytest.raises(pkg.LrdmcError) as e:
        g.init_walkers(torch.tensor(x0, device="cuda"), seed=1, tau=0.01, trace_capacity=2)
    assert e.value.status == pkg.ERR_SINGULAR
    g2 = pkg.LrdmcSystem(system)
    g2.init_walkers(torch.tensor(S.initial_positions(system, 8, 11), device="cuda"), seed=1, tau=0.01,
                    trace_capacity=2)
    g2.step(2, 0.2)
    g2.sync()
    with pytest.raises(pkg.LrdmcError) as e:
        g2.step(1, 0.2)  # trace capacity exhausted
    assert e.value.status == pkg.ERR_ARG
    g2.step(0, 0.2)  # zero steps is a no-op


def test_host_buffers_and_single_walker(pkg, oracle_mod):
    """x0 from host memory, one walker, spin-down block empty (H)."""
    system = S.hydrogen(0.8)
    system.en_b1 = np.array([0.2])
    g = pkg.LrdmcSystem(system)
    x0 = S.initial_positions(system, 1, 12)
    g.init_walkers(x0, seed=12, tau=0.05, e_trial=-0.5, recompute_every=1, trace_capacity=20)
    g.step(20, 0.2, pkg.Spacing(pkg.SINGLE))
    o = oracle_mod.OracleSystem(system)
    pop = oracle_mod.OraclePopulation(o, x0, seed=12, tau=0.05, e_trial=-0.5, recompute_every=1)
    pop.step(oracle_mod.lattice_for(system, 0.2, oracle_mod.SINGLE), 20, 1)
    assert np.allclose(g.energy_trace()[0], pop.trace()[0], rtol=RTOL, atol=0)


# ---------------------------------------------------------------- mixed precision
FP32_RTOL = 2e-4


@pytest.mark.parametrize("name,kind,a", [("He", "this_work", 0.2), ("Ne", "this_work", 0.2),
                                         ("Ar", "this_work", 1 / 63), ("H2O", "this_work", 0.1)])
def test_fp32_evaluation_error(pkg, oracle_mod, name, kind, a):
    """The mixed-precision mode (single-precision evaluation): every ratio
    within 2e-4 of the FP64 oracle relative to max(1, |ratio|), the local
    energy within 2e-4 relative; the measured error is far above FP64 parity
    and far below the statistical noise of a projection."""
    system = S.make_system(name)
    g = pkg.LrdmcSystem(system).set_precision(pkg.PRECISION_FP32)
    o = oracle_mod.OracleSystem(system)
    n = 64
    x = S.initial_positions(system, n, 301)
    R = S.random_rotations(n, 302)
    sp, lat = spacing_pair(pkg, oracle_mod, system, a, kind)
    ratio, T, b, el = (t.cpu().numpy() for t in g.evaluate(torch.tensor(x, device="cuda"),
                                                           torch.tensor(R, device="cuda"), a, sp))
    worst_r = worst_e = 0.0
    for c in range(n):
        ref = o.lattice_eval(lat, x[c], R[c])
        worst_r = max(worst_r, float(np.max(np.abs(ratio[c] - ref["ratio"]) / np.maximum(1.0, np.abs(ref["ratio"])))))
        worst_e = max(worst_e, abs(el[c] - ref["EL"]) / abs(ref["EL"]))
    U.record({"test": f"evaluate {name} {kind} fp32 mode", "kind": "evaluation (mixed precision)",
              "configurations": n, "tolerance_rel": FP32_RTOL, "worst_ratio_rel_max1": worst_r,
              "worst_EL_rel": worst_e})
    assert worst_r < FP32_RTOL and worst_e < FP32_RTOL, (worst_r, worst_e)


@pytest.mark.parametrize("name,a", [("Ne", 0.2), ("Ar", 1 / 63), ("H2O", 0.1)])
def test_fp32_local_energy_is_the_double_float_one(pkg, name, a):
    """The mixed-precision mode forms the local energy in double-float: for
    a Pade guiding function its E_L is bit for bit the double-float mode's
    (which the parity tests hold to the FP64 oracle), while its lattice
    moves keep single-precision ratios."""
    system = S.make_system(name)
    n = 32
    x = torch.tensor(S.initial_positions(system, n, 311), device="cuda")
    R = torch.tensor(S.random_rotations(n, 312), device="cuda")
    sp = pkg.Spacing(pkg.THIS_WORK)
    out = {}
    for prec in (pkg.PRECISION_DF64, pkg.PRECISION_FP32):
        out[prec] = [t.cpu().numpy() for t in pkg.LrdmcSystem(system).set_precision(prec).evaluate(x, R, a, sp)]
    assert np.array_equal(out[pkg.PRECISION_DF64][3], out[pkg.PRECISION_FP32][3])
    # the ratios are the single-precision ones (not the double-float ones)
    assert not np.array_equal(out[pkg.PRECISION_DF64][0], out[pkg.PRECISION_FP32][0])


def test_fp32_projection_energy_matches_fp64(pkg):
    """He, 8192 walkers, 600 intervals after 100 of equilibration: the mixed
    mode's energy agrees with the FP64 mode's within 4 combined standard
    errors plus 0.5 mHa."""
    from paper_1909_01589_gb300 import stats

    system = S.helium()
    res = {}
    for prec in (pkg.PRECISION_FP64, pkg.PRECISION_FP32):
        g = pkg.LrdmcSystem(system).set_precision(prec)
        g.init_walkers(torch.tensor(S.initial_positions(system, 8192, 77), device="cuda"), seed=77, tau=0.02,
                       e_trial=-2.9, recompute_every=5, trace_capacity=700)
        g.step(700, 0.2, pkg.Spacing(pkg.THIS_WORK))
        e, w, _ = g.energy_trace()
        e = e[100:]
        res[prec] = (stats.energy_estimate(e, w[100:], 0), stats.reblock(e)[0])
    (e64, s64), (e32, s32) = res[pkg.PRECISION_FP64], res[pkg.PRECISION_FP32]
    assert abs(e64 - e32) < 4 * np.hypot(s64, s32) + 5e-4, (e64, s64, e32, s32)


@pytest.mark.parametrize("prec", PRECISIONS)
def test_large_system_without_caches(pkg, oracle_mod, prec):
    """48 electrons on 8 centres with 42 AOs: the largest kind of system
    whose four-walker block fits in shared memory only without the
    evaluation caches. Every ratio, rate and local energy of 5
    configurations, then two projection intervals of 6 walkers, against the
    oracle."""
    system = S.cluster(8, 24, 2)
    g = pkg.LrdmcSystem(system).set_precision(_prec(pkg, prec))
    o = oracle_mod.OracleSystem(system)
    n = 5
    x = S.initial_positions(system, n, 11)
    R = S.random_rotations(n, 12)
    sp, lat = spacing_pair(pkg, oracle_mod, system, 0.3, "this_work")
    ratio, T, b, el = (t.cpu().numpy() for t in g.evaluate(torch.tensor(x, device="cuda"),
                                                           torch.tensor(R, device="cuda"), 0.3, sp))
    rec = _EvalWorst()
    for c in range(n):
        ref = o.lattice_eval(lat, x[c], R[c])
        scale = ratio_scale(o, system, lat, x[c], R[c], ref["ratio"])
        err = np.abs(ratio[c] - ref["ratio"]) / (RTOL * scale)
        worst = int(np.argmax(err))
        assert err.max() <= 1.0, (c, worst, float(err.max()), float(ratio[c].flat[worst]),
                                  float(ref["ratio"].flat[worst]))
        tsc = rate_tolerance(lat, ref["w"], scale, w_abs=_w_abs(prec))
        _check_rates(c, T[c], ref, tsc, scale)
        assert abs(b[c] - ref["b"]) <= RTOL * ref["b"]
        assert abs(el[c] - ref["EL"]) <= RTOL * max(1.0, abs(ref["EL"]))
        rec.add(ratio[c], ref["ratio"], scale, T[c], ref["T"], tsc, b[c], ref["b"], el[c], ref["EL"])
    U.record(rec.entry(f"evaluate 48-electron cluster {prec}", n))
    compared, parted = _compare_runs(pkg, oracle_mod, system, "this_work", 0.3, 6, 2, 0.002, 13, 40.0, prec=prec,
                                     label=f"projection 48-electron cluster {prec}")
    assert compared == 2 or parted


def test_large_system_fp32_evaluation(pkg, oracle_mod):
    """The mixed-precision mode on the 48-electron system: its single-precision
    e-e Pade fraction runs over 47 partners a few bohr away, whose product of
    (1 + b r) leaves the float range unless it is rescaled. Every ratio
    within the mode's 2e-4 of the oracle (relative to the magnitude of its
    determinant terms), every local energy within 2e-4 relative, all finite."""
    system = S.cluster(8, 24, 2)
    g = pkg.LrdmcSystem(system).set_precision(pkg.PRECISION_FP32)
    o = oracle_mod.OracleSystem(system)
    n = 5
    x = S.initial_positions(system, n, 11)
    R = S.random_rotations(n, 12)
    sp, lat = spacing_pair(pkg, oracle_mod, system, 0.3, "this_work")
    ratio, T, b, el = (t.cpu().numpy() for t in g.evaluate(torch.tensor(x, device="cuda"),
                                                           torch.tensor(R, device="cuda"), 0.3, sp))
    assert np.all(np.isfinite(ratio)) and np.all(np.isfinite(el)) and np.all(b > 0)
    for c in range(n):
        ref = o.lattice_eval(lat, x[c], R[c])
        scale = ratio_scale(o, system, lat, x[c], R[c], ref["ratio"])
        err = float(np.max(np.abs(ratio[c] - ref["ratio"]) / scale))
        assert err < FP32_RTOL, (c, err)
        assert abs(el[c] - ref["EL"]) < FP32_RTOL * abs(ref["EL"]), (c, el[c], ref["EL"])


HEAVY_FULL = [("Ar", 1 / 63, 2e-4, -527.5), ("Kr", 1 / 126, 3e-5, -2752.0)]


@pytest.mark.parametrize("name,a,tau,et", HEAVY_FULL)
def test_heavy_atoms_evaluate_full_size_sampled(pkg, oracle_mod, name, a, tau, et):
    """The Ar and Kr workloads at full size: 16384 configurations of the
    contracted-Gaussian atoms at a = 1/(3.5 Z) on this work's double grid, in
    the default double-float mode. 16 sampled configurations are checked
    against the oracle one by one; every total rate is positive and finite."""
    system = S.make_system(name)
    g = pkg.LrdmcSystem(system)
    o = oracle_mod.OracleSystem(system)
    n = 16384
    x = S.initial_positions(system, n, 401)
    R = S.random_rotations(n, 402)
    sp, lat = spacing_pair(pkg, oracle_mod, system, a, "this_work")
    ratio, T, b, el = g.evaluate(torch.tensor(x, device="cuda"), torch.tensor(R, device="cuda"), a, sp)
    ratio, b, el = ratio.cpu().numpy(), b.cpu().numpy(), el.cpu().numpy()
    assert np.all(np.isfinite(el)) and np.all(b > 0) and np.all(np.isfinite(b))
    T = T.cpu().numpy()
    worst = _EvalWorst()
    for c in np.random.default_rng(4).choice(n, 16, replace=False):
        ref = o.lattice_eval(lat, x[c], R[c])
        scale = ratio_scale(o, system, lat, x[c], R[c], ref["ratio"])
        assert np.all(np.abs(ratio[c] - ref["ratio"]) <= RTOL * scale), c
        tsc = rate_tolerance(lat, ref["w"], scale, w_abs=_w_abs("df64"))
        _check_rates(c, T[c], ref, tsc, scale)
        assert abs(b[c] - ref["b"]) <= RTOL * ref["b"], c
        assert abs(el[c] - ref["EL"]) <= RTOL * abs(ref["EL"]), c
        worst.add(ratio[c], ref["ratio"], scale, T[c], ref["T"], tsc, b[c], ref["b"], el[c], ref["EL"])
    U.record(worst.entry(f"evaluate {name} full size (16384, 16 sampled) df64", 16))


@pytest.mark.parametrize("name,a,tau,et", HEAVY_FULL)
def test_heavy_atoms_projection_full_size(pkg, oracle_mod, name, a, tau, et):
    """One interval of the Ar and Kr workloads at full size (16384 walkers,
    a = 1/(3.5 Z), this work's double grid, tau for about 9 jumps per
    walker), walker by walker against the oracle's population."""
    compared, parted = _compare_runs(pkg, oracle_mod, S.make_system(name), "this_work", a, 16384, 1, tau, 17, et,
                                     label=f"projection {name} full size (16384) df64")
    assert compared == 1 or parted


@pytest.mark.parametrize("kind", ["single", "this_work"])
def test_helium_workload_full_length(pkg, oracle_mod, kind):
    """The He workload at its full length: 256 walkers, a = 0.2, 2000
    intervals on the single grid and on this work's double grid, walker by
    walker against the oracle after every interval, then the whole energy
    trace. Over about 5 million decisions a parting is accepted only where the
    walker or comb slot that parted had a decision the oracle reports within
    1e-10 of a bin edge; at least 100 intervals must agree before it."""
    compared, parted = _compare_runs(pkg, oracle_mod, S.helium(), kind, 0.2, 256, 2000, 0.02, 23, -2.9,
                                     label=f"projection He workload {kind} (256 walkers, 2000 intervals) df64")
    assert compared == 2000 or (parted and compared >= 100), compared


@pytest.mark.parametrize("kind", ["single", "this_work"])
@pytest.mark.parametrize("a", [0.4, 0.2, 0.1])
def test_neon_workload_lattices(pkg, oracle_mod, a, kind):
    """The Ne workload's lattices at full size: 4096 walkers at a = 0.4, 0.2
    and 0.1 on the single grid and on this work's double grid, tau scaled as
    a^2 (about 10 jumps per walker on the double grid), two intervals walker
    by walker against the oracle."""
    tau = 0.025 * (a / 0.2) ** 2
    compared, parted = _compare_runs(pkg, oracle_mod, S.neon(), kind, a, 4096, 2, tau, 29, -128.9,
                                     label=f"projection Ne workload {kind} a={a} (4096) df64")
    assert compared == 2 or parted


@pytest.mark.parametrize("prec", ["fp64", "df64", "fp32"])
def test_sherman_morrison_residual_trace(pkg, prec):
    """The Sherman-Morrison diagnostic: at every rebuild of the inverse
    Slater matrices (intervals 3 and 6 with recompute_every = 3) the largest
    max|A Ainv - I| of the updated inverses over 512 Ne walkers is recorded;
    it is rounding-sized (the parity modes update in IEEE double) and -1 at
    the other intervals."""
    system = S.neon()
    g = pkg.LrdmcSystem(system).set_precision(_prec(pkg, prec) if prec != "fp32" else pkg.PRECISION_FP32)
    g.init_walkers(torch.tensor(S.initial_positions(system, 512, 81), device="cuda"), seed=82, tau=0.025,
                   e_trial=-128.9, recompute_every=3, trace_capacity=8)
    g.step(8, 0.2, pkg.Spacing(pkg.THIS_WORK))
    r = g.residual_trace()
    assert len(r) == 8
    rebuilt = [k for k in range(8) if k > 0 and k % 3 == 0]
    for k in range(8):
        if k in rebuilt:
            assert 0.0 < r[k] < 1e-8, (k, r[k])
        else:
            assert r[k] == -1.0, (k, r[k])
