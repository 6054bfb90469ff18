"""Paper-style experiments on the GPU path: single vs double grid.

For atoms at the paper's lattice spacing a = 1/(alpha Z) (alpha = 3.5 in
Table I and Fig. 2), the same population is projected with the single grid,
with the double grid of this work (Eq. 3, S-13, Eq. 6/7) and with the
previous double grid (Eq. 2, Eq. 4). Reported per run: the energy and its
blocked error, the mean number of jumps per interval (the acceptance-rate
analogue of the acceleration column of Table S-I), the GPU time, and the
efficiency 1/(sigma^2 t). Ratios to the single grid give the bias (energy
difference) and the acceleration at fixed error (efficiency ratio), the
quantities of Table I, Table S-I and Fig. 2.

The trial functions are this library's synthetic Slater-Jastrow atoms, not
the paper's optimised JAGP wavefunctions, so the numbers show the method's
behaviour on these systems and are context for, not reproductions of, the
paper's tables.

Usage: python -m paper_1909_01589_gb300.experiments [--systems He,Ne,Ar,Kr]
       [--steps 1000] [--out results/single_vs_double.json]
       python -m paper_1909_01589_gb300.experiments --neural --systems Ne,Ar
       [--steps 600] [--out results/neural_vs_pade.json]
       python -m paper_1909_01589_gb300.experiments --mixed --systems Ne,Ar,Kr
       [--out results/mixed_vs_parity.json]
       python -m paper_1909_01589_gb300.experiments --extrapolate [--neural] --systems He
       [--steps 2000] [--out results/extrapolation_he.json]
"""
from __future__ import annotations

import argparse
import json
import os
import time

import numpy as np

from . import LrdmcSystem, Spacing, SINGLE, THIS_WORK, PREVIOUS, PRECISION_DF64
from . import stats

DEFAULTS = {  # system: (walkers, e_trial, target jumps per interval)
    "He": (4096, -2.90, 10.0),
    "Ne": (4096, -128.9, 10.0),
    "Ar": (4096, -527.5, 10.0),
    "Kr": (4096, -2753.0, 10.0),
    "H2O": (4096, -76.0, 10.0),
}


def run(system, a, spacing, W, steps, equil, tau, e_trial, seed=1, precision=PRECISION_DF64, device="cuda",
        neural=None):
    """One projection; returns energy, error, jumps/interval, GPU seconds.
    ``neural`` = (spec, params) installs the neural pair term."""
    import torch

    import lrdmc_synth as S

    g = LrdmcSystem(system).set_precision(precision)
    if neural is not None:
        g.set_neural_jastrow(*neural)
    x0 = S.initial_positions(system, W, seed)
    g.init_walkers(torch.tensor(x0, device=device), seed=seed, tau=tau, e_trial=e_trial, recompute_every=5,
                   trace_capacity=steps + equil + 4)
    g.step(equil, a, spacing)
    g.sync()
    torch.cuda.synchronize()
    m0 = g.moves()
    t0 = time.perf_counter()
    g.step(steps, a, spacing)
    g.sync()
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    moves = g.moves() - m0
    e, w, j = g.energy_trace()
    e, w, j = e[equil:], w[equil:], j[equil:]
    err, _ = stats.reblock(e)
    return {"energy": stats.energy_estimate(e, w, 0), "error": err, "jumps_per_interval": float(np.mean(j)),
            "seconds": dt, "moves": int(moves), "efficiency": stats.efficiency(e, dt), "intervals": steps}


def _tau_for(system, a, spacing, jumps, seed):
    """Interval length giving about ``jumps`` jumps per walker on this
    lattice: jumps / <b>, <b> the mean total rate over 256 start
    configurations (one stateless evaluation)."""
    import lrdmc_synth as S

    from .batch import tau_for

    import paper_1909_01589_gb300 as pkg

    x = S.initial_positions(system, 256, seed)
    return tau_for(pkg, system, a, spacing, jumps, x, S.random_rotations(256, seed + 1))


def single_vs_double(names=("He", "Ne", "Ar", "Kr"), alpha=3.5, steps=1000, equil=200, seed=1):
    """Every lattice gets its own interval length (about 10 jumps per walker
    per interval, so that the intervals are not dominated by the longest
    walker) and the same total projection time: the single grid runs
    ``steps`` intervals of tau_single, each double grid steps * tau_single /
    tau_double intervals (equilibration alike)."""
    import lrdmc_synth as S

    rows = []
    for name in names:
        system = S.make_system(name)
        Z = float(np.max(system.Z))
        a = 1.0 / (alpha * Z)
        W, e_trial, jumps = DEFAULTS[name]
        g = LrdmcSystem(system)
        ratio, rc = g.spacing_params(a, Spacing(THIS_WORK))
        res, taus = {}, {}
        for label, sp in (("single", Spacing(SINGLE)), ("double_this_work", Spacing(THIS_WORK)),
                          ("double_previous", Spacing(PREVIOUS))):
            taus[label] = _tau_for(system, a, sp, jumps, seed)
        for label, sp in (("single", Spacing(SINGLE)), ("double_this_work", Spacing(THIS_WORK)),
                          ("double_previous", Spacing(PREVIOUS))):
            f = taus["single"] / taus[label]
            n_steps = max(64, int(round(steps * f)))
            n_equil = max(16, int(round(equil * f)))
            res[label] = run(system, a, sp, W, n_steps, n_equil, taus[label], e_trial, seed)
            res[label]["tau"] = taus[label]
        s = res["single"]
        row = {"system": name, "Z": Z, "a": a, "alpha": alpha, "aprime_over_a": ratio, "rc": rc,
               "tau": taus["single"], "walkers": W, **{k: v for k, v in res.items()}}
        for label in ("double_this_work", "double_previous"):
            d = res[label]
            row[label + "_bias_mHa"] = 1e3 * (d["energy"] - s["energy"])
            row[label + "_bias_err_mHa"] = 1e3 * float(np.hypot(d["error"], s["error"]))
            # jumps per unit projection time
            row[label + "_acceleration_jumps"] = (s["jumps_per_interval"] / s["tau"]) / max(
                d["jumps_per_interval"] / d["tau"], 1e-300)
            row[label + "_acceleration_efficiency"] = d["efficiency"] / s["efficiency"]
        rows.append(row)
    return rows


# system: (e_trial, a). Ar at a = 0.2 (a Z = 3.6, a lattice coarser than its
# core) gives no stable projection with the synthetic Gaussian-basis trial
# function (the population collapses to about -1650 Ha); a = 0.05 (a Z = 0.9)
NEURAL_DEFAULTS = {"Ne": (-128.9, 0.2), "Ar": (-527.5, 0.05)}


def neural_vs_pade(names=("Ne", "Ar"), W=16384, steps=600, equil=150, n_train=1 << 20, train_steps=600,
                   seed=3):
    """The neural pair Jastrow against the plain Pade Jastrow: configurations
    from a plain projection (a, this work's double grid, W walkers), training
    on the GPU, then a projection with and without the tabulated term over
    the same number of intervals. Reported per system: held-out variance of
    E_L, the walkers' E_L variance in the projection, energy and blocked
    error, walker-moves/s and the efficiency 1/(sigma^2 t)."""
    import torch

    import lrdmc_synth as S

    from . import neural as N

    rows = []
    sp = Spacing(THIS_WORK)
    for name in names:
        system = S.make_system(name)
        e_trial, a = NEURAL_DEFAULTS[name]
        tau = _tau_for(system, a, sp, 10.0, seed)
        spec = S.default_neural_spec(system)
        plain = LrdmcSystem(system)
        t0 = time.perf_counter()
        x = N.sample_configurations(plain, S.initial_positions(system, W, seed), n_train, a, sp, tau, e_trial,
                                    seed=seed, equil=equil)
        grad, e = plain.base_terms(x)
        n_tr = len(x) * 7 // 8
        params, hist = N.train(plain, spec, S.neural_init(spec, seed), x[:n_tr], grad[:n_tr], e[:n_tr],
                               steps=train_steps, seed=seed + 1, log_every=100)
        torch.cuda.synchronize()
        t_train = time.perf_counter() - t0
        el, j = N.evaluate(plain, spec, params, x[n_tr:], grad[n_tr:], e[n_tr:])
        row = {"system": name, "walkers": W, "a": a, "tau": tau, "train_configs": n_tr, "train_steps": train_steps,
               "train_seconds": t_train, "train_loss": hist,
               "heldout_var_pade": float(torch.var(e[n_tr:])),
               "heldout_var_neural": float(N.variance_loss(el, j, clip=0.0))}
        x0 = S.initial_positions(system, W, seed + 7)
        for label, use in (("pade", False), ("neural", True)):
            g = LrdmcSystem(system)
            if use:
                g.set_neural_jastrow(spec, params.cpu().numpy())
            g.init_walkers(torch.tensor(x0, device="cuda"), seed=seed + 8, tau=tau, e_trial=e_trial,
                           recompute_every=5, trace_capacity=steps + equil + 4)
            g.step(equil, a, sp)
            g.sync()
            torch.cuda.synchronize()
            m0 = g.moves()
            t1 = time.perf_counter()
            g.step(steps, a, sp)
            g.sync()
            torch.cuda.synchronize()
            dt = time.perf_counter() - t1
            et, wt, jt = g.energy_trace()
            et, wt = et[equil:], wt[equil:]
            err, _ = stats.reblock(et)
            row[label] = {"energy": stats.energy_estimate(et, wt, 0), "error": err, "seconds": dt,
                          "moves_per_s": (g.moves() - m0) / dt, "efficiency": stats.efficiency(et, dt),
                          "var_EL_walkers": float(np.var(g.walkers()["EL"]))}
        row["efficiency_ratio"] = row["neural"]["efficiency"] / row["pade"]["efficiency"]
        rows.append(row)
        print(f"{name}: held-out var {row['heldout_var_pade']:.2f} -> {row['heldout_var_neural']:.2f}; "
              f"walker var {row['pade']['var_EL_walkers']:.2f} -> {row['neural']['var_EL_walkers']:.2f}; "
              f"E {row['pade']['energy']:.4f}({1e3 * row['pade']['error']:.1f}) -> "
              f"{row['neural']['energy']:.4f}({1e3 * row['neural']['error']:.1f}); "
              f"moves/s {row['pade']['moves_per_s']:.3g} -> {row['neural']['moves_per_s']:.3g}; "
              f"efficiency x{row['efficiency_ratio']:.2f}", flush=True)
    return rows


def extrapolation(name="He", a_values=(0.4, 0.3, 0.2, 0.15, 0.1), W=8192, steps=2000, equil=200, seed=5,
                  neural=False, n_train=1 << 18, train_steps=600, a_train=0.2, proj_time=None):
    """E(a) on the single grid and on this work's double grid at several
    lattice spacings, and the a -> 0 limits from the weighted least-squares
    fit E(a) = E0 + k1 a^2 + k2 a^4 (the three-parameter fit of the paper's
    benzene footnote). For He the guiding function is nodeless, so both
    limits must reach the exact ground-state energy.

    With ``neural`` the neural pair term is trained once on the GPU
    (configurations of a plain projection at a_train on this work's double
    grid) and installed in every run: the guiding function changes E(a) at
    finite a, not the fixed-node limit, so the limits must agree with the
    plain ones.

    With ``proj_time`` every lattice spacing covers the same projection
    time (intervals = proj_time / tau, tau for about 10 jumps per walker per
    interval), so that the points carry comparable errors; otherwise every
    spacing runs ``steps`` intervals."""
    import lrdmc_synth as S

    system = S.make_system(name)
    e_trial = DEFAULTS[name][1]
    out = {"system": name, "a": list(a_values), "walkers": W, "steps": steps, "neural": bool(neural),
           "proj_time": proj_time}
    nj = None
    if neural:
        import torch

        from . import neural as N

        sp = Spacing(THIS_WORK)
        tau = _tau_for(system, a_train, sp, 10.0, seed)
        spec = S.default_neural_spec(system)
        plain = LrdmcSystem(system)
        t0 = time.perf_counter()
        x = N.sample_configurations(plain, S.initial_positions(system, W, seed + 50), n_train, a_train, sp, tau,
                                    e_trial, seed=seed + 50)
        grad, e = plain.base_terms(x)
        n_tr = len(x) * 7 // 8
        params, _ = N.train(plain, spec, S.neural_init(spec, seed), x[:n_tr], grad[:n_tr], e[:n_tr],
                            steps=train_steps, seed=seed + 51)
        torch.cuda.synchronize()
        el, j = N.evaluate(plain, spec, params, x[n_tr:], grad[n_tr:], e[n_tr:])
        out["train"] = {"a": a_train, "configs": n_tr, "steps": train_steps,
                        "seconds": time.perf_counter() - t0,
                        "heldout_var_pade": float(torch.var(e[n_tr:])),
                        "heldout_var_neural": float(N.variance_loss(el, j, clip=0.0))}
        nj = (spec, params.cpu().numpy())
        print(f"{name} neural term: held-out var {out['train']['heldout_var_pade']:.4f} -> "
              f"{out['train']['heldout_var_neural']:.4f} Ha^2", flush=True)
    for label, sp in (("single", Spacing(SINGLE)), ("double_this_work", Spacing(THIS_WORK))):
        E, err = [], []
        for a in a_values:
            tau = _tau_for(system, a, sp, 10.0, seed)
            n_steps = steps if proj_time is None else max(200, int(round(proj_time / tau)))
            r = run(system, a, sp, W, n_steps, equil, tau, e_trial, seed, neural=nj)
            E.append(r["energy"])
            err.append(r["error"])
        fit = fit_a0(a_values, E, err)
        out[label] = {"E": list(map(float, E)), "error": list(map(float, err)), **fit}
        print(f"{name} {label}: E0 = {fit['E0']:.5f} +- {fit['E0_error']:.5f} (chi2/dof "
              f"{fit['chi2_per_dof']:.2f}); E(a) = {np.round(E, 5).tolist()}", flush=True)
    return out


def mixed_vs_parity(names=("Ne", "Ar", "Kr"), steps=None, equil=200, seed=7):
    """Energy of the mixed-precision mode (FP32 evaluation, FP64 state)
    against the FP64-parity form (double-float evaluation, whose
    trajectories equal the FP64 mode's) on the same start population and
    random streams, so the two projections stay correlated while their
    decisions agree: the difference Delta E = mean_k(e32_k - e64_k) and its
    blocked error come from the difference series itself (correlated
    sampling), next to each mode's own energy and error. Workloads: Ne at
    a = 0.2 with 4096 walkers (the bench workload), Ar and Kr at
    a = 1/(3.5 Z) with 16384 walkers, this work's double grid, tau for
    about 10 jumps per walker per interval. Also the evaluation's own error
    on the projected population: the mean shift of the local energy (the
    quantity the mixed estimator averages) and the relative error of the
    total rates, over the parity run's final walkers evaluated in both
    arithmetics."""
    import torch

    import lrdmc_synth as S

    from . import PRECISION_FP32

    work = {"Ne": (4096, 0.2, 20000), "Ar": (16384, 1.0 / 63.0, 3000), "Kr": (16384, 1.0 / 126.0, 1200),
            "He": (4096, 0.2, 20000)}
    rows = []
    for name in names:
        system = S.make_system(name)
        W, a, n_default = work[name]
        n = steps or n_default
        e_trial = DEFAULTS[name][1]
        sp = Spacing(THIS_WORK)
        tau = 0.025 if name == "Ne" else _tau_for(system, a, sp, 10.0, seed)
        x0 = S.initial_positions(system, W, seed)
        res = {}
        for label, prec in (("parity", PRECISION_DF64), ("mixed", PRECISION_FP32)):
            g = LrdmcSystem(system).set_precision(prec)
            g.init_walkers(torch.tensor(x0, device="cuda"), seed=seed, tau=tau, e_trial=e_trial, recompute_every=5,
                           trace_capacity=n + equil + 4)
            g.step(equil, a, sp)
            g.sync()
            torch.cuda.synchronize()
            m0 = g.moves()
            t0 = time.perf_counter()
            g.step(n, a, sp)
            g.sync()
            torch.cuda.synchronize()
            dt = time.perf_counter() - t0
            e, w, j = g.energy_trace()
            e = e[equil:]
            err, _ = stats.reblock(e)
            res[label] = {"energy": float(np.mean(e)), "error": err, "seconds": dt,
                          "moves_per_s": (g.moves() - m0) / dt, "efficiency": stats.efficiency(e, dt), "trace": e}
            if label == "parity":
                x_end = g.walkers()["x"]
        # the evaluation's own error on the projected population: local
        # energies and total rates of the final parity-mode walkers in both
        # arithmetics (the mixed estimator averages E_L over this population)
        xs = torch.tensor(x_end, device="cuda")
        rs = torch.tensor(S.random_rotations(len(x_end), seed + 3), device="cuda")
        ev = {}
        for label, prec in (("parity", PRECISION_DF64), ("mixed", PRECISION_FP32)):
            ev[label] = [t.cpu().numpy() for t in LrdmcSystem(system).set_precision(prec).evaluate(xs, rs, a, sp)]
        del_el = ev["mixed"][3] - ev["parity"][3]
        del_b = (ev["mixed"][2] - ev["parity"][2]) / ev["parity"][2]
        d = res["mixed"]["trace"] - res["parity"]["trace"]
        derr, _ = stats.reblock(d)
        corr = float(np.corrcoef(res["mixed"]["trace"], res["parity"]["trace"])[0, 1])
        row = {"system": name, "walkers": W, "a": a, "tau": tau, "intervals": n, "equilibration": equil,
               "delta_E_Ha": float(np.mean(d)), "delta_E_error_Ha": derr, "trace_correlation": corr,
               "independent_error_Ha": float(np.hypot(res["mixed"]["error"], res["parity"]["error"])),
               "EL_shift_on_population_Ha": float(np.mean(del_el)),
               "EL_shift_error_Ha": float(np.std(del_el, ddof=1) / np.sqrt(len(del_el))),
               "EL_abs_error_mean_Ha": float(np.mean(np.abs(del_el))),
               "b_rel_error_mean": float(np.mean(del_b)), "b_rel_error_rms": float(np.sqrt(np.mean(del_b ** 2))),
               "efficiency_ratio": res["mixed"]["efficiency"] / res["parity"]["efficiency"]}
        for label in ("parity", "mixed"):
            row[label] = {k: v for k, v in res[label].items() if k != "trace"}
        rows.append(row)
        print(f"{name}: E_parity {row['parity']['energy']:.5f}({1e3 * row['parity']['error']:.2f} mHa) "
              f"E_mixed {row['mixed']['energy']:.5f}({1e3 * row['mixed']['error']:.2f}) "
              f"dE {1e3 * row['delta_E_Ha']:+.3f} +- {1e3 * derr:.3f} mHa (corr {corr:.3f}); "
              f"E_L shift {1e3 * row['EL_shift_on_population_Ha']:+.4f} +- {1e3 * row['EL_shift_error_Ha']:.4f} mHa; "
              f"moves/s {row['parity']['moves_per_s']:.3g} -> {row['mixed']['moves_per_s']:.3g}", flush=True)
    return rows


def fit_a0(a_values, E, err):
    """Weighted least-squares fit E(a) = E0 + k1 a^2 + k2 a^4 (the lattice
    error of LRDMC is even in a; the three-parameter form of the paper's
    benzene footnote) to energies E with standard errors err. Returns E0 (the
    a -> 0 limit), its standard error from the fit's covariance, k1, k2 and
    chi^2 per degree of freedom."""
    a = np.asarray(a_values, float)
    E = np.asarray(E, float)
    err = np.asarray(err, float)
    if len(a) < 3 or len(E) != len(a) or len(err) != len(a):
        raise ValueError("fit_a0 needs at least three (a, E, err) points of equal length")
    A = np.stack([np.ones_like(a), a ** 2, a ** 4], 1)
    wt = 1.0 / err ** 2
    cov = np.linalg.inv(A.T @ (A * wt[:, None]))
    coef = cov @ (A.T @ (wt * E))
    chi2 = float(np.sum(wt * (A @ coef - E) ** 2))
    return {"E0": float(coef[0]), "E0_error": float(np.sqrt(cov[0, 0])), "k1": float(coef[1]),
            "k2": float(coef[2]), "chi2_per_dof": chi2 / max(1, len(E) - 3)}


def z_exponent(Z, cost):
    """Exponent x of the least-squares power law cost ~ Z^x (a straight line
    in log-log, as Fig. 2 fits the CPU cost against Z)."""
    return float(np.polyfit(np.log(np.asarray(Z, float)), np.log(np.asarray(cost, float)), 1)[0])


def summarize(rows):
    """Derived quantities of the Fig. 2 analogue: GPU seconds per walker per
    unit of projection time (single grid, this work's double grid, the
    previous double grid), their ratio (the acceleration at equal projection
    time, which equals the acceleration at fixed error when the variance per
    unit projection time is the same for both lattices), the cost at a fixed
    target error (sigma^2 t = 1/efficiency: the GPU seconds that give a
    standard error of 1 Ha, the quantity Fig. 2 plots), and the exponents x
    of least-squares fits cost ~ Z^x over the systems (keys ending in
    "_fixed_error" for the cost at fixed error)."""
    out = []
    labels = ("single", "double_this_work", "double_previous")
    for r in rows:
        W = r["walkers"]
        cost = {k: r[k]["seconds"] / (W * r[k]["intervals"] * r[k].get("tau", r["tau"])) for k in labels}
        cost_err = {k: 1.0 / r[k]["efficiency"] for k in labels}
        out.append({"system": r["system"], "Z": r["Z"], "cost": cost, "cost_fixed_error": cost_err,
                    "acceleration_time": cost["single"] / cost["double_this_work"],
                    "acceleration_fixed_error": cost_err["single"] / cost_err["double_this_work"],
                    "acceleration_jumps": r["double_this_work_acceleration_jumps"]})
    fit = {}
    if len(out) >= 2:
        Zs = [o["Z"] for o in out]
        for k in labels:
            fit[k] = z_exponent(Zs, [o["cost"][k] for o in out])
            fit[k + "_fixed_error"] = z_exponent(Zs, [o["cost_fixed_error"][k] for o in out])
    return out, fit


def markdown(rows):
    derived, fit = summarize(rows)
    lines = ["| system | Z | a | a'/a | E single (Ha) | bias this work (mHa) | bias previous (mHa) | "
             "jumps per unit time single/double | GPU time per unit time single/double | efficiency ratio |",
             "|---|---|---|---|---|---|---|---|---|---|"]
    for r, d in zip(rows, derived):
        lines.append(
            f"| {r['system']} | {r['Z']:.0f} | {r['a']:.5f} | {r['aprime_over_a']:.3f} | "
            f"{r['single']['energy']:.4f} ({1e3 * r['single']['error']:.1f} mHa) | "
            f"{r['double_this_work_bias_mHa']:+.1f} ({r['double_this_work_bias_err_mHa']:.1f}) | "
            f"{r['double_previous_bias_mHa']:+.1f} ({r['double_previous_bias_err_mHa']:.1f}) | "
            f"{d['acceleration_jumps']:.2f} | {d['acceleration_time']:.2f} | "
            f"{r['double_this_work_acceleration_efficiency']:.2f} |")
    if fit:
        lines.append("")
        lines.append("GPU cost per walker per unit projection time ~ Z^x: " +
                     ", ".join(f"{k} x = {v:.2f}" for k, v in fit.items()))
    return "\n".join(lines)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--systems", default="He,Ne,Ar,Kr")
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--equil", type=int, default=200)
    ap.add_argument("--alpha", type=float, default=3.5)
    ap.add_argument("--out", default="results/single_vs_double.json")
    ap.add_argument("--summarize", nargs="*", help="only write the markdown table of these result files")
    ap.add_argument("--neural", action="store_true", help="the neural Jastrow against Pade instead")
    ap.add_argument("--proj-time", type=float, default=None,
                    help="with --extrapolate: the projection time (1/Ha) every lattice spacing covers")
    ap.add_argument("--a-values", default=None, help="with --extrapolate: comma-separated lattice spacings")
    ap.add_argument("--walkers", type=int, default=None, help="with --extrapolate: walkers per run")
    ap.add_argument("--mixed", action="store_true",
                    help="mixed-precision (FP32 evaluation) energy against the FP64-parity form instead")
    ap.add_argument("--extrapolate", action="store_true",
                    help="E(a) and the a -> 0 fit instead (first system); with --neural, with the trained term")
    args = ap.parse_args()
    if args.mixed:
        rows = mixed_vs_parity(args.systems.split(","), steps=args.steps if args.steps != 1000 else None,
                               equil=args.equil)
        os.makedirs(os.path.dirname(args.out) or ".", exist_ok=True)
        json.dump(rows, open(args.out, "w"), indent=1)
        return
    if args.extrapolate:
        kw = {}
        if args.a_values:
            kw["a_values"] = tuple(float(v) for v in args.a_values.split(","))
        if args.walkers:
            kw["W"] = args.walkers
        row = extrapolation(args.systems.split(",")[0], steps=args.steps, equil=args.equil, neural=args.neural,
                            proj_time=args.proj_time, **kw)
        os.makedirs(os.path.dirname(args.out) or ".", exist_ok=True)
        json.dump(row, open(args.out, "w"), indent=1)
        return
    if args.neural:
        rows = neural_vs_pade(args.systems.split(","), steps=args.steps, equil=args.equil)
        os.makedirs(os.path.dirname(args.out) or ".", exist_ok=True)
        json.dump(rows, open(args.out, "w"), indent=1)
        return
    if args.summarize:
        rows = []
        for f in args.summarize:
            rows += json.load(open(f))
        rows.sort(key=lambda r: r["Z"])
        print(markdown(rows))
        return
    rows = single_vs_double(args.systems.split(","), args.alpha, args.steps, args.equil)
    os.makedirs(os.path.dirname(args.out) or ".", exist_ok=True)
    json.dump(rows, open(args.out, "w"), indent=1)
    for r in rows:
        print(f"{r['system']:3s} Z={r['Z']:4.0f} a={r['a']:.5f} a'/a={r['aprime_over_a']:.3f} "
              f"E_single={r['single']['energy']:.5f}({1e3 * r['single']['error']:.1f}mHa) "
              f"bias_this={r['double_this_work_bias_mHa']:+.2f}({r['double_this_work_bias_err_mHa']:.2f}) "
              f"bias_prev={r['double_previous_bias_mHa']:+.2f}({r['double_previous_bias_err_mHa']:.2f}) "
              f"acc_jumps={r['double_this_work_acceleration_jumps']:.2f} "
              f"acc_eff={r['double_this_work_acceleration_efficiency']:.2f}", flush=True)


if __name__ == "__main__":
    main()
