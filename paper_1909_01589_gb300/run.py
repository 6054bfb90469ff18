"""LRDMC projection of a system given as JSON, with the run described by a
second JSON: the command-line face of the library.

    python -m paper_1909_01589_gb300.run --system ne.json --run run.json [--out result.json]
    python -m paper_1909_01589_gb300.run --dump-system Ne --out ne.json

The system file holds the nuclei, charges, spin counts, shells, orbital
coefficients and Pade Jastrow parameters (``lrdmc_synth.system_to_dict``).
The run file holds the projection's parameters:

    {"walkers": 4096, "intervals": 1200, "a": 0.2, "tau": 0.025,
     "e_trial": -128.9, "spacing": "this_work", "seed": 1,
     "recompute_every": 5, "precision": "df64", "equilibration": 200}

``spacing`` is ``single``, ``this_work`` (Eq. 3 with r_c from S-13 and a'/a
from Eq. 6 and 7), ``previous`` (Eq. 2 and Eq. 4) or ``explicit`` (Eq. 3 with
the run's ``rc`` and ``aprime_over_a``). ``precision`` is ``fp64``, ``df64``
(the default) or ``fp32``. The result holds the energy (the mixed
estimator over the intervals after ``equilibration``, with ``mixed_L``
weight factors), its reblocked error, the throughput and the trace.
Every step of the projection runs in the CUDA library; this module only
reads the files, calls the binding and writes the result.
"""
from __future__ import annotations

import argparse
import json
import time
from dataclasses import asdict, dataclass, fields

import numpy as np

SPACINGS = ("single", "this_work", "previous", "explicit")
PRECISIONS = ("fp64", "df64", "fp32")


@dataclass
class RunConfig:
    walkers: int
    intervals: int
    a: float
    tau: float
    e_trial: float
    seed: int = 1
    start_seed: int | None = None  # seed of the start positions (default: seed)
    spacing: str = "this_work"
    rc: float | None = None  # explicit spacing only
    aprime_over_a: float | None = None  # explicit spacing only
    beta: float = 0.75  # S-13
    kappa: float = 2.5  # S-13
    recompute_every: int = 10
    precision: str = "df64"
    equilibration: int = 0
    mixed_L: int = 0


def parse_run(d: dict) -> RunConfig:
    """RunConfig from a dict; ValueError for unknown keys or values out of
    range."""
    names = {f.name for f in fields(RunConfig)}
    unknown = sorted(set(d) - names)
    if unknown:
        raise ValueError(f"run: unknown keys {unknown}")
    for key in ("walkers", "intervals", "a", "tau", "e_trial"):
        if key not in d:
            raise ValueError(f"run: missing '{key}'")
    try:
        cfg = RunConfig(**d)
        cfg.walkers, cfg.intervals = int(cfg.walkers), int(cfg.intervals)
        cfg.a, cfg.tau, cfg.e_trial = float(cfg.a), float(cfg.tau), float(cfg.e_trial)
        cfg.seed, cfg.recompute_every = int(cfg.seed), int(cfg.recompute_every)
        cfg.equilibration, cfg.mixed_L = int(cfg.equilibration), int(cfg.mixed_L)
        cfg.start_seed = cfg.seed if cfg.start_seed is None else int(cfg.start_seed)
        cfg.beta, cfg.kappa = float(cfg.beta), float(cfg.kappa)
    except (TypeError, ValueError) as e:
        raise ValueError(f"run: {e}") from None
    if cfg.walkers < 1 or cfg.intervals < 1:
        raise ValueError("run: need walkers >= 1 and intervals >= 1")
    if not (cfg.a > 0.0 and cfg.tau > 0.0):
        raise ValueError("run: need a > 0 and tau > 0")
    if cfg.recompute_every < 0 or cfg.mixed_L < 0:
        raise ValueError("run: need recompute_every >= 0 and mixed_L >= 0")
    if not 0 <= cfg.equilibration < cfg.intervals:
        raise ValueError("run: need 0 <= equilibration < intervals")
    if cfg.spacing not in SPACINGS:
        raise ValueError(f"run: spacing '{cfg.spacing}' is not one of {SPACINGS}")
    if cfg.precision not in PRECISIONS:
        raise ValueError(f"run: precision '{cfg.precision}' is not one of {PRECISIONS}")
    if cfg.spacing == "explicit":
        if cfg.rc is None or cfg.aprime_over_a is None or not (cfg.rc > 0.0 and cfg.aprime_over_a > 0.0):
            raise ValueError("run: the explicit spacing needs rc > 0 and aprime_over_a > 0")
    elif cfg.rc is not None or cfg.aprime_over_a is not None:
        raise ValueError("run: rc and aprime_over_a belong to the explicit spacing only")
    return cfg


def spacing_of(cfg: RunConfig, lr):
    """The binding's Spacing for the run."""
    kind = {"single": lr.SINGLE, "this_work": lr.THIS_WORK, "previous": lr.PREVIOUS,
            "explicit": lr.EXPLICIT}[cfg.spacing]
    if cfg.spacing == "explicit":
        return lr.Spacing(kind, beta=cfg.beta, kappa=cfg.kappa, rc=cfg.rc, aprime_over_a=cfg.aprime_over_a)
    return lr.Spacing(kind, beta=cfg.beta, kappa=cfg.kappa)


def run(system, cfg: RunConfig, lr=None) -> dict:
    """Projects the system on the GPU with the run's parameters and returns
    the result (energy, error, throughput, trace). ``lr`` is the binding
    module (the package itself by default)."""
    import lrdmc_synth as S

    from . import stats

    if lr is None:
        import paper_1909_01589_gb300 as lr
    prec = {"fp64": lr.PRECISION_FP64, "df64": lr.PRECISION_DF64, "fp32": lr.PRECISION_FP32}[cfg.precision]
    g = lr.LrdmcSystem(system)
    g.set_precision(prec)
    sp = spacing_of(cfg, lr)
    aprime, rc = g.spacing_params(cfg.a, sp)
    x0 = S.initial_positions(system, cfg.walkers, cfg.start_seed)
    g.init_walkers(x0, seed=cfg.seed, tau=cfg.tau, e_trial=cfg.e_trial, recompute_every=cfg.recompute_every,
                   trace_capacity=cfg.intervals)
    t0 = time.perf_counter()
    g.step(cfg.intervals, cfg.a, sp)
    g.sync()
    seconds = time.perf_counter() - t0
    e, wbar, jumps = g.energy_trace(max_n=cfg.intervals)
    moves = g.moves()
    q = cfg.equilibration
    energy = stats.energy_estimate(e[q:], wbar[q:], cfg.mixed_L)
    error, _ = stats.reblock(e[q:])
    return {
        "system": system.name, "config": asdict(cfg), "aprime_over_a": aprime, "rc": rc,
        "energy_Ha": energy, "error_Ha": error, "intervals_used": int(len(e) - q),
        "walker_moves": int(moves), "seconds": seconds,
        "walker_moves_per_s": moves / seconds if seconds > 0 else None,
        "trace": {"e": np.asarray(e).tolist(), "wbar": np.asarray(wbar).tolist(),
                  "mean_jumps": np.asarray(jumps).tolist()},
    }


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--system", help="system JSON (lrdmc_synth.system_to_dict)")
    ap.add_argument("--run", help="run JSON (RunConfig)")
    ap.add_argument("--out", help="result JSON (default: standard output)")
    ap.add_argument("--dump-system", metavar="NAME",
                    help="write the synthetic system NAME (He, Ne, Ar, Kr, H2O, ...) as JSON and exit")
    args = ap.parse_args(argv)
    import lrdmc_synth as S

    if args.dump_system:
        if args.dump_system not in S.SYSTEMS:
            ap.error(f"unknown system {args.dump_system}; one of {sorted(S.SYSTEMS)}")
        text = json.dumps(S.system_to_dict(S.make_system(args.dump_system)), indent=1)
    else:
        if not (args.system and args.run):
            ap.error("--system and --run are needed (or --dump-system)")
        system = S.load_system(args.system)
        with open(args.run) as f:
            cfg = parse_run(json.load(f))
        text = json.dumps(run(system, cfg))
    if args.out:
        with open(args.out, "w") as f:
            f.write(text + "\n")
    else:
        print(text)


if __name__ == "__main__":
    main()
