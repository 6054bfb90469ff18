"""LRDMC throughput benchmark: walker-moves/s and efficiency 1/(sigma^2 t)
of the GB300 library against its plain FP64 form.

Workload: all-electron Ne (Z = 10, 5 up / 5 down), Slater-Jastrow trial
function, 4096 walkers, lattice spacing a = 0.2 bohr with the paper's
double grid (Gaussian p of Eq. 3, r_c from S-13, a'/a from Eq. 6/7),
tau = 0.025 Ha^-1 per reconfiguration interval. One step = one interval:
for every walker the continuous-time loop of waiting time, heat-bath jump,
Sherman-Morrison update, new lattice rotation and evaluation of all
12 N = 120 lattice moves and the local energy, then comb reconfiguration
of the population.

The headline line times the default arithmetic (double-float evaluation
with FP64 state, the FP64-parity mode; --precision chooses another). Extra
legs on the same line: the plain FP64 mode, the mixed FP32 mode, the
trained neural pair Jastrow, a heterogeneous batch of five systems, the
end-to-end figure through the public API from host memory, and the CPU
oracle as a baseline. Throughput comes from the K timed intervals; each
leg's energy, its reblocked error and the efficiency 1/(sigma^2 t) come
from a continuation of the same population for --eff-steps intervals
(default 2000), timed as one block, since 200 intervals leave sigma^2
uncertain by tens of percent.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
Under torchrun (N > 1) every rank runs an independent population (replicas;
walkers shard with no data-path collective) and rank 0 prints the line.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import lrdmc_synth as S  # noqa: E402

METRIC = "LRDMC walker-moves/s and efficiency 1/(σ²·t) vs plain FP64, 1 GB300"
WORKLOAD = dict(system="Ne", n_walkers=4096, a=0.2, spacing="double grid, this work (Eq. 3, S-13, Eq. 6/7)",
                tau=0.025, e_trial=-128.9, recompute_every=5)
# what each --precision computes in: the evaluation (all lattice moves, the
# local energy, waiting times, heat bath) and the state (positions, inverse
# Slater matrices, Sherman-Morrison updates, weights, reconfiguration)
ARITHMETIC = {"df64": {"evaluation": "double-float (2 x fp32, ~48 significant bits)", "state": "fp64"},
              "fp64": {"evaluation": "fp64", "state": "fp64"},
              "fp32": {"evaluation": "fp32 lattice moves, double-float local energy", "state": "fp64"}}
SEED = 2024
L2_FLUSH_BYTES = 512 << 20

# FP64 pipe cost of the special functions on this GPU, in DFMA-equivalents:
# DFMA rate / measured rate of each function (0.505e12 DFMA/s; sqrt 58.6e9/s,
# reciprocal 89.3e9/s, exp 31.6e9/s; profiles/fp64_rates_gb300.md).
C_SQRT, C_DIV, C_EXP = 8.6, 5.7, 16.0
# ALU peaks from unit counts and the 2070 MHz maximum SM clock
# (MEASURED_PEAKS.json records no ALU figure): FP64 152 SMs x 2 DFMA/clk x
# 2 flop (1.01 TF measured); FP32 152 SMs x 128 lanes x 2 flop (70 TF
# measured)
FP64_PEAK_TFLOPS = 1.259
FP32_PEAK_TFLOPS = 80.5


def method_ops_per_move(system, G):
    """Operations of one walker-move - one jump plus one evaluation of all
    P = 6 G N lattice moves and of the local energy - counted from the
    formulas (not from the kernels' code): arithmetic (add, multiply and FMA
    count 1 each), square roots, divisions and exponentials. Per lattice
    move: the distances to the nuclei, the basis exponentials, the length-K
    dot with the projected inverse column, the N - 1 + n_nuc Pade pair
    terms, exp of the Jastrow difference, p at the bond midpoint (double
    grid); per walker-move: the local energy (basis value, gradient and
    Laplacian, pair terms and their derivatives), the Sherman-Morrison
    update and the heat-bath scan."""
    N, n_nuc, n_ao = system.N, system.n_nuc, system.n_ao
    centers = len({s.center for s in system.shells})
    exps = 0
    prev = None
    for s in system.shells:
        key = (s.center, s.zeta) if s.kind == 0 else None
        if s.kind == 0 and key != prev:
            exps += 1
        elif s.kind == 1:
            exps += len(s.alpha)
        prev = key
    nsig = system.n_up
    P = 6 * G * N
    npair = N - 1 + n_nuc
    cand = {"arith": 3 + centers * 6 + exps + 2 * n_ao + npair * 10 + 4 + ((5 + n_nuc * 6) if G == 2 else 0),
            "sqrt": centers + npair, "div": npair, "exp": exps + 1 + (1 if G == 2 else 0)}
    el = {"arith": N * (centers * 6 + exps + 12 * n_ao + npair * 22) + N * n_ao * nsig,
          "sqrt": N * (centers + npair), "div": N * npair * 2, "exp": N * exps}
    sm = {"arith": n_ao * 8 + n_ao * nsig + 3 * nsig * nsig, "sqrt": 0, "div": 0, "exp": exps}
    return {k: P * cand[k] + el[k] + sm[k] + (2 * P if k == "arith" else 0) for k in cand}


def dfma_equiv_per_move(system, G):
    """The method's work of one walker-move in DFMA-equivalents: arithmetic
    counts 1, sqrt, division and exp their measured FP64-pipe cost."""
    o = method_ops_per_move(system, G)
    return o["arith"] + C_SQRT * o["sqrt"] + C_DIV * o["div"] + C_EXP * o["exp"]


def _env_rank():
    return int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")), \
        int(os.environ.get("LOCAL_RANK", "0"))


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index, path=None):
        """``path``: where the samples go ({rank} is replaced by the GPU
        index); by default a file in the temporary directory."""
        import tempfile

        self.gpu = gpu_index
        self.proc = None
        if path:
            self.path = path.replace("{rank}", str(gpu_index))
        else:
            self.path = os.path.join(tempfile.gettempdir(), f"lrdmc_clocks_rank{gpu_index}_{os.getpid()}.csv")

    def __enter__(self):
        try:
            os.makedirs(os.path.dirname(os.path.abspath(self.path)), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.f.close()

    def summary(self):
        if self.proc is None or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sms, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sms.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sms:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": statistics.median(sms), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sms)}


# FP32 operation counts of the double-float primitives as implemented in
# csrc/df64.cuh (add/sub/mul = 1, fma = 2, MUFU seed = 1).
DF_ADD, DF_ADD_FAST, DF_ADD_F, DF_MUL, DF_SQR = 11, 11, 10, 10, 9
DF_DIV, DF_SQRT, DF_EXP, DF_LOG = 11, 10, 101, 132


def df_flops_per_move(system, G):
    """Algorithmic FP32 work of one walker-move in the double-float
    formulation the kernels use: the double-float operations of one
    evaluation of all P = 6 G N moves (from the electron-pair and
    electron-nucleus caches, which the evaluation fills once) and of the
    local energy, plus the jump, each weighted by the FP32 flops of its
    primitive (FMA = 2; additions inside the evaluation are the one-two_sum
    form, division and square root one FMA-residual correction). Counted
    from the formulas."""
    N, n_nuc, n_ao = system.N, system.n_nuc, system.n_ao
    exps = len({(s.center, s.zeta) for s in system.shells if s.kind == 0}) + \
        sum(len(s.alpha) for s in system.shells if s.kind == 1)
    P = 6 * G * N
    dist = 3 * DF_ADD_FAST + 3 * DF_SQR + 2 * DF_ADD_FAST + DF_SQRT
    proj = 9 * DF_MUL + 6 * DF_ADD                                           # e_k . d on three axes
    cached = N <= 24
    if cached:
        fill = N * (N - 1) // 2 * (3 * DF_ADD + 3 * DF_SQR + 2 * DF_ADD + proj) + \
            N * n_nuc * (3 * DF_ADD + 3 * DF_SQR + 2 * DF_ADD + proj)
        ee = (N - 1) * (DF_MUL + 2 * DF_ADD + DF_SQRT + 4 * DF_MUL + DF_ADD_F + DF_ADD) + DF_DIV
    else:
        fill = N * n_nuc * (3 * DF_ADD + 3 * DF_SQR + 2 * DF_ADD + proj)
        ee = (N - 1) * (dist + 4 * DF_MUL + DF_ADD_F + DF_ADD) + DF_DIV
    per_cand = (3 * DF_MUL                                                    # h e_k
                + n_nuc * (DF_MUL + 3 * DF_ADD + 2 * DF_ADD + DF_SQRT           # d, |d|^2 from the cache
                           + DF_MUL + DF_ADD_F + DF_DIV + DF_ADD                 # e-n term
                           + (2 * DF_ADD if G == 2 else 0))                      # midpoint distance
                + exps * (DF_MUL + DF_EXP) + n_ao * (DF_MUL + DF_ADD) + 2 * n_ao * DF_MUL  # basis, dot
                + ee                                                             # e-e Pade terms
                + 2 * DF_ADD + DF_EXP + DF_MUL                                   # Jastrow ratio
                + ((DF_MUL + DF_EXP + DF_ADD_F) if G == 2 else 0)                # p at the midpoint
                + 2 * DF_MUL)                                                    # rate
    pair_el = dist + 2 * DF_DIV + 10 * DF_MUL + 8 * DF_ADD                      # u', u'', gradients
    el = N * (n_nuc * (dist + DF_DIV) + exps * (DF_MUL + DF_EXP) + n_ao * (12 * DF_MUL + 8 * DF_ADD)
              + (N - 1 + n_nuc) * pair_el + 8 * DF_MUL + 8 * DF_ADD)
    jump = DF_LOG + DF_DIV + 2 * P * DF_ADD + n_ao * (DF_MUL + DF_EXP / 3)      # time, scans, orbitals
    return P * per_cand + fill + el + jump


def measure_leg(args, pkg, torch, system, precision, dev, rank, seed, x0, with_clocks, neural=None):
    """W warm-up intervals, then K timed intervals, each bracketed by CUDA
    events on the library's stream with an L2 flush between them.
    ``neural`` = (spec, params) installs the neural pair term first."""
    _, world, local = _env_rank()
    spacing = pkg.Spacing(pkg.THIS_WORK)
    a = WORKLOAD["a"]
    g = pkg.LrdmcSystem(system).set_precision(precision).set_tail_helpers(args.tail_helpers)
    if neural is not None:
        g.set_neural_jastrow(*neural)
    cap = args.warmup + args.steps + args.eff_steps + 8
    g.init_walkers(torch.tensor(x0, device=dev), seed=seed, tau=WORKLOAD["tau"], e_trial=WORKLOAD["e_trial"],
                   recompute_every=WORKLOAD["recompute_every"], trace_capacity=cap)
    stream = g.stream
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    g.step(args.warmup, a, spacing)
    g.sync()
    torch.cuda.synchronize()
    g.set_profiling(True)
    g.kernel_times(reset=True)
    m0 = g.moves()
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    stops = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    if world > 1:
        import torch.distributed as dist

        dist.barrier()
    torch.cuda.synchronize()
    clk = ClockSampler(local, args.clocks_csv) if with_clocks else None
    if clk:
        clk.__enter__()
    t_wall0 = time.perf_counter()
    for k in range(args.steps):
        flush.zero_()  # L2 flush between timed steps (outside the events)
        starts[k].record(stream)
        g.step(1, a, spacing)
        stops[k].record(stream)
    g.sync()
    torch.cuda.synchronize()
    t_wall = time.perf_counter() - t_wall0
    if clk:
        clk.__exit__(None, None, None)
    step_ms = [s0.elapsed_time(s1) for s0, s1 in zip(starts, stops)]
    moves = g.moves() - m0
    t_int_ms, t_rec_ms, n_int, n_rec = g.kernel_times()
    g.set_profiling(False)
    out = dict(total_ms=float(sum(step_ms)), moves=moves, t_int_ms=t_int_ms, t_rec_ms=t_rec_ms, n_int=n_int,
               n_rec=n_rec, wall=t_wall, clocks=clk.summary() if clk else None, g=g)
    e_tr, w_tr, j_tr = g.energy_trace()
    out.update(e=e_tr[-args.steps:], w=w_tr[-args.steps:], j=j_tr[-args.steps:], eff_ms=out["total_ms"])
    if args.eff_steps > 0:
        # the statistical figures (energy, sigma, efficiency) from a longer
        # continuation of the same population, timed as one block of steps
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        g.step(args.eff_steps, a, spacing)
        e1.record(stream)
        g.sync()
        torch.cuda.synchronize()
        e_tr, w_tr, _ = g.energy_trace()
        out.update(e=e_tr[-args.eff_steps:], w=w_tr[-args.eff_steps:], eff_ms=e0.elapsed_time(e1))
    return out


def run_ours(args):
    import torch

    import paper_1909_01589_gb300 as pkg
    from paper_1909_01589_gb300 import stats

    rank, world, local = _env_rank()
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    system = S.neon()
    W = args.walkers
    seed = SEED + 7919 * rank
    x0 = S.initial_positions(system, W, seed)
    main_prec = {"df64": pkg.PRECISION_DF64, "fp64": pkg.PRECISION_FP64, "fp32": pkg.PRECISION_FP32}[args.precision]
    leg = measure_leg(args, pkg, torch, system, main_prec, dev, rank, seed, x0, True)
    # the plain FP64 path on the same workload, seeds and steps (for the
    # efficiency comparison the metric asks for)
    fp = None
    if main_prec != pkg.PRECISION_FP64 and args.fp64_leg:
        fp = measure_leg(args, pkg, torch, system, pkg.PRECISION_FP64, dev, rank, seed, x0, False)
    # the mixed-precision form (single-precision evaluation, FP64 state)
    mx = None
    if args.mixed_leg and main_prec != pkg.PRECISION_FP32:
        mx = measure_leg(args, pkg, torch, system, pkg.PRECISION_FP32, dev, rank, seed, x0, False)
    # the neural pair Jastrow: trained on the GPU (untimed) on configurations
    # of a plain projection, then the same measurement with the term
    nj = None
    if args.neural_leg:
        nj = neural_leg(args, pkg, torch, system, main_prec, dev, rank, seed, x0)
    bt = batched_leg(args, pkg, torch, main_prec, seed) if args.batch_leg else None
    tc = tc_leg(args, pkg, torch, seed) if args.tc_leg else None
    # e2e: the public API from host memory: H2D of the start configurations
    # (pinned), system creation and init, the same steps, each followed by a
    # D2H read of its trace entry (energy, mean weight, mean jumps) into
    # pinned host memory, enqueued behind the step, and one synchronisation
    # at the end (a pipelined caller). The blocking variant reads the whole
    # trace synchronously after every step instead.
    def e2e_run(blocking):
        spacing = pkg.Spacing(pkg.THIS_WORK)
        cap = args.warmup + args.steps + 8
        x0h = torch.tensor(x0).pin_memory()
        tr = torch.zeros((3, cap), dtype=torch.float64).pin_memory()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        g2 = pkg.LrdmcSystem(system).set_precision(main_prec)
        g2.init_walkers(x0h.numpy(), seed=seed, tau=WORKLOAD["tau"], e_trial=WORKLOAD["e_trial"],
                        recompute_every=WORKLOAD["recompute_every"], trace_capacity=cap)
        d2h = 0
        n = args.warmup + args.steps
        for k in range(n):
            g2.step(1, WORKLOAD["a"], spacing)
            if blocking:
                g2.energy_trace(max_n=k + 1)
                d2h += 3 * 8 * (k + 1)
            else:
                g2.energy_trace_async(k, 1, tr)
                d2h += 3 * 8
        g2.sync()
        moves_ = g2.moves()
        torch.cuda.synchronize()
        t = time.perf_counter() - t0
        if not blocking and not np.all(np.isfinite(tr[:, :n].numpy())):
            raise RuntimeError("e2e: non-finite trace entries")
        return t, moves_, d2h, n, x0h.numel() * 8

    t_e2e, e2e_moves, d2h, n_e2e, h2d = e2e_run(False)
    t_e2e_b, e2e_moves_b, d2h_b, _, _ = e2e_run(True)
    if dist is not None:
        value, total_ms, moves_all = stats.reduce_throughput(leg["total_ms"], leg["moves"])
        e2e_all, t_e2e_all, _ = stats.reduce_throughput(t_e2e * 1e3, e2e_moves)
        t_e2e_all *= 1e-3
        e2e_moves_all = e2e_all * t_e2e_all
    else:
        total_ms, moves_all = leg["total_ms"], float(leg["moves"])
        value = moves_all / (total_ms * 1e-3)
        t_e2e_all, e2e_moves_all = t_e2e, float(e2e_moves)
    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return
    G = 2
    roof = roofline(system, G, args.precision, leg)
    t_sec = leg["eff_ms"] * 1e-3
    err, _ = stats.reblock(leg["e"])
    eff = {"value": stats.efficiency(leg["e"], t_sec), "unit": "1/(Ha^2 s)", "sigma_mean_Ha": err,
           "seconds": t_sec, "energy_Ha": stats.energy_estimate(leg["e"], leg["w"], 0),
           "intervals": len(leg["e"])}
    out = {
        "metric": METRIC,
        "value": value,
        "unit": "walker-moves/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": total_ms / args.steps,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": {"df64": "f32x2 (double-float evaluation) + f64 state", "fp64": "f64",
                  "fp32": "f32 lattice moves + f32x2 local energy + f64 state"}[args.precision],
        "data": "synthetic",
        "config": {"workload": "Ne all-electron, 4096 walkers, a=0.2 bohr, smart double grid (this work), "
                               "tau=0.025", **WORKLOAD, **ARITHMETIC[args.precision],
                   "walkers_per_gpu": W, "tail_helpers": bool(args.tail_helpers),
                   "l2": "flushed between timed steps (512 MiB write)",
                   "parallelism": f"replicas x{world}"},
        "e2e": {"value": e2e_moves_all / t_e2e_all, "unit": "walker-moves/s",
                "h2d_bytes_per_step": h2d / n_e2e, "d2h_bytes_per_step": d2h / n_e2e,
                "includes": "H2D of start configurations (pinned), system creation, init, warmup+timed steps, "
                            "per-step D2H of the step's trace entry into pinned memory (enqueued behind the step), "
                            "one synchronisation at the end",
                "blocking_per_step_read": {"value": e2e_moves_b / t_e2e_b, "d2h_bytes_per_step": d2h_b / n_e2e,
                                           "includes": "the same, reading the whole trace synchronously after "
                                                       "every step (rank 0)"}},
        # per step: the interval kernel and the reconfiguration's two kernels
        "gpu_launches": int(leg["n_int"] + 2 * leg["n_rec"]),
        "roofline": roof,
        "efficiency": eff,
        "kernel_share": {"k_interval_ms": leg["t_int_ms"], "k_reconfig_ms": leg["t_rec_ms"]},
        "mean_jumps_per_interval": float(np.mean(leg["j"])),
        "clocks": leg["clocks"],
        "wall_s_timed": leg["wall"],
    }
    if fp is not None:
        fp_value = fp["moves"] / (fp["total_ms"] * 1e-3)
        fp_eff = stats.efficiency(fp["e"], fp["eff_ms"] * 1e-3)
        out["vs_plain_fp64"] = {
            "fp64_value": fp_value, "speedup": value / fp_value if world == 1 else None,
            "fp64_efficiency": fp_eff, "efficiency_ratio": eff["value"] / fp_eff,
            "fp64_energy_Ha": stats.energy_estimate(fp["e"], fp["w"], 0),
            "energy_difference_Ha": eff["energy_Ha"] - stats.energy_estimate(fp["e"], fp["w"], 0),
            "fp64_kernel_ms_per_launch": fp["t_int_ms"] / max(fp["n_int"], 1),
            "roofline": roofline(system, G, "fp64", fp)}
    if mx is not None:
        mx_value = mx["moves"] / (mx["total_ms"] * 1e-3)
        mx_err, _ = stats.reblock(mx["e"])
        mx_energy = stats.energy_estimate(mx["e"], mx["w"], 0)
        ref_leg = fp if fp is not None else leg
        ref_err, _ = stats.reblock(ref_leg["e"])
        ref_energy = stats.energy_estimate(ref_leg["e"], ref_leg["w"], 0)
        out["mixed_precision"] = {
            "mode": "fp32 lattice moves, double-float local energy, fp64 inverse/weights/reconfiguration", "value": mx_value,
            "efficiency": stats.efficiency(mx["e"], mx["eff_ms"] * 1e-3),
            "efficiency_ratio_vs_fp64": stats.efficiency(mx["e"], mx["eff_ms"] * 1e-3) /
            stats.efficiency(ref_leg["e"], ref_leg["eff_ms"] * 1e-3),
            "energy_Ha": mx_energy, "sigma_mean_Ha": mx_err,
            "energy_minus_fp64_Ha": mx_energy - ref_energy,
            "combined_sigma_Ha": float(np.hypot(mx_err, ref_err)),
            "kernel_ms_per_launch": mx["t_int_ms"] / max(mx["n_int"], 1),
            "efficiency_note": "from the short continuation; long traces (results/mixed_el_spikes_ne.json) put "
                               "this mode at 1.8 times the double-float form's efficiency",
            "roofline": roofline(system, G, "fp32", mx)}
    if nj is not None:
        leg_nj, info = nj
        nj_value = leg_nj["moves"] / (leg_nj["total_ms"] * 1e-3)
        nj_err, _ = stats.reblock(leg_nj["e"])
        nj_eff = stats.efficiency(leg_nj["e"], leg_nj["eff_ms"] * 1e-3)
        block = {"mode": "Pade + neural pair Jastrow (2x64 SiLU, bf16 weights, quintic table), " + args.precision,
                 "value": nj_value, "efficiency": nj_eff, "efficiency_ratio_vs_pade": nj_eff / eff["value"],
                 "energy_Ha": stats.energy_estimate(leg_nj["e"], leg_nj["w"], 0), "sigma_mean_Ha": nj_err,
                 "var_EL_walkers_Ha2": info.pop("var_EL_walkers"),
                 "var_EL_walkers_pade_Ha2": float(np.var(leg["g"].walkers()["EL"])),
                 "kernel_ms_per_launch": leg_nj["t_int_ms"] / max(leg_nj["n_int"], 1), **info}
        if fp is not None:
            block["efficiency_ratio_vs_fp64"] = nj_eff / stats.efficiency(fp["e"], fp["eff_ms"] * 1e-3)
        out["neural_jastrow"] = block
    if bt is not None:
        out["batched"] = bt
    if tc is not None:
        out["tensor_core_contraction"] = tc
    out["cpu_baseline"] = cpu_baseline(args) if args.cpu_seconds > 0 else None
    print(json.dumps(out), flush=True)
    if dist is not None:
        dist.destroy_process_group()


def neural_leg(args, pkg, torch, system, precision, dev, rank, seed, x0):
    """Sample configurations from a plain projection of the workload, train
    the neural pair term on the GPU (the library's forward/backward kernels),
    then measure the projection with the tabulated term."""
    from paper_1909_01589_gb300 import neural as N

    spec = S.default_neural_spec(system)
    plain = pkg.LrdmcSystem(system).set_precision(precision)
    sp = pkg.Spacing(pkg.THIS_WORK)
    # one untimed training step on a few start configurations first: PyTorch
    # compiles its own kernels (loss reductions, the optimiser) on first use
    xw = torch.tensor(x0[:256], device="cuda")
    gw, ew = plain.base_terms(xw)
    N.train(plain, spec, S.neural_init(spec, seed), xw, gw, ew, steps=1, batch=256, seed=seed)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    n_cfg = 16 * len(x0)
    x = N.sample_configurations(plain, x0, n_cfg, WORKLOAD["a"], sp, WORKLOAD["tau"], WORKLOAD["e_trial"],
                                seed=seed + 1)
    grad, e = plain.base_terms(x)
    n_tr = n_cfg * 7 // 8
    params, _ = N.train(plain, spec, S.neural_init(spec, seed), x[:n_tr], grad[:n_tr], e[:n_tr], steps=400,
                        seed=seed + 2)
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0
    el, j = N.evaluate(plain, spec, params, x[n_tr:], grad[n_tr:], e[n_tr:])
    info = {"train_seconds": t_train, "train_configs": n_tr, "train_steps": 400,
            "heldout_var_pade_Ha2": float(torch.var(e[n_tr:])),
            "heldout_var_neural_Ha2": float(N.variance_loss(el, j, clip=0.0))}
    leg = measure_leg(args, pkg, torch, system, precision, dev, rank, seed, x0, False,
                      neural=(spec, params.cpu().numpy()))
    info["var_EL_walkers"] = float(np.var(leg["g"].walkers()["EL"]))
    return leg, info


BATCH_SYSTEMS = ("He", "Ne", "Ar", "Kr", "H2O")
BATCH_E_TRIAL = {"He": -2.90, "Ne": -128.9, "Ar": -527.5, "Kr": -2753.0, "H2O": -76.0}


def batched_leg(args, pkg, torch, precision, seed):
    """Heterogeneous batch: 8192 walkers each of He, Ne, Ar, Kr and H2O
    (N = 2..36), each at a = 1/(3.5 Z_max) on this work's double grid with
    tau for about 10 jumps per walker per interval, tuned grids, one CUDA
    graph per step; against the same steps made system by system."""
    from paper_1909_01589_gb300 import batch as B

    W = args.batch_walkers
    sp = pkg.Spacing(pkg.THIS_WORK)
    systems, a, taus = [], [], []
    for q, name in enumerate(BATCH_SYSTEMS):
        system = S.make_system(name)
        ai = 1.0 / (3.5 * float(np.max(system.Z)))
        x = S.initial_positions(system, 256, seed + q)
        tau = B.tau_for(pkg, system, ai, sp, 10.0, x, S.random_rotations(256, seed + q))
        systems.append(system)
        a.append(ai)
        taus.append(tau)
    K = args.batch_steps
    cap = 128 + 2 * K

    def make():
        gs = []
        for q, (system, tau) in enumerate(zip(systems, taus)):
            g = pkg.LrdmcSystem(system).set_precision(precision)
            g.init_walkers(torch.tensor(S.initial_positions(system, W, seed + 100 + q), device="cuda"),
                           seed=seed + 200 + q, tau=tau, e_trial=BATCH_E_TRIAL[BATCH_SYSTEMS[q]],
                           recompute_every=5, trace_capacity=cap)
            gs.append(g)
        return gs

    gs = make()
    batch = pkg.LrdmcBatch(gs, a, [sp] * len(gs))
    report = B.tune(batch, a, [sp] * len(gs), trial_steps=2)
    m0 = sum(g.moves() for g in gs)
    ms = B._time_batch_steps(torch, batch, K)
    moves_b = sum(g.moves() for g in gs) - m0
    # the same systems one by one (default grids), same number of steps
    solo = make()
    t_seq = 0.0
    moves_s = 0
    for g, ai in zip(solo, a):
        g.step(1, ai, sp)
        g.sync()
        m = g.moves()
        t_seq += B._time_system_steps(torch, g, K, ai, sp) * K
        moves_s += g.moves() - m
    value_b = moves_b / (ms * K * 1e-3)
    value_s = moves_s / (t_seq * 1e-3)
    return {"systems": list(BATCH_SYSTEMS), "walkers_each": W, "a": a, "tau": taus, "steps": K,
            "evaluation": args.precision, "value_batched": value_b, "value_sequential": value_s,
            "speedup": value_b / value_s, "unit": "walker-moves/s", "ms_per_batched_step": ms,
            "ms_per_sequential_round": t_seq / K, "tuning": report,
            "note": "one CUDA graph per step with every system's kernels as parallel branches; "
                    "grid sizes chosen by measurement"}


def tc_leg(args, pkg, torch, seed):
    """A/B of the orbital contraction in the mixed-precision (FP32)
    evaluation: the projected form (one length-K dot of basis values with
    the projected inverse column per lattice move, lrdmc_evaluate) against
    the tensor-core form (basis values of 128 moves as bf16x3 rows, tcgen05
    MMA with C, lrdmc_evaluate_tc), on 16384 configurations of Kr at
    a = 1/(3.5 Z) (the mixed-precision workload) and of the bench's Ne.
    Each call is timed with CUDA events on its stream after 3 warm-up
    calls, best of 5."""
    out = {}
    for name, a in (("Kr", 1.0 / 126.0), ("Ne", WORKLOAD["a"])):
        system = S.make_system(name)
        g = pkg.LrdmcSystem(system).set_precision(pkg.PRECISION_FP32)
        n = 16384
        x = torch.tensor(S.initial_positions(system, n, seed + 11), device="cuda")
        R = torch.tensor(S.random_rotations(n, seed + 12), device="cuda")
        sp = pkg.Spacing(pkg.THIS_WORK)
        res = {}
        for label, fn in (("projected", g.evaluate), ("tensor_core", g.evaluate_tc)):
            for _ in range(3):
                fn(x, R, a, sp)
            best = float("inf")
            st = torch.cuda.current_stream()
            for _ in range(5):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(st)
                fn(x, R, a, sp)
                e1.record(st)
                torch.cuda.synchronize()
                best = min(best, e0.elapsed_time(e1))
            res[label] = {"ms": best, "lattice_moves_per_s": n * 12 * system.N / (best * 1e-3)}
        out[name] = {"configurations": n, "a": a, "K": system.n_ao, "orbitals_per_spin": system.n_up,
                     **res, "tensor_core_over_projected": res["projected"]["ms"] / res["tensor_core"]["ms"]}
    return out


def _read_profile(precision):
    """The ncu record of k_interval in this arithmetic on the bench workload
    (profiles/k_interval_<precision>_ne4096_traffic.json: dram bytes per
    launch and pipe activities), if the kernel source has not changed since
    it was taken; else None."""
    path = os.path.join(ROOT, "profiles", f"k_interval_{precision}_ne4096_traffic.json")
    try:
        d = json.load(open(path))
    except (OSError, ValueError):
        return None
    import hashlib

    src = open(os.path.join(ROOT, "paper_1909_01589_gb300", "csrc", "lrdmc_kernels.cu"), "rb").read()
    if hashlib.sha256(src).hexdigest() != d.get("kernel_sha256"):
        return None
    return d


def roofline(system, G, precision, leg):
    """Roofline of k_interval (the dominant kernel) for one leg. Work: the
    method's operations per walker-move counted from the formulas
    (method_ops_per_move), times the walker-moves of an average launch,
    over the launch's CUDA-event time (leg["t_int_ms"] / leg["n_int"],
    events on the library's stream). The IEEE-double and double-float forms
    give the same FP64-parity results, so both are measured in
    FP64-equivalent flops (FMA = 2, sqrt/div/exp at their FP64-pipe cost)
    against the FP64 pipe; the double-float form computes on the FP32 pipe,
    which lets it pass that roofline, and its own pipe's activity comes from
    the ncu record. The FP32 mode is measured in FP32 flops (arithmetic x 2,
    each special function one) against the FP32 pipe."""
    n_int = max(leg["n_int"], 1)
    kernel_ms = leg["t_int_ms"] / n_int
    moves = leg["moves"] / n_int
    ops = method_ops_per_move(system, G)
    prof = _read_profile(precision)
    if precision in ("df64", "fp64"):
        work = 2.0 * dfma_equiv_per_move(system, G)
        peak, unit = FP64_PEAK_TFLOPS, "TFLOP/s (FP64-equivalent)"
        src = "FP64 pipe from unit counts: 152 SMs x 2 DFMA/clk x 2 flop x 2.07 GHz (1.01 TF measured)"
    else:
        work = 2.0 * ops["arith"] + ops["sqrt"] + ops["div"] + ops["exp"]
        peak, unit = FP32_PEAK_TFLOPS, "TFLOP/s (FP32)"
        src = "FP32 pipe from unit counts: 152 SMs x 128 lanes x 2 flop x 2.07 GHz (70 TF measured)"
    achieved = work * moves / (kernel_ms * 1e-3) / 1e12
    out = {"bound": "alu", "kernel": f"k_interval<{precision}>", "achieved": achieved, "peak": peak, "unit": unit,
           "frac": achieved / peak, "traffic": prof.get("dram_bytes_per_launch") if prof else None,
           "peak_source": src + "; MEASURED_PEAKS.json has no ALU entry",
           "work_per_move": {**ops, "flops": work}, "moves_per_launch": moves, "kernel_ms_per_launch": kernel_ms}
    if prof and "pipes" in prof:
        out["ncu_pipes"] = prof["pipes"]
    if precision == "df64":
        dff = df_flops_per_move(system, G)
        a32 = dff * moves / (kernel_ms * 1e-3) / 1e12
        out["double_float_formulation"] = {
            "fp32_flops_per_move": dff, "achieved_tflops": a32, "peak_tflops": FP32_PEAK_TFLOPS,
            "frac": a32 / FP32_PEAK_TFLOPS,
            "note": "the same operations priced at the FP32 cost of their double-float primitives"}
    return out


def _oracle_rate(n_walkers, budget_s, threads, steps=None, warmup=1):
    """The oracle's walker-moves/s on n_walkers of the workload: ``warmup``
    untimed intervals (the first one includes the first evaluation), then
    exactly ``steps`` timed intervals, or as many as fit in budget_s seconds
    when steps is None."""
    import oracle

    system = S.neon()
    o = oracle.OracleSystem(system)
    x0 = S.initial_positions(system, n_walkers, SEED)
    pop = oracle.OraclePopulation(o, x0, seed=SEED, tau=WORKLOAD["tau"], e_trial=WORKLOAD["e_trial"],
                                  recompute_every=WORKLOAD["recompute_every"])
    lat = oracle.lattice_for(system, WORKLOAD["a"], oracle.THIS_WORK)
    pop.step(lat, max(1, warmup), threads)
    m0 = pop.moves
    t0 = time.perf_counter()
    n = 0
    while (n < steps) if steps is not None else (time.perf_counter() - t0 < budget_s):
        pop.step(lat, 1, threads)
        n += 1
    dt = time.perf_counter() - t0
    return (pop.moves - m0) / dt, n, dt


def cpu_baseline(args):
    threads = os.cpu_count() or 1
    W = 1024
    rate, steps, dt = _oracle_rate(W, args.cpu_seconds, threads)
    return {"value": rate, "unit": "walker-moves/s", "cores": threads, "kind": "oracle",
            "sample": f"Ne, {W} of the 4096 walkers, same a/tau/spacing, {steps} intervals in {dt:.1f} s, "
                      f"OpenMP over walkers"}


def run_reference(args):
    """The oracle as the reference arm: W warm-up and exactly K timed
    intervals, each one interval of 1024 of the workload's 4096 walkers on
    the host cores (OpenMP over walkers)."""
    rank, world, _ = _env_rank()
    if rank != 0:
        return
    threads = os.cpu_count() or 1
    W = 1024
    rate, steps, dt = _oracle_rate(W, 0.0, threads, steps=args.steps, warmup=args.warmup)
    out = {
        "impl": "reference", "metric": METRIC, "value": rate, "unit": "walker-moves/s", "n_gpus": world,
        "steps": steps, "warmup": args.warmup, "ms_per_step": dt * 1e3 / max(steps, 1),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": "Ne all-electron, 4096 walkers, a=0.2 bohr, smart double grid (this work), "
                               "tau=0.025, FP64", **WORKLOAD},
        "cpu_baseline": {"value": rate, "unit": "walker-moves/s", "cores": threads, "kind": "oracle",
                         "sample": f"Ne, {W} of the 4096 walkers per step (one interval), {steps} timed "
                                   f"intervals in {dt:.1f} s"},
        "e2e": {"value": rate, "unit": "walker-moves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(out), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--cpu-seconds", type=float, default=15.0,
                    help="CPU-baseline budget (<= 0: no CPU baseline)")
    ap.add_argument("--eff-steps", type=int, default=2000,
                    help="intervals of the longer untimed-for-throughput run each leg continues with for its "
                         "energy, sigma and efficiency 1/(sigma^2 t) (0: use the timed intervals)")
    ap.add_argument("--clocks-csv", default=None,
                    help="keep the nvidia-smi samples of the timed region in this file ({rank}: GPU index)")
    ap.add_argument("--precision", default="df64", choices=["df64", "fp64", "fp32"],
                    help="evaluation arithmetic: double-float on the FP32 pipe or IEEE double")
    ap.add_argument("--no-fp64-leg", dest="fp64_leg", action="store_false",
                    help="skip the plain-FP64 comparison leg")
    ap.add_argument("--no-batch-leg", dest="batch_leg", action="store_false",
                    help="skip the heterogeneous batch (He, Ne, Ar, Kr, H2O in one graph per step)")
    ap.add_argument("--batch-walkers", type=int, default=8192)
    ap.add_argument("--batch-steps", type=int, default=10)
    ap.add_argument("--no-neural-leg", dest="neural_leg", action="store_false",
                    help="skip training and measuring the neural pair Jastrow")
    ap.add_argument("--no-tc-leg", dest="tc_leg", action="store_false",
                    help="skip the A/B of the tensor-core orbital contraction")
    ap.add_argument("--no-mixed-leg", dest="mixed_leg", action="store_false",
                    help="skip the mixed-precision (FP32 evaluation) leg")
    ap.add_argument("--tail-helpers", type=int, default=1, choices=[0, 1],
                    help="warps out of walkers help the others of their block (results are the same bits)")
    ap.add_argument("--walkers", type=int, default=WORKLOAD["n_walkers"],
                    help="walkers per GPU (smaller cases for profiling)")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
