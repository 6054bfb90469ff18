"""LRDMC throughput benchmark: walker-moves/s of the GB300 FP64 path.

Workload: all-electron Ne (Z = 10, 5 up / 5 down), Slater-Jastrow trial
function, 4096 walkers, lattice spacing a = 0.2 bohr with the paper's
double grid (Gaussian p of Eq. 3, r_c from S-13, a'/a from Eq. 6/7),
tau = 0.025 Ha^-1 per reconfiguration interval, FP64. One step = one
interval: for every walker the continuous-time loop of waiting time,
heat-bath jump, Sherman-Morrison update, new lattice rotation and
evaluation of all 12 N = 120 lattice moves and the local energy, then comb
reconfiguration of the population.

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
                tau=0.025, e_trial=-128.9, recompute_every=5, precision="fp64")
SEED = 2024
L2_FLUSH_BYTES = 512 << 20

# FP64 pipe cost of the special functions on this GPU, in DFMA-equivalents:
# DFMA rate / measured rate of each function (0.505e12 DFMA/s; sqrt 58.6e9/s,
# reciprocal 89.3e9/s, exp 31.6e9/s, measured with csrc/fp64_rates.cu).
C_SQRT, C_DIV, C_EXP = 8.6, 5.7, 16.0
FP64_PEAK_TFLOPS = 1.259  # 152 SMs x 2 DFMA/clk x 2 flop x 2.07 GHz (nominal 1.25 TF)


def dfma_equiv_per_move(system, G):
    """Algorithmic FP64 work of one walker-move (one jump plus one evaluation
    of all P = 6 G N lattice moves and of the local energy), in DFMA
    equivalents: adds, multiplies and FMAs count 1, sqrt/div/exp their
    measured cost. Counted from the formulas, not from the kernels' code."""
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
    pair = 6 + C_SQRT + 2 + C_DIV + 2  # distance, Pade term
    per_cand = (3 + centers * (6 + C_SQRT) + exps * (1 + C_EXP) + 2 * n_ao
                + (N - 1 + n_nuc) * pair + 2 + C_EXP + 2
                + ((3 + n_nuc * 6 + C_EXP + 2) if G == 2 else 0))
    el = N * (centers * (6 + C_SQRT) + exps * (1 + C_EXP) + 12 * n_ao
              + (N - 1 + n_nuc) * (pair + C_DIV + 12)) + N * n_ao * nsig
    sm = n_ao * 8 + exps * C_EXP + n_ao * nsig + nsig * nsig + 2 * nsig * nsig
    scan = 2 * P
    return P * per_cand + el + sm + scan


def _env_rank():
    return int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")), \
        int(os.environ.get("LOCAL_RANK", "0"))


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = os.path.join(ROOT, "gpurun_out", f"clocks_bench_rank{gpu_index}.csv")

    def __enter__(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
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


def run_ours(args):
    import torch

    import paper_1909_01589_gb300 as pkg

    rank, world, local = _env_rank()
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    system = S.neon()
    W = args.walkers
    spacing = pkg.Spacing(pkg.THIS_WORK)
    a = WORKLOAD["a"]
    seed = SEED + 7919 * rank
    x0 = S.initial_positions(system, W, seed)
    prec = pkg.PRECISION_DF64 if args.precision == "df64" else pkg.PRECISION_FP64
    g = pkg.LrdmcSystem(system).set_precision(prec)
    cap = args.warmup + args.steps + 8
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
    step_ms = []
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    stops = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        t_wall0 = time.perf_counter()
        for k in range(args.steps):
            flush.zero_()  # L2 flush between timed steps (outside the events)
            starts[k].record(stream)
            g.step(1, a, spacing)
            stops[k].record(stream)
        g.sync()
        torch.cuda.synchronize()
        t_wall = time.perf_counter() - t_wall0
    if dist is not None:
        dist.barrier()
    step_ms = [s.elapsed_time(e) for s, e in zip(starts, stops)]
    moves = g.moves() - m0
    t_int_ms, t_rec_ms, n_int, n_rec = g.kernel_times()
    total_ms = float(sum(step_ms))
    local_rate = moves / (total_ms * 1e-3)
    # e2e: the public API from host memory: H2D of the start configurations,
    # init, the same K steps, each followed by a D2H read of the trace.
    x0h = torch.tensor(x0).pin_memory()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    g2 = pkg.LrdmcSystem(system).set_precision(prec)
    g2.init_walkers(x0h.numpy(), seed=seed, tau=WORKLOAD["tau"], e_trial=WORKLOAD["e_trial"],
                    recompute_every=WORKLOAD["recompute_every"], trace_capacity=cap)
    d2h = 0
    for k in range(args.warmup + args.steps):
        g2.step(1, a, spacing)
        e_tr, _, _ = g2.energy_trace(max_n=k + 1)
        d2h += 3 * 8 * (k + 1)
    e2e_moves = g2.moves()
    torch.cuda.synchronize()
    t_e2e = time.perf_counter() - t0
    n_e2e = args.warmup + args.steps
    e2e_rate = e2e_moves / t_e2e
    e_trace, w_trace, j_trace = g.energy_trace()
    if dist is not None:
        t = torch.tensor([total_ms, float(moves), t_e2e, float(e2e_moves)], dtype=torch.float64, device=dev)
        gathered = [torch.zeros_like(t) for _ in range(world)]
        dist.all_gather(gathered, t)
        gathered = torch.stack(gathered).cpu().numpy()
        total_ms = float(gathered[:, 0].max())
        moves_all = float(gathered[:, 1].sum())
        t_e2e_all = float(gathered[:, 2].max())
        e2e_all = float(gathered[:, 3].sum())
    else:
        moves_all, t_e2e_all, e2e_all = float(moves), t_e2e, float(e2e_moves)
    value = moves_all / (total_ms * 1e-3)
    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return
    G = 2
    flop_per_move = 2.0 * dfma_equiv_per_move(system, G)
    moves_per_launch = moves / max(n_int, 1)
    achieved_tflops = flop_per_move * moves_per_launch / (t_int_ms / max(n_int, 1) * 1e-3) / 1e12
    traffic = _read_traffic()
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
        "dtype": "f32x2 (double-float evaluation) + f64 state" if args.precision == "df64" else "f64",
        "data": "synthetic",
        "config": {"workload": "Ne all-electron, 4096 walkers, a=0.2 bohr, smart double grid (this work), "
                               "tau=0.025, FP64-parity arithmetic", **WORKLOAD, "evaluation": args.precision,
                   "walkers_per_gpu": W, "l2": "flushed between timed steps (512 MiB write)",
                   "parallelism": f"replicas x{world}"},
        "e2e": {"value": e2e_all / t_e2e_all, "unit": "walker-moves/s",
                "h2d_bytes_per_step": x0.nbytes / n_e2e, "d2h_bytes_per_step": d2h / n_e2e,
                "includes": "H2D of start configurations, init, warmup+timed steps, per-step trace D2H"},
        "gpu_launches": int(n_int + n_rec),
        "roofline": {"bound": "alu", "kernel": "k_interval", "achieved": achieved_tflops,
                     "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                     "frac": achieved_tflops / FP64_PEAK_TFLOPS,
                     "peak_source": "nominal FP64 (recipe: 1.25 TF = 152 SM x 2 DFMA/clk x 2 x 2.07 GHz); "
                                    "no FP64 entry in MEASURED_PEAKS.json",
                     "flop_per_move": flop_per_move, "kernel_ms_per_launch": t_int_ms / max(n_int, 1),
                     "traffic": traffic},
        "kernel_share": {"k_interval_ms": t_int_ms, "k_reconfig_ms": t_rec_ms},
        "mean_jumps_per_interval": float(np.mean(j_trace[-args.steps:])),
        "energy_mean_timed": float(np.mean(e_trace[-args.steps:])),
        "clocks": clk.summary(),
        "wall_s_timed": t_wall,
    }
    out["cpu_baseline"] = cpu_baseline(args) if args.cpu_seconds > 0 else None
    print(json.dumps(out), flush=True)
    if dist is not None:
        dist.destroy_process_group()


def _read_traffic():
    """dram bytes per k_interval launch from the committed ncu summary, if the
    kernel source has not changed since it was taken; else None."""
    path = os.path.join(ROOT, "profiles", "k_interval_ne4096_traffic.json")
    try:
        d = json.load(open(path))
    except (OSError, ValueError):
        return None
    import hashlib

    src = open(os.path.join(ROOT, "paper_1909_01589_gb300", "csrc", "lrdmc_kernels.cu"), "rb").read()
    if hashlib.sha256(src).hexdigest() != d.get("kernel_sha256"):
        return None
    return d.get("dram_bytes_per_launch")


def _oracle_rate(n_walkers, budget_s, threads):
    import oracle

    system = S.neon()
    o = oracle.OracleSystem(system)
    x0 = S.initial_positions(system, n_walkers, SEED)
    pop = oracle.OraclePopulation(o, x0, seed=SEED, tau=WORKLOAD["tau"], e_trial=WORKLOAD["e_trial"],
                                  recompute_every=WORKLOAD["recompute_every"])
    lat = oracle.lattice_for(system, WORKLOAD["a"], oracle.THIS_WORK)
    pop.step(lat, 1, threads)  # first evaluation and one interval, untimed
    m0 = pop.moves
    t0 = time.perf_counter()
    steps = 0
    while time.perf_counter() - t0 < budget_s:
        pop.step(lat, 1, threads)
        steps += 1
    dt = time.perf_counter() - t0
    return (pop.moves - m0) / dt, steps, dt


def cpu_baseline(args):
    threads = os.cpu_count() or 1
    W = 1024
    rate, steps, dt = _oracle_rate(W, args.cpu_seconds, threads)
    return {"value": rate, "unit": "walker-moves/s", "cores": threads, "kind": "oracle",
            "sample": f"Ne, {W} of the 4096 walkers, same a/tau/spacing, {steps} intervals in {dt:.1f} s, "
                      f"OpenMP over walkers"}


def run_reference(args):
    rank, world, _ = _env_rank()
    if rank != 0:
        return
    threads = os.cpu_count() or 1
    W = 1024
    _oracle_rate(W, 2.0, threads)  # warm-up
    rate, steps, dt = _oracle_rate(W, args.cpu_seconds, threads)
    out = {
        "impl": "reference", "metric": METRIC, "value": rate, "unit": "walker-moves/s", "n_gpus": world,
        "steps": steps, "warmup": args.warmup, "ms_per_step": dt * 1e3 / max(steps, 1),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": "Ne all-electron, 4096 walkers, a=0.2 bohr, smart double grid (this work), "
                               "tau=0.025, FP64", **WORKLOAD},
        "cpu_baseline": {"value": rate, "unit": "walker-moves/s", "cores": threads, "kind": "oracle",
                         "sample": f"Ne, {W} walkers per interval, {steps} intervals in {dt:.1f} s"},
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
    ap.add_argument("--precision", default="df64", choices=["df64", "fp64"],
                    help="evaluation arithmetic: double-float on the FP32 pipe or IEEE double")
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
