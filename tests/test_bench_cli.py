"""CPU checks of bench.py's contract: the reference arm (the oracle timed on
the host cores) prints one JSON line with the keys the contract names, the
warm-up floor is enforced, and the clock samples are summarised as the
timing rules read them (median SM clock, throttle reasons)."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench(*args, timeout=600):
    return subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), *args], capture_output=True, text=True,
                          timeout=timeout, cwd=ROOT)


def test_reference_arm_prints_one_contract_line():
    r = _bench("--impl", "reference", "--steps", "1", "--warmup", "3")
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.strip().startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["unit"] == "walker-moves/s" and d["value"] > 0
    assert d["n_gpus"] == 1 and d["steps"] == 1 and d["warmup"] == 3 and d["higher_is_better"] is True
    assert d["ms_per_step"] > 0 and d["dtype"] == "f64" and d["data"] == "synthetic"
    assert d["config"]["n_walkers"] == 4096 and d["config"]["system"] == "Ne" and "workload" in d["config"]
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and cb["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}


def test_warmup_floor_is_enforced():
    r = _bench("--impl", "reference", "--steps", "1", "--warmup", "2", timeout=120)
    assert r.returncode != 0 and "--warmup must be >= 3" in r.stderr


def test_clock_summary_reads_median_and_reasons(tmp_path):
    sys.path.insert(0, ROOT)
    import bench

    path = tmp_path / "clocks_rank0.csv"
    rows = [
        "0, 2070, 2070, 900.1, 0x0, Not Active, Not Active, Not Active, Not Active",
        "0, 2055, 2070, 1200.4, 0x4, Not Active, Not Active, Not Active, Active",
        "0, 1980, 2070, 1390.0, 0x4, Not Active, Not Active, Not Active, Active",
        "garbled line",
        "0, [N/A], 2070, 0, 0x0, Not Active, Not Active, Not Active, Not Active",
    ]
    path.write_text("\n".join(rows) + "\n")
    clk = bench.ClockSampler(0, str(tmp_path / "clocks_rank{rank}.csv"))
    assert clk.path == str(path)
    clk.proc = object()  # as if nvidia-smi had run
    s = clk.summary()
    assert s["sm_mhz"] == 2055.0 and s["sm_max_mhz"] == 2070.0 and s["samples"] == 3
    assert s["reasons"] == ["sw_power_cap"]
    rows[2] = "0, 1500, 2070, 1390.0, 0x8, Not Active, Active, Not Active, Not Active"
    path.write_text("\n".join(rows) + "\n")
    assert clk.summary()["reasons"] == ["hw_thermal_slowdown", "sw_power_cap"]


def test_clock_sampler_defaults_to_a_temporary_file():
    sys.path.insert(0, ROOT)
    import tempfile

    import bench

    clk = bench.ClockSampler(3)
    assert clk.path.startswith(tempfile.gettempdir()) and "rank3" in clk.path
    with pytest.raises(AttributeError):
        clk.f  # nothing opened before the timed region starts


def test_roofline_reproduces_by_hand():
    """The bench line's roofline from the method's work: Ne on the double
    grid counts 20 253 arithmetic operations, 1430 square roots, 1400
    divisions and 502 exponentials per walker-move; at 8.6, 5.7 and 16.0
    DFMA-equivalents for sqrt, division and exp that is 97 126 FP64-equivalent
    flops. A launch of 34 058 walker-moves in 1.373 ms then achieves
    97 126 x 34 058 / 1.373 ms = 2.409 TFLOP/s, 1.91 of the 1.259 TFLOP/s FP64
    pipe (152 SMs x 2 DFMA/clk x 2 flop x 2.07 GHz)."""
    import bench
    import lrdmc_synth as S

    ne = S.neon()
    assert bench.method_ops_per_move(ne, 2) == {"arith": 20253, "sqrt": 1430, "div": 1400, "exp": 502}
    flops = 2 * (20253 + 8.6 * 1430 + 5.7 * 1400 + 16.0 * 502)
    assert abs(flops - 97126) < 0.5 and abs(2 * bench.dfma_equiv_per_move(ne, 2) - flops) < 1e-6
    assert abs(bench.FP64_PEAK_TFLOPS - 152 * 2 * 2 * 2.07e9 / 1e12) < 1e-3
    leg = {"t_int_ms": 10 * 1.373, "n_int": 10, "moves": 10 * 34058}
    r = bench.roofline(ne, 2, "df64", leg)
    assert abs(r["achieved"] - flops * 34058 / 1.373e-3 / 1e12) < 1e-9
    assert abs(r["achieved"] - 2.409) < 1e-3 and abs(r["frac"] - 2.409 / 1.259) < 1e-3
    assert r["bound"] == "alu" and r["peak"] == bench.FP64_PEAK_TFLOPS

