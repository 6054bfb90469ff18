"""Child process of test_gpu_bounds.py (test code). It runs with
LRDMC_LIBRARY pointing at the bounds-checked build, steps the tiny
populations that the test compares with the oracle and the default build,
loads a checkpoint with one parent index out of range, and prints one JSON
line with what it saw."""
import json
import os
import struct
import sys
import tempfile

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(HERE))
sys.path.insert(0, HERE)

import lrdmc_synth as S  # noqa: E402

# tiny populations: 8 walkers of 2 (He) and 4 (tiny_mixed) electrons
W, N_INT, A, TAU = 8, 6, 0.2, 0.05
CASES = [("He", 11), ("tiny_mixed", 12)]


def run_case(name, seed, precision, e_trial):
    """N_INT intervals of one population: trace and final positions."""
    import torch

    import paper_1909_01589_gb300 as pkg

    system = S.make_system(name)
    g = pkg.LrdmcSystem(system)
    g.set_precision(precision)
    x0 = S.initial_positions(system, W, seed)
    g.init_walkers(torch.tensor(x0, device="cuda"), seed=seed, tau=TAU, e_trial=e_trial, recompute_every=2,
                   trace_capacity=N_INT + 2)
    g.step(N_INT, A, pkg.Spacing(pkg.THIS_WORK))
    g.sync()
    e, w, j = g.energy_trace()
    return dict(e=e.tolist(), w=w.tolist(), j=j.tolist(), x=g.walkers()["x"].ravel().tolist())


def corrupt_parent(path, slot, value):
    """Overwrites parent index `slot` of a checkpoint written by lrdmc_save:
    the file ends with the W parents (int32), the 4 x cap trace (doubles)
    and the move count (uint64); W and cap are header words 1 and 3."""
    data = bytearray(open(path, "rb").read())
    w, cap = struct.unpack_from("<q", data, 8)[0], struct.unpack_from("<q", data, 24)[0]
    off = len(data) - 8 - 8 * 4 * cap - 4 * w
    struct.pack_into("<i", data, off + 4 * slot, value)
    open(path, "wb").write(bytes(data))


def bad_parent_case(precision, tmp):
    """A checkpoint whose parent of slot 3 is W (one past the population):
    loaded, then stepped; the status of the synchronising call."""
    import torch

    import paper_1909_01589_gb300 as pkg

    system = S.helium()
    g = pkg.LrdmcSystem(system)
    g.set_precision(precision)
    g.init_walkers(torch.tensor(S.initial_positions(system, W, 21), device="cuda"), seed=21, tau=TAU,
                   e_trial=-2.9, recompute_every=2, trace_capacity=8)
    sp = pkg.Spacing(pkg.THIS_WORK)
    g.step(2, A, sp)
    path = os.path.join(tmp, f"bad_{precision}.bin")
    g.save(path)
    corrupt_parent(path, 3, W)
    g.load(path)
    g.step(1, A, sp)
    try:
        g.sync()
        return dict(status=pkg.OK, message="")
    except pkg.LrdmcError as e:
        return dict(status=e.status, message=str(e))


def main():
    import paper_1909_01589_gb300 as pkg

    e_trials = json.loads(sys.argv[1])
    out = dict(flags=pkg.build_flags(), runs={}, bad_parent={})
    for name, seed in CASES:
        for prec in (pkg.PRECISION_FP64, pkg.PRECISION_DF64):
            out["runs"][f"{name}/{prec}"] = run_case(name, seed, prec, e_trials[name])
    with tempfile.TemporaryDirectory() as tmp:
        for prec in (pkg.PRECISION_FP64, pkg.PRECISION_DF64):
            out["bad_parent"][str(prec)] = bad_parent_case(prec, tmp)
    # the context is still usable after the reported error
    out["after"] = run_case("He", 31, pkg.PRECISION_DF64, e_trials["He"])["j"]
    print(json.dumps(out))


if __name__ == "__main__":
    main()
