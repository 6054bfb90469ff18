"""The tensor-core form of the orbital contraction (lrdmc_evaluate_tc):
basis values of every lattice move in FP32, split into bfloat16 high and low
parts, contracted with the MO coefficients by tcgen05 MMAs (FP32
accumulation in tensor memory). Checked against the FP64 oracle at the
mixed-precision mode's tolerance (2e-4 of each ratio's floating-point
scale; the measured error, about 1e-5, is recorded in the parity report),
and against the FP32 mode's projected-orbital evaluation: the same local
energies bit for bit (the same code computes them) and rates that differ
only by the bfloat16-split rounding."""
import numpy as np
import pytest

import lrdmc_synth as S
import _parity_util as U
from _parity_util import ratio_scale

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 2e-4


@pytest.fixture(scope="module")
def pkg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1909_01589_gb300 import build

    build.build()
    import paper_1909_01589_gb300 as p

    p.load_library()
    return p


def _lattice(pkg, oracle_mod, system, a):
    return pkg.Spacing(pkg.THIS_WORK), oracle_mod.lattice_for(system, a, oracle_mod.THIS_WORK)


CASES = [("He", 0.2), ("Ne", 0.2), ("Ar", 1 / 63), ("Kr", 1 / 126), ("H2O", 0.1), ("tiny_mixed", 0.3)]


@pytest.mark.parametrize("name,a", CASES)
def test_tc_evaluation_matches_oracle(pkg, oracle_mod, name, a):
    """37 configurations (nine blocks of four, a ragged last block), every
    ratio within TOL of its scale and every local energy within TOL
    relative of the oracle; local energies identical to the FP32 mode's,
    total rates within TOL of them."""
    system = S.make_system(name)
    g = pkg.LrdmcSystem(system).set_precision(pkg.PRECISION_FP32)
    o = oracle_mod.OracleSystem(system)
    n = 37
    x = torch.tensor(S.initial_positions(system, n, 131), device="cuda")
    R = torch.tensor(S.random_rotations(n, 132), device="cuda")
    sp, lat = _lattice(pkg, oracle_mod, system, a)
    ratio, T, b, el = (t.cpu().numpy() for t in g.evaluate_tc(x, R, a, sp))
    r32, T32, b32, el32 = (t.cpu().numpy() for t in g.evaluate(x, R, a, sp))
    assert np.array_equal(el, el32)
    assert np.all(np.abs(b - b32) <= TOL * b32)
    xs = x.cpu().numpy()
    Rs = R.cpu().numpy()
    worst_r = worst_e = 0.0
    for c in range(n):
        ref = o.lattice_eval(lat, xs[c], Rs[c])
        scale = ratio_scale(o, system, lat, xs[c], Rs[c], ref["ratio"])
        err = float(np.max(np.abs(ratio[c] - ref["ratio"]) / scale))
        worst_r = max(worst_r, err)
        worst_e = max(worst_e, abs(el[c] - ref["EL"]) / abs(ref["EL"]))
    U.record({"test": f"evaluate_tc {name} this_work a={a:.6g}", "kind": "evaluation (tensor-core contraction)",
              "configurations": n, "tolerance": TOL, "worst_ratio_scaled": worst_r, "worst_EL_rel": worst_e,
              "worst_b_rel_vs_fp32_mode": float(np.max(np.abs(b - b32) / b32))})
    assert worst_r < TOL and worst_e < TOL, (worst_r, worst_e)


def test_tc_evaluation_full_size_kr(pkg, oracle_mod):
    """The Kr workload at full size (16384 configurations, a = 1/(3.5 Z),
    this work's double grid): every rate finite and every total rate
    positive, 16 sampled configurations against the oracle."""
    system = S.krypton()
    g = pkg.LrdmcSystem(system).set_precision(pkg.PRECISION_FP32)
    o = oracle_mod.OracleSystem(system)
    n = 16384
    a = 1 / 126
    x = torch.tensor(S.initial_positions(system, n, 141), device="cuda")
    R = torch.tensor(S.random_rotations(n, 142), device="cuda")
    sp, lat = _lattice(pkg, oracle_mod, system, a)
    ratio, T, b, el = (t.cpu().numpy() for t in g.evaluate_tc(x, R, a, sp))
    assert np.all(np.isfinite(ratio)) and np.all(np.isfinite(el)) and np.all(b > 0)
    xs = x.cpu().numpy()
    Rs = R.cpu().numpy()
    for c in np.random.default_rng(5).choice(n, 16, replace=False):
        ref = o.lattice_eval(lat, xs[c], Rs[c])
        scale = ratio_scale(o, system, lat, xs[c], Rs[c], ref["ratio"])
        assert float(np.max(np.abs(ratio[c] - ref["ratio"]) / scale)) < TOL, c
        assert abs(el[c] - ref["EL"]) < TOL * abs(ref["EL"]), c


def test_tc_rejects_what_does_not_fit(pkg):
    """More than 32 orbitals per spin cannot use the 32-column accumulator:
    rejected with LRDMC_ERR_ARG before any GPU work."""
    system = S.cluster(8, 24, 2)  # 24 orbitals per spin, 42 AOs: tiles do not fit beside its block
    g = pkg.LrdmcSystem(system)
    x = torch.tensor(S.initial_positions(system, 4, 1), device="cuda")
    R = torch.tensor(S.random_rotations(4, 2), device="cuda")
    with pytest.raises(pkg.LrdmcError) as e:
        g.evaluate_tc(x, R, 0.3, pkg.Spacing(pkg.THIS_WORK))
    assert e.value.status == pkg.ERR_ARG
