"""Tail helpers of the interval kernel: warps that run out of walkers take
chunks of the lattice moves of walkers other warps of their block still run.
Which warp computes which move depends on timing, so the results must not:
projections with the helpers on and off are compared bit for bit, in the
double-float and FP32 modes, on populations small enough that most warps
are helpers most of the time, on one large enough for blocks of 16 warps,
and on a heavy atom whose evaluations span many chunks."""
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


CASES = [  # name, walkers, a, tau, e_trial, intervals
    ("He", 300, 0.2, 0.05, -2.9, 6),
    ("Ne", 700, 0.2, 0.025, -128.9, 4),
    ("Ne", 4096, 0.2, 0.025, -128.9, 3),
    ("H2O", 200, 0.1, 0.01, -76.0, 3),
    ("Kr", 24, 1 / 126, 3e-5, -2752.0, 2),
]


def _run(pkg, name, W, a, tau, et, n, prec, helpers, blocks=0):
    system = S.make_system(name)
    g = pkg.LrdmcSystem(system).set_precision(prec).set_tail_helpers(helpers)
    if blocks:
        g.set_interval_blocks(blocks)
    g.init_walkers(torch.tensor(S.initial_positions(system, W, 61), device="cuda"), seed=62, tau=tau,
                   e_trial=et, recompute_every=3, trace_capacity=n)
    g.step(n, a, pkg.Spacing(pkg.THIS_WORK))
    w = g.walkers()
    e, wb, j = g.energy_trace()
    return w, e, wb, j, g.moves()


def _same(off, on):
    for key in ("x", "EL", "b", "T", "logw_pre", "jumps_pre", "parent"):
        assert np.array_equal(off[0][key], on[0][key]), key
    for q in (1, 2, 3):
        assert np.array_equal(off[q], on[q])
    assert off[4] == on[4]


@pytest.mark.parametrize("prec", ["df64", "fp32"])
@pytest.mark.parametrize("name,W,a,tau,et,n", CASES)
def test_helpers_do_not_change_results(pkg, name, W, a, tau, et, n, prec):
    p = pkg.PRECISION_DF64 if prec == "df64" else pkg.PRECISION_FP32
    _same(_run(pkg, name, W, a, tau, et, n, p, False), _run(pkg, name, W, a, tau, et, n, p, True))


def test_helpers_with_a_few_blocks(pkg):
    """Two blocks of four warps for 40 walkers: every warp runs several
    walkers and then helps; the result equals the run without helpers."""
    off = _run(pkg, "Ne", 40, 0.2, 0.025, -128.9, 3, pkg.PRECISION_DF64, False, blocks=2)
    on = _run(pkg, "Ne", 40, 0.2, 0.025, -128.9, 3, pkg.PRECISION_DF64, True, blocks=2)
    assert np.array_equal(off[0]["x"], on[0]["x"]) and np.array_equal(off[1], on[1])


def test_helpers_neural_and_no_cache_variants(pkg):
    """The kernel variants with the neural pair term (double-float) and
    without the evaluation caches (the 48-electron cluster): helpers on and
    off give the same bits."""
    system = S.neon()
    spec = S.default_neural_spec(system)
    params = S.neural_init(spec, 3, out_scale=0.5)
    runs = []
    for helpers in (False, True):
        g = pkg.LrdmcSystem(system).set_tail_helpers(helpers)
        g.set_neural_jastrow(spec, params)
        g.init_walkers(torch.tensor(S.initial_positions(system, 600, 71), device="cuda"), seed=72, tau=0.025,
                       e_trial=-128.9, recompute_every=3, trace_capacity=3)
        g.step(3, 0.2, pkg.Spacing(pkg.THIS_WORK))
        runs.append((g.walkers()["x"], g.energy_trace()[0]))
    assert np.array_equal(runs[0][0], runs[1][0]) and np.array_equal(runs[0][1], runs[1][1])
    system = S.cluster(8, 24, 2)
    runs = []
    for helpers in (False, True):
        g = pkg.LrdmcSystem(system).set_tail_helpers(helpers)
        g.init_walkers(torch.tensor(S.initial_positions(system, 40, 73), device="cuda"), seed=74, tau=0.002,
                       e_trial=40.0, recompute_every=3, trace_capacity=2)
        g.step(2, 0.3, pkg.Spacing(pkg.THIS_WORK))
        runs.append((g.walkers()["x"], g.energy_trace()[0]))
    assert np.array_equal(runs[0][0], runs[1][0]) and np.array_equal(runs[0][1], runs[1][1])
