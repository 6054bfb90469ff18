"""lrdmc_evaluate_static: the evaluation entry point that allocates no device
memory, for callers that cannot call cudaMalloc when they evaluate (code
inside another framework's reserved memory budget, processes that forbid
allocation after start-up). Its scratch is a static device array shared by
all calls. It must give the same results as lrdmc_evaluate, on consecutive
calls, whether it runs alone in a fresh process or after other tests."""
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


def test_static_evaluate_matches_allocating_evaluate(pkg):
    system = S.neon()
    g = pkg.LrdmcSystem(system)
    sp = pkg.Spacing(pkg.THIS_WORK)
    for call, (n, seed) in enumerate([(300, 41), (77, 42)]):  # two calls in a row
        x = torch.tensor(S.initial_positions(system, n, seed), device="cuda")
        R = torch.tensor(S.random_rotations(n, seed + 100), device="cuda")
        ref = [t.cpu().numpy() for t in g.evaluate(x, R, 0.2, sp)]
        got = [t.cpu().numpy() for t in g.evaluate_static(x, R, 0.2, sp)]
        # the two entry points run the same device body on the same inputs:
        # the results are the same bits
        for r, o in zip(ref, got):
            assert r.shape == o.shape
            assert np.array_equal(o, r), f"call {call}"


def test_static_evaluate_limits_and_errors(pkg):
    system = S.neon()
    g = pkg.LrdmcSystem(system)
    sp = pkg.Spacing(pkg.SINGLE)
    n = pkg.STATIC_EVAL_MAX + 1
    x = torch.zeros((n, system.N, 3), dtype=torch.float64, device="cuda")
    R = torch.zeros((n, 9), dtype=torch.float64, device="cuda")
    with pytest.raises(pkg.LrdmcError) as e:
        g.evaluate_static(x, R, 0.2, sp)
    assert e.value.status == pkg.ERR_ARG
    # a singular configuration is reported, and the next call starts clean
    xs = S.initial_positions(system, 5, 43)
    xs[2, 1] = xs[2, 0]
    Rs = torch.tensor(S.random_rotations(5, 44), device="cuda")
    with pytest.raises(pkg.LrdmcError) as e:
        g.evaluate_static(torch.tensor(xs, device="cuda"), Rs, 0.2, sp)
    assert e.value.status == pkg.ERR_SINGULAR
    assert "first at configuration 2" in str(e.value)
    ok = torch.tensor(S.initial_positions(system, 5, 45), device="cuda")
    g.evaluate_static(ok, Rs, 0.2, sp)
