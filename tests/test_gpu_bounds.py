"""The bounds-checked build (liblrdmc_bounds.so, -DLRDMC_BOUNDS) on tiny
populations of 8 walkers with 2 and 4 electrons. Its trajectories match the
oracle and the default build. A checkpoint whose parent index is one past
the population is rejected by the default build on the host; the
bounds-checked build leaves it to the kernels, whose checks report
LRDMC_ERR_BOUNDS and keep the access inside the record array (the index
becomes 0), after which the context still works. The bounds-checked build
runs in a child process (tests/_bounds_case.py) with LRDMC_LIBRARY set."""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

import lrdmc_synth as S
from _bounds_case import CASES, TAU, A, W, N_INT, corrupt_parent, run_case

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)


@pytest.fixture(scope="module")
def pkg():
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    from paper_1909_01589_gb300 import build

    build.build()
    import paper_1909_01589_gb300 as p

    p.load_library()
    return p


def _e_trial(oracle_mod, name, seed):
    """Mean local energy of the start configurations (oracle)."""
    system = S.make_system(name)
    osys = oracle_mod.OracleSystem(system)
    lat = oracle_mod.lattice_for(system, A, oracle_mod.THIS_WORK)
    x0 = S.initial_positions(system, W, seed)
    R = S.random_rotations(W, seed)
    return float(np.mean([osys.lattice_eval(lat, x0[c], R[c])["EL"] for c in range(W)]))


@pytest.fixture(scope="module")
def bounds_run(pkg, oracle_mod):
    from paper_1909_01589_gb300 import build

    lib = build.build(bounds=True)
    e_trials = {name: _e_trial(oracle_mod, name, seed) for name, seed in CASES}
    env = dict(os.environ, LRDMC_LIBRARY=lib)
    r = subprocess.run([sys.executable, os.path.join(HERE, "_bounds_case.py"), json.dumps(e_trials)], env=env,
                       cwd=ROOT, capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stderr[-4000:]
    return e_trials, json.loads(r.stdout.strip().splitlines()[-1])


def test_bounds_build_is_loaded_in_the_child(bounds_run, pkg):
    _, out = bounds_run
    assert out["flags"] == pkg.BUILD_BOUNDS
    if not os.environ.get("LRDMC_LIBRARY"):
        assert pkg.build_flags() == 0  # this process runs the default build


@pytest.mark.parametrize("name,seed", CASES)
def test_bounds_build_matches_oracle_and_default_build(bounds_run, pkg, oracle_mod, name, seed):
    e_trials, out = bounds_run
    system = S.make_system(name)
    osys = oracle_mod.OracleSystem(system)
    lat = oracle_mod.lattice_for(system, A, oracle_mod.THIS_WORK)
    x0 = S.initial_positions(system, W, seed)
    pop = oracle_mod.OraclePopulation(osys, x0, seed=seed, tau=TAU, e_trial=e_trials[name], recompute_every=2)
    pop.step(lat, N_INT)
    e_ref, w_ref, j_ref = pop.trace()
    x_ref = pop.walkers(lat.G)["x"].ravel()
    for prec in (pkg.PRECISION_FP64, pkg.PRECISION_DF64):
        got = out["runs"][f"{name}/{prec}"]
        ref = run_case(name, seed, prec, e_trials[name])  # the default build, in this process
        # move counts exact; energies and weights within the parity bar
        assert np.array_equal(got["j"], j_ref[:N_INT]) and np.array_equal(got["j"], ref["j"])
        assert np.allclose(got["e"], e_ref[:N_INT], rtol=1e-10, atol=0), (prec, got["e"], e_ref)
        assert np.allclose(got["w"], w_ref[:N_INT], rtol=1e-10, atol=0), (prec, got["w"], w_ref)
        assert np.allclose(got["x"], x_ref, rtol=0, atol=1e-9)
        # the checks add no arithmetic: the default build's numbers to rounding
        assert np.allclose(got["e"], ref["e"], rtol=1e-12, atol=0)
        assert np.allclose(got["w"], ref["w"], rtol=1e-12, atol=0)
        assert np.allclose(got["x"], ref["x"], rtol=0, atol=1e-12)


def test_out_of_range_parent_is_reported_not_accessed(bounds_run, pkg):
    _, out = bounds_run
    for prec, r in out["bad_parent"].items():
        assert r["status"] == pkg.ERR_BOUNDS, (prec, r)
        assert "out of range" in r["message"]
    assert len(out["after"]) == N_INT  # a fresh system stepped after the error


def test_default_build_rejects_the_same_checkpoint_on_the_host(pkg, tmp_path):
    system = S.helium()
    g = pkg.LrdmcSystem(system)
    g.init_walkers(torch.tensor(S.initial_positions(system, W, 21), device="cuda"), seed=21, tau=TAU,
                   e_trial=-2.9, recompute_every=2, trace_capacity=8)
    g.step(2, A, pkg.Spacing(pkg.THIS_WORK))
    path = str(tmp_path / "bad.bin")
    g.save(path)
    corrupt_parent(path, 3, W)
    with pytest.raises(pkg.LrdmcError) as e:
        g.load(path)
    assert e.value.status == pkg.ERR_ARG and "parent" in str(e.value)
