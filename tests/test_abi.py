"""CPU checks of the C ABI: the library loads, exports every entry point the
header declares, validates its arguments and computes the double-grid
parameters (host logic) like the oracle."""
import ctypes as ct
import os
import re

import numpy as np
import pytest

import lrdmc_synth as S

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def pkg():
    from paper_1909_01589_gb300 import build

    build.build()
    import paper_1909_01589_gb300 as p

    p.load_library()
    return p


def declared_functions():
    text = open(os.path.join(ROOT, "include", "lrdmc.h")).read()
    return sorted(set(re.findall(r"LRDMC_API\s+[\w\s\*]+?\b(lrdmc_\w+)\s*\(", text)))


def test_every_declared_symbol_is_exported(pkg):
    names = declared_functions()
    assert len(names) >= 13
    lib = ct.CDLL(pkg.LIB_PATH)
    for n in names:
        assert hasattr(lib, n), n
    assert set(names) == set(pkg.EXPORTED)


def test_create_system_rejects_bad_sizes(pkg):
    s = S.neon()
    s.n_up, s.n_dn = 40, 5  # beyond LRDMC_MAX_SPIN
    with pytest.raises(pkg.LrdmcError) as e:
        pkg.LrdmcSystem(s)
    assert e.value.status == pkg.ERR_ARG
    s = S.neon()
    s.shells = s.shells[:-1]  # n_ao no longer matches C
    with pytest.raises(pkg.LrdmcError):
        pkg.LrdmcSystem(s)


def test_create_system_rejects_a_layout_beyond_shared_memory(pkg):
    """A block of four walkers of 64 electrons with 62 AOs needs more than
    227 KB of shared memory: rejected at creation with a message that says
    so. 48 electrons with 42 AOs fit (without the evaluation caches)."""
    with pytest.raises(pkg.LrdmcError) as e:
        pkg.LrdmcSystem(S.cluster(8, 32, 6))
    assert e.value.status == pkg.ERR_ARG and "shared memory" in str(e.value)
    pkg.LrdmcSystem(S.cluster(8, 24, 2))


def test_step_before_init_is_a_state_error(pkg):
    g = pkg.LrdmcSystem(S.helium())
    with pytest.raises(pkg.LrdmcError) as e:
        g.step(1, 0.2)
    assert e.value.status == pkg.ERR_STATE


@pytest.mark.parametrize("name,Z", [("He", 2), ("Ne", 10)])
@pytest.mark.parametrize("a", [0.4, 0.2, 0.1, 0.02857142857142857])
def test_spacing_params_match_oracle(pkg, oracle_mod, name, Z, a):
    """S-13, Eq. 6 and Eq. 7 in the library (Gauss-Legendre quadrature,
    its own Slater's-rule code) agree with the oracle (Simpson rule)."""
    s = S.make_system(name)
    g = pkg.LrdmcSystem(s)
    ratio, rc = g.spacing_params(a, pkg.Spacing(pkg.THIS_WORK))
    assert abs(rc - oracle_mod.rc_this_work(a, Z)) < 1e-15 * max(1, rc)
    q = oracle_mod.aprime_over_a_this_work(Z, a)
    assert abs(ratio - q) < 1e-11 * q
    r2, rc2 = g.spacing_params(a, pkg.Spacing(pkg.PREVIOUS))
    assert abs(r2 - oracle_mod.aprime_over_a_previous(Z)) < 1e-15 * r2 and rc2 == Z / 2
    r3, rc3 = g.spacing_params(a, pkg.Spacing(pkg.SINGLE))
    assert r3 == 1.0


@pytest.mark.parametrize("Z", [4, 18, 36, 54])
def test_spacing_params_heavier_atoms(pkg, oracle_mod, Z):
    s = S.hydrogenic_ion(Z)
    g = pkg.LrdmcSystem(s)
    a = 1.0 / (3.5 * Z)
    ratio, rc = g.spacing_params(a, pkg.Spacing(pkg.THIS_WORK))
    q = oracle_mod.aprime_over_a_this_work(Z, a)
    assert abs(ratio - q) < 1e-9 * q


def test_spacing_rejects_bad_arguments(pkg):
    g = pkg.LrdmcSystem(S.neon())
    with pytest.raises(pkg.LrdmcError):
        g.spacing_params(-0.1, pkg.Spacing(pkg.SINGLE))
    with pytest.raises(pkg.LrdmcError):
        g.spacing_params(0.1, pkg.Spacing(pkg.EXPLICIT, rc=0.0, aprime_over_a=2.0))
    with pytest.raises(pkg.LrdmcError):
        g.spacing_params(0.1, pkg.Spacing(7))


def test_workspace_bytes_grow_with_walkers(pkg):
    g = pkg.LrdmcSystem(S.neon())
    b1, b2 = g.workspace_bytes(100, 10), g.workspace_bytes(1000, 10)
    assert b2 > 9 * b1 / 2 and b1 % 256 == 0


def test_population_limit_matches_header(pkg):
    """LRDMC_MAX_WALKERS walkers are accepted, one more is LRDMC_ERR_ARG;
    the limit is read from the header."""
    hdr = open(os.path.join(os.path.dirname(__file__), "..", "include", "lrdmc.h")).read()
    limit = int(re.search(r"#define LRDMC_MAX_WALKERS (\d+)", hdr).group(1))
    g = pkg.LrdmcSystem(S.helium())
    assert g.workspace_bytes(limit, 4) > 0
    with pytest.raises(pkg.LrdmcError) as e:
        g.workspace_bytes(limit + 1, 4)
    assert e.value.status == pkg.ERR_ARG


def test_evaluate_argument_checks_before_the_library(pkg):
    """evaluate / evaluate_static refuse tensors the kernels would overrun
    or misread - wrong shape, dtype or device, a short output - with a
    ValueError, before any pointer reaches the library (checked here with
    CPU tensors, which both paths reject)."""
    torch = pytest.importorskip("torch")
    s = S.neon()
    g = pkg.LrdmcSystem(s)
    sp = pkg.Spacing(pkg.THIS_WORK)
    x = torch.zeros((4, s.N, 3), dtype=torch.float64)
    R = torch.zeros((4, 9), dtype=torch.float64)
    for fn in (g.evaluate, g.evaluate_static):
        with pytest.raises(ValueError):
            fn(x, R, 0.2, sp)  # not on a CUDA device
        with pytest.raises(ValueError):
            fn(torch.zeros((4, s.N + 1, 3), dtype=torch.float64), R, 0.2, sp)
        with pytest.raises(ValueError):
            fn(x, torch.zeros((3, 9), dtype=torch.float64), 0.2, sp)
        with pytest.raises(ValueError):
            fn(x.float(), R, 0.2, sp)
    P = 12 * s.N
    short = (torch.zeros((4, P - 1), dtype=torch.float64), torch.zeros((4, P), dtype=torch.float64),
             torch.zeros(4, dtype=torch.float64), torch.zeros(4, dtype=torch.float64))
    with pytest.raises(ValueError):
        g._eval_args(x, R, P, short)


def test_static_eval_limit_matches_header(pkg):
    """The binding's STATIC_EVAL_MAX is the header's LRDMC_STATIC_EVAL_MAX."""
    text = open(os.path.join(ROOT, "include", "lrdmc.h")).read()
    m = re.search(r"#define\s+LRDMC_STATIC_EVAL_MAX\s+(\d+)", text)
    assert m and int(m.group(1)) == pkg.STATIC_EVAL_MAX



def test_batch_binding_methods(pkg):
    """The batch binding's setters are methods and its stream a property."""
    for name in ("step", "sync", "set_groups", "set_carveout", "set_pipelined"):
        assert callable(getattr(pkg.LrdmcBatch, name)), name
    assert isinstance(pkg.LrdmcBatch.stream_ptr, property)


def test_set_tail_helpers_arguments(pkg):
    """The tail-helper switch takes 0 or 1; anything else is LRDMC_ERR_ARG."""
    g = pkg.LrdmcSystem(S.helium())
    g.set_tail_helpers(False).set_tail_helpers(True)
    with pytest.raises(pkg.LrdmcError) as e:
        g._check(pkg.load_library().lrdmc_set_tail_helpers(g.h, 2))
    assert e.value.status == pkg.ERR_ARG


def test_energy_trace_async_arguments(pkg):
    """The asynchronous trace read: before init_walkers it is a state error;
    the binding checks the host buffer's type and shape before the library."""
    g = pkg.LrdmcSystem(S.helium())
    out = np.zeros((3, 4))
    with pytest.raises(pkg.LrdmcError) as e:
        g.energy_trace_async(0, 1, out)
    assert e.value.status == pkg.ERR_STATE
    for bad in (np.zeros((3, 4), np.float32), np.zeros((2, 4)), np.zeros((4, 3)).T):
        with pytest.raises(ValueError):
            g.energy_trace_async(0, 1, bad)
    with pytest.raises(ValueError):
        g.energy_trace_async(3, 2, out)



def test_status_codes_match_header(pkg):
    text = open(os.path.join(ROOT, "include", "lrdmc.h")).read()
    codes = {m.group(1): int(m.group(2)) for m in re.finditer(r"LRDMC_(OK|ERR_\w+)\s*=\s*(\d+)", text)}
    assert codes == {"OK": pkg.OK, "ERR_ARG": pkg.ERR_ARG, "ERR_CUDA": pkg.ERR_CUDA,
                     "ERR_SINGULAR": pkg.ERR_SINGULAR, "ERR_NONFINITE": pkg.ERR_NONFINITE,
                     "ERR_TIMEOUT": pkg.ERR_TIMEOUT, "ERR_STATE": pkg.ERR_STATE, "ERR_BOUNDS": pkg.ERR_BOUNDS}
    assert int(re.search(r"#define LRDMC_BUILD_BOUNDS (\d+)", text).group(1)) == pkg.BUILD_BOUNDS


def test_bounds_checked_build_exports_the_same_abi(pkg):
    """liblrdmc_bounds.so (-DLRDMC_BOUNDS) exports every declared entry point
    and reports LRDMC_BUILD_BOUNDS; the default library reports no flag."""
    from paper_1909_01589_gb300 import build

    path = build.build(bounds=True)
    lib = ct.CDLL(path)
    for n in declared_functions():
        assert hasattr(lib, n), n
    lib.lrdmc_build_flags.restype = ct.c_int
    assert lib.lrdmc_build_flags() == pkg.BUILD_BOUNDS
    default = ct.CDLL(build.LIB)
    default.lrdmc_build_flags.restype = ct.c_int
    assert default.lrdmc_build_flags() == 0


def test_init_walkers_validates_start_positions_before_device_work(pkg):
    """Fault injection on the host: NaN start positions, a wrong shape and a
    wrong dtype are rejected before the library or the device is touched."""
    import torch

    system = S.helium()
    g = pkg.LrdmcSystem(system)
    x0 = S.initial_positions(system, 8, 1)
    bad = x0.copy()
    bad[3, 1, 2] = np.nan
    cases = [(bad, "finite"), (x0[:, :1], r"\[W\]\[2\]\[3\]"), (x0.reshape(8, 6), r"\[W\]\[2\]\[3\]"),
             (x0[:0], "W >= 1"), (x0.astype(np.int64), "floating point"),
             (torch.tensor(x0, dtype=torch.float32), "float64"), (torch.tensor(bad), "finite")]
    inf = x0.copy()
    inf[0, 0, 0] = np.inf
    cases.append((inf, "finite"))
    for x, msg in cases:
        with pytest.raises(ValueError, match=msg):
            g.init_walkers(x, seed=1, tau=0.02, e_trial=-2.9)
    assert g._ws is None  # nothing was allocated


def test_create_system_rejects_non_finite_or_unphysical_input(pkg):
    """Host validation before any allocation: NaN or infinite coordinates,
    Jastrow parameters and MO coefficients, a charge <= 0 and two nuclei at
    one point fail with LRDMC_ERR_ARG; every synthetic system still passes."""
    def broken(change):
        s = S.make_system("H2O")
        s.nuc_xyz = np.array(s.nuc_xyz, float)
        s.Z = np.array(s.Z, float)
        s.C = np.array(s.C, float)
        s.en_b1 = np.array(s.en_b1, float)
        change(s)
        return s

    cases = [
        lambda s: s.nuc_xyz.__setitem__((1, 0), np.nan),
        lambda s: s.nuc_xyz.__setitem__((2, 2), np.inf),
        lambda s: s.Z.__setitem__(1, 0.0),
        lambda s: s.Z.__setitem__(0, -8.0),
        lambda s: s.C.__setitem__((3, 1), np.nan),
        lambda s: s.en_b1.__setitem__(2, np.inf),
        lambda s: setattr(s, "b_ee", np.nan),
        lambda s: setattr(s, "c_anti", np.inf),
        lambda s: s.nuc_xyz.__setitem__(2, s.nuc_xyz[1]),
    ]
    for change in cases:
        with pytest.raises(pkg.LrdmcError) as e:
            pkg.LrdmcSystem(broken(change))
        assert e.value.status == pkg.ERR_ARG
    for name in S.SYSTEMS:
        pkg.LrdmcSystem(S.make_system(name))
    for Z in (1, 4, 18, 36, 54):
        pkg.LrdmcSystem(S.hydrogenic_ion(Z))
    pkg.LrdmcSystem(S.cluster(8, 24, 2))
