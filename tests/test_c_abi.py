"""The C ABI from a plain C99 program (CPU): tests/c_abi_host.c includes
include/lrdmc.h, is compiled with gcc -std=c99 -pedantic -Werror, links
liblrdmc.so and calls the entry points that need no GPU (build flags,
system creation, double-grid parameters, workspace size, error statuses).
Its double-grid parameters must agree with the oracle's S-13 and Eq. 6/7."""
import os
import shutil
import subprocess

import pytest

import lrdmc_synth as S

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)


@pytest.fixture(scope="module")
def c_output(tmp_path_factory):
    if shutil.which("gcc") is None:
        pytest.skip("needs gcc")
    from paper_1909_01589_gb300 import build

    lib = build.build()
    libdir = os.path.dirname(lib)
    exe = str(tmp_path_factory.mktemp("cabi") / "c_abi_host")
    cmd = ["gcc", "-std=c99", "-Wall", "-Wextra", "-Werror", "-pedantic", "-I", os.path.join(ROOT, "include"),
           os.path.join(HERE, "c_abi_host.c"), "-L", libdir, "-llrdmc", f"-Wl,-rpath,{libdir}", "-o", exe]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    r = subprocess.run([exe], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stdout + r.stderr
    return dict(line.split("=", 1) for line in r.stdout.splitlines() if "=" in line)


def test_c_caller_statuses(c_output):
    import paper_1909_01589_gb300 as pkg

    out = c_output
    assert int(out["build_flags"]) == 0
    assert int(out["create"]) == pkg.OK and int(out["spacing"]) == pkg.OK and int(out["workspace"]) == pkg.OK
    assert int(out["bad_walkers"]) == pkg.ERR_ARG
    assert int(out["step_before_init"]) == pkg.ERR_STATE and "init" in out["message"]
    assert int(out["too_many_electrons"]) == pkg.ERR_ARG


def test_c_caller_double_grid_matches_oracle(c_output, oracle_mod):
    ratio, rc = float(c_output["aprime_over_a"]), float(c_output["rc"])
    assert abs(rc - oracle_mod.rc_this_work(0.2, 2)) < 1e-15
    q = oracle_mod.aprime_over_a_this_work(2, 0.2)
    assert abs(ratio - q) < 1e-11 * q


def test_c_caller_workspace_matches_binding(c_output):
    import paper_1909_01589_gb300 as pkg

    pkg.load_library()
    g = pkg.LrdmcSystem(S.helium())
    assert int(c_output["bytes"]) == g.workspace_bytes(256, 100)
