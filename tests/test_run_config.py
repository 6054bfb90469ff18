"""CPU checks of the JSON inputs: the system file round trip (every synthetic
system, checked through the oracle's evaluation), its validation, the run
file's validation, and the runner's calls into the binding (a recording
stand-in for the binding, so no GPU is needed)."""
import json
import types

import numpy as np
import pytest

import lrdmc_synth as S
from paper_1909_01589_gb300 import run as R
from paper_1909_01589_gb300 import stats


@pytest.mark.parametrize("name", sorted(S.SYSTEMS))
def test_system_json_round_trip(name, oracle_mod, tmp_path):
    s = S.make_system(name)
    path = str(tmp_path / "s.json")
    S.save_system(s, path)
    t = S.load_system(path)
    for a, b in zip(s.shell_arrays(), t.shell_arrays()):
        assert np.array_equal(a, b)
    assert np.array_equal(t.C, s.C) and np.array_equal(t.Z, np.asarray(s.Z, float))
    assert (t.n_up, t.n_dn, t.ee_on, t.orbital_shell, t.exact_energy) == \
        (s.n_up, s.n_dn, s.ee_on, s.orbital_shell, s.exact_energy)
    # the oracle sees the same trial function: identical lattice evaluations
    lat = oracle_mod.lattice_for(s, 0.2, oracle_mod.THIS_WORK)
    lat_t = oracle_mod.lattice_for(t, 0.2, oracle_mod.THIS_WORK)
    x = S.initial_positions(s, 2, 5)
    Rm = S.random_rotations(2, 6)
    for c in range(2):
        r1 = oracle_mod.OracleSystem(s).lattice_eval(lat, x[c], Rm[c])
        r2 = oracle_mod.OracleSystem(t).lattice_eval(lat_t, x[c], Rm[c])
        assert np.array_equal(r1["ratio"], r2["ratio"]) and r1["EL"] == r2["EL"]


def test_system_json_rejects_malformed_input():
    good = S.system_to_dict(S.neon())
    S.system_from_dict(good)
    cases = [
        ("C", lambda d: d.__setitem__("C", d["C"][:-1]), "'C' must be"),
        ("kind", lambda d: d["shells"][0].__setitem__("kind", "sgo"), "kind"),
        ("centre", lambda d: d["shells"][0].__setitem__("center", 3), "out of range"),
        ("zeta", lambda d: d["shells"][0].__setitem__("zeta", 0.0), "zeta > 0"),
        ("en_b1", lambda d: d["jastrow"].__setitem__("en_b1", [0.1, 0.2]), "en_b1"),
        ("missing", lambda d: d.pop("n_up"), "missing 'n_up'"),
        ("orbital", lambda d: d.__setitem__("orbital_shell", [0, 99]), "orbital_shell"),
    ]
    for label, change, msg in cases:
        d = json.loads(json.dumps(good))
        change(d)
        with pytest.raises(ValueError, match=msg):
            S.system_from_dict(d)


BASE = {"walkers": 64, "intervals": 10, "a": 0.2, "tau": 0.02, "e_trial": -2.9}


def test_run_config_defaults_and_checks():
    cfg = R.parse_run(dict(BASE))
    assert (cfg.spacing, cfg.precision, cfg.seed, cfg.start_seed, cfg.equilibration) == \
        ("this_work", "df64", 1, 1, 0)
    bad = [({"walkers": 0}, "walkers"), ({"tau": -1.0}, "tau"), ({"spacing": "double"}, "spacing"),
           ({"precision": "bf16"}, "precision"), ({"equilibration": 10}, "equilibration"),
           ({"spacing": "explicit"}, "explicit"), ({"rc": 0.5}, "explicit spacing only"),
           ({"colour": 1}, "unknown keys"), ({"walkers": "many"}, "run:")]
    for change, msg in bad:
        with pytest.raises(ValueError, match=msg):
            R.parse_run({**BASE, **change})
    with pytest.raises(ValueError, match="missing 'tau'"):
        R.parse_run({k: v for k, v in BASE.items() if k != "tau"})
    cfg = R.parse_run({**BASE, "spacing": "explicit", "rc": 0.4, "aprime_over_a": 2.0, "start_seed": 7})
    assert (cfg.rc, cfg.aprime_over_a, cfg.start_seed) == (0.4, 2.0, 7)


class _FakeSystem:
    """Records the runner's calls; returns a fixed trace."""

    calls = []

    def __init__(self, system):
        self.calls.append(("create", system.name))

    def set_precision(self, p):
        self.calls.append(("precision", p))

    def spacing_params(self, a, sp):
        self.calls.append(("spacing_params", a, sp))
        return 1.5, 0.4

    def init_walkers(self, x0, **kw):
        self.calls.append(("init", x0.shape, kw))

    def step(self, n, a, sp):
        self.calls.append(("step", n, a, sp))

    def sync(self):
        self.calls.append(("sync",))

    def energy_trace(self, max_n=1 << 20):
        assert max_n == 10  # the whole trace of the run, not a default length
        k = np.arange(10.0)
        return -2.9 + 0.01 * np.sin(k), 1.0 + 0.001 * np.cos(k), 3.0 + 0 * k

    def moves(self):
        return 4096


def _fake_binding():
    import paper_1909_01589_gb300 as real

    lr = types.SimpleNamespace(**{k: getattr(real, k) for k in (
        "SINGLE", "THIS_WORK", "PREVIOUS", "EXPLICIT", "PRECISION_FP64", "PRECISION_DF64", "PRECISION_FP32",
        "Spacing")})
    lr.LrdmcSystem = _FakeSystem
    return lr


def test_runner_calls_the_binding_in_order():
    lr = _fake_binding()
    _FakeSystem.calls = []
    cfg = R.parse_run({**BASE, "precision": "fp64", "spacing": "previous", "equilibration": 4, "mixed_L": 2,
                       "recompute_every": 3, "seed": 9, "start_seed": 5})
    out = R.run(S.helium(), cfg, lr=lr)
    names = [c[0] for c in _FakeSystem.calls]
    assert names == ["create", "precision", "spacing_params", "init", "step", "sync"]
    assert _FakeSystem.calls[1][1] == lr.PRECISION_FP64
    sp = _FakeSystem.calls[4][3]
    assert sp.kind == lr.PREVIOUS and _FakeSystem.calls[4][1:3] == (10, 0.2)
    shape, kw = _FakeSystem.calls[3][1], _FakeSystem.calls[3][2]
    assert shape == (64, 2, 3)
    assert kw == {"seed": 9, "tau": 0.02, "e_trial": -2.9, "recompute_every": 3, "trace_capacity": 10}
    e, w, _ = _FakeSystem.energy_trace(None, 10)
    assert out["energy_Ha"] == stats.energy_estimate(e[4:], w[4:], 2)
    assert out["error_Ha"] == stats.reblock(e[4:])[0]
    assert out["intervals_used"] == 6 and out["walker_moves"] == 4096
    assert (out["aprime_over_a"], out["rc"]) == (1.5, 0.4)
    json.dumps(out)  # the result is plain JSON


def test_dump_system_writes_a_loadable_file(tmp_path):
    path = str(tmp_path / "ne.json")
    R.main(["--dump-system", "Ne", "--out", path])
    t = S.load_system(path)
    assert t.N == 10 and t.n_ao == S.neon().n_ao
