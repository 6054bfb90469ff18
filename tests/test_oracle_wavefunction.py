"""Pins of the oracle's trial function, local energy, Sherman-Morrison update
and lattice evaluation against closed forms, exact eigenstates, brute force
and invariances."""
import math

import numpy as np
import pytest

import lrdmc_synth as S


def _osys(oracle_mod, name_or_sys, **kw):
    s = S.make_system(name_or_sys, **kw) if isinstance(name_or_sys, str) else name_or_sys
    return s, oracle_mod.OracleSystem(s)


def test_ao_derivatives_finite_difference(oracle_mod):
    """Gradient and Laplacian of every atomic orbital (STO s/p/d, contracted
    Gaussian) agree with 4th-order central differences of the values."""
    s, o = _osys(oracle_mod, "tiny_mixed")
    rng = np.random.default_rng(0)
    h = 1e-3
    for _ in range(20):
        r = rng.normal(size=3)
        chi, g, lp = o.ao_values(r)
        gfd = np.zeros_like(g)
        lfd = np.zeros_like(lp)
        for k in range(3):
            e = np.zeros(3)
            e[k] = h
            f = [o.ao_values(r + m * e)[0] for m in (-2, -1, 1, 2)]
            gfd[:, k] = (f[0] - 8 * f[1] + 8 * f[2] - f[3]) / (12 * h)
            lfd += (-f[0] + 16 * f[1] - 30 * chi + 16 * f[2] - f[3]) / (12 * h * h)
        assert np.allclose(g, gfd, rtol=1e-7, atol=1e-8)
        assert np.allclose(lp, lfd, rtol=1e-5, atol=1e-6)


def test_d_shell_spans_rotation_invariant_space(oracle_mod):
    """The five l = 2 functions span a rotation-invariant space (a complete
    set of degree-2 harmonics): values at rotated points are a fixed linear
    map of values at the original points; the p set rotates as a vector."""
    s, o = _osys(oracle_mod, "tiny_mixed")
    rng = np.random.default_rng(1)
    Q = S.random_rotations(1, 4).reshape(3, 3)
    pts = rng.normal(size=(12, 3))
    d_idx = slice(5, 10)
    p_idx = slice(1, 4)
    A = np.array([o.ao_values(p)[0][d_idx] for p in pts])
    B = np.array([o.ao_values(Q @ p)[0][d_idx] for p in pts])
    D, res, *_ = np.linalg.lstsq(A, B, rcond=None)
    assert np.max(np.abs(A @ D - B)) < 1e-12 * np.max(np.abs(B))
    for p in pts:
        assert np.allclose(o.ao_values(Q @ p)[0][p_idx], Q @ o.ao_values(p)[0][p_idx], rtol=1e-12, atol=1e-15)


def _one_electron(Z, n, l, zeta):
    sys = S.hydrogenic_ion(Z)
    sys.shells = [S.Shell(0, l, S.STO, float(n), zeta)]
    sys.C = np.zeros((2 * l + 1, 1))
    sys.C[0, 0] = 1.0
    return sys


@pytest.mark.parametrize("Z,n,l,m", [(1, 1, 0, 0), (2, 1, 0, 0), (1, 2, 1, 0), (1, 2, 1, 2),
                                     (1, 3, 2, 0), (3, 3, 2, 3), (1, 3, 2, 4)])
def test_exact_hydrogenic_states(oracle_mod, Z, n, l, m):
    """r^l Y_lm exp(-Z r / n) with n = l + 1 is an exact eigenstate of the
    hydrogenic ion: E_L = -Z^2 / (2 n^2) at every point (pins the radial
    derivatives, the (l+1) term of the Laplacian and the potential)."""
    sys = _one_electron(Z, n, l, Z / n)
    sys.C[:, 0] = 0.0
    sys.C[m, 0] = 1.0
    o = oracle_mod.OracleSystem(sys)
    rng = np.random.default_rng(2)
    for _ in range(20):
        x = rng.normal(size=(1, 3)) * n
        assert abs(o.local_energy(x) + Z * Z / (2.0 * n * n)) < 1e-11 * Z * Z


def test_be_bare_exact(oracle_mod):
    """Four non-interacting electrons in exact 1s/2s orbitals of Z = 4:
    E_L = -20 everywhere, including both determinants with their 2s node."""
    s, o = _osys(oracle_mod, "Be_bare")
    x = S.initial_positions(s, 50, 3)
    for w in range(50):
        assert abs(o.local_energy(x[w]) + 20.0) < 1e-10


def test_ee_cusp_cancels_coulomb_singularity(oracle_mod):
    """Antiparallel Pade factor with c = 1/2 satisfies Kato's cusp: the
    1/r_12 of V cancels against the Jastrow Laplacian, so E_L stays finite
    as the two He electrons meet; with c = 1/4 it would diverge."""
    s, o = _osys(oracle_mod, "He")
    base = np.array([0.7, -0.2, 0.4])
    d = np.array([0.3, 0.5, -0.8]) / np.linalg.norm([0.3, 0.5, -0.8])
    E = [o.local_energy(np.array([base, base + eps * d])) for eps in (1e-4, 1e-6, 1e-8)]
    assert abs(E[1] - E[2]) < 1e-5 and abs(E[0] - E[1]) < 1e-2
    s2 = S.helium()
    s2.c_anti = 0.25
    o2 = oracle_mod.OracleSystem(s2)
    E2 = [o2.local_energy(np.array([base, base + eps * d])) for eps in (1e-6, 1e-8)]
    # 1/r12 - 2 c / r12 with c = 1/4 leaves +1/(2 r12)
    assert abs(E2[1] * 1e-8 - 0.5) < 1e-3
    assert abs(E2[1] - E2[0]) > 1e6


def test_en_cusp(oracle_mod):
    """H with orbital exp(-0.7 r) and e-n factor -0.3 r/(1 + r): the slopes
    add to -Z, so E_L is finite at the nucleus."""
    sys = S.hydrogen(0.7)
    sys.en_b1 = np.array([0.3])
    o = oracle_mod.OracleSystem(sys)
    d = np.array([0.2, -0.6, 0.3]) / np.linalg.norm([0.2, -0.6, 0.3])
    E = [o.local_energy((eps * d)[None, :]) for eps in (1e-4, 1e-6, 1e-8)]
    assert abs(E[1] - E[2]) < 1e-5 and abs(E[0] - E[1]) < 1e-3


@pytest.mark.parametrize("name", ["He", "Ne", "tiny_mixed", "Be_bare", "Ar", "H2O"])
def test_lattice_ratios_match_brute_force(oracle_mod, name):
    """Every psi_G(x')/psi_G(x) of the lattice evaluation (inverse-column
    route) equals the ratio of brute-force determinants and Jastrow sums."""
    s, o = _osys(oracle_mod, name)
    x = S.initial_positions(s, 4, 11)
    R = S.random_rotations(4, 12)
    lat = oracle_mod.lattice_for(s, 0.3, oracle_mod.EXPLICIT, rc=0.4, aprime_over_a=1.7)
    for w in range(4):
        ev = o.lattice_eval(lat, x[w], R[w])
        la0, sg0 = o.log_psi(x[w])
        Rm = R[w].reshape(3, 3)
        for c in range(len(ev["ratio"])):
            sg, k, g, i = c % 2, (c // 2) % 3, (c // 6) % 2, c // 12
            h = lat.a if g == 0 else lat.ap
            xp = x[w].copy()
            xp[i] += (1 if sg == 0 else -1) * h * Rm[:, k]
            la, sgn = o.log_psi(xp)
            brute = sgn * sg0 * np.exp(la - la0)
            assert abs(ev["ratio"][c] - brute) < 1e-10 * max(1.0, abs(brute))


def test_ratios_invariant_under_orbital_mixing(oracle_mod):
    """det(A M) = det(A) det(M): mixing the orbitals with any invertible M
    (C -> C M) leaves every ratio, rate and local energy unchanged."""
    s = S.neon()
    o = oracle_mod.OracleSystem(s)
    rng = np.random.default_rng(5)
    M = rng.normal(size=(5, 5)) + 3 * np.eye(5)
    s2 = S.neon()
    s2.C = s.C @ M
    o2 = oracle_mod.OracleSystem(s2)
    x = S.initial_positions(s, 3, 6)
    R = S.random_rotations(3, 7)
    lat = oracle_mod.lattice_for(s, 0.2, oracle_mod.THIS_WORK)
    for w in range(3):
        a, b = o.lattice_eval(lat, x[w], R[w]), o2.lattice_eval(lat, x[w], R[w])
        assert np.allclose(a["ratio"], b["ratio"], rtol=1e-9, atol=1e-12)
        assert abs(a["EL"] - b["EL"]) < 1e-9 * abs(a["EL"])


def test_sherman_morrison_against_recompute(oracle_mod):
    """A chain of 30 single-electron moves updated by Sherman-Morrison ends
    at the inverse of the final Slater matrix; each returned ratio is the
    brute-force determinant ratio."""
    s, o = _osys(oracle_mod, "tiny_mixed")
    rng = np.random.default_rng(8)
    x = S.initial_positions(s, 1, 9)[0]
    Au, Ad = o.inverses(x)
    for _ in range(30):
        i = rng.integers(0, s.N)
        xn = x.copy()
        xn[i] += rng.normal(scale=0.3, size=3)
        spin, l = (0, i) if i < s.n_up else (1, i - s.n_up)
        la0, sg0 = o.log_psi(x)
        la1, sg1 = o.log_psi(xn)
        J = lambda y: 0.0  # noqa: E731  (Jastrow cancels below)
        A_new, ratio, rc = o.sm_update(spin, Au if spin == 0 else Ad, l, xn[i])
        assert rc == 0
        # brute-force determinant ratio: psi ratio divided by the Jastrow ratio
        ev_x = x.copy()
        jx = _jastrow(s, ev_x)
        jn = _jastrow(s, xn)
        brute = sg1 * sg0 * np.exp(la1 - la0 - (jn - jx))
        assert abs(ratio - brute) < 1e-10 * max(1, abs(brute))
        if spin == 0:
            Au = A_new
        else:
            Ad = A_new
        x = xn
        del J
    Au2, Ad2 = o.inverses(x)
    assert np.allclose(Au, Au2, rtol=1e-9, atol=1e-10)
    assert np.allclose(Ad, Ad2, rtol=1e-9, atol=1e-10)


def _jastrow(s, x):
    """Brute-force J(x) = sum_{i<j} u_ee + sum_iI u_en with the Pade forms."""
    J = 0.0
    for i in range(s.N):
        for j in range(i + 1, s.N):
            c = s.c_par if (i < s.n_up) == (j < s.n_up) else s.c_anti
            r = np.linalg.norm(x[i] - x[j])
            J += c * r / (1 + s.b_ee * r)
        for I in range(s.n_nuc):
            r = np.linalg.norm(x[i] - s.nuc_xyz[I])
            J += -s.en_b1[I] * r / (1 + s.en_b2 * r)
    return J


@pytest.mark.parametrize("name", ["He", "Ne", "tiny_mixed"])
@pytest.mark.parametrize("double", [False, True])
def test_lattice_laplacian_converges_quadratically(oracle_mod, name, double):
    """Eq. 1: sum_c (w_c / h_c^2)(rho_c - 1) = Delta^{a,a'} psi / psi tends to
    the analytic lap psi / psi with error O(a^2) (a'/a fixed): halving a cuts
    the error by ~4."""
    s, o = _osys(oracle_mod, name)
    x = S.initial_positions(s, 1, 21)[0]
    R = S.random_rotations(1, 22)[0]
    lap, _ = o.laplacian_terms(x)
    errs = []
    for a in (0.02, 0.01, 0.005):
        if double:
            lat = oracle_mod.lattice_for(s, a, oracle_mod.EXPLICIT, rc=0.6, aprime_over_a=1.8)
        else:
            lat = oracle_mod.lattice_for(s, a, oracle_mod.SINGLE)
        ev = o.lattice_eval(lat, x, R)
        G = lat.G
        h = np.array([lat.a if (c // 6) % G == 0 else lat.ap for c in range(len(ev["ratio"]))])
        errs.append(abs(np.sum(ev["w"] / h ** 2 * (ev["ratio"] - 1.0)) - lap))
    assert 3.0 < errs[0] / errs[1] < 5.0 and 3.0 < errs[1] / errs[2] < 5.0
    assert errs[2] < 5e-3 * max(1.0, abs(lap))


def test_double_grid_limits(oracle_mod):
    """Eq. 1 limits: with p = 1 everywhere (r_c -> infinity) the a' grid
    drops out and the a grid equals the single grid; with a' = a the two
    grids add up to the single grid move by move."""
    s, o = _osys(oracle_mod, "Ne")
    x = S.initial_positions(s, 1, 31)[0]
    R = S.random_rotations(1, 32)[0]
    single = o.lattice_eval(oracle_mod.lattice_for(s, 0.1, oracle_mod.SINGLE), x, R)
    big = o.lattice_eval(oracle_mod.lattice_for(s, 0.1, oracle_mod.EXPLICIT, rc=1e9, aprime_over_a=2.0), x, R)
    Tb = big["T"].reshape(s.N, 2, 6)
    assert np.allclose(Tb[:, 0, :].ravel(), single["T"], rtol=1e-14, atol=0)
    assert np.all(Tb[:, 1, :] == 0.0)
    same = o.lattice_eval(oracle_mod.lattice_for(s, 0.1, oracle_mod.EXPLICIT, rc=0.2, aprime_over_a=1.0), x, R)
    Ts = same["T"].reshape(s.N, 2, 6)
    assert np.allclose(Ts.sum(axis=1).ravel(), single["T"], rtol=1e-13, atol=0)
    assert abs(same["b"] - single["b"]) < 1e-12 * single["b"]


def test_lattice_hamiltonian_symmetric(oracle_mod):
    """p is taken at the bond midpoint, so the kinetic element of H^a between
    x and a neighbour x' is the same from both ends: w(x -> x') = w(x' -> x)
    and psi(x')/psi(x) * psi(x)/psi(x') = 1."""
    s, o = _osys(oracle_mod, "Ne")
    x = S.initial_positions(s, 1, 41)[0]
    R = S.random_rotations(1, 42)[0]
    Rm = R.reshape(3, 3)
    lat = oracle_mod.lattice_for(s, 0.2, oracle_mod.THIS_WORK)
    ev = o.lattice_eval(lat, x, R)
    for c in range(0, len(ev["w"]), 7):
        sg, k, g, i = c % 2, (c // 2) % 3, (c // 6) % 2, c // 12
        h = lat.a if g == 0 else lat.ap
        xp = x.copy()
        xp[i] += (1 if sg == 0 else -1) * h * Rm[:, k]
        back = o.lattice_eval(lat, xp, R)
        cb = c ^ 1  # same electron, grid and axis, opposite sign
        assert abs(back["w"][cb] - ev["w"][c]) < 1e-14
        assert abs(back["ratio"][cb] * ev["ratio"][c] - 1.0) < 1e-10


def test_rates_and_sign_flip(oracle_mod):
    """T_c = w_c / (2 h^2) max(rho_c, 0): moves that cross the fixed node
    (rho < 0) get no rate; b is the sum of the rates."""
    s, o = _osys(oracle_mod, "Be_bare")
    x = S.initial_positions(s, 40, 51)
    R = S.random_rotations(40, 52)
    lat = oracle_mod.lattice_for(s, 0.4, oracle_mod.EXPLICIT, rc=0.5, aprime_over_a=1.5)
    flips = 0
    for w in range(40):
        ev = o.lattice_eval(lat, x[w], R[w])
        h = np.array([lat.a if (c // 6) % 2 == 0 else lat.ap for c in range(len(ev["w"]))])
        expect = np.where(ev["ratio"] > 0, ev["w"] / (2 * h * h) * ev["ratio"], 0.0)
        assert np.allclose(ev["T"], expect, rtol=1e-15, atol=0)
        assert abs(ev["b"] - np.sum(ev["T"])) < 1e-12 * ev["b"]
        flips += int(np.sum(ev["ratio"] < 0))
    assert flips > 0


def test_heavy_atom_rule_polyatomic(oracle_mod):
    """Large systems: R_c runs over the heaviest atoms only, so near an H of
    H2O p is still the Gaussian of the distance to O."""
    s, o = _osys(oracle_mod, "H2O")
    lat = oracle_mod.lattice_for(s, 0.1, oracle_mod.THIS_WORK)
    near_h = S.WATER_H[0] + np.array([0.05, -0.02, 0.01])
    d2 = float(np.sum(near_h ** 2))
    assert abs(o.p(lat, near_h) - np.exp(-d2 / (2 * lat.rc ** 2))) < 1e-15
    # r_c and a'/a come from the heaviest atom (Z = 8)
    assert abs(lat.rc - oracle_mod.rc_this_work(0.1, 8.0)) < 1e-15


@pytest.mark.parametrize("name", ["Ar", "Kr", "H2O"])
def test_gaussian_atoms_cusp_and_laplacian(oracle_mod, name):
    """STO-6G-style atoms: the e-n factor carries the whole nuclear cusp, so
    E_L stays finite as an electron reaches a nucleus; the analytic Laplacian
    matches second differences of the brute-force psi."""
    s, o = _osys(oracle_mod, name)
    x = S.initial_positions(s, 1, 61)[0]
    d = np.array([0.3, -0.5, 0.81]) / np.linalg.norm([0.3, -0.5, 0.81])
    E = []
    for eps in (1e-5, 1e-7):
        y = x.copy()
        y[0] = s.nuc_xyz[0] + eps * d
        E.append(o.local_energy(y))
    assert abs(E[0] - E[1]) < 1e-2 * max(1.0, abs(E[1]))
    lap, _ = o.laplacian_terms(x)
    h = 1e-4
    la0, _ = o.log_psi(x)
    fd = 0.0
    for i in range(s.N):
        for k in range(3):
            for sg in (1, -1):
                y = x.copy()
                y[i, k] += sg * h
                la, sgn = o.log_psi(y)
                fd += np.exp(la - la0)
    fd = (fd - 6 * s.N) / (h * h)
    assert abs(fd - lap) < 1e-4 * max(1.0, abs(lap))


def _unit_vectors(n, seed):
    v = np.random.default_rng(seed).normal(size=(n, 3))
    return v / np.linalg.norm(v, axis=1, keepdims=True)


@pytest.mark.parametrize("name,a", [("He", 0.2), ("Ne", 0.2), ("Ne", 0.05), ("Kr", 1 / 126)])
def test_gaussian_p_characteristic_values(oracle_mod, name, a):
    """Eq. 3 (this work): p(r) = exp(-|r - R_c|^2 / (2 r_c^2)) with r_c a
    length from S-13. Its defining values, along any direction: 1 at the
    nucleus, exp(-1/2) at one r_c, exp(-2) at two, 1/2 at r_c sqrt(2 ln 2).
    A dropped square, a missing factor 2 or r_c read as an inverse length
    moves every one of them."""
    s, o = _osys(oracle_mod, name)
    lat = oracle_mod.lattice_for(s, a, oracle_mod.THIS_WORK)
    assert lat.pkind == 0 and lat.G == 2
    assert abs(lat.rc - oracle_mod.rc_this_work(a, float(s.Z[0]))) < 1e-15
    Rc = np.asarray(s.nuc_xyz, float).reshape(-1, 3)[0]
    assert o.p(lat, Rc) == 1.0
    for u in _unit_vectors(8, 5):
        assert abs(o.p(lat, Rc + lat.rc * u) - math.exp(-0.5)) < 1e-14
        assert abs(o.p(lat, Rc + 2.0 * lat.rc * u) - math.exp(-2.0)) < 1e-14
        assert abs(o.p(lat, Rc + lat.rc * math.sqrt(2.0 * math.log(2.0)) * u) - 0.5) < 1e-14
    # the a' grid's weight 1 - p vanishes at the nucleus and tends to 1 far out
    assert o.p(lat, Rc + 20.0 * lat.rc * np.array([0.0, 0.0, 1.0])) < 1e-80


@pytest.mark.parametrize("name", ["He", "Ne", "Ar", "Kr"])
def test_pade_p_characteristic_values(oracle_mod, name):
    """Eq. 2 (the previous scheme): p(r) = 1/(1 + r_c^2 |r - R_c|^2) with r_c
    an inverse length, r_c = Z/2 (the choice that Eq. 4 pairs with
    a'/a = sqrt(Z^2/4 + 1)). Its defining values: 1 at the nucleus, 1/2 at
    distance 1/r_c = 2/Z, and the far tail p (r_c d)^2 -> 1. r_c in place
    of r_c^2, or 2 r_c^2, fails the half-value point for every Z != 2."""
    s, o = _osys(oracle_mod, name)
    Z = float(s.Z[0])
    lat = oracle_mod.lattice_for(s, 0.1, oracle_mod.PREVIOUS)
    assert lat.pkind == 1 and lat.G == 2
    assert lat.rc == Z / 2.0
    assert abs(lat.ap / lat.a - math.sqrt(Z * Z / 4.0 + 1.0)) < 1e-14
    Rc = np.asarray(s.nuc_xyz, float).reshape(-1, 3)[0]
    assert o.p(lat, Rc) == 1.0
    for u in _unit_vectors(8, 6):
        assert abs(o.p(lat, Rc + (2.0 / Z) * u) - 0.5) < 1e-14
        assert abs(o.p(lat, Rc + (6.0 / Z) * u) - 0.1) < 1e-14  # 1/(1 + 3^2)
        d = 1e3 * 2.0 / Z
        assert abs(o.p(lat, Rc + d * u) * (Z / 2.0 * d) ** 2 - 1.0) < 2e-6


def test_pade_p_polyatomic_uses_heaviest_atom(oracle_mod):
    """For H2O the previous scheme takes r_c = Z_max/2 = 4 from O, and the
    distance to O, not to the nearer H: p = 1/2 at 1/4 bohr from O, and
    next to an H p is the Pade value of its distance to O."""
    s, o = _osys(oracle_mod, "H2O")
    lat = oracle_mod.lattice_for(s, 0.1, oracle_mod.PREVIOUS)
    assert lat.rc == 4.0
    assert abs(o.p(lat, np.array([0.25, 0.0, 0.0])) - 0.5) < 1e-14
    near_h = S.WATER_H[0] + np.array([0.05, -0.02, 0.01])
    d2 = float(np.sum(near_h ** 2))
    assert abs(o.p(lat, near_h) - 1.0 / (1.0 + 16.0 * d2)) < 1e-15
