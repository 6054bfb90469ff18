"""Pins of the oracle's neural pair Jastrow: bfloat16 rounding against the
library conversion, radial derivatives against finite differences, the
quintic Hermite table against closed forms, the energy decomposition
against the oracle's direct Laplacian, and the objective's gradient
against finite differences."""
import numpy as np
import pytest
import torch

import lrdmc_synth as S


@pytest.fixture(scope="module")
def nn():
    from oracle import neural

    return neural


def _trained_like(spec, seed=3, scale=0.5):
    """Parameters with a non-zero output layer (an untrained network is
    identically zero by construction)."""
    return S.neural_init(spec, seed, out_scale=scale)


def test_bf16_round_matches_library_conversion(nn):
    rng = np.random.default_rng(0)
    v = np.concatenate([rng.normal(size=2000) * 10.0 ** rng.integers(-8, 8, size=2000),
                        [0.0, -0.0, 1.0, 1.0 + 2 ** -8, 1.0 + 3 * 2 ** -8, 1.0 + 2 ** -9, -(1.0 + 2 ** -8)]])
    t = torch.tensor(v, dtype=torch.float32)
    ref = t.to(torch.bfloat16).to(torch.float64)
    assert torch.equal(nn.bf16_round(t.to(torch.float64)), ref)
    # ties go to the even neighbour: 1 + 2^-8 lies halfway between 1 and 1 + 2^-7
    assert float(nn.bf16_round(torch.tensor([1.0 + 2 ** -8]))[0]) == 1.0
    assert float(nn.bf16_round(torch.tensor([1.0 + 3 * 2 ** -8]))[0]) == 1.0 + 2 ** -6


@pytest.mark.parametrize("bf16", [False, True])
def test_radial_derivatives_finite_difference(nn, bf16):
    spec = S.default_neural_spec(S.neon())
    th = _trained_like(spec)
    r = np.array([0.013, 0.05, 0.2, 0.7, 1.5, 3.0, 4.6])
    h = 1e-4
    for c in range(spec.n_ch):
        ch = np.full(len(r), c)
        g, g1, g2 = (t.numpy() for t in nn.radial(th, spec, r, ch, bf16))
        f = [nn.radial(th, spec, r + m * h, ch, bf16)[0].numpy() for m in (-2, -1, 1, 2)]
        d1 = (f[0] - 8 * f[1] + 8 * f[2] - f[3]) / (12 * h)
        d2 = (-f[0] + 16 * f[1] - 30 * g + 16 * f[2] - f[3]) / (12 * h * h)
        scale = np.max(np.abs(g)) + 1e-3
        assert np.allclose(g1, d1, atol=1e-7 * scale / h, rtol=1e-6)
        assert np.allclose(g2, d2, atol=1e-5 * scale / h, rtol=1e-4)


def test_radial_cusp_and_cutoff(nn):
    """g'(0) = 0 (the Pade cusps are kept); g, g', g'' vanish from r_cut on."""
    spec = S.default_neural_spec(S.water())
    th = _trained_like(spec)
    for c in range(spec.n_ch):
        g, g1, g2 = nn.radial(th, spec, np.array([0.0]), np.array([c]))
        assert float(g1[0]) == 0.0
        rc = spec.r_cut[c]
        g, g1, g2 = nn.radial(th, spec, np.array([rc, rc * 1.5]), np.array([c, c]))
        assert torch.all(g == 0) and torch.all(g1 == 0) and torch.all(g2 == 0)
        g, g1, g2 = nn.radial(th, spec, np.array([rc * (1 - 1e-4)]), np.array([c]))
        assert abs(float(g[0])) < 1e-9 and abs(float(g1[0])) < 1e-6 and abs(float(g2[0])) < 1e-2


def test_quintic_table_reproduces_polynomials(oracle_mod, nn):
    """The interpolant is exact for a polynomial of degree 5 in r (each cell
    maps r affinely to t), and zero from r_cut on."""
    s = S.helium()
    o = oracle_mod.OracleSystem(s)
    coef = np.array([0.3, -1.2, 0.8, -0.25, 0.04, -0.002])
    rc, n = 4.0, 16
    k = np.arange(n + 1)
    rk = rc * (k / n) ** 2
    P = np.polynomial.Polynomial(coef)
    nodes = np.zeros((3, n + 1, 3))
    for c in range(3):
        nodes[c, :, 0] = P(rk) * (c + 1)
        nodes[c, :, 1] = P.deriv(1)(rk) * (c + 1)
        nodes[c, :, 2] = P.deriv(2)(rk) * (c + 1)
    tab = nn.Table(np.full(3, rc), np.array([0], dtype=np.int32), n, nodes)
    o.set_neural(tab)
    rng = np.random.default_rng(5)
    for r in np.concatenate([rng.uniform(0, rc, 200), rk[:-1], [1e-9]]):
        for c in range(3):
            g, g1, g2 = o.neural_pair(c, r)
            assert abs(g - (c + 1) * P(r)) < 1e-12
            assert abs(g1 - (c + 1) * P.deriv(1)(r)) < 1e-10
            assert abs(g2 - (c + 1) * P.deriv(2)(r)) < 1e-8
    assert o.neural_pair(1, rc) == (0.0, 0.0, 0.0)
    assert o.neural_pair(1, rc + 1.0) == (0.0, 0.0, 0.0)


def test_table_interpolates_network(oracle_mod, nn):
    """At the nodes the table returns the network's values; between them it
    is within a small interpolation error; across a node it is continuous
    to second order."""
    s = S.neon()
    spec = S.default_neural_spec(s)
    th = _trained_like(spec)
    tab = nn.table(th, spec)
    o = oracle_mod.OracleSystem(s).set_neural(tab)
    n = tab.n_cells
    for c in range(spec.n_ch):
        rc = spec.r_cut[c]
        for k in (1, 7, 100, n // 2, n - 3):
            rk = rc * (k / n) ** 2
            g = o.neural_pair(c, rk)
            assert np.allclose(g, tab.nodes[c, k], rtol=1e-12, atol=1e-12)
            lo = o.neural_pair(c, rk * (1 - 1e-13))
            assert np.allclose(lo, g, rtol=1e-8, atol=1e-9)
        rng = np.random.default_rng(c)
        r = rng.uniform(0, rc, 300) ** 1.0
        ref = nn.radial(th, spec, r, np.full(len(r), c))
        got = np.array([o.neural_pair(c, v) for v in r])
        scale = np.max(np.abs(tab.nodes[c, :, 0])) + 1e-3
        assert np.max(np.abs(got[:, 0] - ref[0].numpy())) < 1e-8 * scale
        assert np.max(np.abs(got[:, 1] - ref[1].numpy())) < 1e-5 * scale


@pytest.mark.parametrize("name", ["He", "Ne", "H2O"])
def test_energy_decomposition_matches_direct_laplacian(oracle_mod, nn, name):
    """E_L and J_NN assembled from the base terms and the pair derivatives
    equal the oracle's own local energy and log|psi| with the table
    installed (the table is fine enough that interpolation error is below
    the tolerance); the direct local energy in turn matches second
    differences of the brute-force log|psi| (the pair term is in both)."""
    s = S.make_system(name)
    spec = S.default_neural_spec(s, n_cells=2048)
    th = _trained_like(spec, scale=0.8)
    o = oracle_mod.OracleSystem(s)
    x = S.initial_positions(s, 6, 71)
    gb, eb = nn.base_terms(o, x)
    la0 = np.array([o.log_psi(xx)[0] for xx in x])
    EL, J = nn.energy_terms(th, spec, x, s.n_up, s.nuc_xyz, gb, eb)
    o.set_neural(nn.table(th, spec))
    direct = np.array([o.local_energy(xx) for xx in x])
    la1 = np.array([o.log_psi(xx)[0] for xx in x])
    assert np.allclose(J.numpy(), la1 - la0, rtol=1e-9, atol=1e-9)
    assert np.allclose(EL.numpy(), direct, rtol=1e-7, atol=1e-6)
    # the pair term changes E_L (the check above is not vacuous)
    assert np.max(np.abs(EL.numpy() - eb)) > 1e-2
    # direct Laplacian with the table against second differences
    xx = x[0]
    lap, _ = o.laplacian_terms(xx)
    h = 1e-4
    fd = 0.0
    for i in range(s.N):
        for k in range(3):
            for sg in (1, -1):
                y = xx.copy()
                y[i, k] += sg * h
                fd += np.exp(o.log_psi(y)[0] - la1[0])
    fd = (fd - 6 * s.N) / (h * h)
    assert abs(fd - lap) < 1e-4 * max(1.0, abs(lap))


def test_objective_gradient_finite_difference(oracle_mod, nn):
    s = S.neon()
    spec = S.default_neural_spec(s)
    th = _trained_like(spec, scale=0.3).astype(np.float64)
    o = oracle_mod.OracleSystem(s)
    x = S.initial_positions(s, 24, 5)
    gb, eb = nn.base_terms(o, x)
    L0, grad, _, _ = nn.loss_and_grad(th, spec, x, s.n_up, s.nuc_xyz, gb, eb, bf16=False)
    rng = np.random.default_rng(9)
    for _ in range(4):
        v = rng.normal(size=th.shape)
        v /= np.linalg.norm(v)
        eps = 1e-5
        lp = nn.loss_and_grad(th + eps * v, spec, x, s.n_up, s.nuc_xyz, gb, eb, bf16=False)[0]
        lm = nn.loss_and_grad(th - eps * v, spec, x, s.n_up, s.nuc_xyz, gb, eb, bf16=False)[0]
        fd = (lp - lm) / (2 * eps)
        assert abs(fd - grad @ v) < 1e-6 * max(1.0, abs(fd))
    # the weights of every layer receive gradient
    H, D = spec.hidden, spec.n_in
    assert np.abs(grad[:H * D]).max() > 0 and np.abs(grad[-H - 1:-1]).max() > 0
