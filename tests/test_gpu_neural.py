"""Neural pair Jastrow on the GPU, through the C ABI, against the oracle:

* the tabulated term in the lattice evaluation and in the projection
  (FP64 and double-float: the bar of the plain path, 1e-10 relative);
* the FP64 base terms of the objective;
* the FP32 training forward (E_L, J_NN) and the hand-written backward
  (gradient of the reweighted variance) against the oracle's float64
  autograd gradient, and against finite differences of the GPU objective;
* what training gains: lower local-energy variance of the projection with
  the trained term than without it.
"""
import numpy as np
import pytest

import lrdmc_synth as S
from _parity_util import ratio_scale

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

RTOL = 1e-10


@pytest.fixture(scope="module")
def pkg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1909_01589_gb300 import build

    build.build()
    import paper_1909_01589_gb300 as p

    p.load_library()
    return p


@pytest.fixture(scope="module")
def nn():
    from oracle import neural

    return neural


def _prec(pkg, name):
    return pkg.PRECISION_FP64 if name == "fp64" else pkg.PRECISION_DF64


def _lattice(pkg, oracle_mod, system, a):
    return pkg.Spacing(pkg.THIS_WORK), oracle_mod.lattice_for(system, a, oracle_mod.THIS_WORK)


@pytest.mark.parametrize("prec", ["fp64", "df64"])
@pytest.mark.parametrize("name,a", [("He", 0.2), ("Ne", 0.2), ("H2O", 0.1), ("Ar", 1 / 63)])
def test_evaluate_with_neural_term(pkg, oracle_mod, nn, name, a, prec):
    system = S.make_system(name)
    spec = S.default_neural_spec(system)
    params = S.neural_init(spec, 11, out_scale=0.6)
    g = pkg.LrdmcSystem(system).set_precision(_prec(pkg, prec)).set_neural_jastrow(spec, params)
    o = oracle_mod.OracleSystem(system).set_neural(nn.table(params, spec))
    n = 37
    x = S.initial_positions(system, n, 301)
    R = S.random_rotations(n, 302)
    sp, lat = _lattice(pkg, oracle_mod, system, a)
    ratio, T, b, el = (t.cpu().numpy() for t in g.evaluate(torch.tensor(x, device="cuda"),
                                                           torch.tensor(R, device="cuda"), a, sp))
    plain = oracle_mod.OracleSystem(system)
    moved = 0.0
    for c in range(n):
        ref = o.lattice_eval(lat, x[c], R[c])
        scale = ratio_scale(o, system, lat, x[c], R[c], ref["ratio"])
        assert np.all(np.abs(ratio[c] - ref["ratio"]) <= RTOL * scale)
        assert np.all(np.abs(T[c] - ref["T"]) <= RTOL * np.max(ref["T"] * scale))
        assert abs(b[c] - ref["b"]) <= RTOL * ref["b"]
        assert abs(el[c] - ref["EL"]) <= RTOL * max(1.0, abs(ref["EL"]))
        moved = max(moved, abs(ref["EL"] - plain.local_energy(x[c])))
    assert moved > 1e-3  # the term is active
    # removing the term restores the plain evaluation
    g.set_neural_jastrow(None, None)
    el0 = g.evaluate(torch.tensor(x, device="cuda"), torch.tensor(R, device="cuda"), a, sp)[3].cpu().numpy()
    assert abs(el0[0] - plain.local_energy(x[0])) <= RTOL * abs(el0[0])


@pytest.mark.parametrize("name,a", [("Ne", 0.2), ("Ar", 0.05)])
def test_evaluate_with_neural_term_full_size_sampled(pkg, oracle_mod, nn, name, a):
    """The neural workload at full size: 16384 configurations with the
    tabulated term (weights with a non-zero output layer), this work's
    double grid, the default double-float mode; 16 sampled configurations
    against the oracle with the same table installed."""
    system = S.make_system(name)
    spec = S.default_neural_spec(system)
    params = S.neural_init(spec, 13, out_scale=0.6)
    g = pkg.LrdmcSystem(system).set_neural_jastrow(spec, params)
    o = oracle_mod.OracleSystem(system).set_neural(nn.table(params, spec))
    n = 16384
    x = S.initial_positions(system, n, 311)
    R = S.random_rotations(n, 312)
    sp, lat = _lattice(pkg, oracle_mod, system, a)
    ratio, T, b, el = g.evaluate(torch.tensor(x, device="cuda"), torch.tensor(R, device="cuda"), a, sp)
    ratio, b, el = ratio.cpu().numpy(), b.cpu().numpy(), el.cpu().numpy()
    assert np.all(np.isfinite(el)) and np.all(b > 0)
    for c in np.random.default_rng(5).choice(n, 16, replace=False):
        ref = o.lattice_eval(lat, x[c], R[c])
        scale = ratio_scale(o, system, lat, x[c], R[c], ref["ratio"])
        assert np.all(np.abs(ratio[c] - ref["ratio"]) <= RTOL * scale), c
        assert abs(b[c] - ref["b"]) <= RTOL * ref["b"], c
        assert abs(el[c] - ref["EL"]) <= RTOL * max(1.0, abs(ref["EL"])), c


@pytest.mark.parametrize("prec", ["fp64", "df64"])
def test_projection_with_neural_term(pkg, oracle_mod, nn, prec):
    """Ne, 64 walkers, three intervals with the term installed: walker by
    walker identical to the oracle's projection with the same table."""
    system = S.neon()
    spec = S.default_neural_spec(system)
    params = S.neural_init(spec, 12, out_scale=0.4)
    g = pkg.LrdmcSystem(system).set_precision(_prec(pkg, prec)).set_neural_jastrow(spec, params)
    o = oracle_mod.OracleSystem(system).set_neural(nn.table(params, spec))
    W, a, tau = 64, 0.2, 0.02
    x0 = S.initial_positions(system, W, 13)
    sp, lat = _lattice(pkg, oracle_mod, system, a)
    g.init_walkers(torch.tensor(x0, device="cuda"), seed=14, tau=tau, e_trial=-128.9, recompute_every=2,
                   trace_capacity=4)
    pop = oracle_mod.OraclePopulation(o, x0, seed=14, tau=tau, e_trial=-128.9, recompute_every=2)
    for k in range(3):
        g.step(1, a, sp)
        pop.step(lat, 1, 8)
        gw, ow = g.walkers(), pop.walkers(lat.G)
        mw, mc = pop.margins()
        if min(np.min(mw), mc) < 1e-9:
            pytest.skip("a decision within 1e-9 of a bin edge")
        assert np.array_equal(gw["jumps_pre"], ow["jumps_pre"]) and np.array_equal(gw["parent"], ow["parent"])
        assert np.all(np.abs(gw["x"] - ow["x"]) <= RTOL * np.maximum(1.0, np.abs(ow["x"])))
        assert np.all(np.abs(gw["EL"] - ow["EL"]) <= RTOL * np.maximum(1.0, np.abs(ow["EL"])))
    e_g, w_g, _ = g.energy_trace()
    e_o, w_o, _ = pop.trace()
    assert np.allclose(e_g, e_o, rtol=RTOL, atol=0) and np.allclose(w_g, w_o, rtol=RTOL, atol=0)


@pytest.mark.parametrize("name", ["Ne", "H2O"])
def test_base_terms_match_oracle(pkg, oracle_mod, nn, name):
    system = S.make_system(name)
    g = pkg.LrdmcSystem(system)
    # an installed term must not enter the base terms
    spec = S.default_neural_spec(system)
    g.set_neural_jastrow(spec, S.neural_init(spec, 1, out_scale=1.0))
    o = oracle_mod.OracleSystem(system)
    x = S.initial_positions(system, 41, 7)
    grad, e = g.base_terms(torch.tensor(x, device="cuda"))
    gb, eb = nn.base_terms(o, x)
    assert np.allclose(grad.cpu().numpy(), gb, rtol=1e-10, atol=1e-10 * np.max(np.abs(gb)))
    assert np.allclose(e.cpu().numpy(), eb, rtol=1e-10, atol=0)


def _training_inputs(pkg, oracle_mod, nn, name, n, seed):
    system = S.make_system(name)
    spec = S.default_neural_spec(system)
    g = pkg.LrdmcSystem(system)
    o = oracle_mod.OracleSystem(system)
    x = S.initial_positions(system, n, seed)
    gb, eb = nn.base_terms(o, x)
    return system, spec, g, x, gb, eb


@pytest.mark.parametrize("name,bf16", [("Ne", True), ("Ne", False), ("H2O", True)])
def test_training_forward_matches_oracle(pkg, oracle_mod, nn, name, bf16):
    system, spec, g, x, gb, eb = _training_inputs(pkg, oracle_mod, nn, name, 53, 21)
    params = S.neural_init(spec, 5, out_scale=0.5)
    el, j, q, pairs = g.nj_forward(spec, torch.tensor(params, device="cuda"), torch.tensor(x, device="cuda"),
                                   torch.tensor(gb, device="cuda"), torch.tensor(eb, device="cuda"), bf16)
    EL, J = nn.energy_terms(params.astype(np.float64), spec, x, system.n_up, system.nuc_xyz, gb, eb, bf16)
    EL, J = EL.numpy(), J.numpy()
    scale = np.abs(EL - eb).max()
    assert scale > 1e-2
    assert np.max(np.abs(el.cpu().numpy() - EL)) < 2e-4 * max(1.0, np.abs(EL).max()) + 1e-3 * scale
    assert np.max(np.abs(j.cpu().numpy() - J)) < 1e-4 * max(1.0, np.abs(J).max())


@pytest.mark.parametrize("name", ["Ne", "H2O"])
def test_training_backward_matches_oracle_gradient(pkg, oracle_mod, nn, name):
    """Gradient of the reweighted variance through the hand-written backward
    kernel against the oracle's float64 autograd gradient (same bfloat16
    weights, same configurations)."""
    from paper_1909_01589_gb300 import neural as N

    system, spec, g, x, gb, eb = _training_inputs(pkg, oracle_mod, nn, name, 96, 22)
    params = S.neural_init(spec, 6, out_scale=0.5)
    p = torch.tensor(params, device="cuda", requires_grad=True)
    xt, gbt, ebt = (torch.tensor(v, device="cuda") for v in (x, gb, eb))
    el, j = N.NeuralJastrowTerms.apply(p, g, spec, xt, gbt, ebt, True)
    loss = N.variance_loss(el, j)
    loss.backward()
    ref_loss, ref_grad, _, _ = nn.loss_and_grad(params.astype(np.float64), spec, x, system.n_up, system.nuc_xyz,
                                                gb, eb, bf16=True)
    got = p.grad.cpu().numpy().astype(np.float64)
    assert abs(float(loss) - ref_loss) < 1e-3 * ref_loss
    err = np.linalg.norm(got - ref_grad) / np.linalg.norm(ref_grad)
    assert err < 2e-3, err
    # every block of parameters is checked, not only the largest
    H, D = spec.hidden, spec.n_in
    blocks = [slice(0, H * D), slice(H * D, H * D + H), slice(H * D + H, H * D + H + H * H),
              slice(H * D + H + H * H, H * D + 2 * H + H * H), slice(-H - 1, -1), slice(-1, None)]
    for bl in blocks:
        r = ref_grad[bl]
        if np.linalg.norm(r) > 0:
            assert np.linalg.norm(got[bl] - r) / np.linalg.norm(r) < 1e-2


def test_training_backward_finite_difference(pkg, oracle_mod, nn):
    """Directional derivatives of the GPU objective (float32 weights, no
    rounding) against central differences of the same GPU objective."""
    from paper_1909_01589_gb300 import neural as N

    system, spec, g, x, gb, eb = _training_inputs(pkg, oracle_mod, nn, "Ne", 256, 23)
    params = S.neural_init(spec, 7, out_scale=0.5)
    xt, gbt, ebt = (torch.tensor(v, device="cuda") for v in (x, gb, eb))

    def loss_at(th):
        el, j, _, _ = g.nj_forward(spec, th, xt, gbt, ebt, False)
        return float(N.variance_loss(el, j))

    p = torch.tensor(params, device="cuda", requires_grad=True)
    el, j = N.NeuralJastrowTerms.apply(p, g, spec, xt, gbt, ebt, False)
    N.variance_loss(el, j).backward()
    grad = p.grad.double()
    rng = np.random.default_rng(8)
    for _ in range(3):
        v = torch.tensor(rng.normal(size=params.shape), device="cuda")
        v /= v.norm()
        eps = 3e-3
        fd = (loss_at((p.detach().double() + eps * v).float()) - loss_at((p.detach().double() - eps * v).float())) / (
            2 * eps)
        an = float(grad @ v)
        assert abs(fd - an) < 3e-2 * max(abs(an), 1e-3 * float(grad.norm())), (fd, an)


def test_training_is_bitwise_repeatable(pkg, oracle_mod, nn):
    """The backward kernel sums in a fixed order: the same inputs give the
    same gradient bits (over 4096 configurations, so many blocks contribute),
    and a 30-step training run repeated from the same start ends at the same
    parameters."""
    from paper_1909_01589_gb300 import neural as N

    system = S.neon()
    spec = S.default_neural_spec(system)
    params = torch.tensor(S.neural_init(spec, 3, out_scale=0.5), device="cuda")
    g = pkg.LrdmcSystem(system)
    x = torch.tensor(S.initial_positions(system, 4096, 91), device="cuda")
    gb, eb = g.base_terms(x)
    el, j, q, _ = g.nj_forward(spec, params, x, gb, eb)
    gen = torch.Generator(device="cuda").manual_seed(5)
    d_el = torch.randn(4096, device="cuda", generator=gen)
    d_j = torch.randn(4096, device="cuda", generator=gen)
    g1 = g.nj_backward(spec, params, x, q, d_el, d_j)
    g2 = g.nj_backward(spec, params, x, q, d_el, d_j)
    assert torch.count_nonzero(g1) > 0 and torch.equal(g1, g2)
    runs = [N.train(g, spec, S.neural_init(spec, 3), x, gb, eb, steps=30, batch=1024, seed=7)[0] for _ in range(2)]
    assert torch.equal(runs[0], runs[1])


def test_training_gain_on_neon(pkg, oracle_mod, nn):
    """What the trained term gains: 65536 configurations from a plain
    projection of Ne (a = 0.2, double grid), 400 Adam steps on the GPU
    (reweighted variance, local energies clipped at the median +- 5 mean
    absolute deviations), then the variance of E_L on held-out
    configurations and over a fresh projection with the tabulated term,
    both against the plain Pade Jastrow."""
    from paper_1909_01589_gb300 import neural as N

    system = S.neon()
    spec = S.default_neural_spec(system)
    plain = pkg.LrdmcSystem(system)
    sp = pkg.Spacing(pkg.THIS_WORK)
    x = N.sample_configurations(plain, S.initial_positions(system, 4096, 31), 65536, 0.2, sp, 0.02, -128.9, seed=31)
    grad, e = plain.base_terms(x)
    train_idx, hold = slice(0, 57344), slice(57344, None)
    params, _ = N.train(plain, spec, S.neural_init(spec, 32), x[train_idx], grad[train_idx], e[train_idx],
                        steps=400, seed=33)
    el, j = N.evaluate(plain, spec, params, x[hold], grad[hold], e[hold])
    var_plain = float(torch.var(e[hold]))
    var_nn = float(N.variance_loss(el, j, clip=0.0))
    assert var_nn < 0.85 * var_plain, (var_nn, var_plain)
    # the projection with the trained term has a smaller local-energy spread
    x0 = S.initial_positions(system, 4096, 34)
    spreads = []
    for use in (False, True):
        gsys = pkg.LrdmcSystem(system)
        if use:
            gsys.set_neural_jastrow(spec, params.cpu().numpy())
        gsys.init_walkers(torch.tensor(x0, device="cuda"), seed=35, tau=0.02, e_trial=-128.9, recompute_every=5,
                          trace_capacity=200)
        gsys.step(60, 0.2, sp)
        v = []
        for _ in range(10):
            gsys.step(4, 0.2, sp)
            v.append(np.var(gsys.walkers()["EL"]))
        spreads.append(np.median(v))
    assert spreads[1] < 0.8 * spreads[0], spreads
