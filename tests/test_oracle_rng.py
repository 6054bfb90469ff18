"""Pins of the oracle's counter-based generator, uniform conversion, lattice
rotation, heat bath and comb."""
import numpy as np


def test_philox4x64_matches_numpy(oracle_mod):
    """Philox4x64-10 against NumPy's independent implementation: NumPy bumps
    the 256-bit counter before each block, so its first block for counter c-1
    is Philox(c)."""
    rng = np.random.default_rng(1)
    for _ in range(200):
        key = rng.integers(0, 2**63, size=2, dtype=np.uint64)
        ctr = rng.integers(1, 2**63, size=4, dtype=np.uint64)
        prev = ctr.copy()
        prev[0] -= np.uint64(1)
        g = np.random.Philox(counter=prev, key=key)
        assert np.array_equal(g.random_raw(4).astype(np.uint64), oracle_mod.philox4x64(ctr, key))


def test_uniform_open_interval(oracle_mod):
    """(top 52 bits + 1/2) 2^-52 is exact and stays strictly inside (0, 1)."""
    assert oracle_mod.uniform(0) == 2.0 ** -53
    assert oracle_mod.uniform(2**12 - 1) == 2.0 ** -53
    top = oracle_mod.uniform(2**64 - 1)
    assert top < 1.0 and top == 1.0 - 2.0 ** -53
    assert oracle_mod.uniform(2**63) == 0.5 + 2.0 ** -53


def test_rotation_haar(oracle_mod):
    """Rotations from uniform quaternions are proper orthogonal and uniformly
    distributed: E[R] = 0, E[R_ij^2] = 1/3, E[R_00 R_11] = 0 (Haar moments)."""
    rng = np.random.default_rng(3)
    Rs = np.array([oracle_mod.rotation(*rng.random(3)).reshape(3, 3) for _ in range(20000)])
    eye = np.einsum("nki,nkj->nij", Rs, Rs)
    assert np.max(np.abs(eye - np.eye(3))) < 1e-14
    assert np.max(np.abs(np.linalg.det(Rs) - 1)) < 1e-13
    assert np.max(np.abs(Rs.mean(0))) < 0.02
    assert np.max(np.abs((Rs ** 2).mean(0) - 1 / 3)) < 0.02
    assert abs(np.mean(Rs[:, 0, 0] * Rs[:, 1, 1])) < 0.02


def test_rotation_special_cases(oracle_mod):
    """u1 = 0, u2 = 1/4: q = (1, 0, 0, 0), a rotation by pi about x."""
    R = oracle_mod.rotation(0.0, 0.25, 0.0).reshape(3, 3)
    assert np.allclose(R, np.diag([1.0, -1.0, -1.0]), atol=1e-15)
    R = oracle_mod.rotation(1.0, 0.0, 0.0).reshape(3, 3)  # q = (0,0,0,1): identity
    assert np.allclose(R, np.eye(3), atol=1e-15)


def test_heat_bath_normalised_and_frequencies(oracle_mod):
    """Bin probabilities T_c / b sum to one and the picks of 2e5 uniforms are
    chi-square consistent with them; zero-rate moves are never picked."""
    rng = np.random.default_rng(5)
    T = rng.random(24) * (rng.random(24) > 0.3)
    b = np.sum(T)
    assert abs(np.sum(T / b) - 1) < 1e-15
    n = 200000
    counts = np.zeros(24)
    for u in rng.random(n):
        c, _ = oracle_mod.heat_bath(T, b, u)
        counts[c] += 1
    assert np.all(counts[T == 0] == 0)
    p = T[T > 0] / b
    chi2 = np.sum((counts[T > 0] - n * p) ** 2 / (n * p))
    dof = int(np.sum(T > 0)) - 1
    assert chi2 < dof + 6 * np.sqrt(2 * dof)


def test_heat_bath_edges(oracle_mod):
    T = np.array([0.25, 0.0, 0.25, 0.5])
    assert oracle_mod.heat_bath(T, 1.0, 0.0)[0] == 0
    assert oracle_mod.heat_bath(T, 1.0, 0.25)[0] == 2  # u b on an edge goes up
    assert oracle_mod.heat_bath(T, 1.0, 0.49)[0] == 2
    assert oracle_mod.heat_bath(T, 1.0, 0.999)[0] == 3
    c, m = oracle_mod.heat_bath(T, 1.0, 0.26)
    assert c == 2 and abs(m - 0.01) < 1e-12


def test_comb_identity_and_expectation(oracle_mod):
    """Equal weights give the identity for every offset; over offsets the
    expected copy count of slot s is exactly W w_s / sum(w)."""
    W = 37
    for xi in [1e-9, 0.3, 0.999999]:
        parent, _ = oracle_mod.comb(np.ones(W), xi)
        assert np.array_equal(parent, np.arange(W))
    rng = np.random.default_rng(9)
    w = rng.exponential(size=W)
    counts = np.zeros(W)
    K = 4000
    for xi in (np.arange(K) + 0.5) / K:
        parent, _ = oracle_mod.comb(w, xi)
        assert np.all(np.diff(parent) >= 0)
        c = np.bincount(parent, minlength=W)
        expect = W * w / w.sum()
        assert np.all((c == np.floor(expect)) | (c == np.ceil(expect)))
        counts += c
    assert np.max(np.abs(counts / K - W * w / w.sum())) < 2e-3
