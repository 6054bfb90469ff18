"""Seeded synthetic inputs for LRDMC: trial-function systems and walker starts.

This module builds the inputs that both the CUDA library and the CPU oracle
consume. It holds none of the projection method's arithmetic: it only
writes down trial functions (nuclei, Slater-type or contracted-Gaussian
shells, orbital coefficients, Pade Jastrow parameters) and draws the first
electron positions from a seeded generator.

The paper's own guiding functions (optimised JSD/JAGP with cc-pVDZ or ADZP
bases, supplement Sec. III) are not reproducible here, so the systems are
the simple Slater-Jastrow atoms of the workloads this library is measured on:

* ``helium``: 1s Slater orbital exp(-1.6875 r) for each spin, Pade e-e
  Jastrow r / (2 (1 + r)).
* ``neon``: a single determinant of 1s/2s/2p Slater-type orbitals with
  exponents from Slater's rules, Pade e-e and e-n Jastrow factors.
* ``hydrogen``, ``hydrogenic_ion`` and ``be_bare`` are exactly solvable
  checks: with the exact orbital the local energy is constant.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

MAX_PRIM = 16

STO = 0
GTO = 1


@dataclass
class Shell:
    center: int
    l: int
    kind: int = STO
    n_eff: float = 1.0
    zeta: float = 1.0
    alpha: list = field(default_factory=list)
    coef: list = field(default_factory=list)


@dataclass
class System:
    name: str
    nuc_xyz: np.ndarray
    Z: np.ndarray
    n_up: int
    n_dn: int
    shells: list
    C: np.ndarray  # [n_ao][n_mo]
    b_ee: float = 1.0
    c_par: float = 0.25
    c_anti: float = 0.5
    en_b1: np.ndarray = None
    en_b2: float = 1.0
    ee_on: bool = True
    # shell whose radial density seeds the start radius of each orbital
    orbital_shell: list = None
    exact_energy: float | None = None

    @property
    def N(self) -> int:
        return self.n_up + self.n_dn

    @property
    def n_nuc(self) -> int:
        return len(self.Z)

    @property
    def n_ao(self) -> int:
        return sum(2 * s.l + 1 for s in self.shells)

    @property
    def n_mo(self) -> int:
        return self.C.shape[1]

    def shell_arrays(self):
        """Flat arrays describing the shells (prim arrays padded to MAX_PRIM)."""
        ns = len(self.shells)
        center = np.array([s.center for s in self.shells], dtype=np.int32)
        l = np.array([s.l for s in self.shells], dtype=np.int32)
        kind = np.array([s.kind for s in self.shells], dtype=np.int32)
        nprim = np.array([len(s.alpha) for s in self.shells], dtype=np.int32)
        neff = np.array([s.n_eff for s in self.shells], dtype=np.float64)
        zeta = np.array([s.zeta for s in self.shells], dtype=np.float64)
        alpha = np.zeros((ns, MAX_PRIM))
        coef = np.zeros((ns, MAX_PRIM))
        for q, s in enumerate(self.shells):
            alpha[q, : len(s.alpha)] = s.alpha
            coef[q, : len(s.coef)] = s.coef
        return center, l, kind, nprim, neff, zeta, alpha, coef


def _atom(Z: float):
    return np.zeros((1, 3)), np.array([float(Z)])


def hydrogen(zeta: float = 1.0) -> System:
    """H atom, psi = exp(-zeta r); exact for zeta = 1 (E = -0.5)."""
    return hydrogenic_ion(1, zeta)


def hydrogenic_ion(Z: int, zeta: float | None = None) -> System:
    """One electron around charge Z, psi = exp(-zeta r); exact when zeta = Z."""
    zeta = float(Z) if zeta is None else zeta
    xyz, Zs = _atom(Z)
    return System(
        name=f"Z{Z}_1e", nuc_xyz=xyz, Z=Zs, n_up=1, n_dn=0,
        shells=[Shell(0, 0, STO, 1.0, zeta)], C=np.eye(1),
        c_par=0.0, c_anti=0.0, en_b1=np.zeros(1), orbital_shell=[0],
        exact_energy=-0.5 * Z * Z if zeta == Z else None,
    )


def helium(zeta: float = 1.6875) -> System:
    """He, 1s exp(-zeta r) per spin times the e-e Pade factor r / (2 (1 + r))
    and the e-n factor exp(-(2 - zeta) r / (1 + r)), whose slope completes the
    nuclear cusp (without it E_L ~ -(2 - zeta)/r near the nucleus and the
    lattice Hamiltonian, whose kinetic part is bounded, has no ground state)."""
    xyz, Zs = _atom(2)
    return System(
        name="He", nuc_xyz=xyz, Z=Zs, n_up=1, n_dn=1,
        shells=[Shell(0, 0, STO, 1.0, zeta)], C=np.eye(1),
        b_ee=1.0, c_par=0.25, c_anti=0.5, en_b1=np.array([2.0 - zeta]), en_b2=1.0,
        orbital_shell=[0],
    )


def be_bare() -> System:
    """Be nucleus with four non-interacting electrons in the exact hydrogenic
    1s = exp(-4 r) and 2s = (1 - 2 r) exp(-2 r) orbitals: E = 2(-8) + 2(-2) = -20
    for every configuration; the 2s node makes fixed-node sign flips occur."""
    xyz, Zs = _atom(4)
    shells = [Shell(0, 0, STO, 1.0, 4.0), Shell(0, 0, STO, 1.0, 2.0), Shell(0, 0, STO, 2.0, 2.0)]
    C = np.array([[1.0, 0.0], [0.0, 1.0], [0.0, -2.0]])
    return System(
        name="Be_bare", nuc_xyz=xyz, Z=Zs, n_up=2, n_dn=2, shells=shells, C=C,
        c_par=0.0, c_anti=0.0, en_b1=np.zeros(1), ee_on=False,
        orbital_shell=[0, 2], exact_energy=-20.0,
    )


# Slater's-rule exponents for the closed-shell atoms used here.
# Ne: 1s (10 - 0.30) / 1 = 9.70; 2s2p (10 - 7*0.35 - 2*0.85) / 2 = 2.925.
NE_ZETA_1S = 9.70
NE_ZETA_2SP = 2.925


def neon() -> System:
    """Ne, one determinant per spin of hydrogenic-style orbitals with
    Slater's-rule exponents: 1s = exp(-z1 r), 2s = (1 + (z2 - z1) r) exp(-z2 r),
    2p = (x, y, z) exp(-z2 r), z1 = 9.70, z2 = 2.925. Both s orbitals have the
    slope -z1 at the nucleus, so the e-n factor -(10 - z1) r / (1 + r)
    completes the nuclear cusp for every configuration; the e-e Pade factor
    has 1/2 (antiparallel) and 1/4 (parallel), b = 1."""
    xyz, Zs = _atom(10)
    z1, z2 = NE_ZETA_1S, NE_ZETA_2SP
    shells = [
        Shell(0, 0, STO, 1.0, z1),
        Shell(0, 0, STO, 1.0, z2),
        Shell(0, 0, STO, 2.0, z2),
        Shell(0, 1, STO, 2.0, z2),
    ]
    C = np.zeros((6, 5))
    C[0, 0] = 1.0
    C[1, 1] = 1.0
    C[2, 1] = z2 - z1
    C[3, 2] = C[4, 3] = C[5, 4] = 1.0
    return System(
        name="Ne", nuc_xyz=xyz, Z=Zs, n_up=5, n_dn=5, shells=shells, C=C,
        b_ee=1.0, c_par=0.25, c_anti=0.5, en_b1=np.array([10.0 - z1]), en_b2=1.0,
        orbital_shell=[0, 2, 3, 3, 3],
    )


def tiny_mixed(seed: int = 7) -> System:
    """Four-electron check system (2 up, 2 down) on two nuclei with mixed
    s/p/d Slater shells, one contracted-Gaussian shell and a dense,
    well-conditioned orbital-coefficient matrix: used for brute-force checks."""
    rng = np.random.default_rng(seed)
    xyz = np.array([[0.0, 0.0, 0.0], [0.3, -0.4, 1.1]])
    Zs = np.array([3.0, 1.0])
    shells = [
        Shell(0, 0, STO, 1.0, 2.7),
        Shell(0, 1, STO, 2.0, 1.3),
        Shell(1, 0, GTO, alpha=[3.1, 0.62, 0.17], coef=[0.2, 0.5, 0.4]),
        Shell(0, 2, STO, 3.0, 1.1),
    ]
    n_ao = 1 + 3 + 1 + 5
    C = np.zeros((n_ao, 2))
    C[:, 0] = rng.normal(0, 0.3, n_ao)
    C[:, 1] = rng.normal(0, 0.3, n_ao)
    C[0, 0] += 1.0
    C[1, 1] += 1.0
    return System(
        name="tiny_mixed", nuc_xyz=xyz, Z=Zs, n_up=2, n_dn=2, shells=shells, C=C,
        b_ee=0.8, c_par=0.25, c_anti=0.5, en_b1=np.array([0.2, 0.1]), en_b2=1.3,
        orbital_shell=[0, 1],
    )


def cluster(n_centers: int = 8, n_per_spin: int = 24, d_shells: int = 0, seed: int = 3) -> System:
    """Synthetic many-centre system for size checks: nuclei (Z = 3) on a
    cube-like grid 2.5 bohr apart, each with a 1s (zeta 2.2) and a 2p
    (zeta 1.1) Slater shell, 3d shells (zeta 0.9) on the first d_shells
    centres; n_per_spin electrons per spin in the first orbitals of a
    diagonally dominant coefficient matrix (orbital m is AO m plus small
    admixtures), e-n factors with the 1s cusp."""
    rng = np.random.default_rng(seed)
    pts = [(i, j, k) for i in range(2) for j in range(2) for k in range(2)]
    pts += [(i, j, 2) for i in range(2) for j in range(2)]
    xyz = 2.5 * np.array(pts[:n_centers], dtype=np.float64)
    Zs = np.full(n_centers, 3.0)
    shells = []
    for c in range(n_centers):
        shells.append(Shell(c, 0, STO, 1.0, 2.2))
        shells.append(Shell(c, 1, STO, 2.0, 1.1))
    for c in range(d_shells):
        shells.append(Shell(c, 2, STO, 3.0, 0.9))
    n_ao = sum(2 * sh.l + 1 for sh in shells)
    if n_per_spin > n_ao:
        raise ValueError("more electrons per spin than orbitals")
    C = 0.05 * rng.normal(size=(n_ao, n_per_spin))
    for m in range(n_per_spin):
        C[m, m] += 1.0
    owner = []
    for q, sh in enumerate(shells):
        owner += [q] * (2 * sh.l + 1)
    return System(
        name="cluster", nuc_xyz=xyz, Z=Zs, n_up=n_per_spin, n_dn=n_per_spin, shells=shells, C=C,
        b_ee=1.0, c_par=0.25, c_anti=0.5, en_b1=np.full(n_centers, 3.0 - 2.2), en_b2=1.0,
        orbital_shell=owner[:n_per_spin],
    )


# ---------------------------------------------------------------- Gaussian fits
_FIT_CACHE = {}


def sto_gaussian_fit(m: float, l: int, n: int = 6):
    """Even-tempered least-squares fit of a Slater radial function r^m e^(-r)
    (zeta = 1) by n Gaussians sum_p c_p exp(-alpha_p r^2), alpha_p =
    alpha_0 beta^p, weighted by the volume element of the whole function
    r^(2 + 2l). The even-tempered form keeps the exponents apart so the
    coefficients stay well conditioned. For exponent zeta the primitives
    are alpha_p zeta^2 with coefficients c_p zeta^m (the radial part scales
    as zeta^-m (zeta r)^m e^(-zeta r))."""
    key = (float(m), int(l), int(n))
    if key in _FIT_CACHE:
        return _FIT_CACHE[key]
    from scipy.optimize import least_squares

    r = np.concatenate([np.linspace(1e-4, 0.5, 300), np.linspace(0.5, 30.0, 1500)])
    wgt = r ** (1 + l)
    target = r ** m * np.exp(-r)

    def solve(p):
        a = np.exp(p[0]) * np.exp(p[1]) ** np.arange(n)
        G = np.exp(-np.outer(r * r, a))
        c, *_ = np.linalg.lstsq(G * wgt[:, None], target * wgt, rcond=None)
        return a, c, (G @ c - target) * wgt

    res = least_squares(lambda p: solve(p)[2], [np.log(0.04), np.log(3.0)],
                        bounds=([np.log(1e-3), np.log(1.6)], [np.log(10.0), np.log(8.0)]),
                        xtol=1e-12, ftol=1e-12)
    a, c, _ = solve(res.x)
    _FIT_CACHE[key] = (a, c)
    return a, c


def gto_shell(center: int, l: int, n_eff: float, zeta: float) -> Shell:
    """Contracted-Gaussian stand-in for the Slater shell r^(n-1-l) e^(-zeta r)."""
    m = n_eff - 1.0 - l
    a, c = sto_gaussian_fit(m, l)
    # n_eff and zeta record the Slater shell the contraction stands in for
    # (start positions use its radial density); the evaluation reads only
    # the Gaussian exponents and coefficients of a GTO shell
    return Shell(center, l, GTO, n_eff=n_eff, zeta=zeta, alpha=list(a * zeta * zeta), coef=list(c * zeta ** m))


def _slater_atom_shells(Z: int):
    """(n, l, n*, zeta, electrons) of a closed-shell atom by Slater's rules
    (occupations in Madelung order)."""
    nstar = {1: 1.0, 2: 2.0, 3: 3.0, 4: 3.7, 5: 4.0}
    groups = {  # Z -> list of (n, kind, occupation) in Slater's order
        18: [(1, "sp", 2), (2, "sp", 8), (3, "sp", 8)],
        36: [(1, "sp", 2), (2, "sp", 8), (3, "sp", 8), (3, "d", 10), (4, "sp", 8)],
        8: [(1, "sp", 2), (2, "sp", 6)],
    }[Z]
    out = []
    for gi, (n, kind, occ) in enumerate(groups):
        s = (occ - 1) * (0.30 if n == 1 else 0.35)
        for gj, (n2, kind2, occ2) in enumerate(groups):
            if gj == gi:
                continue
            if kind == "sp":
                if n2 == n - 1:
                    s += 0.85 * occ2
                elif n2 < n - 1:
                    s += occ2
            elif gj < gi:
                s += occ2
        zeta = (Z - s) / nstar[n]
        if kind == "sp":
            out.append((n, 0, nstar[n], zeta))
            if occ > 2:
                out.append((n, 1, nstar[n], zeta))
        else:
            out.append((n, 2, nstar[n], zeta))
    return out


def _gto_atom(Z: int, name: str) -> System:
    """Closed-shell atom Z with one determinant of STO-6G-style orbitals
    (Slater's-rule exponents, each Slater function fitted by 6 Gaussians);
    Gaussians have no nuclear cusp, so the e-n factor -Z r/(1 + Z r) supplies
    all of it (slope -Z at the nucleus, bounded far away)."""
    xyz, Zs = _atom(Z)
    shells = [gto_shell(0, l, nst, zeta) for (n, l, nst, zeta) in _slater_atom_shells(Z)]
    n_ao = sum(2 * s.l + 1 for s in shells)
    nel = Z // 2
    C = np.eye(n_ao)[:, :nel]
    orbital_shell = []
    for q, s in enumerate(shells):
        orbital_shell += [q] * (2 * s.l + 1)
    return System(
        name=name, nuc_xyz=xyz, Z=Zs, n_up=nel, n_dn=nel, shells=shells, C=C,
        b_ee=1.0, c_par=0.25, c_anti=0.5, en_b1=np.array([float(Z)]), en_b2=float(Z),
        orbital_shell=orbital_shell[:nel],
    )


def argon() -> System:
    """Ar (Z = 18, 9 up / 9 down): 1s, 2s, 2p, 3s, 3p STO-6G-style orbitals."""
    return _gto_atom(18, "Ar")


def krypton() -> System:
    """Kr (Z = 36, 18 up / 18 down): 1s ... 4s, 4p and 3d STO-6G-style
    orbitals; the 4s/4p Slater functions have the non-integer n* = 3.7."""
    return _gto_atom(36, "Kr")


WATER_H = np.array([[1.430, 1.107, 0.0], [-1.430, 1.107, 0.0]])


def water() -> System:
    """H2O: O at the origin, H at (+-1.430, 1.107, 0) bohr; STO-6G-style O 1s,
    2s, 2p (Slater's rules) and H 1s (zeta = 1.24) Gaussians; five doubly
    occupied orbitals from a fixed, non-degenerate mixing; e-n factors with
    the full cusps -Z_I r/(1 + 4 r)."""
    xyz = np.vstack([np.zeros(3), WATER_H])
    Zs = np.array([8.0, 1.0, 1.0])
    oshells = [gto_shell(0, l, nst, zeta) for (n, l, nst, zeta) in _slater_atom_shells(8)]
    shells = oshells + [gto_shell(1, 0, 1.0, 1.24), gto_shell(2, 0, 1.0, 1.24)]
    # AOs: O1s, O2s, O2px, O2py, O2pz, H1 1s, H2 1s
    C = np.zeros((7, 5))
    C[0, 0] = 1.0
    C[1, 1], C[5, 1], C[6, 1] = 1.0, 0.3, 0.3
    C[2, 2], C[5, 2], C[6, 2] = 1.0, 0.4, -0.4
    C[3, 3], C[5, 3], C[6, 3] = 1.0, 0.25, 0.25
    C[4, 4] = 1.0
    return System(
        name="H2O", nuc_xyz=xyz, Z=Zs, n_up=5, n_dn=5, shells=shells, C=C,
        b_ee=1.0, c_par=0.25, c_anti=0.5, en_b1=Zs.copy(), en_b2=4.0,
        orbital_shell=[0, 1, 2, 2, 2],
    )


SYSTEMS = {
    "H": hydrogen,
    "He": helium,
    "Ne": neon,
    "Be_bare": be_bare,
    "tiny_mixed": tiny_mixed,
    "Ar": argon,
    "Kr": krypton,
    "H2O": water,
}


def make_system(name: str, **kw) -> System:
    return SYSTEMS[name](**kw)


def initial_positions(system: System, n_walkers: int, seed: int) -> np.ndarray:
    """Start configurations [W][N][3]: electron i of a spin block occupies
    orbital i of that block; its distance from the orbital's centre is drawn
    from the radial density r^(2n) exp(-2 zeta r) of the Slater shell seeding
    that orbital (a Gamma(2n + 1, 1/(2 zeta)) variate; a Gaussian shell uses
    the Slater shell its contraction was fitted to), its direction uniformly
    on the sphere."""
    rng = np.random.default_rng(np.random.PCG64(seed))
    N = system.N
    x = np.empty((n_walkers, N, 3))
    orbital_shell = system.orbital_shell or [0]  # a system without the map seeds from its first shell
    for i in range(N):
        m = i if i < system.n_up else i - system.n_up
        sh = system.shells[orbital_shell[m % len(orbital_shell)]]
        r = rng.gamma(2.0 * sh.n_eff + 1.0, 1.0 / (2.0 * sh.zeta), n_walkers)
        v = rng.normal(size=(n_walkers, 3))
        v /= np.linalg.norm(v, axis=1, keepdims=True)
        x[:, i, :] = system.nuc_xyz[sh.center][None, :] + r[:, None] * v
    return x


def random_rotations(n: int, seed: int) -> np.ndarray:
    """Uniformly random 3x3 rotation matrices [n][9] (row-major, column k is
    the rotated axis e_k), drawn with SciPy: inputs for single-evaluation
    checks that bypass the in-kernel rotation draw."""
    from scipy.spatial.transform import Rotation

    return Rotation.random(n, random_state=seed).as_matrix().reshape(n, 9).copy()


# ---------------------------------------------------------------- neural pair Jastrow: data only
@dataclass
class NeuralSpec:
    """Shape of the neural pair term of the Jastrow factor (data only).

    Channels: 0 = electron pairs of equal spin, 1 = opposite spins,
    2 + s = electron-nucleus pairs of nucleus species s (``species[I]`` per
    nucleus). The network reads the radial features r^2/(r^2 + ell_k^2) and
    a one-hot channel code; ``r_cut`` per channel ends the term smoothly;
    the lattice projection interpolates it on ``n_cells`` cells per channel.
    Parameters are a flat float32 vector: W1 [hidden][n_in], b1 [hidden],
    W2 [hidden][hidden], b2 [hidden], w3 [hidden], b3 [1]."""

    ell: tuple
    r_cut: tuple
    species: tuple
    hidden: int = 64
    n_cells: int = 512

    @property
    def n_ch(self) -> int:
        return len(self.r_cut)

    @property
    def n_in(self) -> int:
        return len(self.ell) + self.n_ch

    @property
    def n_params(self) -> int:
        H, D = self.hidden, self.n_in
        return H * D + H + H * H + H + H + 1


def default_neural_spec(system: System, n_cells: int = 512) -> NeuralSpec:
    """Six feature lengths from 0.5/Z_max to 4 bohr (geometric), e-e terms cut
    at 6 bohr, e-n terms at 5 bohr; one e-n channel per distinct Z (heaviest
    first)."""
    Zs = sorted({float(z) for z in system.Z}, reverse=True)
    species = tuple(Zs.index(float(z)) for z in system.Z)
    lo, hi = 0.5 / Zs[0], 4.0
    ell = tuple(float(lo * (hi / lo) ** (k / 5.0)) for k in range(6))
    r_cut = (6.0, 6.0) + tuple(5.0 for _ in Zs)
    return NeuralSpec(ell=ell, r_cut=r_cut, species=species, n_cells=n_cells)


def neural_init(spec: NeuralSpec, seed: int, out_scale: float = 0.0) -> np.ndarray:
    """Seeded initial parameters (float32): W1 ~ N(0, 1/n_in), W2 ~ N(0, 1/hidden),
    biases 0, w3 ~ out_scale * N(0, 1/hidden) (0: the term starts at zero)."""
    rng = np.random.default_rng(seed)
    H, D = spec.hidden, spec.n_in
    parts = [rng.normal(size=H * D) / np.sqrt(D), np.zeros(H), rng.normal(size=H * H) / np.sqrt(H), np.zeros(H),
             out_scale * rng.normal(size=H) / np.sqrt(H), np.zeros(1)]
    return np.concatenate(parts).astype(np.float32)


# ---------------------------------------------------------------- JSON form of a system
def system_to_dict(system: System) -> dict:
    """The system as plain JSON types: nuclei, charges, spin counts, shells,
    orbital coefficients [n_ao][n_mo] and the Pade Jastrow parameters."""
    def shell(s):
        d = {"center": int(s.center), "l": int(s.l), "kind": "sto" if s.kind == STO else "gto"}
        if s.kind == STO:
            d.update(n_eff=float(s.n_eff), zeta=float(s.zeta))
        else:
            d.update(alpha=[float(v) for v in s.alpha], coef=[float(v) for v in s.coef],
                     n_eff=float(s.n_eff), zeta=float(s.zeta))
        return d

    return {
        "name": system.name,
        "nuclei": np.asarray(system.nuc_xyz, float).reshape(-1, 3).tolist(),
        "Z": np.asarray(system.Z, float).tolist(),
        "n_up": int(system.n_up), "n_dn": int(system.n_dn),
        "shells": [shell(s) for s in system.shells],
        "C": np.asarray(system.C, float).tolist(),
        "jastrow": {"b_ee": float(system.b_ee), "c_par": float(system.c_par), "c_anti": float(system.c_anti),
                    "en_b1": None if system.en_b1 is None else np.asarray(system.en_b1, float).tolist(),
                    "en_b2": float(system.en_b2), "ee_on": bool(system.ee_on)},
        "orbital_shell": None if system.orbital_shell is None else [int(q) for q in system.orbital_shell],
        "exact_energy": system.exact_energy,
    }


def system_from_dict(d: dict) -> System:
    """Inverse of system_to_dict; raises ValueError for a malformed system
    (shapes, shell kinds, centres, coefficient rows against the shells)."""
    def need(obj, key, where):
        if key not in obj:
            raise ValueError(f"system: missing '{key}' in {where}")
        return obj[key]

    nuc = np.asarray(need(d, "nuclei", "system"), dtype=np.float64)
    Z = np.asarray(need(d, "Z", "system"), dtype=np.float64)
    if nuc.ndim != 2 or nuc.shape[1] != 3 or len(Z) != len(nuc) or len(Z) == 0:
        raise ValueError("system: 'nuclei' must be [n_nuc][3] and 'Z' [n_nuc]")
    n_up, n_dn = int(need(d, "n_up", "system")), int(need(d, "n_dn", "system"))
    if n_up < 1 or n_dn < 0:
        raise ValueError("system: need n_up >= 1 and n_dn >= 0")
    shells = []
    for q, s in enumerate(need(d, "shells", "system")):
        where = f"shell {q}"
        center, l = int(need(s, "center", where)), int(need(s, "l", where))
        if not 0 <= center < len(Z) or not 0 <= l <= 2:
            raise ValueError(f"system: {where} has centre {center} or l = {l} out of range")
        kind = need(s, "kind", where)
        if kind == "sto":
            zeta = float(need(s, "zeta", where))
            if zeta <= 0.0:
                raise ValueError(f"system: {where} needs zeta > 0")
            shells.append(Shell(center, l, STO, float(need(s, "n_eff", where)), zeta))
        elif kind == "gto":
            alpha, coef = list(need(s, "alpha", where)), list(need(s, "coef", where))
            if not 1 <= len(alpha) <= MAX_PRIM or len(coef) != len(alpha) or min(alpha) <= 0.0:
                raise ValueError(f"system: {where} needs 1..{MAX_PRIM} positive exponents with one coefficient each")
            shells.append(Shell(center, l, GTO, float(s.get("n_eff", 1.0)), float(s.get("zeta", 1.0)),
                                [float(v) for v in alpha], [float(v) for v in coef]))
        else:
            raise ValueError(f"system: {where} has kind '{kind}' (sto or gto)")
    C = np.asarray(need(d, "C", "system"), dtype=np.float64)
    n_ao = sum(2 * s.l + 1 for s in shells)
    if C.ndim != 2 or C.shape[0] != n_ao or C.shape[1] < max(n_up, n_dn):
        raise ValueError(f"system: 'C' must be [{n_ao}][>= {max(n_up, n_dn)}] for these shells")
    j = need(d, "jastrow", "system")
    en_b1 = j.get("en_b1")
    if en_b1 is not None and len(en_b1) != len(Z):
        raise ValueError("system: 'en_b1' needs one value per nucleus")
    orb = d.get("orbital_shell")
    if orb is not None and any(not 0 <= int(q) < len(shells) for q in orb):
        raise ValueError("system: 'orbital_shell' names a shell that does not exist")
    return System(
        name=str(d.get("name", "system")), nuc_xyz=nuc, Z=Z, n_up=n_up, n_dn=n_dn, shells=shells, C=C,
        b_ee=float(j.get("b_ee", 1.0)), c_par=float(j.get("c_par", 0.25)), c_anti=float(j.get("c_anti", 0.5)),
        en_b1=None if en_b1 is None else np.asarray(en_b1, dtype=np.float64), en_b2=float(j.get("en_b2", 1.0)),
        ee_on=bool(j.get("ee_on", True)), orbital_shell=None if orb is None else [int(q) for q in orb],
        exact_energy=d.get("exact_energy"),
    )


def save_system(system: System, path: str) -> None:
    import json

    with open(path, "w") as f:
        json.dump(system_to_dict(system), f, indent=1)


def load_system(path: str) -> System:
    import json

    with open(path) as f:
        return system_from_dict(json.load(f))
