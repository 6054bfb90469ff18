"""ctypes wrapper of the plain FP64 CPU oracle (lrdmc_oracle.c).

TEST INFRASTRUCTURE ONLY: imported by the tests, by ``__graft_entry__.smoke``
and by the CPU-baseline leg of ``bench.py``. The product package never
imports it, and it imports nothing from the product package.

Everything here is argument marshalling around the C functions; the
arithmetic lives in lrdmc_oracle.c, each function citing the passage of
arXiv:1909.01589 (or of the LRDMC method it cites) that it follows.
"""
from __future__ import annotations

import ctypes as ct
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lrdmc_oracle.c")
_LIB = os.path.join(_HERE, "liblrdmc_oracle.so")

MAX_PRIM = 16
SINGLE, THIS_WORK, PREVIOUS, EXPLICIT = 0, 1, 2, 3


def build(force: bool = False) -> str:
    """Compile the oracle into a shared library next to its source."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < max(
        os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_HERE, "lrdmc_oracle.h"))
    ):
        cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared", "-o", _LIB + ".tmp", _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(_LIB + ".tmp", _LIB)
    return _LIB


_lib = None


def lib():
    global _lib
    if _lib is None:
        build()
        L = ct.CDLL(_LIB)
        d, i, u64, vp = ct.c_double, ct.c_int, ct.c_uint64, ct.c_void_p
        L.orc_rc_this_work.restype = d
        L.orc_rc_this_work.argtypes = [d, d, d, d]
        L.orc_slater_groups.restype = i
        L.orc_slater_groups.argtypes = [i, vp, vp, vp, vp, vp, i]
        L.orc_ncore.restype = d
        L.orc_ncore.argtypes = [i, d]
        L.orc_aprime_over_a_this_work.restype = d
        L.orc_aprime_over_a_this_work.argtypes = [i, d, d, d]
        L.orc_aprime_over_a_previous.restype = d
        L.orc_aprime_over_a_previous.argtypes = [d]
        L.orc_speedup.restype = d
        L.orc_speedup.argtypes = [d, d, d]
        L.orc_philox4x64.argtypes = [vp, vp, vp]
        L.orc_uniform.restype = d
        L.orc_uniform.argtypes = [u64]
        L.orc_rotation.argtypes = [d, d, d, vp]
        L.orc_system_create.restype = vp
        L.orc_system_create.argtypes = [i, vp, vp, i, i, i, vp, vp, vp, vp, vp, vp, vp, vp,
                                        i, i, vp, d, d, d, vp, d, i]
        L.orc_system_destroy.argtypes = [vp]
        L.orc_n_ao.restype = i
        L.orc_n_ao.argtypes = [vp]
        L.orc_ao_values.argtypes = [vp, vp, vp, vp, vp]
        L.orc_log_psi.restype = i
        L.orc_log_psi.argtypes = [vp, vp, vp, vp]
        L.orc_inverses.restype = i
        L.orc_inverses.argtypes = [vp, vp, vp, vp]
        L.orc_laplacian_terms.argtypes = [vp, vp, vp, vp, vp, vp]
        L.orc_local_energy.restype = d
        L.orc_local_energy.argtypes = [vp, vp, vp, vp]
        L.orc_sm_update.restype = i
        L.orc_sm_update.argtypes = [vp, i, vp, i, vp, vp]
        L.orc_grad_log_psi.argtypes = [vp, vp, vp, vp, vp]
        L.orc_system_set_neural.restype = i
        L.orc_system_set_neural.argtypes = [vp, i, i, vp, vp, vp]
        L.orc_neural_pair.argtypes = [vp, i, d, vp, vp, vp]
        L.orc_n_candidates.restype = i
        L.orc_n_candidates.argtypes = [vp, i]
        L.orc_p.restype = d
        L.orc_p.argtypes = [vp, vp, vp]
        L.orc_lattice_eval.argtypes = [vp, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp]
        L.orc_heat_bath.restype = i
        L.orc_heat_bath.argtypes = [vp, i, d, d, vp]
        L.orc_comb.argtypes = [i, vp, d, vp, vp, vp]
        L.orc_pop_create.restype = vp
        L.orc_pop_create.argtypes = [vp, i, vp, u64, d, d, i]
        L.orc_pop_destroy.argtypes = [vp]
        L.orc_pop_step.restype = i
        L.orc_pop_step.argtypes = [vp, vp, i, i]
        L.orc_pop_trace.restype = i
        L.orc_pop_trace.argtypes = [vp, vp, vp, vp, i]
        L.orc_pop_walkers.argtypes = [vp, vp, vp, vp, vp, vp, vp, vp]
        L.orc_pop_margins.argtypes = [vp, vp, vp, vp]
        L.orc_pop_moves.restype = ct.c_longlong
        L.orc_pop_moves.argtypes = [vp]
        L.orc_pop_error.restype = i
        L.orc_pop_error.argtypes = [vp]
        _lib = L
    return _lib


def _p(a):
    return None if a is None else a.ctypes.data_as(ct.c_void_p)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


# ---------------------------------------------------------------- parameters
def rc_this_work(a, Z, beta=0.75, kappa=2.5):
    return lib().orc_rc_this_work(a, float(Z), beta, kappa)


def slater_groups(Z):
    n = np.zeros(16, np.int32)
    t = np.zeros(16, np.int32)
    occ = np.zeros(16, np.int32)
    neff = np.zeros(16)
    zeta = np.zeros(16)
    k = lib().orc_slater_groups(int(Z), _p(n), _p(t), _p(neff), _p(zeta), _p(occ), 16)
    return [dict(n=int(n[j]), type=int(t[j]), n_eff=float(neff[j]), zeta=float(zeta[j]), occ=int(occ[j]))
            for j in range(k)]


def ncore(Z, rc):
    return lib().orc_ncore(int(Z), float(rc))


def aprime_over_a_this_work(Z, a, beta=0.75, kappa=2.5):
    return lib().orc_aprime_over_a_this_work(int(Z), a, beta, kappa)


def aprime_over_a_previous(Z):
    return lib().orc_aprime_over_a_previous(float(Z))


def speedup(Z, n_core, ratio):
    return lib().orc_speedup(float(Z), n_core, ratio)


# ---------------------------------------------------------------- RNG
def philox4x64(ctr, key):
    c = np.asarray(ctr, dtype=np.uint64)
    k = np.asarray(key, dtype=np.uint64)
    o = np.zeros(4, dtype=np.uint64)
    lib().orc_philox4x64(_p(c), _p(k), _p(o))
    return o


def uniform(bits):
    return lib().orc_uniform(int(bits))


def rotation(u1, u2, u3):
    R = np.zeros(9)
    lib().orc_rotation(u1, u2, u3, _p(R))
    return R


def heat_bath(T, b, u):
    T = _f64(T)
    m = ct.c_double()
    c = lib().orc_heat_bath(_p(T), len(T), float(b), float(u), ct.byref(m))
    return c, m.value


def comb(wt, xi):
    wt = _f64(wt)
    parent = np.zeros(len(wt), np.int32)
    m = ct.c_double()
    lib().orc_comb(len(wt), _p(wt), float(xi), _p(parent), ct.byref(m), None)
    return parent, m.value


# ---------------------------------------------------------------- lattice
class Lattice(ct.Structure):
    _fields_ = [("a", ct.c_double), ("ap", ct.c_double), ("G", ct.c_int),
                ("pkind", ct.c_int), ("rc", ct.c_double)]


def lattice_for(system, a, kind=SINGLE, beta=0.75, kappa=2.5, rc=None, aprime_over_a=None):
    """Lattice parameters for spacing kind: single grid, this work (Eq. 3 with
    S-13 and Eq. 6), previous (Eq. 2 with r_c = Z/2 and Eq. 4) or explicit.
    For a polyatomic system r_c and a'/a come from the heaviest atom."""
    Zmax = float(np.max(system.Z))
    if kind == SINGLE:
        return Lattice(a, a, 1, 0, 1.0)
    if kind == THIS_WORK:
        r = rc_this_work(a, Zmax, beta, kappa)
        ratio = aprime_over_a_this_work(int(round(Zmax)), a, beta, kappa)
        return Lattice(a, a * ratio, 2, 0, r)
    if kind == PREVIOUS:
        return Lattice(a, a * aprime_over_a_previous(Zmax), 2, 1, Zmax / 2.0)
    if kind == EXPLICIT:
        return Lattice(a, a * aprime_over_a, 2, 0, rc)
    raise ValueError(kind)


# ---------------------------------------------------------------- system
class OracleSystem:
    def __init__(self, system):
        L = lib()
        self.sys = system
        center, l, kind, nprim, neff, zeta, alpha, coef = system.shell_arrays()
        self._keep = [center, l, kind, nprim, neff, zeta, alpha, coef]
        en_b1 = _f64(system.en_b1 if system.en_b1 is not None else np.zeros(system.n_nuc))
        C = _f64(system.C)
        xyz = _f64(system.nuc_xyz)
        Z = _f64(system.Z)
        self._keep += [en_b1, C, xyz, Z]
        self.h = L.orc_system_create(
            system.n_nuc, _p(xyz), _p(Z), system.n_up, system.n_dn,
            len(system.shells), _p(center), _p(l), _p(kind), _p(nprim), _p(neff), _p(zeta),
            _p(alpha), _p(coef), system.n_ao, system.n_mo, _p(C),
            system.b_ee, system.c_par, system.c_anti, _p(en_b1), system.en_b2, int(system.ee_on))
        if not self.h:
            raise ValueError("oracle rejected the system")
        self.N = system.N
        self.n_up, self.n_dn = system.n_up, system.n_dn

    def __del__(self):
        if getattr(self, "h", None):
            lib().orc_system_destroy(self.h)
            self.h = None

    def ao_values(self, r):
        n = self.sys.n_ao
        chi, g, lp = np.zeros(n), np.zeros((n, 3)), np.zeros(n)
        lib().orc_ao_values(self.h, _p(_f64(r)), _p(chi), _p(g), _p(lp))
        return chi, g, lp

    def log_psi(self, x):
        la, sg = ct.c_double(), ct.c_double()
        lib().orc_log_psi(self.h, _p(_f64(x)), ct.byref(la), ct.byref(sg))
        return la.value, sg.value

    def inverses(self, x):
        Au = np.zeros((self.n_up, self.n_up))
        Ad = np.zeros((max(self.n_dn, 1), max(self.n_dn, 1)))
        rc = lib().orc_inverses(self.h, _p(_f64(x)), _p(Au), _p(Ad))
        if rc:
            raise ValueError("singular Slater matrix")
        return Au, Ad

    def laplacian_terms(self, x, Au=None, Ad=None):
        if Au is None:
            Au, Ad = self.inverses(x)
        lap, V = ct.c_double(), ct.c_double()
        lib().orc_laplacian_terms(self.h, _p(_f64(x)), _p(Au), _p(Ad), ct.byref(lap), ct.byref(V))
        return lap.value, V.value

    def local_energy(self, x, Au=None, Ad=None):
        if Au is None:
            Au, Ad = self.inverses(x)
        return lib().orc_local_energy(self.h, _p(_f64(x)), _p(Au), _p(Ad))

    def grad_log_psi(self, x, Au=None, Ad=None):
        """grad_i log|psi_G| for every electron, [N][3]."""
        if Au is None:
            Au, Ad = self.inverses(x)
        g = np.zeros((self.N, 3))
        lib().orc_grad_log_psi(self.h, _p(_f64(x)), _p(Au), _p(Ad), _p(g))
        return g

    def set_neural(self, table):
        """Install (or, with None, remove) the tabulated neural pair term:
        ``table`` is an oracle.neural.Table."""
        if table is None:
            rc = lib().orc_system_set_neural(self.h, 0, 0, None, None, None)
            self._nj = None
        else:
            rcut = _f64(table.r_cut)
            species = np.ascontiguousarray(table.species, dtype=np.int32)
            nodes = _f64(table.nodes)
            self._nj = (rcut, species, nodes)
            rc = lib().orc_system_set_neural(self.h, len(rcut), table.n_cells, _p(rcut), _p(species), _p(nodes))
        if rc:
            raise ValueError("oracle rejected the neural table")
        return self

    def neural_pair(self, channel, r):
        g, g1, g2 = ct.c_double(), ct.c_double(), ct.c_double()
        lib().orc_neural_pair(self.h, channel, float(r), ct.byref(g), ct.byref(g1), ct.byref(g2))
        return g.value, g1.value, g2.value

    def sm_update(self, spin, Ainv, l, r_new):
        A = np.ascontiguousarray(Ainv, dtype=np.float64).copy()
        ratio = ct.c_double()
        rc = lib().orc_sm_update(self.h, spin, _p(A), l, _p(_f64(r_new)), ct.byref(ratio))
        return A, ratio.value, rc

    def n_candidates(self, G):
        return lib().orc_n_candidates(self.h, G)

    def p(self, lat, r):
        return lib().orc_p(self.h, ct.byref(lat), _p(_f64(r)))

    def lattice_eval(self, lat, x, R):
        x = _f64(x)
        Au, Ad = self.inverses(x)
        P = self.n_candidates(lat.G)
        ratio, w, T = np.zeros(P), np.zeros(P), np.zeros(P)
        b, EL = ct.c_double(), ct.c_double()
        lib().orc_lattice_eval(self.h, ct.byref(lat), _p(x), _p(Au), _p(Ad), _p(_f64(R)),
                               _p(ratio), _p(w), _p(T), ct.byref(b), ct.byref(EL))
        return dict(ratio=ratio, w=w, T=T, b=b.value, EL=EL.value)


class OraclePopulation:
    """W walkers projected with the continuous-time lattice Green's function."""

    def __init__(self, osys: OracleSystem, x0, seed, tau, e_trial=0.0, recompute_every=10):
        self.osys = osys
        x0 = _f64(x0)
        self.W = x0.shape[0]
        self.h = lib().orc_pop_create(osys.h, self.W, _p(x0), int(seed), float(tau),
                                      float(e_trial), int(recompute_every))
        if not self.h:
            raise ValueError("oracle rejected the population")
        err = lib().orc_pop_error(self.h)
        if err:
            raise ValueError(f"oracle init error {err}")

    def __del__(self):
        if getattr(self, "h", None):
            lib().orc_pop_destroy(self.h)
            self.h = None

    def step(self, lat, n_steps=1, n_threads=1):
        rc = lib().orc_pop_step(self.h, ct.byref(lat), int(n_steps), int(n_threads))
        if rc:
            raise RuntimeError(f"oracle step error {rc}")

    def trace(self, max_n=1 << 20):
        e, w, j = np.zeros(max_n), np.zeros(max_n), np.zeros(max_n)
        n = lib().orc_pop_trace(self.h, _p(e), _p(w), _p(j), max_n)
        return e[:n].copy(), w[:n].copy(), j[:n].copy()

    def walkers(self, G):
        W, N = self.W, self.osys.N
        P = self.osys.n_candidates(G)
        x = np.zeros((W, N, 3))
        EL, b = np.zeros(W), np.zeros(W)
        T = np.zeros((W, P))
        logw, jumps, parent = np.zeros(W), np.zeros(W, np.int32), np.zeros(W, np.int32)
        lib().orc_pop_walkers(self.h, _p(x), _p(EL), _p(b), _p(T), _p(logw), _p(jumps), _p(parent))
        return dict(x=x, EL=EL, b=b, T=T, logw_pre=logw, jumps_pre=jumps, parent=parent)

    def margins(self, teeth=False):
        """Distances of the last interval's decisions from their bin edges:
        per walker slot (smallest over its waiting-time and heat-bath
        decisions, relative to tau and to b), the comb's smallest (relative
        to the total weight) and, with teeth, the comb's per new slot."""
        m = np.zeros(self.W)
        mt = np.zeros(self.W)
        mc = ct.c_double()
        lib().orc_pop_margins(self.h, _p(m), ct.byref(mc), _p(mt))
        return (m, mc.value, mt) if teeth else (m, mc.value)

    @property
    def moves(self):
        return lib().orc_pop_moves(self.h)
