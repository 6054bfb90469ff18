"""Python binding of liblrdmc.so, the GB300 (sm_103a) LRDMC library.

Argument marshalling only: every step of the projection runs in the CUDA
kernels behind the C ABI of include/lrdmc.h. PyTorch provides the device
memory (the population workspace, configuration and output buffers) and
the CUDA stream. There is no CPU fallback: importing the binding fails
loudly when the compiled library is missing.
"""
from __future__ import annotations

import ctypes as ct
import os
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
# LRDMC_LIBRARY selects another build of the library, such as the
# bounds-checked liblrdmc_bounds.so (build.build(bounds=True))
LIB_PATH = os.environ.get("LRDMC_LIBRARY") or os.path.join(_HERE, "liblrdmc.so")

MAX_NUC = 8
MAX_SHELL = 32
MAX_PRIM = 8
MAX_AO = 64
MAX_SPIN = 32
STATIC_EVAL_MAX = 262144

OK, ERR_ARG, ERR_CUDA, ERR_SINGULAR, ERR_NONFINITE, ERR_TIMEOUT, ERR_STATE, ERR_BOUNDS = range(8)
BUILD_BOUNDS = 1
SINGLE, THIS_WORK, PREVIOUS, EXPLICIT = 0, 1, 2, 3
PRECISION_FP64, PRECISION_DF64, PRECISION_FP32 = 0, 1, 2

EXPORTED = [
    "lrdmc_create_system", "lrdmc_spacing_params", "lrdmc_workspace_bytes", "lrdmc_init_walkers",
    "lrdmc_step", "lrdmc_sync", "lrdmc_get_energy_trace", "lrdmc_get_energy_trace_async", "lrdmc_get_residual_trace",
    "lrdmc_get_walkers",
    "lrdmc_moves", "lrdmc_evaluate",
    "lrdmc_evaluate_static", "lrdmc_evaluate_tc",
    "lrdmc_save", "lrdmc_load", "lrdmc_set_precision", "lrdmc_set_profiling", "lrdmc_kernel_times", "lrdmc_last_error",
    "lrdmc_destroy", "lrdmc_nj_n_params", "lrdmc_set_neural_jastrow", "lrdmc_base_terms", "lrdmc_nj_forward",
    "lrdmc_nj_backward", "lrdmc_set_interval_blocks", "lrdmc_interval_blocks", "lrdmc_set_tail_helpers",
    "lrdmc_batch_create",
    "lrdmc_batch_step", "lrdmc_batch_sync", "lrdmc_batch_stream", "lrdmc_batch_last_error", "lrdmc_batch_destroy",
    "lrdmc_batch_set_groups", "lrdmc_batch_set_carveout", "lrdmc_batch_set_pipelined", "lrdmc_build_flags",
]
NJ_MAX_CH, NJ_MAX_FEAT, NJ_HIDDEN, NJ_MAX_CELLS = 8, 12, 64, 8192


class LrdmcError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"lrdmc status {status}: {msg}")
        self.status = status


class _Shell(ct.Structure):
    _fields_ = [("center", ct.c_int), ("l", ct.c_int), ("kind", ct.c_int), ("n_prim", ct.c_int),
                ("n_eff", ct.c_double), ("zeta", ct.c_double),
                ("alpha", ct.c_double * MAX_PRIM), ("coef", ct.c_double * MAX_PRIM)]


class _Jastrow(ct.Structure):
    _fields_ = [("b_ee", ct.c_double), ("c_par", ct.c_double), ("c_anti", ct.c_double),
                ("en_b2", ct.c_double), ("en_b1", ct.c_double * MAX_NUC), ("ee_on", ct.c_int)]


class _Spacing(ct.Structure):
    _fields_ = [("kind", ct.c_int), ("beta", ct.c_double), ("kappa", ct.c_double),
                ("rc", ct.c_double), ("aprime_over_a", ct.c_double)]


class _NjSpec(ct.Structure):
    _fields_ = [("n_feat", ct.c_int), ("ell", ct.c_void_p), ("n_ch", ct.c_int), ("r_cut", ct.c_void_p),
                ("species", ct.c_void_p), ("hidden", ct.c_int), ("bf16", ct.c_int), ("n_cells", ct.c_int)]


def _nj_spec(spec, bf16):
    """ctypes image of a neural-term spec (any object with ell, r_cut,
    species, hidden, n_cells); the arrays are kept alive on the result."""
    ell = np.ascontiguousarray(spec.ell, dtype=np.float64)
    rcut = np.ascontiguousarray(spec.r_cut, dtype=np.float64)
    species = np.ascontiguousarray(spec.species, dtype=np.int32)
    c = _NjSpec(len(ell), _np_ptr(ell), len(rcut), _np_ptr(rcut), _np_ptr(species), int(spec.hidden), int(bool(bf16)),
                int(spec.n_cells))
    c._keep = (ell, rcut, species)
    return c


@dataclass(frozen=True)
class Spacing:
    """Lattice spacing function: SINGLE, THIS_WORK (Eq. 3, S-13, Eq. 6),
    PREVIOUS (Eq. 2, Eq. 4) or EXPLICIT (Gaussian p with given r_c, a'/a)."""
    kind: int = SINGLE
    beta: float = 0.75
    kappa: float = 2.5
    rc: float = 0.0
    aprime_over_a: float = 0.0

    def c(self):
        return _Spacing(self.kind, self.beta, self.kappa, self.rc, self.aprime_over_a)


_lib = None


def load_library():
    """Load liblrdmc.so (built by ``__graft_entry__.build()``); raises if absent."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"the CUDA library {LIB_PATH} is not built; run __graft_entry__.build()")
    L = ct.CDLL(LIB_PATH)
    i, d, vp, sz = ct.c_int, ct.c_double, ct.c_void_p, ct.c_size_t
    L.lrdmc_create_system.restype = i
    L.lrdmc_create_system.argtypes = [i, vp, vp, i, i, vp, i, vp, i, i, vp, ct.POINTER(vp)]
    L.lrdmc_spacing_params.restype = i
    L.lrdmc_spacing_params.argtypes = [vp, d, vp, ct.POINTER(d), ct.POINTER(d)]
    L.lrdmc_workspace_bytes.restype = i
    L.lrdmc_workspace_bytes.argtypes = [vp, i, i, ct.POINTER(sz)]
    L.lrdmc_init_walkers.restype = i
    L.lrdmc_init_walkers.argtypes = [vp, i, vp, ct.c_uint64, d, d, i, i, vp, sz, vp]
    L.lrdmc_step.restype = i
    L.lrdmc_step.argtypes = [vp, i, d, vp]
    L.lrdmc_sync.restype = i
    L.lrdmc_sync.argtypes = [vp]
    L.lrdmc_get_energy_trace.restype = i
    L.lrdmc_get_energy_trace.argtypes = [vp, vp, vp, vp, i, ct.POINTER(i)]
    L.lrdmc_get_energy_trace_async.restype = i
    L.lrdmc_get_energy_trace_async.argtypes = [vp, i, i, vp, vp, vp]
    L.lrdmc_get_residual_trace.restype = i
    L.lrdmc_get_residual_trace.argtypes = [vp, vp, i, ct.POINTER(i)]
    L.lrdmc_get_walkers.restype = i
    L.lrdmc_get_walkers.argtypes = [vp, vp, vp, vp, vp, vp, vp, vp]
    L.lrdmc_moves.restype = i
    L.lrdmc_moves.argtypes = [vp, ct.POINTER(ct.c_longlong)]
    L.lrdmc_evaluate.restype = i
    L.lrdmc_evaluate.argtypes = [vp, i, vp, vp, d, vp, vp, vp, vp, vp, vp]
    L.lrdmc_evaluate_static.restype = i
    L.lrdmc_evaluate_static.argtypes = [vp, i, vp, vp, d, vp, vp, vp, vp, vp, vp]
    L.lrdmc_evaluate_tc.restype = i
    L.lrdmc_evaluate_tc.argtypes = [vp, i, vp, vp, d, vp, vp, vp, vp, vp, vp]
    L.lrdmc_save.restype = i
    L.lrdmc_save.argtypes = [vp, ct.c_char_p]
    L.lrdmc_load.restype = i
    L.lrdmc_load.argtypes = [vp, ct.c_char_p]
    L.lrdmc_set_precision.restype = i
    L.lrdmc_set_precision.argtypes = [vp, i]
    L.lrdmc_set_profiling.restype = i
    L.lrdmc_set_profiling.argtypes = [vp, i]
    L.lrdmc_kernel_times.restype = i
    L.lrdmc_kernel_times.argtypes = [vp, ct.POINTER(d), ct.POINTER(d), ct.POINTER(ct.c_longlong),
                                     ct.POINTER(ct.c_longlong), i]
    L.lrdmc_last_error.restype = ct.c_char_p
    L.lrdmc_last_error.argtypes = [vp]
    L.lrdmc_build_flags.restype = i
    L.lrdmc_build_flags.argtypes = []
    L.lrdmc_destroy.restype = None
    L.lrdmc_destroy.argtypes = [vp]
    L.lrdmc_nj_n_params.restype = i
    L.lrdmc_nj_n_params.argtypes = [vp]
    L.lrdmc_set_neural_jastrow.restype = i
    L.lrdmc_set_neural_jastrow.argtypes = [vp, vp, vp]
    L.lrdmc_base_terms.restype = i
    L.lrdmc_base_terms.argtypes = [vp, i, vp, vp, vp, vp]
    L.lrdmc_nj_forward.restype = i
    L.lrdmc_nj_forward.argtypes = [vp, vp, vp, i, vp, vp, vp, vp, vp, vp, vp, vp]
    L.lrdmc_nj_backward.restype = i
    L.lrdmc_nj_backward.argtypes = [vp, vp, vp, i, vp, vp, vp, vp, vp, vp]
    L.lrdmc_set_interval_blocks.restype = i
    L.lrdmc_set_interval_blocks.argtypes = [vp, i]
    L.lrdmc_set_tail_helpers.restype = i
    L.lrdmc_set_tail_helpers.argtypes = [vp, i]
    L.lrdmc_interval_blocks.restype = i
    L.lrdmc_interval_blocks.argtypes = [vp, ct.POINTER(i), ct.POINTER(i)]
    L.lrdmc_batch_create.restype = i
    L.lrdmc_batch_create.argtypes = [vp, i, vp, vp, ct.POINTER(vp)]
    L.lrdmc_batch_step.restype = i
    L.lrdmc_batch_step.argtypes = [vp, i]
    L.lrdmc_batch_sync.restype = i
    L.lrdmc_batch_sync.argtypes = [vp]
    L.lrdmc_batch_set_carveout.restype = i
    L.lrdmc_batch_set_carveout.argtypes = [vp, i]
    L.lrdmc_batch_set_pipelined.restype = i
    L.lrdmc_batch_set_pipelined.argtypes = [vp, i]
    L.lrdmc_batch_set_groups.restype = i
    L.lrdmc_batch_set_groups.argtypes = [vp, vp]
    L.lrdmc_batch_stream.restype = i
    L.lrdmc_batch_stream.argtypes = [vp, ct.POINTER(vp)]
    L.lrdmc_batch_last_error.restype = ct.c_char_p
    L.lrdmc_batch_last_error.argtypes = [vp]
    L.lrdmc_batch_destroy.restype = None
    L.lrdmc_batch_destroy.argtypes = [vp]
    _lib = L
    return L


def build_flags() -> int:
    """lrdmc_build_flags of the loaded library (BUILD_BOUNDS for the
    bounds-checked build)."""
    return load_library().lrdmc_build_flags()


def _np_ptr(a):
    return a.ctypes.data_as(ct.c_void_p) if a is not None else None


def _t_ptr(t):
    return ct.c_void_p(t.data_ptr()) if t is not None else None


class LrdmcSystem:
    """A trial function and, after ``init_walkers``, a walker population."""

    def __init__(self, system):
        L = load_library()
        self.sys = system
        n_shell = len(system.shells)
        shells = (_Shell * n_shell)()
        for q, s in enumerate(system.shells):
            sh = shells[q]
            sh.center, sh.l, sh.kind, sh.n_prim = s.center, s.l, s.kind, len(s.alpha)
            sh.n_eff, sh.zeta = s.n_eff, s.zeta
            for p, (a, c) in enumerate(zip(s.alpha, s.coef)):
                sh.alpha[p], sh.coef[p] = a, c
        jas = _Jastrow()
        jas.b_ee, jas.c_par, jas.c_anti, jas.en_b2 = system.b_ee, system.c_par, system.c_anti, system.en_b2
        en_b1 = system.en_b1 if system.en_b1 is not None else np.zeros(system.n_nuc)
        for I in range(system.n_nuc):
            jas.en_b1[I] = float(en_b1[I])
        jas.ee_on = int(system.ee_on)
        xyz = np.ascontiguousarray(system.nuc_xyz, dtype=np.float64)
        Z = np.ascontiguousarray(system.Z, dtype=np.float64)
        C = np.ascontiguousarray(system.C, dtype=np.float64)
        h = ct.c_void_p()
        st = L.lrdmc_create_system(system.n_nuc, _np_ptr(xyz), _np_ptr(Z), system.n_up, system.n_dn,
                                   ct.cast(shells, ct.c_void_p), n_shell, _np_ptr(C), C.shape[0],
                                   C.shape[1], ct.byref(jas), ct.byref(h))
        if st != OK:
            raise LrdmcError(st, L.lrdmc_last_error(None).decode())
        self.h = h
        self.N = system.N
        self._ws = None
        self.W = 0
        self.stream = None
        self.lattice_G = None

    def __del__(self):
        if getattr(self, "h", None):
            load_library().lrdmc_destroy(self.h)
            self.h = None

    def _check(self, st):
        if st != OK:
            raise LrdmcError(st, load_library().lrdmc_last_error(self.h).decode())

    # ---------------------------------------------------------------- host
    def spacing_params(self, a, spacing: Spacing):
        r, rc = ct.c_double(), ct.c_double()
        sp = spacing.c()
        self._check(load_library().lrdmc_spacing_params(self.h, a, ct.byref(sp), ct.byref(r), ct.byref(rc)))
        return r.value, rc.value

    def workspace_bytes(self, n_walkers, trace_capacity):
        b = ct.c_size_t()
        self._check(load_library().lrdmc_workspace_bytes(self.h, n_walkers, trace_capacity, ct.byref(b)))
        return b.value

    # ---------------------------------------------------------------- population
    def init_walkers(self, x0, seed, tau, e_trial=0.0, recompute_every=10, trace_capacity=4096,
                     stream=None, device="cuda"):
        """x0: [W][N][3] float64, a CUDA tensor on the workspace's device or a
        host array (copied). Raises ValueError, before any device work, for
        another shape or dtype, non-finite positions or a tensor on another
        device."""
        import torch

        shape = tuple(x0.shape)
        if len(shape) != 3 or shape[1:] != (self.N, 3) or shape[0] < 1:
            raise ValueError(f"init_walkers: x0 must be [W][{self.N}][3] with W >= 1, got {shape}")
        if isinstance(x0, np.ndarray):
            if not np.issubdtype(x0.dtype, np.floating):
                raise ValueError(f"init_walkers: x0 must be floating point, got {x0.dtype}")
            finite = bool(np.isfinite(x0).all())
        else:
            if x0.dtype != torch.float64:
                raise ValueError(f"init_walkers: x0 must be float64, got {x0.dtype}")
            finite = bool(torch.isfinite(x0).all())
        if not finite:
            raise ValueError("init_walkers: start positions must be finite")
        W = shape[0]
        nbytes = self.workspace_bytes(W, trace_capacity)
        self._ws = torch.empty(nbytes + 256, dtype=torch.uint8, device=device)
        if not isinstance(x0, np.ndarray) and x0.is_cuda and x0.device != self._ws.device:
            raise ValueError(f"init_walkers: x0 is on {x0.device}, the workspace on {self._ws.device}")
        base = self._ws.data_ptr()
        ptr = (base + 255) & ~255
        if stream is None:
            stream = torch.cuda.current_stream(self._ws.device)
        self.stream = stream
        if isinstance(x0, np.ndarray):
            x0 = np.ascontiguousarray(x0, dtype=np.float64)
            xp = _np_ptr(x0)
        else:
            x0 = x0.contiguous()
            xp = _t_ptr(x0)
        self._x0_keep = x0
        st = load_library().lrdmc_init_walkers(self.h, W, xp, int(seed), float(tau), float(e_trial),
                                               int(recompute_every), int(trace_capacity),
                                               ct.c_void_p(ptr), nbytes, ct.c_void_p(stream.cuda_stream))
        self._check(st)
        self.W = W
        return self

    def step(self, n_steps, a, spacing: Spacing = Spacing()):
        sp = spacing.c()
        self._check(load_library().lrdmc_step(self.h, int(n_steps), float(a), ct.byref(sp)))
        self.lattice_G = 1 if spacing.kind == SINGLE else 2

    def sync(self):
        """Wait for the enqueued steps and raise any error they reported."""
        self._check(load_library().lrdmc_sync(self.h))

    def energy_trace(self, max_n=1 << 20):
        n = ct.c_int()
        cap = max_n
        e, w, j = np.zeros(cap), np.zeros(cap), np.zeros(cap)
        self._check(load_library().lrdmc_get_energy_trace(self.h, _np_ptr(e), _np_ptr(w), _np_ptr(j), cap,
                                                          ct.byref(n)))
        k = n.value
        return e[:k].copy(), w[:k].copy(), j[:k].copy()

    def energy_trace_async(self, first, n, out):
        """Enqueues the copy of trace entries [first, first + n) into
        out[0..2, first:first + n] (energy, mean weight, mean jumps) without
        waiting; ``out`` is a contiguous (3, m) float64 CPU tensor or array,
        pinned for the copies to be asynchronous, valid until ``sync()``."""
        import torch

        if isinstance(out, torch.Tensor):
            if out.device.type != "cpu" or out.dtype != torch.float64 or not out.is_contiguous():
                raise ValueError("energy_trace_async: out must be a contiguous float64 CPU tensor")
            base = out.data_ptr()
        else:
            if not (isinstance(out, np.ndarray) and out.dtype == np.float64 and out.flags.c_contiguous):
                raise ValueError("energy_trace_async: out must be a contiguous float64 array")
            base = out.ctypes.data
        if out.ndim != 2 or out.shape[0] != 3 or first < 0 or n < 0 or first + n > out.shape[1]:
            raise ValueError("energy_trace_async: out must have shape (3, m) with first + n <= m")
        m = int(out.shape[1])
        ptrs = [ct.c_void_p(base + 8 * (r * m + first)) for r in range(3)]
        self._check(load_library().lrdmc_get_energy_trace_async(self.h, int(first), int(n), *ptrs))

    def residual_trace(self, max_n=1 << 20):
        """Largest Sherman-Morrison residual max|A Ainv - I| per interval,
        measured at each rebuild of the inverses (-1 where none)."""
        n = ct.c_int()
        r = np.zeros(max_n)
        self._check(load_library().lrdmc_get_residual_trace(self.h, _np_ptr(r), max_n, ct.byref(n)))
        return r[:n.value].copy()

    def walkers(self):
        W, N = self.W, self.N
        P = 6 * N * (self.lattice_G or 1)
        x = np.zeros((W, N, 3))
        el, b = np.zeros(W), np.zeros(W)
        T = np.zeros((W, P))
        logw, jumps, parent = np.zeros(W), np.zeros(W, np.int32), np.zeros(W, np.int32)
        self._check(load_library().lrdmc_get_walkers(self.h, _np_ptr(x), _np_ptr(el), _np_ptr(b),
                                                     _np_ptr(T) if self.lattice_G else None,
                                                     _np_ptr(logw), _np_ptr(jumps), _np_ptr(parent)))
        return dict(x=x, EL=el, b=b, T=T, logw_pre=logw, jumps_pre=jumps, parent=parent)

    def moves(self):
        m = ct.c_longlong()
        self._check(load_library().lrdmc_moves(self.h, ct.byref(m)))
        return m.value

    def set_precision(self, precision):
        """PRECISION_FP64 (IEEE double everywhere), PRECISION_DF64 (default:
        double-float evaluation on the FP32 pipe, FP64 state and updates) or
        PRECISION_FP32 (mixed: single-precision evaluation, FP64 state)."""
        self._check(load_library().lrdmc_set_precision(self.h, int(precision)))
        return self

    def set_profiling(self, on=True):
        self._check(load_library().lrdmc_set_profiling(self.h, int(on)))

    def kernel_times(self, reset=False):
        """Accumulated (interval_ms, reconfig_ms, interval_launches, reconfig_launches)."""
        a, b = ct.c_double(), ct.c_double()
        na, nb = ct.c_longlong(), ct.c_longlong()
        self._check(load_library().lrdmc_kernel_times(self.h, ct.byref(a), ct.byref(b), ct.byref(na),
                                                      ct.byref(nb), int(reset)))
        return a.value, b.value, na.value, nb.value

    def save(self, path):
        self._check(load_library().lrdmc_save(self.h, path.encode()))

    def load(self, path):
        self._check(load_library().lrdmc_load(self.h, path.encode()))

    # ---------------------------------------------------------------- stateless
    def _eval_args(self, x, rot, P, out=None):
        """Checks of the arguments of evaluate / evaluate_static before any
        pointer reaches the library: x [n][N][3] and rot [n][9] float64 on
        one CUDA device; out = (ratio [n][P], T [n][P], b [n], el [n]),
        float64, contiguous, on the same device (the kernels write exactly
        these extents, so a smaller or differently typed buffer is refused
        here rather than overrun on the device)."""
        import torch

        if not (isinstance(x, torch.Tensor) and isinstance(rot, torch.Tensor)):
            raise ValueError("x and rot must be torch tensors")
        if x.dim() != 3 or tuple(x.shape[1:]) != (self.N, 3):
            raise ValueError(f"x must be [n][{self.N}][3], got {tuple(x.shape)}")
        n = int(x.shape[0])
        if tuple(rot.shape) != (n, 9):
            raise ValueError(f"rot must be [{n}][9], got {tuple(rot.shape)}")
        for name, t in (("x", x), ("rot", rot)):
            if t.dtype != torch.float64 or not t.is_cuda:
                raise ValueError(f"{name} must be a float64 CUDA tensor")
        if rot.device != x.device:
            raise ValueError("x and rot must be on the same device")
        if out is not None:
            if len(out) != 4:
                raise ValueError("out must be (ratio, T, b, el)")
            for name, t, shape in zip(("ratio", "T", "b", "el"), out, ((n, P), (n, P), (n,), (n,))):
                if not isinstance(t, torch.Tensor) or tuple(t.shape) != shape:
                    raise ValueError(f"out {name} must have shape {shape}")
                if t.dtype != torch.float64 or t.device != x.device or not t.is_contiguous():
                    raise ValueError(f"out {name} must be a contiguous float64 tensor on {x.device}")
        return n

    def evaluate_static(self, x, rot, a, spacing: Spacing = Spacing(), stream=None, out=None):
        """Like evaluate, through lrdmc_evaluate_static: the library allocates
        no device memory (its scratch is a static device array shared by all
        calls; at most STATIC_EVAL_MAX configurations). ``out`` may pass
        preallocated (ratio, T, b, el) CUDA tensors."""
        import torch

        G = 1 if spacing.kind == SINGLE else 2
        P = 6 * self.N * G
        n = self._eval_args(x, rot, P, out)
        x = x.contiguous()
        rot = rot.contiguous()
        if out is None:
            out = (torch.empty((n, P), dtype=torch.float64, device=x.device),
                   torch.empty((n, P), dtype=torch.float64, device=x.device),
                   torch.empty(n, dtype=torch.float64, device=x.device),
                   torch.empty(n, dtype=torch.float64, device=x.device))
        ratio, T, b, el = out
        if stream is None:
            stream = torch.cuda.current_stream(x.device)
        sp = spacing.c()
        self._check(load_library().lrdmc_evaluate_static(self.h, n, _t_ptr(x), _t_ptr(rot), float(a),
                                                         ct.byref(sp), _t_ptr(ratio), _t_ptr(T), _t_ptr(b),
                                                         _t_ptr(el), ct.c_void_p(stream.cuda_stream)))
        return ratio, T, b, el

    def evaluate(self, x, rot, a, spacing: Spacing = Spacing(), stream=None):
        """One evaluation of every lattice move of n configurations.
        x: [n][N][3] and rot: [n][9] float64 CUDA tensors. Returns CUDA tensors
        ratio [n][P], T [n][P], b [n], el [n]."""
        return self._evaluate_with("lrdmc_evaluate", x, rot, a, spacing, stream)

    def evaluate_tc(self, x, rot, a, spacing: Spacing = Spacing(), stream=None):
        """Like evaluate, through lrdmc_evaluate_tc: the FP32 mode's
        evaluation with the basis x MO contraction on the tensor cores
        (bf16x3 operands, FP32 accumulation)."""
        return self._evaluate_with("lrdmc_evaluate_tc", x, rot, a, spacing, stream)

    def _evaluate_with(self, entry, x, rot, a, spacing, stream):
        import torch

        G = 1 if spacing.kind == SINGLE else 2
        P = 6 * self.N * G
        n = self._eval_args(x, rot, P)
        x = x.contiguous()
        rot = rot.contiguous()
        ratio = torch.empty((n, P), dtype=torch.float64, device=x.device)
        T = torch.empty((n, P), dtype=torch.float64, device=x.device)
        b = torch.empty(n, dtype=torch.float64, device=x.device)
        el = torch.empty(n, dtype=torch.float64, device=x.device)
        if stream is None:
            stream = torch.cuda.current_stream(x.device)
        sp = spacing.c()
        fn = getattr(load_library(), entry)
        self._check(fn(self.h, n, _t_ptr(x), _t_ptr(rot), float(a), ct.byref(sp), _t_ptr(ratio), _t_ptr(T),
                       _t_ptr(b), _t_ptr(el), ct.c_void_p(stream.cuda_stream)))
        return ratio, T, b, el

    def set_tail_helpers(self, on=True):
        """Warps out of walkers help the warps of their block that still run
        one (default on; results are bit for bit the same either way)."""
        self._check(load_library().lrdmc_set_tail_helpers(self.h, int(bool(on))))
        return self

    def set_interval_blocks(self, blocks):
        """Persistent grid size of the interval kernel (0 = occupancy default)."""
        self._check(load_library().lrdmc_set_interval_blocks(self.h, int(blocks)))
        return self

    def interval_blocks(self):
        """(current setting, occupancy default) of the interval grid."""
        c, d = ct.c_int(), ct.c_int()
        self._check(load_library().lrdmc_interval_blocks(self.h, ct.byref(c), ct.byref(d)))
        return c.value, d.value

    # ---------------------------------------------------------------- neural pair term
    def set_neural_jastrow(self, spec, params, bf16=True):
        """Install the neural pair term (params: float32 array or tensor of
        lrdmc_nj_n_params entries) in the projection and every evaluation;
        ``spec=None`` removes it."""
        if spec is None:
            self._check(load_library().lrdmc_set_neural_jastrow(self.h, None, None))
            return self
        p = np.ascontiguousarray(params.detach().cpu().numpy() if hasattr(params, "detach") else params,
                                 dtype=np.float32)
        c = _nj_spec(spec, bf16)
        self._check(load_library().lrdmc_set_neural_jastrow(self.h, ct.byref(c), _np_ptr(p)))
        return self

    def nj_n_params(self, spec):
        return load_library().lrdmc_nj_n_params(ct.byref(_nj_spec(spec, True)))

    def base_terms(self, x, stream=None):
        """grad_i log|psi_G| [n][N][3] and E_L [n] without the neural term, in
        FP64, for configurations x [n][N][3] (float64 CUDA tensor)."""
        import torch

        x = x.contiguous()
        n = int(x.shape[0])
        grad = torch.empty((n, self.N, 3), dtype=torch.float64, device=x.device)
        e = torch.empty(n, dtype=torch.float64, device=x.device)
        if stream is None:
            stream = torch.cuda.current_stream(x.device)
        self._check(load_library().lrdmc_base_terms(self.h, n, _t_ptr(x), _t_ptr(grad), _t_ptr(e),
                                                    ct.c_void_p(stream.cuda_stream)))
        return grad, e

    def nj_forward(self, spec, params, x, grad_base, e_base, bf16=True, stream=None):
        """Training forward pass (FP32): E_L [n], J_NN [n], q = a + G [n][N][3]
        and the pair values [n][n_pairs][3]."""
        import torch

        n = int(x.shape[0])
        n_pairs = self.N * (self.N - 1) // 2 + self.N * self.sys.n_nuc
        dev = x.device
        el = torch.empty(n, dtype=torch.float32, device=dev)
        j = torch.empty(n, dtype=torch.float32, device=dev)
        q = torch.empty((n, self.N, 3), dtype=torch.float32, device=dev)
        pairs = torch.empty((n, n_pairs, 3), dtype=torch.float32, device=dev)
        if stream is None:
            stream = torch.cuda.current_stream(dev)
        c = _nj_spec(spec, bf16)
        p = params.detach().contiguous()
        assert p.dtype == torch.float32 and p.is_cuda
        self._check(load_library().lrdmc_nj_forward(
            self.h, ct.byref(c), _t_ptr(p), n, _t_ptr(x.contiguous()), _t_ptr(grad_base.contiguous()),
            _t_ptr(e_base.contiguous()), _t_ptr(el), _t_ptr(j), _t_ptr(q), _t_ptr(pairs),
            ct.c_void_p(stream.cuda_stream)))
        return el, j, q, pairs

    def nj_backward(self, spec, params, x, q, d_el, d_j, bf16=True, stream=None):
        """Gradient of sum(d_el E_L + d_j J_NN) with respect to the parameters
        (float32 CUDA tensor)."""
        import torch

        n = int(x.shape[0])
        p = params.detach().contiguous()
        grad = torch.empty_like(p)
        if stream is None:
            stream = torch.cuda.current_stream(x.device)
        c = _nj_spec(spec, bf16)
        self._check(load_library().lrdmc_nj_backward(
            self.h, ct.byref(c), _t_ptr(p), n, _t_ptr(x.contiguous()), _t_ptr(q.contiguous()),
            _t_ptr(d_el.contiguous()), _t_ptr(d_j.contiguous()), _t_ptr(grad), ct.c_void_p(stream.cuda_stream)))
        return grad


class LrdmcBatch:
    """Several systems projected together, one CUDA graph per step (see
    lrdmc_batch_create). ``systems`` are LrdmcSystem objects with
    populations; ``a`` and ``spacing`` give each system's lattice."""

    def __init__(self, systems, a, spacing):
        L = load_library()
        n = len(systems)
        self.systems = list(systems)
        hs = (ct.c_void_p * n)(*[s.h for s in systems])
        av = np.ascontiguousarray(a, dtype=np.float64)
        sp = (_Spacing * n)(*[x.c() for x in spacing])
        h = ct.c_void_p()
        st = L.lrdmc_batch_create(ct.cast(hs, ct.c_void_p), n, _np_ptr(av), ct.cast(sp, ct.c_void_p), ct.byref(h))
        if st != OK:
            raise LrdmcError(st, "batch_create failed (systems need populations; no duplicates; valid lattices)")
        self.h = h
        self._G = [1 if x.kind == SINGLE else 2 for x in spacing]
        for s, G in zip(self.systems, self._G):
            s.lattice_G = G

    def __del__(self):
        if getattr(self, "h", None):
            load_library().lrdmc_batch_destroy(self.h)
            self.h = None

    def _check(self, st):
        if st != OK:
            raise LrdmcError(st, load_library().lrdmc_batch_last_error(self.h).decode())

    def step(self, n_steps):
        self._check(load_library().lrdmc_batch_step(self.h, int(n_steps)))

    def sync(self):
        self._check(load_library().lrdmc_batch_sync(self.h))

    def set_groups(self, groups):
        """Execution groups: systems of one group run concurrently, groups
        one after another (in increasing number)."""
        gv = np.ascontiguousarray(groups, dtype=np.int32)
        self._check(load_library().lrdmc_batch_set_groups(self.h, _np_ptr(gv)))

    def set_carveout(self, carveout):
        """Preferred shared-memory carveout (percent) of the batched interval
        launches, or -1 for the default."""
        self._check(load_library().lrdmc_batch_set_carveout(self.h, int(carveout)))

    def set_pipelined(self, on=True):
        """Chain the systems' interval kernels on one stream with
        programmatic stream serialization (each starts while the previous
        one drains its walkers); off: the fork/join groups."""
        self._check(load_library().lrdmc_batch_set_pipelined(self.h, int(bool(on))))

    @property
    def stream_ptr(self):
        p = ct.c_void_p()
        self._check(load_library().lrdmc_batch_stream(self.h, ct.byref(p)))
        return p.value


def create_system(system) -> LrdmcSystem:
    return LrdmcSystem(system)
