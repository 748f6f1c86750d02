"""Thin ctypes binding of libfks.so (include/fks.h).

Argument marshalling only: tensors are passed as device pointers with the
caller's current CUDA stream; every step of the computation runs in the
library's kernels.  There is no fallback: if the library or a GPU is
missing, the calls raise.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

from . import build as _build

FKS_FP64 = 0
FKS_FP32 = 1
FKS_BF16X3 = 2   # split-BF16 tensor-core transforms, FP32 storage
FKS_FP32X2 = 3   # double-float arithmetic (the last escalation tier)
HARD_SPHERE = 0
MAXWELL = 1
BGK = 2
VHS = 3          # variable hard spheres B = C|g|^alpha (Config.alpha, Config.terms)
PERIODIC = 0
SPECULAR = 1

_STATUS = {0: "ok", 1: "invalid argument", 2: "unsupported configuration", 3: "out of device memory",
           4: "CUDA error", 5: "numerical health check failed", 6: "timeout"}


class FKSError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"fks status {status} ({_STATUS.get(status, '?')}): {msg}")
        self.status = status


class _Grid(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
                ("x0", ctypes.c_double * 3), ("x1", ctypes.c_double * 3), ("bc", ctypes.c_int * 3)]


class _VBox(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int), ("L", ctypes.c_double)]


class _Kernel(ctypes.Structure):
    _fields_ = [("type", ctypes.c_int), ("C", ctypes.c_double), ("knudsen", ctypes.c_double),
                ("alpha", ctypes.c_double), ("terms", ctypes.c_int)]


class _Dirs(ctypes.Structure):
    _fields_ = [("A1", ctypes.c_int), ("A2", ctypes.c_int), ("rule", ctypes.c_int)]


_lib = None

# every symbol include/fks.h declares
EXPORTS = ["fks_init", "fks_collide", "fks_transport", "fks_step", "fks_moments", "fks_check",
           "fks_get_offsets", "fks_set_offsets", "fks_ncells", "fks_nv", "fks_cluster_size",
           "fks_set_cluster_size", "fks_launch_count", "fks_kernel_transform", "fks_destroy",
           "fks_last_error", "fks_status_string", "fks_transport_noalloc",
           "fks_batch_init", "fks_batch_collide", "fks_batch_step", "fks_batch_run", "fks_batch_check",
           "fks_batch_cluster_size", "fks_batch_set_cluster_size", "fks_batch_launch_count",
           "fks_batch_destroy", "fks_batch_last_error",
           "fks_net_init", "fks_net_num_params", "fks_net_set_params", "fks_net_get_params", "fks_net_forward",
           "fks_net_gradient", "fks_net_train_step", "fks_net_launch_count", "fks_net_last_error",
           "fks_net_destroy", "fks_surrogate_inputs", "fks_surrogate_collide", "fks_surrogate_indicator",
           "fks_net_infer", "fks_net_check", "fks_selftest_wait", "fks_set_dealias", "fks_step_host", "fks_vhs_factor",
           "fks_step_strang", "fks_alu_peak", "fks_step_exp", "fks_relax", "fks_surrogate_step", "fks_set_profiling", "fks_get_profile", "fks_set_schedule", "fks_radix",
           "fks_batch_set_schedule", "fks_batch_radix", "fks_set_escalation", "fks_get_escalation", "fks_set_escalation_arith",
           "fks_batch_set_escalation", "fks_batch_get_escalation", "fks_set_escalation_direct"]


def lib(build: bool = True):
    """Load libfks.so (building it first if it is missing or stale)."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.build() if build else _build.LIB
    if not os.path.exists(path):
        raise FileNotFoundError(f"{path} is missing: run paper_1701_01608_gb300.build.build()")
    L = ctypes.CDLL(path)
    P = ctypes.c_void_p
    D = ctypes.c_double
    I = ctypes.c_int
    L.fks_init.argtypes = [ctypes.POINTER(_Grid), ctypes.POINTER(_VBox), ctypes.POINTER(_Kernel),
                           ctypes.POINTER(_Dirs), I, ctypes.POINTER(P)]
    for name in ("fks_collide",):
        getattr(L, name).argtypes = [P, P, P, P]
    L.fks_transport.argtypes = [P, P, P, D, P]
    L.fks_step.argtypes = [P, P, P, D, P]
    L.fks_relax.argtypes = [P, P, P, D, P]
    L.fks_step_strang.argtypes = [P, P, P, P, D, P]
    L.fks_step_exp.argtypes = [P, P, P, D, P]
    L.fks_moments.argtypes = [P, P, P, P]
    L.fks_check.argtypes = [P, P, ctypes.POINTER(I)]
    L.fks_get_offsets.argtypes = [P, P]
    L.fks_set_offsets.argtypes = [P, P]
    L.fks_ncells.argtypes = [P]
    L.fks_ncells.restype = ctypes.c_long
    L.fks_nv.argtypes = [P]
    L.fks_cluster_size.argtypes = [P]
    L.fks_set_cluster_size.argtypes = [P, I]
    L.fks_set_schedule.argtypes = [P, I, I]
    L.fks_radix.argtypes = [P]
    L.fks_launch_count.argtypes = [P]
    L.fks_launch_count.restype = ctypes.c_long
    L.fks_kernel_transform.argtypes = [I, D, D, D, ctypes.POINTER(D), ctypes.POINTER(D)]
    L.fks_vhs_factor.argtypes = [D, D, D, I, I, I, D, D, ctypes.POINTER(D), ctypes.POINTER(I), ctypes.POINTER(D)]
    L.fks_transport_noalloc.argtypes = [ctypes.POINTER(_Grid), ctypes.POINTER(_VBox), I, P, D, P, P, P]
    PP = ctypes.POINTER(ctypes.c_void_p)
    PD = ctypes.POINTER(ctypes.c_double)
    PI = ctypes.POINTER(ctypes.c_int)
    L.fks_batch_init.argtypes = [I, PI, PD, PI, PD, PD, ctypes.POINTER(_Dirs), I, PP]
    L.fks_batch_collide.argtypes = [P, PP, PP, P]
    L.fks_batch_step.argtypes = [P, PP, PP, PD, P]
    L.fks_batch_run.argtypes = [P, PP, PP, PD, I, P]
    L.fks_batch_check.argtypes = [P, P, PI]
    L.fks_batch_set_escalation.argtypes = [P, D]
    L.fks_batch_get_escalation.argtypes = [P, ctypes.POINTER(D), ctypes.POINTER(ctypes.c_long)]
    L.fks_batch_cluster_size.argtypes = [P, I]
    L.fks_batch_set_cluster_size.argtypes = [P, I, I]
    L.fks_batch_set_schedule.argtypes = [P, I, I, I]
    L.fks_batch_radix.argtypes = [P, I]
    L.fks_batch_launch_count.argtypes = [P]
    L.fks_batch_launch_count.restype = ctypes.c_long
    L.fks_batch_destroy.argtypes = [P]
    L.fks_batch_destroy.restype = None
    L.fks_batch_last_error.argtypes = [P]
    L.fks_batch_last_error.restype = ctypes.c_char_p
    L.fks_net_init.argtypes = [I, I, ctypes.c_ulonglong, PP]
    L.fks_net_num_params.argtypes = [P]
    L.fks_net_num_params.restype = ctypes.c_long
    L.fks_net_set_params.argtypes = [P, P, ctypes.c_long]
    L.fks_net_get_params.argtypes = [P, P, ctypes.c_long]
    L.fks_net_forward.argtypes = [P, I, P, P, P]
    L.fks_net_gradient.argtypes = [P, I, P, P, P, P]
    L.fks_net_infer.argtypes = [P, I, P, P, P]
    L.fks_net_check.argtypes = [P, P]
    L.fks_net_train_step.argtypes = [P, I, P, P, ctypes.c_float, P, P]
    L.fks_net_launch_count.argtypes = [P]
    L.fks_net_launch_count.restype = ctypes.c_long
    L.fks_net_last_error.argtypes = [P]
    L.fks_net_last_error.restype = ctypes.c_char_p
    L.fks_net_destroy.argtypes = [P]
    L.fks_net_destroy.restype = None
    L.fks_surrogate_inputs.argtypes = [I, D, ctypes.c_long, P, P, P, P, P]
    L.fks_surrogate_collide.argtypes = [P, P, P, P, D, D, D, ctypes.POINTER(ctypes.c_long), P]
    L.fks_surrogate_indicator.argtypes = [P, P, ctypes.c_long]
    L.fks_surrogate_step.argtypes = [P, P, P, P, P, D, D, D, D, ctypes.POINTER(ctypes.c_long), P]
    L.fks_selftest_wait.argtypes = [ctypes.c_long, P]
    L.fks_alu_peak.argtypes = [I, ctypes.POINTER(D), P]
    L.fks_set_dealias.argtypes = [P, I]
    L.fks_set_escalation.argtypes = [P, D]
    L.fks_set_profiling.argtypes = [P, I]
    L.fks_get_profile.argtypes = [P, P, P]
    L.fks_set_escalation_arith.argtypes = [P, I]
    L.fks_set_escalation_direct.argtypes = [P, I]
    L.fks_get_escalation.argtypes = [P, ctypes.POINTER(D), ctypes.POINTER(ctypes.c_long)]
    L.fks_step_host.argtypes = [P, P, P, D, P]
    L.fks_destroy.argtypes = [P]
    L.fks_destroy.restype = None
    L.fks_last_error.argtypes = [P]
    L.fks_last_error.restype = ctypes.c_char_p
    L.fks_status_string.argtypes = [I]
    L.fks_status_string.restype = ctypes.c_char_p
    _lib = L
    return L


def kernel_transform(ktype: int, C: float, L: float, s: float) -> tuple[float, float]:
    """phi_R(s), psi_R(s) as the library's table kernel evaluates them (host)."""
    phi = ctypes.c_double()
    psi = ctypes.c_double()
    st = lib().fks_kernel_transform(ktype, C, L, s, ctypes.byref(phi), ctypes.byref(psi))
    if st != 0:
        raise FKSError(st, "fks_kernel_transform")
    return phi.value, psi.value


def vhs_factor(alpha: float, C: float, L: float, n: int, precision: int, terms: int, t: float,
               u: float) -> tuple[float, int, float]:
    """(H(t, u), term count, truncation estimate) of the library's VHS expansion (host)."""
    H = ctypes.c_double()
    S = ctypes.c_int()
    e = ctypes.c_double()
    st = lib().fks_vhs_factor(alpha, C, L, n, precision, terms, t, u, ctypes.byref(H), ctypes.byref(S),
                              ctypes.byref(e))
    if st != 0:
        raise FKSError(st, "fks_vhs_factor")
    return H.value, S.value, e.value


def _stream_ptr(stream) -> int:
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return int(s.cuda_stream)


def _dptr(t, dtype) -> int:
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError("expected a CUDA tensor")
    if t.dtype != dtype or not t.is_contiguous():
        raise TypeError(f"expected a contiguous {dtype} tensor, got {t.dtype}")
    return int(t.data_ptr())


@dataclass
class Config:
    ncell: tuple = (1, 1, 1)
    x0: tuple = (0.0, 0.0, 0.0)
    x1: tuple = (1.0, 1.0, 1.0)
    bc: tuple = (0, 0, 0)
    n: int = 16
    L: float = 8.0
    kernel: int = HARD_SPHERE
    C: float = 0.25
    kn: float = 1.0
    A1: int = 4
    A2: int = 4
    rule: int = 0
    precision: int = FKS_FP32
    dealias: bool = False   # variant B: 2n-padded (de-aliased) operator, n = 8 or 16
    alpha: float = 1.0      # VHS exponent (kernel=VHS only)
    terms: int = 0          # VHS separable terms, 0 = automatic


class Context:
    """One fks_ctx: spectral tables, offsets and flags on the current device."""

    def __init__(self, cfg: Config):
        import torch
        self.cfg = cfg
        self._L = lib()
        g = _Grid(cfg.ncell[0], cfg.ncell[1], cfg.ncell[2], (ctypes.c_double * 3)(*cfg.x0),
                  (ctypes.c_double * 3)(*cfg.x1), (ctypes.c_int * 3)(*cfg.bc))
        vb = _VBox(cfg.n, cfg.L)
        k = _Kernel(cfg.kernel, cfg.C, cfg.kn, cfg.alpha, cfg.terms)
        d = _Dirs(cfg.A1, cfg.A2, cfg.rule)
        h = ctypes.c_void_p()
        st = self._L.fks_init(ctypes.byref(g), ctypes.byref(vb), ctypes.byref(k), ctypes.byref(d),
                              cfg.precision, ctypes.byref(h))
        if st != 0:
            raise FKSError(st, "fks_init")
        self._h = h
        self.dtype = torch.float64 if cfg.precision == FKS_FP64 else torch.float32
        if cfg.dealias:
            self.set_dealias(True)

    def step_host(self, f, f_out, dt: float, stream=None):
        """fks_step with host (CPU, preferably pinned) tensors, copies pipelined with the step."""
        for t in (f, f_out):
            if t.device.type != "cpu" or t.dtype != self.dtype or not t.is_contiguous():
                raise TypeError(f"expected a contiguous CPU tensor of {self.dtype}")
        self._check(self._L.fks_step_host(self._h, ctypes.c_void_p(f.data_ptr()), ctypes.c_void_p(f_out.data_ptr()),
                                          float(dt), _stream_ptr(stream)), "fks_step_host")

    def set_escalation(self, tol: float):
        """Precision escalation: cells whose error bound exceeds tol * ||Q|| are recomputed at
        higher precision (0: off)."""
        self._check(self._L.fks_set_escalation(self._h, float(tol)), "fks_set_escalation")

    def set_escalation_arith(self, arith: int):
        """Arithmetic of the last escalation tier: FKS_FP32X2 (double-float, default) or FKS_FP64."""
        self._check(self._L.fks_set_escalation_arith(self._h, int(arith)), "fks_set_escalation_arith")

    def set_escalation_direct(self, on: bool):
        """Direct routes to the last escalation tier (default on): split-BF16 cells beyond the FP32
        tier's reach, and in the surrogate step cells this close to equilibrium that every earlier
        tier must fail them (identical results, less work)."""
        self._check(self._L.fks_set_escalation_direct(self._h, int(bool(on))), "fks_set_escalation_direct")

    def escalation(self) -> tuple[float, tuple[int, int]]:
        """(tolerance, cells sent to the first and second tier by the last collision or step)."""
        tol = ctypes.c_double()
        counts = (ctypes.c_long * 2)()
        self._check(self._L.fks_get_escalation(self._h, ctypes.byref(tol), counts), "fks_get_escalation")
        return tol.value, (counts[0], counts[1])

    def set_profiling(self, on: bool = True):
        """Record CUDA events around each collision launch (stage 0 own kernel, 1 and 2 escalation tiers)."""
        self._check(self._L.fks_set_profiling(self._h, 1 if on else 0), "fks_set_profiling")

    def profile(self) -> tuple[list, list]:
        """(ms per stage, launches per stage) since the last call; synchronises the device."""
        ms = (ctypes.c_double * 3)()
        n = (ctypes.c_long * 3)()
        self._check(self._L.fks_get_profile(self._h, ms, n), "fks_get_profile")
        return list(ms), list(n)

    def set_dealias(self, on: bool = True):
        """Variant B: the 2n-padded (de-aliased) operator for this context's collisions."""
        self._check(self._L.fks_set_dealias(self._h, 1 if on else 0), "fks_set_dealias")

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            self._L.fks_destroy(h)
            self._h = None

    def _check(self, st: int, what: str):
        if st != 0:
            raise FKSError(st, f"{what}: {self._L.fks_last_error(self._h).decode()}")

    @property
    def ncells(self) -> int:
        return self._L.fks_ncells(self._h)

    @property
    def cluster_size(self) -> int:
        return self._L.fks_cluster_size(self._h)

    def set_cluster_size(self, C: int):
        self._check(self._L.fks_set_cluster_size(self._h, C), "fks_set_cluster_size")

    def set_schedule(self, C: int, radix: int = 0):
        """Cluster size and radix schedule (top radix of the length-n transforms, 0 = default)."""
        self._check(self._L.fks_set_schedule(self._h, C, radix), "fks_set_schedule")

    @property
    def radix(self) -> int:
        return self._L.fks_radix(self._h)

    @property
    def launches(self) -> int:
        return self._L.fks_launch_count(self._h)

    def collide(self, f, Q, stream=None):
        self._check(self._L.fks_collide(self._h, _dptr(f, self.dtype), _dptr(Q, self.dtype),
                                        _stream_ptr(stream)), "fks_collide")

    def transport(self, f, f_out, dt: float, stream=None):
        self._check(self._L.fks_transport(self._h, _dptr(f, self.dtype), _dptr(f_out, self.dtype), float(dt),
                                          _stream_ptr(stream)), "fks_transport")

    def step(self, f, f_out, dt: float, stream=None):
        self._check(self._L.fks_step(self._h, _dptr(f, self.dtype), _dptr(f_out, self.dtype), float(dt),
                                     _stream_ptr(stream)), "fks_step")

    def relax(self, f, f_out, dt: float, stream=None):
        """Collision sub-step alone (space-homogeneous cells): f_out = f + dt Q(f)."""
        self._check(self._L.fks_relax(self._h, _dptr(f, self.dtype), _dptr(f_out, self.dtype), float(dt),
                                      _stream_ptr(stream)), "fks_relax")

    def step_exp(self, f, f_out, dt: float, stream=None):
        """Stiff BGK step: transport, then the exact BGK relaxation over dt (BGK contexts)."""
        self._check(self._L.fks_step_exp(self._h, _dptr(f, self.dtype), _dptr(f_out, self.dtype), float(dt),
                                         _stream_ptr(stream)), "fks_step_exp")

    def step_strang(self, f, f_out, work, dt: float, stream=None):
        """Second-order step: Strang splitting with a Heun collision sub-step (work: scratch like f)."""
        self._check(self._L.fks_step_strang(self._h, _dptr(f, self.dtype), _dptr(f_out, self.dtype),
                                            _dptr(work, self.dtype), float(dt), _stream_ptr(stream)),
                    "fks_step_strang")

    def moments(self, f, U, stream=None):
        import torch
        self._check(self._L.fks_moments(self._h, _dptr(f, self.dtype), _dptr(U, torch.float64),
                                        _stream_ptr(stream)), "fks_moments")

    def check(self, stream=None) -> int:
        bits = ctypes.c_int()
        st = self._L.fks_check(self._h, _stream_ptr(stream), ctypes.byref(bits))
        self._check(st, "fks_check")
        return bits.value

    def surrogate_collide(self, net: "Net", f, Q, out_scale: float, ind_scale: float, threshold: float,
                          stream=None) -> int:
        """Q by the learned surrogate, cells over the indicator threshold by the spectral operator;
        returns the number of routed cells."""
        nr = ctypes.c_long()
        self._check(self._L.fks_surrogate_collide(self._h, net._h, _dptr(f, self.dtype), _dptr(Q, self.dtype),
                                                  float(out_scale), float(ind_scale), float(threshold),
                                                  ctypes.byref(nr), _stream_ptr(stream)), "fks_surrogate_collide")
        return nr.value

    def surrogate_step(self, net: "Net", f, f_out, work, dt: float, out_scale: float, ind_scale: float,
                       threshold: float, stream=None) -> int:
        """One step with the surrogate (transport into work, then f* + dt Q); returns the routed count."""
        nr = ctypes.c_long()
        self._check(self._L.fks_surrogate_step(self._h, net._h, _dptr(f, self.dtype), _dptr(f_out, self.dtype),
                                               _dptr(work, self.dtype), float(dt), float(out_scale), float(ind_scale),
                                               float(threshold), ctypes.byref(nr), _stream_ptr(stream)),
                    "fks_surrogate_step")
        return nr.value

    def indicator(self) -> np.ndarray:
        out = np.empty(self.ncells, dtype=np.float32)
        self._check(self._L.fks_surrogate_indicator(self._h, out.ctypes.data_as(ctypes.c_void_p), self.ncells),
                    "fks_surrogate_indicator")
        return out

    def offsets(self) -> np.ndarray:
        s = np.empty((3, self.cfg.n))
        self._check(self._L.fks_get_offsets(self._h, s.ctypes.data_as(ctypes.c_void_p)), "fks_get_offsets")
        return s

    def set_offsets(self, s):
        s = np.ascontiguousarray(s, dtype=np.float64).reshape(3, self.cfg.n)
        self._check(self._L.fks_set_offsets(self._h, s.ctypes.data_as(ctypes.c_void_p)), "fks_set_offsets")


class Batch:
    """fks_batch: independent homogeneous problems of uneven size.

    problems: list of dicts with keys n, L, kernel, C (default 0.25), kn."""

    def __init__(self, problems, A1=4, A2=8, rule=0, precision=FKS_FP32):
        import torch
        self._L = lib()
        k = len(problems)
        self.problems = problems
        self.n = [int(p["n"]) for p in problems]
        arr = lambda t, xs: (t * k)(*xs)
        d = _Dirs(A1, A2, rule)
        h = ctypes.c_void_p()
        st = self._L.fks_batch_init(k, arr(ctypes.c_int, self.n), arr(ctypes.c_double, [p["L"] for p in problems]),
                                    arr(ctypes.c_int, [int(p.get("kernel", 0)) for p in problems]),
                                    arr(ctypes.c_double, [float(p.get("C", 0.25)) for p in problems]),
                                    arr(ctypes.c_double, [float(p["kn"]) for p in problems]), ctypes.byref(d),
                                    precision, ctypes.byref(h))
        if st != 0:
            raise FKSError(st, "fks_batch_init")
        self._h = h
        self.dtype = torch.float64 if precision == FKS_FP64 else torch.float32

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            self._L.fks_batch_destroy(h)
            self._h = None

    def _check(self, st, what):
        if st != 0:
            raise FKSError(st, f"{what}: {self._L.fks_batch_last_error(self._h).decode()}")

    def _ptrs(self, ts):
        if len(ts) != len(self.n):
            raise ValueError("one tensor per problem")
        for t, n in zip(ts, self.n):
            _dptr(t, self.dtype)
            if t.numel() != n ** 3:
                raise ValueError("problem tensor must hold n^3 values")
        return (ctypes.c_void_p * len(ts))(*[t.data_ptr() for t in ts])

    def _dts(self, dt):
        if isinstance(dt, (int, float)):
            dt = [float(dt)] * len(self.n)
        return (ctypes.c_double * len(self.n))(*dt)

    def collide(self, fs, Qs, stream=None):
        self._check(self._L.fks_batch_collide(self._h, self._ptrs(fs), self._ptrs(Qs), _stream_ptr(stream)),
                    "fks_batch_collide")

    def step(self, fs, outs, dt, stream=None):
        self._check(self._L.fks_batch_step(self._h, self._ptrs(fs), self._ptrs(outs), self._dts(dt),
                                           _stream_ptr(stream)), "fks_batch_step")

    def run(self, fa, fb, dt, nsteps: int, stream=None):
        """nsteps ping-pong steps through one CUDA graph; result in fb if nsteps is odd else fa."""
        self._check(self._L.fks_batch_run(self._h, self._ptrs(fa), self._ptrs(fb), self._dts(dt), int(nsteps),
                                          _stream_ptr(stream)), "fks_batch_run")

    def check(self, stream=None) -> int:
        bits = ctypes.c_int()
        self._check(self._L.fks_batch_check(self._h, _stream_ptr(stream), ctypes.byref(bits)), "fks_batch_check")
        return bits.value

    def cluster_size(self, n: int) -> int:
        return self._L.fks_batch_cluster_size(self._h, n)

    def set_escalation(self, tol: float):
        """Precision escalation of FP32 batches (0: off)."""
        self._check(self._L.fks_batch_set_escalation(self._h, float(tol)), "fks_batch_set_escalation")

    def escalation(self) -> tuple[float, int]:
        """(tolerance, problems recomputed in FP64 by the last launch)."""
        tol = ctypes.c_double()
        cnt = ctypes.c_long()
        self._check(self._L.fks_batch_get_escalation(self._h, ctypes.byref(tol), ctypes.byref(cnt)),
                    "fks_batch_get_escalation")
        return tol.value, cnt.value

    def set_cluster_size(self, n: int, C: int):
        self._check(self._L.fks_batch_set_cluster_size(self._h, n, C), "fks_batch_set_cluster_size")

    def set_schedule(self, n: int, C: int, radix: int = 0):
        self._check(self._L.fks_batch_set_schedule(self._h, n, C, radix), "fks_batch_set_schedule")

    def radix(self, n: int) -> int:
        return self._L.fks_batch_radix(self._h, n)

    @property
    def launches(self) -> int:
        return self._L.fks_batch_launch_count(self._h)


class Net:
    """fks_net: the convolutional collision surrogate (BF16 weights, FP32 accumulation)."""

    def __init__(self, n: int, max_batch: int, seed: int = 0):
        self._L = lib()
        h = ctypes.c_void_p()
        st = self._L.fks_net_init(n, max_batch, seed, ctypes.byref(h))
        if st != 0:
            raise FKSError(st, "fks_net_init")
        self._h = h
        self.n = n
        self.max_batch = max_batch
        self.num_params = int(self._L.fks_net_num_params(h))

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            self._L.fks_net_destroy(h)
            self._h = None

    def _check(self, st, what):
        if st != 0:
            raise FKSError(st, f"{what}: {self._L.fks_net_last_error(self._h).decode()}")

    def get_params(self) -> np.ndarray:
        out = np.empty(self.num_params, dtype=np.float32)
        self._check(self._L.fks_net_get_params(self._h, out.ctypes.data_as(ctypes.c_void_p), self.num_params),
                    "fks_net_get_params")
        return out

    def set_params(self, p):
        p = np.ascontiguousarray(p, dtype=np.float32)
        self._check(self._L.fks_net_set_params(self._h, p.ctypes.data_as(ctypes.c_void_p), p.size),
                    "fks_net_set_params")

    def forward(self, x, y, stream=None):
        import torch
        self._check(self._L.fks_net_forward(self._h, x.shape[0], _dptr(x, torch.float32), _dptr(y, torch.float32),
                                            _stream_ptr(stream)), "fks_net_forward")

    def infer(self, x, y, stream=None):
        """Tensor-core inference (BF16 activations, FP32 accumulation)."""
        import torch
        self._check(self._L.fks_net_infer(self._h, x.shape[0], _dptr(x, torch.float32), _dptr(y, torch.float32),
                                          _stream_ptr(stream)), "fks_net_infer")

    def check(self, stream=None):
        self._check(self._L.fks_net_check(self._h, _stream_ptr(stream)), "fks_net_check")

    def gradient(self, x, gy, grad, stream=None):
        import torch
        self._check(self._L.fks_net_gradient(self._h, x.shape[0], _dptr(x, torch.float32),
                                             _dptr(gy, torch.float32), _dptr(grad, torch.float32),
                                             _stream_ptr(stream)), "fks_net_gradient")

    def train_step(self, x, target, lr: float, loss, stream=None):
        import torch
        self._check(self._L.fks_net_train_step(self._h, x.shape[0], _dptr(x, torch.float32),
                                               _dptr(target, torch.float32), float(lr), _dptr(loss, torch.float32),
                                               _stream_ptr(stream)), "fks_net_train_step")

    @property
    def launches(self) -> int:
        return self._L.fks_net_launch_count(self._h)


def surrogate_inputs(n: int, L: float, f, x, rho, dist, stream=None):
    """x = (f/rho, M[f]/rho), rho (FP64), dist = ||f/rho - M/rho|| / ||M/rho|| for every cell of f."""
    import torch
    st = lib().fks_surrogate_inputs(n, float(L), f.shape[0], _dptr(f, torch.float32), _dptr(x, torch.float32),
                                    _dptr(rho, torch.float64), _dptr(dist, torch.float32), _stream_ptr(stream))
    if st != 0:
        raise FKSError(st, "fks_surrogate_inputs")


def alu_peak(precision: int, stream=None) -> float:
    """Measured FMA throughput (TFLOP/s) of the FP32 or FP64 pipe."""
    t = ctypes.c_double()
    st = lib().fks_alu_peak(precision, ctypes.byref(t), _stream_ptr(stream))
    if st != 0:
        raise FKSError(st, "fks_alu_peak")
    return t.value


def selftest_wait(polls: int = 4096, stream=None) -> int:
    """Run the bounded-wait self-test (a wait that nothing completes); returns its
    status: FKS_ERR_TIMEOUT (6) is the expected result."""
    return lib().fks_selftest_wait(int(polls), _stream_ptr(stream))
