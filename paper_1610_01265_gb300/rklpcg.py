"""Thin ctypes binding of the rklpcg C ABI (``include/rklpcg.h``).

Argument marshalling only: every step of the computation runs in the CUDA library
``_build/librklpcg.so``.  Arrays may be torch tensors (CUDA or CPU) or numpy arrays,
contiguous float64; their data pointers are handed to the library unchanged (host
arrays are staged by the library itself).  The library must have been built
(``paper_1610_01265_gb300.build.build()``); importing the binding never falls back to
anything else.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

RKL_OK = 0
RKL_EINVAL = -1
RKL_ENOMEM = -2
RKL_ECUDA = -3
RKL_ENONFINITE = -4
RKL_ENOTCONV = -5
RKL_EBREAKDOWN = -6
RKL_ESTATE = -7
RKL_OP_CONDUCTION = 0
RKL_OP_VISCOSITY = 1
RKL_PC_JACOBI = 1
RKL_PC_BILU0 = 2
RKL_F64 = 0
RKL_F32MIX = 1
RKL_BETA_TCUT = 1
RKL_FLUX_FORM = 2
RKL_ACROSS_POLE = 4
RKL_FORCE_ODD = 1

EXPORTED = ("rkl_create", "rkl_destroy", "rkl_set_stream", "rkl_strerror", "rkl_last_error",
            "rkl_kernel_launches", "rkl2_stage_count", "set_coeffs", "apply_F", "rkl2_superstep",
            "be_pcg_solve", "rkl2_superstep_noalloc", "rkl_profile_enable", "rkl_profile_read",
            "sts_advance", "rkl_fp64_peak")
RKL_SCHEME_RKL2 = 0
RKL_SCHEME_RKL1 = 1

KERNELS = ("setup", "apply_F", "rkl2_first", "rkl2_stage", "pcg_init", "spmv", "pcg_update",
           "pcg_pupdate", "bilu_factor", "bilu_apply")


class RklError(RuntimeError):
    def __init__(self, code: int, where: str, detail: str = ""):
        self.code = code
        msg = f"{where}: {strerror(code)} ({code})"
        if detail:
            msg += f": {detail}"
        super().__init__(msg)


class StsOptions(ctypes.Structure):
    _fields_ = [("scheme", ctypes.c_int), ("cycles", ctypes.c_int), ("extra_stages", ctypes.c_int),
                ("euler_fraction", ctypes.c_double), ("flags", ctypes.c_int)]


class _Grid(ctypes.Structure):
    _fields_ = [("nr", ctypes.c_int), ("nth", ctypes.c_int), ("nph", ctypes.c_int),
                ("r_faces", ctypes.POINTER(ctypes.c_double)), ("rsun_cm", ctypes.c_double)]


_lib = None


def library_path() -> str:
    return _build.LIB


def load(path: str | None = None):
    """Load librklpcg.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or library_path()
    if not os.path.exists(path):
        raise RuntimeError(f"rklpcg CUDA library not built ({path}); run paper_1610_01265_gb300.build.build()")
    lib = ctypes.CDLL(path)
    P, I, D = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
    lib.rkl_create.argtypes = [ctypes.POINTER(P), ctypes.POINTER(_Grid), I, P]
    lib.rkl_destroy.argtypes = [P]
    lib.rkl_set_stream.argtypes = [P, P]
    lib.rkl_strerror.argtypes = [I]
    lib.rkl_strerror.restype = ctypes.c_char_p
    lib.rkl_last_error.argtypes = [P]
    lib.rkl_last_error.restype = ctypes.c_char_p
    lib.rkl_kernel_launches.argtypes = [P]
    lib.rkl_kernel_launches.restype = ctypes.c_longlong
    lib.rkl2_stage_count.argtypes = [D, I]
    lib.set_coeffs.argtypes = [P, I, P, P, P, D, I, ctypes.POINTER(D)]
    lib.apply_F.argtypes = [P, P, P, I]
    lib.rkl2_superstep.argtypes = [P, P, I, D, D, I, I, ctypes.POINTER(I)]
    lib.be_pcg_solve.argtypes = [P, P, I, D, I, ctypes.POINTER(I), D, I, P, ctypes.POINTER(I),
                                 ctypes.POINTER(D)]
    lib.sts_advance.argtypes = [P, P, I, D, D, ctypes.POINTER(StsOptions), ctypes.POINTER(I)]
    lib.rkl_profile_enable.argtypes = [P, I]
    lib.rkl_profile_read.argtypes = [P, I, ctypes.POINTER(D), ctypes.POINTER(ctypes.c_longlong)]
    lib.rkl2_superstep_noalloc.argtypes = [ctypes.POINTER(_Grid), P, P, P, D, I, P, D, I, I, P,
                                           ctypes.POINTER(D), ctypes.POINTER(I)]
    lib.rkl_fp64_peak.argtypes = [P, ctypes.POINTER(D)]
    _lib = lib
    return lib


def strerror(code: int) -> str:
    return load().rkl_strerror(int(code)).decode()


def rkl2_stage_count(dt_over_dt_exp: float, flags: int = 0) -> int:
    s = load().rkl2_stage_count(float(dt_over_dt_exp), int(flags))
    if s < 0:
        raise RklError(s, "rkl2_stage_count")
    return s


def rkl2_superstep_noalloc(r_faces, nth: int, nph: int, T, bhat, n, u, dt: float, kappa0: float = 9e-7,
                           beta_tcut: bool = False, s: int = 0, force_odd: bool = False, stream=None):
    """Conduction set-up + one RKL2 super-step with no device allocation (device arrays only);
    for callers whose memory is owned elsewhere.  Returns (s_used, dt_exp)."""
    lib = load()
    rf = np.ascontiguousarray(r_faces, dtype=np.float64)
    nr = len(rf) - 1
    N = nr * int(nth) * int(nph)
    g = _Grid(nr, int(nth), int(nph), rf.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    dte = ctypes.c_double(0.0)
    used = ctypes.c_int(0)
    code = lib.rkl2_superstep_noalloc(ctypes.byref(g), _ptr(T, N), _ptr(bhat, 3 * N), _ptr(n, N), float(kappa0),
                                      RKL_BETA_TCUT if beta_tcut else 0, _ptr(u, N), float(dt), int(s),
                                      RKL_FORCE_ODD if force_odd else 0,
                                      stream if stream is not None else _current_stream(),
                                      ctypes.byref(dte), ctypes.byref(used))
    if code != RKL_OK:
        raise RklError(code, "rkl2_superstep_noalloc")
    return used.value, dte.value


def fp64_peak(stream=None) -> float:
    """Measured FP64 FMA throughput of the current device, TFLOP/s (instrumentation)."""
    tf = ctypes.c_double(0.0)
    code = load().rkl_fp64_peak(stream if stream is not None else _current_stream(), ctypes.byref(tf))
    if code != RKL_OK:
        raise RklError(code, "rkl_fp64_peak")
    return tf.value


def _ptr(a, n: int | None = None):
    """Data pointer of a contiguous float64 torch tensor / numpy array (None -> NULL)."""
    if a is None:
        return None
    if isinstance(a, int):
        return a
    if isinstance(a, np.ndarray):
        if a.dtype != np.float64 or not a.flags["C_CONTIGUOUS"]:
            raise TypeError("arrays must be contiguous float64")
        if n is not None and a.size < n:
            raise ValueError(f"array too small: {a.size} < {n}")
        return a.ctypes.data
    import torch  # noqa: PLC0415 - only needed when tensors are passed

    if not isinstance(a, torch.Tensor):
        raise TypeError(f"unsupported array type {type(a)!r}")
    if a.dtype != torch.float64 or not a.is_contiguous():
        raise TypeError("tensors must be contiguous float64")
    if n is not None and a.numel() < n:
        raise ValueError(f"tensor too small: {a.numel()} < {n}")
    return a.data_ptr()


def _current_stream():
    try:
        import torch  # noqa: PLC0415

        if torch.cuda.is_available():
            return torch.cuda.current_stream().cuda_stream
    except ImportError:
        pass
    return None


class Context:
    """One grid on the current CUDA device; mirrors rkl_create .. rkl_destroy."""

    def __init__(self, r_faces, nth: int, nph: int, stream=None, prec: int = RKL_F64, rsun_cm: float = 0.0):
        """prec = RKL_F64, or RKL_F32MIX for the mixed-precision path (FP32 operator and
        stages, FP64 coefficients of the recurrence, dot products and residual correction).
        rsun_cm: length unit of r_faces in cm (0: R_sun = 6.96e10 cm)."""
        self._lib = load()
        rf = np.ascontiguousarray(r_faces, dtype=np.float64)
        self.nr, self.nth, self.nph = len(rf) - 1, int(nth), int(nph)
        self.N = self.nr * self.nth * self.nph
        self._rf = rf
        g = _Grid(self.nr, self.nth, self.nph, rf.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), float(rsun_cm))
        h = ctypes.c_void_p()
        if stream is None:
            stream = _current_stream()
        code = self._lib.rkl_create(ctypes.byref(h), ctypes.byref(g), int(prec), stream)
        if code != RKL_OK:
            raise RklError(code, "rkl_create")
        self._h = h

    @property
    def handle(self):
        return self._h

    def close(self):
        if getattr(self, "_h", None):
            self._lib.rkl_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def _check(self, code: int, where: str):
        if code != RKL_OK:
            raise RklError(code, where, self._lib.rkl_last_error(self._h).decode())

    @property
    def kernel_launches(self) -> int:
        return int(self._lib.rkl_kernel_launches(self._h))

    def profile_enable(self, on: bool = True):
        """Start (clearing the counters) or stop per-kernel event timing."""
        self._check(self._lib.rkl_profile_enable(self._h, 1 if on else 0), "rkl_profile_enable")

    def profile(self) -> dict:
        """{kernel family: (total ms, counted launches)} (synchronises the stream)."""
        out = {}
        for k, name in enumerate(KERNELS):
            ms = ctypes.c_double(0.0)
            n = ctypes.c_longlong(0)
            self._check(self._lib.rkl_profile_read(self._h, k, ctypes.byref(ms), ctypes.byref(n)),
                        "rkl_profile_read")
            out[name] = (ms.value, n.value)
        return out

    def set_stream(self, stream):
        self._check(self._lib.rkl_set_stream(self._h, stream), "rkl_set_stream")

    def set_coeffs(self, op: int, a, b, c, kappa0: float = 9e-7, flags: int = 0) -> float:
        dt = ctypes.c_double(0.0)
        N = self.N
        code = self._lib.set_coeffs(self._h, int(op), _ptr(a, N), _ptr(b, 3 * N), _ptr(c, N),
                                    float(kappa0), int(flags), ctypes.byref(dt))
        self._check(code, "set_coeffs")
        return dt.value

    def set_conduction(self, T, bhat, n, kappa0: float = 9e-7, beta_tcut: bool = False,
                       flux_form: bool = False, across_pole: bool = False) -> float:
        flags = ((RKL_BETA_TCUT if beta_tcut else 0) | (RKL_FLUX_FORM if flux_form else 0)
                 | (RKL_ACROSS_POLE if across_pole else 0))
        return self.set_coeffs(RKL_OP_CONDUCTION, T, bhat, n, kappa0, flags)

    def set_viscosity(self, rho, nu) -> float:
        return self.set_coeffs(RKL_OP_VISCOSITY, rho, None, nu)

    def apply_F(self, u, Fu, ncomp: int = 1):
        n = self.N * ncomp
        self._check(self._lib.apply_F(self._h, _ptr(u, n), _ptr(Fu, n), int(ncomp)), "apply_F")
        return Fu

    def rkl2_superstep(self, u, dt: float, dt_exp: float = 0.0, s: int = 0, force_odd: bool = False,
                       ncomp: int = 1) -> int:
        used = ctypes.c_int(0)
        code = self._lib.rkl2_superstep(self._h, _ptr(u, self.N * ncomp), int(ncomp), float(dt),
                                        float(dt_exp), int(s), RKL_FORCE_ODD if force_odd else 0,
                                        ctypes.byref(used))
        self._check(code, "rkl2_superstep")
        return used.value

    def sts_advance(self, u, dt: float, dt_exp: float, scheme: int = RKL_SCHEME_RKL2, cycles: int = 1,
                    extra_stages: int = 0, euler_fraction: float = 0.0, force_odd: bool = False,
                    ncomp: int = 1) -> int:
        """Sec. 6 damping variants (Euler prefix, sub-cycles, RKL1, extra stages); returns the
        number of operator applications."""
        opt = StsOptions(int(scheme), int(cycles), int(extra_stages), float(euler_fraction),
                         RKL_FORCE_ODD if force_odd else 0)
        used = ctypes.c_int(0)
        code = self._lib.sts_advance(self._h, _ptr(u, self.N * ncomp), int(ncomp), float(dt), float(dt_exp),
                                     ctypes.byref(opt), ctypes.byref(used))
        self._check(code, "sts_advance")
        return used.value

    def be_pcg_solve(self, u, dt: float, pc: int = RKL_PC_JACOBI, block=(8, 8, 8), rtol: float = 1e-10,
                     maxit: int = 100000, x0=None, ncomp: int = 1):
        """Returns (code, iters[ncomp], relres[ncomp]); code is RKL_OK, RKL_ENOTCONV or
        RKL_EBREAKDOWN (other failures raise)."""
        blk = (ctypes.c_int * 3)(*[int(b) for b in block])
        its = (ctypes.c_int * ncomp)()
        rel = (ctypes.c_double * ncomp)()
        n = self.N * ncomp
        code = self._lib.be_pcg_solve(self._h, _ptr(u, n), int(ncomp), float(dt), int(pc), blk,
                                      float(rtol), int(maxit), _ptr(x0, n), its, rel)
        if code not in (RKL_OK, RKL_ENOTCONV, RKL_EBREAKDOWN):
            self._check(code, "be_pcg_solve")
        return code, list(its), list(rel)
