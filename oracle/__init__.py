"""FP64 CPU oracle for the parabolic operators and integrators of arXiv:1610.01265.

TEST INFRASTRUCTURE ONLY: imported by the tests, by the smoke check and by the
benchmark's CPU-baseline leg, never by the product path.  The arithmetic lives in
``oracle.c`` (plain loops, written from the paper); this module only compiles it
(gcc, in-tree under ``oracle/_build``) and marshals numpy arrays through ctypes.

Layout: scalar fields are float64 arrays of shape (nph, nth, nr) (r fastest);
operators are full 24-slot rows, shape (N, 24): slot s < 19 the neighbour at offsets()[s],
slots 19..23 (pole rows with the across-pole option only) the antipodal cells
(i + di, j, k + nph/2 + dk) for (di, dk) in pole_offsets().
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

NSLOT = 24   # slots per stored row
NS19 = 19    # the 19-point stencil
NPOLE = 5    # antipodal couplings of a pole cell (across-pole option)
PC_JACOBI = 1
PC_BILU0 = 2
STATUS = {0: "converged", 1: "not converged", 2: "breakdown", -1: "bad arguments"}


def build(force: bool = False) -> str:
    """Compile oracle.c into oracle/_build/liboracle.so (OpenMP when gcc supports it)."""
    src = os.path.join(_HERE, "oracle.c")
    if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(src):
        return _LIB_PATH
    os.makedirs(_BUILD, exist_ok=True)
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    base = ["gcc", "-O2", "-std=c99", "-fPIC", "-shared", src, "-o", tmp, "-lm"]
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True, capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB_PATH)
            D = ctypes.c_double
            P = ctypes.c_void_p
            I = ctypes.c_int
            lib.or_assemble_conduction.argtypes = [I, I, I, P, P, P, P, D, I, P, P]
            lib.or_assemble_viscosity.argtypes = [I, I, I, P, P, P, P, P]
            lib.or_energy_conduction.argtypes = [I, I, I, P, P, P, P, D, I, P]
            lib.or_energy_conduction.restype = D
            lib.or_apply_F.argtypes = [I, I, I, P, P, P, P, P]
            lib.or_gershgorin_dt.argtypes = [I, I, I, P, P, P, P]
            lib.or_gershgorin_dt.restype = D
            lib.or_rkl2_stages.argtypes = [D, I]
            lib.or_rkl2_coeffs.argtypes = [I, P, P, P, P]
            lib.or_rkl2_superstep.argtypes = [I, I, I, P, P, P, P, D, I]
            lib.or_rkl1_stages.argtypes = [D]
            lib.or_rkl1_coeffs.argtypes = [I, P, P, P]
            lib.or_rkl1_superstep.argtypes = [I, I, I, P, P, P, P, D, I]
            lib.or_bilu0_factor.argtypes = [I, I, I, P, P, I, P, P]
            lib.or_bilu0_apply.argtypes = [I, I, I, P, P, I, P, P, P]
            lib.or_be_pcg.argtypes = [I, I, I, P, P, P, P, D, I, P, I, D, I, P, I, P, P]
            lib.or_offsets.argtypes = [P]
            lib.or_pole_offsets.argtypes = [P, P]
            lib.or_num_threads.restype = I
            lib.or_set_num_threads.argtypes = [I]
            _lib = lib
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


class Grid:
    """nr x nth x nph cell-centred spherical grid; rf = nr+1 radial faces in R_sun."""

    def __init__(self, rf, nth: int, nph: int):
        self.rf = _f64(rf)
        self.nr = len(self.rf) - 1
        self.nth = int(nth)
        self.nph = int(nph)

    @property
    def shape(self):
        return (self.nph, self.nth, self.nr)

    @property
    def N(self):
        return self.nr * self.nth * self.nph

    def _dims(self):
        return (self.nr, self.nth, self.nph, _ptr(self.rf))


def offsets() -> np.ndarray:
    """(19, 3) neighbour offsets of the stencil slots."""
    out = np.zeros((NS19, 3), dtype=np.int32)
    _load().or_offsets(_ptr(out))
    return out


def pole_offsets() -> np.ndarray:
    """(5, 2) offsets (di, dk) of the antipodal slots 19..23 from (i, k + nph/2)."""
    di = np.zeros(NPOLE, dtype=np.int32)
    dk = np.zeros(NPOLE, dtype=np.int32)
    _load().or_pole_offsets(_ptr(di), _ptr(dk))
    return np.stack([di, dk], axis=1)


def num_threads() -> int:
    return _load().or_num_threads()


def set_num_threads(n: int) -> None:
    """Host threads of the parallel loops (timing only)."""
    _load().or_set_num_threads(int(n))


def assemble_conduction(g: Grid, T, bhat, n, kappa0: float = 9e-7, beta_tcut: bool = False,
                        isotropic: bool = False, flux_form: bool = False, across_pole: bool = False):
    """S (N,24) = Hessian of the discrete energy (flux_form: minus the divergence of the
    face fluxes, non-symmetric, whose symmetric part is that Hessian), W (N,) = 3 k_B n V.
    across_pole: theta-ghosts beyond a pole at phi + pi (needs nth >= 2, even nph >= 6)."""
    T, bhat, n = _f64(T), _f64(bhat), _f64(n)
    S = np.empty((g.N, NSLOT))
    W = np.empty(g.N)
    flags = (1 if beta_tcut else 0) | (2 if isotropic else 0) | (4 if flux_form else 0) | (8 if across_pole else 0)
    rc = _load().or_assemble_conduction(*g._dims(), _ptr(T), _ptr(bhat), _ptr(n), kappa0, flags,
                                        _ptr(S), _ptr(W))
    if rc != 0:
        raise ValueError("bad grid for the oracle (needs nr>=1, nth>=1, nph>=3; across-pole: nth>=2, even nph>=6)")
    return S, W


def assemble_viscosity(g: Grid, rho, nu):
    rho, nu = _f64(rho), _f64(nu)
    S = np.empty((g.N, NSLOT))
    W = np.empty(g.N)
    rc = _load().or_assemble_viscosity(*g._dims(), _ptr(rho), _ptr(nu), _ptr(S), _ptr(W))
    if rc != 0:
        raise ValueError("bad grid for the oracle")
    return S, W


def energy_conduction(g: Grid, T, bhat, n, u, kappa0: float = 9e-7, beta_tcut: bool = False,
                      isotropic: bool = False, across_pole: bool = False) -> float:
    T, bhat, n, u = _f64(T), _f64(bhat), _f64(n), _f64(u)
    flags = (1 if beta_tcut else 0) | (2 if isotropic else 0) | (8 if across_pole else 0)
    return _load().or_energy_conduction(*g._dims(), _ptr(T), _ptr(bhat), _ptr(n), kappa0, flags,
                                        _ptr(u))


def apply_F(g: Grid, S, W, u) -> np.ndarray:
    S, W, u = _f64(S), _f64(W), _f64(u)
    out = np.empty(g.N)
    _load().or_apply_F(*g._dims(), _ptr(S), _ptr(W), _ptr(u), _ptr(out))
    return out.reshape(np.shape(u))


def gershgorin_dt(g: Grid, S, W):
    """(dt_Euler, |lambda|max bound) from App. B's row-sum Gershgorin bound."""
    S, W = _f64(S), _f64(W)
    lam = ctypes.c_double(0.0)
    dt = _load().or_gershgorin_dt(*g._dims(), _ptr(S), _ptr(W), ctypes.byref(lam))
    return dt, lam.value


def rkl2_stages(ratio: float, force_odd: bool = False) -> int:
    return _load().or_rkl2_stages(float(ratio), 1 if force_odd else 0)


def rkl2_coeffs(s: int):
    """(mu, nu, mu~, gamma~) arrays indexed by stage j = 0..s."""
    arrs = [np.zeros(s + 1) for _ in range(4)]
    _load().or_rkl2_coeffs(int(s), *[_ptr(a) for a in arrs])
    return tuple(arrs)


def rkl2_superstep(g: Grid, S, W, u, dt: float, s: int) -> np.ndarray:
    S, W = _f64(S), _f64(W)
    out = _f64(u).copy()
    rc = _load().or_rkl2_superstep(*g._dims(), _ptr(S), _ptr(W), _ptr(out), float(dt), int(s))
    if rc != 0:
        raise ValueError("s must be >= 2")
    return out


def rkl1_stages(ratio: float) -> int:
    """Smallest s with (s^2 + s)/2 >= dt/dt_E (at least 1)."""
    return _load().or_rkl1_stages(float(ratio))


def rkl1_coeffs(s: int):
    """(mu, nu, mu~) of RKL1 indexed by stage j = 0..s."""
    arrs = [np.zeros(s + 1) for _ in range(3)]
    _load().or_rkl1_coeffs(int(s), *[_ptr(a) for a in arrs])
    return tuple(arrs)


def rkl1_superstep(g: Grid, S, W, u, dt: float, s: int) -> np.ndarray:
    S, W = _f64(S), _f64(W)
    out = _f64(u).copy()
    if _load().or_rkl1_superstep(*g._dims(), _ptr(S), _ptr(W), _ptr(out), float(dt), int(s)) != 0:
        raise ValueError("s must be >= 1")
    return out


def euler_step(g: Grid, S, W, u, h: float) -> np.ndarray:
    """One explicit Euler step u + h F(u)."""
    return _f64(u) + h * apply_F(g, S, W, u)


def build_A(S, W, dt: float) -> np.ndarray:
    A = np.asarray(S, dtype=np.float64) * dt
    A[:, 0] += W
    return A


def bilu0_factor(g: Grid, A, block, pattern: int = 19) -> np.ndarray:
    """Zero-fill ILU of every block; pattern = 19 (conduction) or 7 (viscosity)."""
    A = _f64(A)
    blk = np.asarray(block, dtype=np.int32)
    LU = np.empty_like(A)
    rc = _load().or_bilu0_factor(*g._dims(), _ptr(blk), int(pattern), _ptr(A), _ptr(LU))
    if rc != 0:
        raise ValueError("grid not divisible by block")
    return LU


def bilu0_apply(g: Grid, LU, block, r, pattern: int = 19) -> np.ndarray:
    LU, r = _f64(LU), _f64(r)
    blk = np.asarray(block, dtype=np.int32)
    z = np.empty(g.N)
    _load().or_bilu0_apply(*g._dims(), _ptr(blk), int(pattern), _ptr(LU), _ptr(r), _ptr(z))
    return z.reshape(np.shape(r))


def be_pcg(g: Grid, S, W, u, dt: float, pc: int = PC_JACOBI, block=(8, 8, 8), rtol: float = 1e-10,
           maxit: int = 10000, x0=None, fixed_iters: int = 0, pattern: int = 19):
    """BE step by PCG; returns (x, iters, relres, status).  pattern: 19 (conduction) or 7
    (viscosity), the structural pattern kept by the PC2 zero-fill ILU."""
    S, W = _f64(S), _f64(W)
    x = _f64(u).copy()
    blk = np.asarray(block, dtype=np.int32)
    x0a = _f64(x0) if x0 is not None else None
    x0p = _ptr(x0a) if x0a is not None else None
    it = ctypes.c_int(0)
    rel = ctypes.c_double(0.0)
    st = _load().or_be_pcg(*g._dims(), _ptr(S), _ptr(W), _ptr(x), float(dt), int(pc), _ptr(blk),
                           int(pattern), float(rtol), int(maxit), x0p, int(fixed_iters), ctypes.byref(it),
                           ctypes.byref(rel))
    if st < 0:
        raise ValueError("bad PCG arguments")
    return x, it.value, rel.value, st


def dense(g: Grid, S) -> np.ndarray:
    """Dense N x N matrix of a stored operator (tiny grids only)."""
    off = offsets()
    poff = pole_offsets()
    N = g.N
    Dm = np.zeros((N, N))
    nr, nth, nph = g.nr, g.nth, g.nph
    for k in range(nph):
        for j in range(nth):
            for i in range(nr):
                c = (k * nth + j) * nr + i
                for s in range(NS19):
                    ii, jj, kk = i + off[s, 0], j + off[s, 1], (k + off[s, 2]) % nph
                    if 0 <= ii < nr and 0 <= jj < nth:
                        Dm[c, (kk * nth + jj) * nr + ii] += S[c, s]
                if j in (0, nth - 1):
                    for q in range(NPOLE):
                        ii, kk = i + poff[q, 0], (k + nph // 2 + poff[q, 1]) % nph
                        if 0 <= ii < nr:
                            Dm[c, (kk * nth + j) * nr + ii] += S[c, NS19 + q]
    return Dm
