"""Thin ctypes binding of the learned-initial-guess C ABI (``include/warmstart.h``).

Argument marshalling only: the net's forward and backward passes, the loss, Adam and
the guess x0 = T + scale * y all run in ``_build/librklpcg.so``.  Device arrays are torch
CUDA tensors (float32 for net inputs/outputs, float64 for T, bhat and x0); parameter and
gradient vectors may be numpy float32 arrays.
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import rklpcg as R

EXPORTED = ("ws_num_params", "ws_create", "ws_destroy", "ws_set_stream", "ws_last_error",
            "ws_kernel_launches", "ws_set_params", "ws_get_params", "ws_get_grads", "ws_set_grads",
            "ws_forward", "ws_loss_grad", "ws_adam", "ws_features", "ws_guess", "ws_target", "ws_check")
LAYERS = ((5, 32), (32, 32), (32, 32), (32, 1))

_bound = False


def load():
    global _bound
    lib = R.load()
    if not _bound:
        P, I, D = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
        IA = ctypes.POINTER(ctypes.c_int)
        lib.ws_num_params.argtypes = []
        lib.ws_create.argtypes = [ctypes.POINTER(P), ctypes.c_ulonglong, P]
        lib.ws_destroy.argtypes = [P]
        lib.ws_set_stream.argtypes = [P, P]
        lib.ws_last_error.argtypes = [P]
        lib.ws_last_error.restype = ctypes.c_char_p
        lib.ws_kernel_launches.argtypes = [P]
        lib.ws_kernel_launches.restype = ctypes.c_longlong
        for name in ("ws_set_params", "ws_get_params", "ws_get_grads", "ws_set_grads"):
            getattr(lib, name).argtypes = [P, P, I]
        lib.ws_forward.argtypes = [P, IA, I, I, P, P]
        lib.ws_loss_grad.argtypes = [P, IA, I, I, P, P, P, ctypes.POINTER(D)]
        lib.ws_adam.argtypes = [P, D]
        lib.ws_features.argtypes = [P, ctypes.POINTER(R._Grid), P, P, D, P]
        lib.ws_guess.argtypes = [P, ctypes.POINTER(R._Grid), P, P, D, D, P]
        lib.ws_target.argtypes = [P, ctypes.c_longlong, P, P, D, P]
        lib.ws_check.argtypes = [P]
        _bound = True
    return lib


def num_params() -> int:
    return load().ws_num_params()


def _p(a, dtype, n: int | None = None):
    """Data pointer of a contiguous array of the given dtype (numpy or torch)."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        if a.dtype != np.dtype(dtype) or not a.flags["C_CONTIGUOUS"]:
            raise TypeError(f"arrays must be contiguous {np.dtype(dtype)}")
        if n is not None and a.size < n:
            raise ValueError(f"array too small: {a.size} < {n}")
        return a.ctypes.data
    import torch  # noqa: PLC0415

    tdt = {np.float32: torch.float32, np.float64: torch.float64}[dtype]
    if not isinstance(a, torch.Tensor) or a.dtype != tdt or not a.is_contiguous():
        raise TypeError(f"tensors must be contiguous {tdt}")
    if n is not None and a.numel() < n:
        raise ValueError(f"tensor too small: {a.numel()} < {n}")
    return a.data_ptr()


class Net:
    """One net on the current CUDA device (ws_create .. ws_destroy)."""

    def __init__(self, seed: int = 0, stream=None):
        self._lib = load()
        h = ctypes.c_void_p()
        code = self._lib.ws_create(ctypes.byref(h), int(seed), stream if stream is not None else R._current_stream())
        if code != R.RKL_OK:
            raise R.RklError(code, "ws_create")
        self._h = h
        self.nparam = self._lib.ws_num_params()

    def _check(self, code, where):
        if code != R.RKL_OK:
            detail = self._lib.ws_last_error(self._h).decode() if self._h else ""
            raise R.RklError(code, where, detail)

    def close(self):
        if getattr(self, "_h", None):
            self._lib.ws_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:  # noqa: BLE001
            pass

    def set_stream(self, stream):
        self._check(self._lib.ws_set_stream(self._h, stream), "ws_set_stream")

    def kernel_launches(self) -> int:
        return int(self._lib.ws_kernel_launches(self._h))

    def params(self) -> np.ndarray:
        out = np.empty(self.nparam, dtype=np.float32)
        self._check(self._lib.ws_get_params(self._h, out.ctypes.data, self.nparam), "ws_get_params")
        return out

    def set_params(self, p):
        p = np.ascontiguousarray(p, dtype=np.float32)
        self._check(self._lib.ws_set_params(self._h, p.ctypes.data, p.size), "ws_set_params")

    def grads(self) -> np.ndarray:
        out = np.empty(self.nparam, dtype=np.float32)
        self._check(self._lib.ws_get_grads(self._h, out.ctypes.data, self.nparam), "ws_get_grads")
        return out

    def set_grads(self, g):
        g = np.ascontiguousarray(g, dtype=np.float32)
        self._check(self._lib.ws_set_grads(self._h, g.ctypes.data, g.size), "ws_set_grads")

    @staticmethod
    def _box(box):
        b = (ctypes.c_int * 3)(*[int(v) for v in box])
        return b, int(box[0]) * int(box[1]) * int(box[2])

    def forward(self, box, feats, y, nbox: int = 1, periodic: bool = True):
        """y (float32 CUDA, nbox*cells) = net(feats (float32 CUDA, [5][nbox*cells]))."""
        b, nc = self._box(box)
        n = nc * nbox
        self._check(self._lib.ws_forward(self._h, b, int(nbox), int(bool(periodic)), _p(feats, np.float32, 5 * n),
                                         _p(y, np.float32, n)), "ws_forward")

    def loss_grad(self, box, feats, target, weight=None, nbox: int = 1, periodic: bool = True,
                  want_loss: bool = True):
        b, nc = self._box(box)
        n = nc * nbox
        loss = ctypes.c_double(0.0)
        self._check(self._lib.ws_loss_grad(self._h, b, int(nbox), int(bool(periodic)), _p(feats, np.float32, 5 * n),
                                           _p(target, np.float32, n), _p(weight, np.float32, n),
                                           ctypes.byref(loss) if want_loss else None), "ws_loss_grad")
        return loss.value if want_loss else None

    def adam(self, lr: float):
        self._check(self._lib.ws_adam(self._h, float(lr)), "ws_adam")

    @staticmethod
    def _grid(nr, nth, nph):
        return R._Grid(int(nr), int(nth), int(nph), None)

    def features(self, shape, T, bhat, dt: float, feat):
        """feat (float32 CUDA [5][N]) from T, bhat (float64 CUDA) of a whole grid of shape (nph, nth, nr)."""
        nph, nth, nr = shape
        N = nr * nth * nph
        g = self._grid(nr, nth, nph)
        self._check(self._lib.ws_features(self._h, ctypes.byref(g), _p(T, np.float64, N), _p(bhat, np.float64, 3 * N),
                                          float(dt), _p(feat, np.float32, 5 * N)), "ws_features")

    def guess(self, shape, T, bhat, dt: float, scale: float, x0):
        """x0 = T + scale * net(T, bhat, dt) on a whole grid (float64 CUDA arrays)."""
        nph, nth, nr = shape
        N = nr * nth * nph
        g = self._grid(nr, nth, nph)
        self._check(self._lib.ws_guess(self._h, ctypes.byref(g), _p(T, np.float64, N), _p(bhat, np.float64, 3 * N),
                                       float(dt), float(scale), _p(x0, np.float64, N)), "ws_guess")

    def target(self, x, base, unit: float, out):
        """out (float32 CUDA) = (x - base) / unit for float64 CUDA arrays x, base."""
        n = x.numel()
        self._check(self._lib.ws_target(self._h, n, _p(x, np.float64, n), _p(base, np.float64, n), float(unit),
                                        _p(out, np.float32, n)), "ws_target")

    def check(self):
        """Drain the stream; raise if a tensor-core convolution since the last check gave up
        waiting for its MMAs (its outputs would not be valid)."""
        self._check(self._lib.ws_check(self._h), "ws_check")
