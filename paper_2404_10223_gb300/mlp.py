"""ctypes binding of the proposal network (include/tnqe_mlp.h).

Argument marshalling only: forward, gradient and Adam run in the library's
CUDA kernels (csrc/mlp.cu).  Loading fails loudly when the library is absent.
"""
from __future__ import annotations

import ctypes
from typing import Optional

import numpy as np

from . import tnqe

EXPORTED = ["tnqe_mlp_create", "tnqe_mlp_param_count", "tnqe_mlp_set_params", "tnqe_mlp_get_params",
            "tnqe_mlp_forward", "tnqe_mlp_gradient", "tnqe_mlp_adam_step", "tnqe_mlp_last_launches",
            "tnqe_mlp_last_error", "tnqe_mlp_destroy"]

_bound = None


def load(path: str = tnqe.LIB_PATH) -> ctypes.CDLL:
    global _bound
    lib = tnqe.load(path)
    if _bound is lib:
        return lib
    P, I, F, LL = ctypes.c_void_p, ctypes.c_int, ctypes.c_float, ctypes.c_longlong
    lib.tnqe_mlp_create.argtypes = [I, I, I, I, P, ctypes.POINTER(P)]
    lib.tnqe_mlp_create.restype = I
    lib.tnqe_mlp_param_count.argtypes = [P]
    lib.tnqe_mlp_param_count.restype = LL
    lib.tnqe_mlp_set_params.argtypes = [P, P]
    lib.tnqe_mlp_get_params.argtypes = [P, P]
    lib.tnqe_mlp_forward.argtypes = [P, P, I, P]
    lib.tnqe_mlp_gradient.argtypes = [P, P, P, P, I, ctypes.POINTER(F), P]
    lib.tnqe_mlp_adam_step.argtypes = [P, P, P, P, I, F, F, F, F, ctypes.POINTER(F)]
    lib.tnqe_mlp_last_launches.argtypes = [P]
    lib.tnqe_mlp_last_launches.restype = I
    lib.tnqe_mlp_last_error.argtypes = [P]
    lib.tnqe_mlp_last_error.restype = ctypes.c_char_p
    lib.tnqe_mlp_destroy.argtypes = [P]
    lib.tnqe_mlp_destroy.restype = None
    for n in ("tnqe_mlp_set_params", "tnqe_mlp_get_params", "tnqe_mlp_forward", "tnqe_mlp_gradient",
              "tnqe_mlp_adam_step"):
        getattr(lib, n).restype = I
    _bound = lib
    return lib


def _f32(a, shape=None) -> np.ndarray:
    a = np.ascontiguousarray(np.asarray(a, dtype=np.float32))
    if shape is not None and a.shape != shape:
        a = a.reshape(shape)
    return a


class Mlp:
    """The n_in -> n_h -> n_h -> n_out GELU network on the GPU."""

    def __init__(self, n_in: int, n_h: int, n_out: int, max_batch: int = 4096, stream: Optional[int] = None):
        lib = load()
        self.n_in, self.n_h, self.n_out, self.max_batch = n_in, n_h, n_out, max_batch
        h = ctypes.c_void_p()
        st = lib.tnqe_mlp_create(n_in, n_h, n_out, max_batch, ctypes.c_void_p(stream or 0), ctypes.byref(h))
        if st != 0:
            raise tnqe.TnqeError(st, "tnqe_mlp_create failed")
        self.h = h
        self.count = int(lib.tnqe_mlp_param_count(h))

    def _check(self, st: int):
        if st != 0:
            raise tnqe.TnqeError(st, load().tnqe_mlp_last_error(self.h).decode())

    def set_params(self, flat):
        flat = _f32(flat)
        assert flat.size == self.count
        self._check(load().tnqe_mlp_set_params(self.h, flat.ctypes.data_as(ctypes.c_void_p)))

    def get_params(self) -> np.ndarray:
        out = np.zeros(self.count, dtype=np.float32)
        self._check(load().tnqe_mlp_get_params(self.h, out.ctypes.data_as(ctypes.c_void_p)))
        return out

    def forward(self, X) -> np.ndarray:
        X = _f32(X)
        B = X.shape[0]
        Y = np.zeros((B, self.n_out), dtype=np.float32)
        self._check(load().tnqe_mlp_forward(self.h, X.ctypes.data_as(ctypes.c_void_p), B,
                                            Y.ctypes.data_as(ctypes.c_void_p)))
        return Y

    def gradient(self, X, T, w=None):
        X, T = _f32(X), _f32(T)
        wp = None if w is None else _f32(w)
        g = np.zeros(self.count, dtype=np.float32)
        loss = ctypes.c_float()
        self._check(load().tnqe_mlp_gradient(self.h, X.ctypes.data_as(ctypes.c_void_p),
                                             T.ctypes.data_as(ctypes.c_void_p),
                                             None if wp is None else wp.ctypes.data_as(ctypes.c_void_p),
                                             X.shape[0], ctypes.byref(loss), g.ctypes.data_as(ctypes.c_void_p)))
        return float(loss.value), g

    def adam_step(self, X, T, w=None, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8) -> float:
        X, T = _f32(X), _f32(T)
        wp = None if w is None else _f32(w)
        loss = ctypes.c_float()
        self._check(load().tnqe_mlp_adam_step(self.h, X.ctypes.data_as(ctypes.c_void_p),
                                              T.ctypes.data_as(ctypes.c_void_p),
                                              None if wp is None else wp.ctypes.data_as(ctypes.c_void_p),
                                              X.shape[0], lr, beta1, beta2, eps, ctypes.byref(loss)))
        return float(loss.value)

    def last_launches(self) -> int:
        return int(load().tnqe_mlp_last_launches(self.h))

    def close(self):
        if self.h:
            load().tnqe_mlp_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
