"""ctypes binding of include/fno.h (argument marshalling only).

:class:`Fno` owns one network handle; every computation (features, forward,
loss, backward, Adam) runs in the CUDA library.  Device buffers are torch
tensors or raw device pointers.
"""
from __future__ import annotations

import ctypes as C

import numpy as np

from .lb import LBError, load_library


class fno_config(C.Structure):
    _fields_ = [("width", C.c_int32), ("hidden", C.c_int32), ("layers", C.c_int32),
                ("modes_x", C.c_int32), ("modes_y", C.c_int32), ("outputs", C.c_int32),
                ("batch_max", C.c_int32),
                ("nx_max", C.c_int32), ("ny_max", C.c_int32), ("gemm_bf16", C.c_int32),
                ("stream", C.c_void_p)]


_ready = False


def _lib():
    global _ready
    lib = load_library()
    if not _ready:
        P = C.c_void_p
        lib.fno_create.argtypes = [C.POINTER(fno_config), C.POINTER(P)]
        lib.fno_param_count.argtypes = [P]
        lib.fno_param_count.restype = C.c_int64
        for n in ("fno_set_params", "fno_get_params", "fno_get_grads"):
            getattr(lib, n).argtypes = [P, P]
        lib.fno_forward.argtypes = [P, C.c_int32, C.c_int32, C.c_int32, P, P]
        lib.fno_backward.argtypes = [P, P, C.POINTER(C.c_double)]
        lib.fno_adam.argtypes = [P, C.c_float, C.c_float, C.c_float, C.c_float, C.c_int32]
        lib.fno_fields.argtypes = [P, P, C.c_int32, C.c_int32, C.c_int32, C.POINTER(C.c_double), C.c_double, P]
        lib.fno_destroy.argtypes = [P]
        lib.fno_last_error.argtypes = [P]
        lib.fno_last_error.restype = C.c_char_p
        lib.fno_gemm_bf16.argtypes = [P, C.c_int32, C.c_int64, P, C.c_int32, C.c_int64, P, C.c_int64,
                                      C.c_int64, C.c_int64, C.c_int32, C.c_int32, C.c_int32, C.c_int32,
                                      C.c_float, P, P]
        lib.fno_gemm_bf16.restype = C.c_int
        for n in ("fno_create", "fno_set_params", "fno_get_params", "fno_get_grads", "fno_forward",
                  "fno_backward", "fno_adam", "fno_fields", "fno_destroy"):
            getattr(lib, n).restype = C.c_int
        _ready = True
    return lib


def _ptr(a):
    if a is None:
        return None
    if isinstance(a, int):
        return a
    if isinstance(a, np.ndarray):
        return a.ctypes.data
    return a.data_ptr()


def _check(rc, h):
    if rc != 0:
        s = _lib().fno_last_error(h)
        raise LBError(rc, s.decode() if s else "")


def fno_create(cfg: fno_config) -> int:
    h = C.c_void_p()
    _check(_lib().fno_create(C.byref(cfg), C.byref(h)), None)
    return h.value


class Fno:
    """Network handle: width, hidden, layers, modes and workspace bounds."""

    def __init__(self, *, width=32, hidden=64, layers=4, modes_x=16, modes_y=8, outputs=3,
                 batch_max=16, nx_max=512, ny_max=128, gemm_bf16=True, stream=None):
        self.cfg = fno_config(width, hidden, layers, modes_x, modes_y, outputs, batch_max, nx_max,
                              ny_max, int(bool(gemm_bf16)), stream)
        self.outputs = outputs
        self.h = fno_create(self.cfg)
        self.n_params = int(_lib().fno_param_count(self.h))
        self.t = 0

    def set_params(self, flat: np.ndarray):
        flat = np.ascontiguousarray(flat, dtype=np.float32)
        assert flat.size == self.n_params
        _check(_lib().fno_set_params(self.h, _ptr(flat)), self.h)
        return self

    def get_params(self) -> np.ndarray:
        out = np.empty(self.n_params, dtype=np.float32)
        _check(_lib().fno_get_params(self.h, _ptr(out)), self.h)
        return out

    def get_grads(self) -> np.ndarray:
        out = np.empty(self.n_params, dtype=np.float32)
        _check(_lib().fno_get_grads(self.h, _ptr(out)), self.h)
        return out

    def forward(self, params_dev, nx: int, ny: int, out) -> None:
        """params_dev: device float [B][4] (U_w, A0, lambda, T_r); out: device [B][outputs][ny][nx]."""
        B = params_dev.shape[0] if hasattr(params_dev, "shape") else 1
        _check(_lib().fno_forward(self.h, B, nx, ny, _ptr(params_dev), _ptr(out)), self.h)

    def backward(self, target, want_loss: bool = True):
        loss = C.c_double(0.0)
        _check(_lib().fno_backward(self.h, _ptr(target), C.byref(loss) if want_loss else None), self.h)
        return loss.value if want_loss else None

    def adam(self, lr: float, beta1: float = 0.9, beta2: float = 0.999, eps: float = 1e-8):
        self.t += 1
        _check(_lib().fno_adam(self.h, lr, beta1, beta2, eps, self.t), self.h)

    def fields(self, out, nx: int, ny: int, scales, rho_mean: float, fields) -> None:
        """Solver fields [B][3][ny][nx] (device float64) from the network
        output `out` (device [B][outputs][ny][nx]); see fno_fields."""
        fno_fields(self.h, out, out.shape[0], nx, ny, scales, rho_mean, fields)

    def close(self):
        if self.h:
            _lib().fno_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---------------------------------------------------- same-name wrappers

def fno_param_count(h) -> int:
    return int(_lib().fno_param_count(h))


def fno_set_params(h, host: np.ndarray):
    _check(_lib().fno_set_params(h, _ptr(np.ascontiguousarray(host, dtype=np.float32))), h)


def fno_get_params(h, host: np.ndarray):
    _check(_lib().fno_get_params(h, _ptr(host)), h)


def fno_get_grads(h, host: np.ndarray):
    _check(_lib().fno_get_grads(h, _ptr(host)), h)


def fno_forward(h, batch: int, nx: int, ny: int, params_dev, out):
    _check(_lib().fno_forward(h, batch, nx, ny, _ptr(params_dev), _ptr(out)), h)


def fno_backward(h, target) -> float:
    loss = C.c_double(0.0)
    _check(_lib().fno_backward(h, _ptr(target), C.byref(loss)), h)
    return loss.value


def fno_adam(h, lr: float, beta1: float, beta2: float, eps: float, t: int):
    _check(_lib().fno_adam(h, lr, beta1, beta2, eps, t), h)


def fno_fields(h, out, batch: int, nx: int, ny: int, scales, rho_mean: float, fields):
    sc = (C.c_double * 3)(*[float(v) for v in scales])
    _check(_lib().fno_fields(h, _ptr(out), batch, nx, ny, sc, rho_mean, _ptr(fields)), h)


def fno_destroy(h):
    return _lib().fno_destroy(h)


def fno_last_error(h) -> str:
    s = _lib().fno_last_error(h)
    return s.decode() if s else ""


def fno_gemm_bf16(X, ldx: int, sX: int, Y, ldy: int, sY: int, Cout, cm: int, cn: int, sC: int,
                  M: int, N: int, K: int, batch: int, beta: float, err, stream=None):
    """C[b](m, n) = sum_k X[b](m, k) Y[b](n, k) + beta C[b](m, n) on the
    tensor cores (BF16 operands, FP32 result); device buffers."""
    rc = _lib().fno_gemm_bf16(_ptr(X), ldx, sX, _ptr(Y), ldy, sY, _ptr(Cout), cm, cn, sC, M, N, K, batch,
                              beta, _ptr(err), stream)
    if rc != 0:
        raise LBError(rc, "fno_gemm_bf16: bad arguments or CUDA error")
