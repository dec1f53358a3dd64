"""FP64 CPU oracle of the vdW lattice Boltzmann step (arXiv:1307.6703, Sec. II).

TEST INFRASTRUCTURE ONLY: the test suite, the smoke check and the benchmark's
CPU-baseline / reference leg are the only callers.  The CUDA product path never
imports this package, and this package imports nothing from the product.

The arithmetic lives in ``lb_oracle.c`` (plain C, FP64, no fused multiply-add);
this module builds it with gcc and exposes it through ctypes on numpy arrays.
Analysis helpers that are not part of the step (Maxwell construction,
observables) live in ``oracle.maxwell`` and ``oracle.analysis``.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lb_oracle.c")
_LIB = os.path.join(_HERE, "_build", "liblb_oracle.so")


def build(force: bool = False) -> str:
    """Compile lb_oracle.c into oracle/_build/liblb_oracle.so (gcc, OpenMP).

    ``-ffp-contract=off`` keeps every multiply and add separately rounded,
    which the documented evaluation order relies on (aarch64 gcc would fuse
    them by default).
    """
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c99", "-fPIC", "-shared", "-fopenmp",
           "-ffp-contract=off", "-fno-fast-math", "-Wall", "-Wno-unknown-pragmas",
           _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


class _Params(C.Structure):
    _fields_ = [("nx", C.c_int32), ("ny", C.c_int32), ("walls", C.c_int32),
                ("nthreads", C.c_int32),
                ("a", C.c_double), ("b", C.c_double), ("T", C.c_double),
                ("kappa", C.c_double), ("tau", C.c_double),
                ("A0", C.c_double), ("lam", C.c_double),
                ("u_bot", C.c_double), ("u_top", C.c_double),
                ("N", C.c_double), ("Q", C.c_double)]


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(build())
        dp = C.POINTER(C.c_double)
        _lib.orc_feq.argtypes = [C.c_double] * 4 + [dp]
        _lib.orc_forcing.argtypes = [C.c_double] * 9 + [dp]
        _lib.orc_pressure_diff.argtypes = [C.c_double] * 4
        _lib.orc_pressure_diff.restype = C.c_double
        _lib.orc_stencils.argtypes = [C.c_double, C.c_double, dp, dp, dp, dp]
        _lib.orc_wall.argtypes = [C.c_int, C.c_double, C.c_double, C.c_double,
                                  dp, dp, dp]
        _lib.orc_noise_field.argtypes = [C.c_int, C.c_int, C.c_uint64,
                                         C.c_double, C.c_double, dp]
        _lib.orc_init.argtypes = [C.POINTER(_Params), dp, dp, dp, dp]
        _lib.orc_step.argtypes = [C.POINTER(_Params), dp, C.c_int64]
        _lib.orc_step.restype = C.c_int
        _lib.orc_moments.argtypes = [C.POINTER(_Params), dp, dp, dp, dp, dp, dp]
        _lib.orc_moments.restype = C.c_int
        _lib.orc_round_sig.argtypes = [C.c_double, C.c_int, C.c_int]
        _lib.orc_round_sig.restype = C.c_double
        _lib.orc_quantize.argtypes = [C.c_int, C.c_int, C.c_double, C.c_size_t, dp, dp]
    return _lib


def _ptr(a: np.ndarray | None):
    if a is None:
        return None
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(C.POINTER(C.c_double))


@dataclass
class Params:
    """Physical and numerical parameters, lattice units (T0 = 1/3)."""
    nx: int
    ny: int
    walls: bool = True
    a: float = 9.0 / 49.0
    b: float = 2.0 / 21.0
    T: float = 0.9 * 4.0 / 7.0
    kappa: float = 0.0490
    tau: float = 1.0
    A0: float = 0.0
    lam: float = 0.0
    u_bot: float = 0.0
    u_top: float = 0.0
    N: float = 0.5
    Q: float = 1.0
    nthreads: int = field(default_factory=lambda: int(os.environ.get("ORACLE_THREADS", "0")))

    def c(self) -> _Params:
        return _Params(self.nx, self.ny, int(self.walls), int(self.nthreads),
                       self.a, self.b, self.T, self.kappa, self.tau, self.A0,
                       self.lam, self.u_bot, self.u_top, self.N, self.Q)


# ---------------------------------------------------------------- pieces

def feq(n: float, ux: float, uy: float, T: float) -> np.ndarray:
    out = np.zeros(9)
    lib().orc_feq(n, ux, uy, T, _ptr(out))
    return out


def forcing(tau, T, ux, uy, Fx, Fy, dnx, dny, divJ) -> np.ndarray:
    out = np.zeros(9)
    lib().orc_forcing(tau, T, ux, uy, Fx, Fy, dnx, dny, divJ, _ptr(out))
    return out


def pressure_diff(a, b, T, n) -> float:
    return lib().orc_pressure_diff(a, b, T, n)


def stencils(N: float, Q: float, phi9) -> tuple[float, float, float]:
    phi = np.ascontiguousarray(phi9, dtype=np.float64)
    dx, dy, lap = C.c_double(), C.c_double(), C.c_double()
    lib().orc_stencils(N, Q, _ptr(phi), C.byref(dx), C.byref(dy), C.byref(lap))
    return dx.value, dy.value, lap.value


def wall(top: bool, U: float, Fx: float, Fy: float, f9, g9):
    f = np.array(f9, dtype=np.float64)
    g = np.array(g9, dtype=np.float64)
    nh = C.c_double()
    lib().orc_wall(int(top), U, Fx, Fy, _ptr(f), _ptr(g), C.byref(nh))
    return f, nh.value


def noise_field(nx: int, ny: int, seed: int, rho_mean: float, amp: float) -> np.ndarray:
    out = np.zeros((ny, nx))
    lib().orc_noise_field(nx, ny, seed, rho_mean, amp, _ptr(out))
    return out


# 16-bit deviation storage formats: (significant bits, smallest exponent).
FORMATS = {"bf16": (8, -126), "fp16": (11, -14)}


def round_sig(x: float, fmt: str) -> float:
    """x rounded to the format's precision (nearest, ties to even)."""
    p, emin = FORMATS[fmt]
    return lib().orc_round_sig(float(x), p, emin)


def quantize(f: np.ndarray, fmt: str, rho_ref: float, want_unrounded: bool = False):
    """State f[9][...] after a store in the 16-bit deviation format (in place
    on a copy); optionally also the deviations before rounding."""
    p, emin = FORMATS[fmt]
    out = np.ascontiguousarray(f, dtype=np.float64).copy()
    S = out.size // 9
    dev = np.zeros((8,) + out.shape[1:]) if want_unrounded else None
    lib().orc_quantize(p, emin, float(rho_ref), S, _ptr(out), _ptr(dev))
    return (out, dev) if want_unrounded else out


def reference_pops(rho_ref: float) -> np.ndarray:
    """Reference populations r_i of the deviation format (FP32-rounded)."""
    r = np.zeros(9)
    r[1:5] = np.float32(rho_ref / 9.0)
    r[5:9] = np.float32(rho_ref / 36.0)
    return r


# ---------------------------------------------------------------- solver

class Oracle:
    """State holder: post-collision populations f*[9][ny][nx] (FP64)."""

    def __init__(self, p: Params):
        self.p = p
        self._cp = p.c()
        self.f = np.zeros((9, p.ny, p.nx))
        self.t = 0

    def init_fields(self, n0, ux0=None, uy0=None):
        n0 = np.ascontiguousarray(n0, dtype=np.float64).reshape(self.p.ny, self.p.nx)
        ux0 = None if ux0 is None else np.ascontiguousarray(ux0, dtype=np.float64)
        uy0 = None if uy0 is None else np.ascontiguousarray(uy0, dtype=np.float64)
        lib().orc_init(C.byref(self._cp), _ptr(n0), _ptr(ux0), _ptr(uy0), _ptr(self.f))
        self.t = 0
        return self

    def init_noise(self, seed: int, rho_mean: float, amp: float):
        return self.init_fields(noise_field(self.p.nx, self.p.ny, seed, rho_mean, amp))

    def set_state(self, f):
        self.f = np.ascontiguousarray(f, dtype=np.float64).reshape(9, self.p.ny, self.p.nx).copy()
        return self

    def step(self, nsteps: int = 1, storage: tuple[str, float] | None = None):
        """Advance nsteps.  With storage = (fmt, rho_ref) every stored state
        (after each step) goes through the 16-bit deviation format."""
        if storage is None:
            rc = lib().orc_step(C.byref(self._cp), _ptr(self.f), int(nsteps))
            if rc != 0:
                raise RuntimeError("oracle step failed (bad parameters or out of memory)")
        else:
            for _ in range(int(nsteps)):
                if lib().orc_step(C.byref(self._cp), _ptr(self.f), 1) != 0:
                    raise RuntimeError("oracle step failed (bad parameters or out of memory)")
                self.quantize(*storage)
        self.t += nsteps
        return self

    def quantize(self, fmt: str, rho_ref: float):
        """Pass the current state through the 16-bit deviation format."""
        self.f = quantize(self.f, fmt, rho_ref)
        return self

    def moments(self, forces: bool = False):
        ny, nx = self.p.ny, self.p.nx
        n, ux, uy = np.zeros((ny, nx)), np.zeros((ny, nx)), np.zeros((ny, nx))
        Fx = np.zeros((ny, nx)) if forces else None
        Fy = np.zeros((ny, nx)) if forces else None
        rc = lib().orc_moments(C.byref(self._cp), _ptr(self.f), _ptr(n), _ptr(ux),
                               _ptr(uy), _ptr(Fx), _ptr(Fy))
        if rc != 0:
            raise RuntimeError("oracle moments failed")
        return (n, ux, uy, Fx, Fy) if forces else (n, ux, uy)

    def mass(self) -> float:
        import math
        return math.fsum(self.f.ravel())
