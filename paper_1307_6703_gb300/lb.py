"""ctypes binding of the C ABI in include/lb.h (argument marshalling only).

Every function here has the name of the C entry point it calls; the
:class:`Solver` convenience class only strings those calls together.  All
computation happens in the CUDA library; loading fails loudly when it is
missing or when no CUDA device is usable -- there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

LB_OK = 0
LB_ERR_ARG = -1
LB_ERR_CUDA = -2
LB_ERR_OOM = -3
LB_ERR_UNSTABLE = -4
LB_ERR_TIMEOUT = -5
LB_ERR_STATE = -6

LB_FP64 = 0
LB_FP32 = 1
LB_BF16DEV = 2
LB_FP16DEV = 3

LB_DTYPE_F64 = 0
LB_DTYPE_F32 = 1

_ERR_NAMES = {LB_ERR_ARG: "LB_ERR_ARG", LB_ERR_CUDA: "LB_ERR_CUDA", LB_ERR_OOM: "LB_ERR_OOM",
              LB_ERR_UNSTABLE: "LB_ERR_UNSTABLE", LB_ERR_TIMEOUT: "LB_ERR_TIMEOUT",
              LB_ERR_STATE: "LB_ERR_STATE"}

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "liblb.so")


class lb_params(C.Structure):
    _fields_ = [("nx", C.c_int32), ("ny", C.c_int32), ("walls", C.c_int32),
                ("precision", C.c_int32),
                ("a", C.c_double), ("b", C.c_double), ("T", C.c_double),
                ("kappa", C.c_double), ("tau", C.c_double),
                ("A0", C.c_double), ("lambda_", C.c_double),
                ("u_bot", C.c_double), ("u_top", C.c_double),
                ("N", C.c_double), ("Q", C.c_double), ("rho_ref", C.c_double),
                ("stream", C.c_void_p)]


class LBError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{_ERR_NAMES.get(code, code)}: {msg}")
        self.code = code


_lib = None


def load_library(path: str = LIB_PATH) -> C.CDLL:
    """Load liblb.so (built by paper_1307_6703_gb300.build); raises if absent."""
    global _lib
    if _lib is None:
        if not os.path.exists(path):
            raise FileNotFoundError(
                f"CUDA library not built: {path} (run __graft_entry__.build())")
        lib = C.CDLL(path)
        P = C.c_void_p
        lib.lb_create.argtypes = [C.POINTER(lb_params), C.POINTER(P)]
        lib.lb_init.argtypes = [P, C.c_int, C.c_uint64, C.c_double, C.c_double, P, P, P]
        lib.lb_step.argtypes = [P, C.c_int64]
        lib.lb_moments.argtypes = [P, P, P, P, C.c_int, C.c_int]
        lib.lb_reduce.argtypes = [P, C.POINTER(C.c_double)]
        lib.lb_reduce_async.argtypes = [P, P]
        lib.lb_monitor.argtypes = [P, P, C.c_int32]
        lib.lb_get_state.argtypes = [P, P, C.POINTER(C.c_size_t)]
        lib.lb_set_state.argtypes = [P, P, C.c_size_t, C.c_int64]
        lib.lb_get_step.argtypes = [P, C.POINTER(C.c_int64)]
        lib.lb_destroy.argtypes = [P]
        lib.lb_last_error.argtypes = [P]
        lib.lb_last_error.restype = C.c_char_p
        lib.lb_reduce_noalloc.argtypes = [P, C.c_int, C.c_int32, C.c_int32, C.c_double, P, P, P]
        lib.lb_autotune.argtypes = [P, C.c_int, C.POINTER(C.c_int32)]
        lib.lb_set_seg_h.argtypes = [P, C.c_int32]
        lib.lb_get_tiling.argtypes = [P, C.POINTER(C.c_int32), C.POINTER(C.c_int32)]
        lib.lb_set_tiling.argtypes = [P, C.c_int32, C.c_int32]
        lib.lb_sweep_dependencies.argtypes = [C.c_int32, C.c_int32, C.c_int32, C.c_int32, C.c_int32, C.c_int32,
                                              P, P, C.c_int64, C.POINTER(C.c_int64)]
        lib.lb_batch_create.argtypes = [C.POINTER(lb_params), C.c_int32, C.POINTER(P)]
        lib.lb_batch_handle.argtypes = [P, C.c_int32]
        lib.lb_batch_handle.restype = P
        lib.lb_batch_step.argtypes = [P, C.c_int64]
        lib.lb_batch_autotune.argtypes = [P, C.c_int, C.POINTER(C.c_int32)]
        lib.lb_batch_destroy.argtypes = [P]
        lib.lb_batch_last_error.argtypes = [P]
        lib.lb_batch_last_error.restype = C.c_char_p
        for name in ("lb_create", "lb_init", "lb_step", "lb_moments", "lb_reduce",
                     "lb_get_state", "lb_set_state", "lb_get_step", "lb_destroy",
                     "lb_reduce_noalloc", "lb_autotune", "lb_get_tiling", "lb_set_tiling", "lb_sweep_dependencies",
                     "lb_batch_create", "lb_batch_step",
                     "lb_batch_autotune", "lb_batch_destroy"):
            getattr(lib, name).restype = C.c_int
        _lib = lib
    return _lib


def _check(rc: int, h) -> int:
    if rc != LB_OK:
        raise LBError(rc, lb_last_error(h))
    return rc


def _addr(a) -> int | None:
    """Address of a numpy array, a torch tensor, or a raw integer pointer."""
    if a is None:
        return None
    if isinstance(a, int):
        return a
    if isinstance(a, np.ndarray):
        return a.ctypes.data
    if hasattr(a, "data_ptr"):
        return a.data_ptr()
    raise TypeError(f"cannot take the address of {type(a)}")


# ------------------------------------------------------- same-name wrappers

def lb_create(p: lb_params) -> int:
    h = C.c_void_p()
    _check(load_library().lb_create(C.byref(p), C.byref(h)), None)
    return h.value


def lb_init(h, mode: int, seed: int = 0, rho_mean: float = 0.0, noise_amp: float = 0.0,
            rho0=None, ux0=None, uy0=None) -> int:
    for a in (rho0, ux0, uy0):
        if isinstance(a, np.ndarray):
            assert a.dtype == np.float64 and a.flags.c_contiguous
        elif hasattr(a, "data_ptr"):
            assert str(a.dtype) == "torch.float64" and a.is_contiguous()
    return _check(load_library().lb_init(h, mode, seed, rho_mean, noise_amp, _addr(rho0),
                                         _addr(ux0), _addr(uy0)), h)


def lb_step(h, nsteps: int) -> int:
    return _check(load_library().lb_step(h, nsteps), h)


def lb_moments(h, rho, ux, uy, dtype: int, on_device: int) -> int:
    return _check(load_library().lb_moments(h, _addr(rho), _addr(ux), _addr(uy), dtype,
                                            on_device), h)


def lb_reduce(h, out=None):
    """Returns (rc, [mass, momx, momy]); LB_ERR_UNSTABLE is returned, not raised."""
    buf = (C.c_double * 3)()
    rc = load_library().lb_reduce(h, buf)
    if rc not in (LB_OK, LB_ERR_UNSTABLE):
        _check(rc, h)
    vals = [buf[0], buf[1], buf[2]]
    if out is not None:
        out[:] = vals
    return rc, vals


def lb_reduce_async(h, out) -> None:
    """Enqueue the sums of lb_reduce and their copy into `out`, five HOST
    doubles (mass, momx, momy, unstable flag, wait/layout error flag) --
    a pinned torch tensor or a numpy array; valid after a stream sync."""
    _check(load_library().lb_reduce_async(h, _addr(out)), h)


def lb_monitor(h, ring=None, capacity: int = 0) -> None:
    """Register `ring` (page-locked HOST memory of capacity x 6 doubles, e.g.
    a pinned torch tensor) for per-step records written by the step kernel:
    (mass, momx, momy, unstable flag, wait/layout error flag, step); None
    switches monitoring off."""
    if ring is not None and capacity == 0:
        capacity = int(ring.numel() if hasattr(ring, "numel") else ring.size) // 6
    _check(load_library().lb_monitor(h, _addr(ring), capacity if ring is not None else 0), h)


def lb_get_state(h, buf=None) -> int:
    n = C.c_size_t(0 if buf is None else buf.nbytes)
    _check(load_library().lb_get_state(h, _addr(buf), C.byref(n)), h)
    return n.value


def lb_set_state(h, buf, step: int = 0) -> int:
    return _check(load_library().lb_set_state(h, _addr(buf), buf.nbytes, step), h)


def lb_get_step(h) -> int:
    t = C.c_int64()
    _check(load_library().lb_get_step(h, C.byref(t)), h)
    return t.value


def lb_destroy(h) -> int:
    return load_library().lb_destroy(h)


def lb_reduce_noalloc(f, precision: int, nx: int, ny: int, b: float, out, flag=None,
                      stream=None) -> int:
    """Allocation-free reduction over a caller-owned DEVICE population buffer;
    `out` (3 doubles) and `flag` (1 int) are DEVICE buffers.  Asynchronous."""
    rc = load_library().lb_reduce_noalloc(_addr(f), precision, nx, ny, b, _addr(out),
                                          _addr(flag), stream)
    if rc != LB_OK:
        raise LBError(rc, "lb_reduce_noalloc failed")
    return rc


def lb_autotune(h, steps: int = 20) -> int:
    """Returns the chosen segment height (0: tile kernel, nothing to tune)."""
    seg = C.c_int32(0)
    _check(load_library().lb_autotune(h, steps, C.byref(seg)), h)
    return seg.value


def lb_set_seg_h(h, seg_h: int) -> None:
    """Fix the sweep kernel's segment height (rows per CTA) without tuning."""
    _check(load_library().lb_set_seg_h(h, seg_h), h)


def lb_get_tiling(h) -> tuple[int, int]:
    """(strip count, segment height) of the sweep kernel's tiling."""
    ns, sh = C.c_int32(0), C.c_int32(0)
    _check(load_library().lb_get_tiling(h, C.byref(ns), C.byref(sh)), h)
    return ns.value, sh.value


def lb_set_tiling(h, nstrips: int, seg_h: int) -> None:
    """Fix the sweep kernel's strip count and segment height without tuning."""
    _check(load_library().lb_set_tiling(h, nstrips, seg_h), h)


def lb_sweep_dependencies(precision: int, nx: int, ny: int, walls: int, nstrips: int, seg_h: int):
    """(ofs, idx): the multi-step sweep's dependency lists in CSR form, tile
    t = strip + nstrips * segment waiting for idx[ofs[t]:ofs[t + 1]] (host
    computation; no GPU needed)."""
    lib = load_library()
    nseg = -(-ny // min(seg_h, ny)) if seg_h >= 1 else 1
    ofs = np.zeros(max(nstrips, 0) * nseg + 1, dtype=np.int32)
    count = C.c_int64(0)
    rc = lib.lb_sweep_dependencies(precision, nx, ny, walls, nstrips, seg_h, ofs.ctypes.data, None, 0,
                                   C.byref(count))
    if rc != LB_OK and count.value == 0:
        raise LBError(rc, "lb_sweep_dependencies: lattice or tiling not taken by the sweep")
    idx = np.zeros(count.value, dtype=np.int32)
    rc = lib.lb_sweep_dependencies(precision, nx, ny, walls, nstrips, seg_h, ofs.ctypes.data, idx.ctypes.data,
                                   count.value, C.byref(count))
    if rc != LB_OK:
        raise LBError(rc, "lb_sweep_dependencies failed")
    return ofs, idx


def _bcheck(rc: int, b) -> int:
    if rc != LB_OK:
        s = load_library().lb_batch_last_error(b)
        raise LBError(rc, s.decode() if s else "")
    return rc


def lb_batch_create(ps) -> int:
    arr = (lb_params * len(ps))(*ps)
    b = C.c_void_p()
    _bcheck(load_library().lb_batch_create(arr, len(ps), C.byref(b)), None)
    return b.value


def lb_batch_handle(b, i: int) -> int:
    h = load_library().lb_batch_handle(b, i)
    if not h:
        raise LBError(LB_ERR_ARG, f"lb_batch_handle: no instance {i}")
    return h


def lb_batch_step(b, nsteps: int) -> int:
    return _bcheck(load_library().lb_batch_step(b, nsteps), b)


def lb_batch_autotune(b, steps: int, count: int) -> list[int]:
    seg = (C.c_int32 * count)()
    _bcheck(load_library().lb_batch_autotune(b, steps, seg), b)
    return list(seg)


def lb_batch_destroy(b) -> int:
    return load_library().lb_batch_destroy(b)


def lb_batch_last_error(b) -> str:
    s = load_library().lb_batch_last_error(b)
    return s.decode() if s else ""


def lb_last_error(h) -> str:
    s = load_library().lb_last_error(h)
    return s.decode() if s else ""


# ------------------------------------------------------------ convenience

class Solver:
    """Owns one lb_handle.  Arguments are lattice-unit parameters as in lb.h."""

    def __init__(self, nx: int, ny: int, *, walls: bool = True, precision: int = LB_FP32,
                 a: float, b: float, T: float, kappa: float, tau: float,
                 A0: float = 0.0, lam: float = 0.0, u_bot: float = 0.0, u_top: float = 0.0,
                 N: float = 0.5, Q: float = 1.0, rho_ref: float = 0.0, stream: int | None = None):
        self.nx, self.ny, self.precision = nx, ny, precision
        self.params = lb_params(nx, ny, int(walls), precision, a, b, T, kappa, tau, A0, lam,
                                u_bot, u_top, N, Q, rho_ref, stream)
        self.h = lb_create(self.params)
        self.dtype = np.float64 if precision == LB_FP64 else np.float32
        self.dev16 = precision in (LB_BF16DEV, LB_FP16DEV)

    def init_noise(self, seed: int, rho_mean: float, amp: float):
        lb_init(self.h, 0, seed, rho_mean, amp)
        return self

    def init_fields(self, rho0, ux0=None, uy0=None):
        """Host arrays (converted to contiguous float64) or contiguous
        float64 device tensors, which lb_init reads in place."""
        def c(a):
            if a is None or hasattr(a, "data_ptr"):
                return a
            return np.ascontiguousarray(a, dtype=np.float64)
        lb_init(self.h, 1, 0, 0.0, 0.0, c(rho0), c(ux0), c(uy0))
        return self

    def step(self, nsteps: int = 1):
        lb_step(self.h, nsteps)
        return self

    def moments(self, dtype=np.float64):
        shape = (self.ny, self.nx)
        n, u, v = (np.empty(shape, dtype=dtype) for _ in range(3))
        code = LB_DTYPE_F64 if dtype == np.float64 else LB_DTYPE_F32
        lb_moments(self.h, n, u, v, code, 0)
        return n, u, v

    def reduce(self):
        return lb_reduce(self.h)

    def autotune(self, steps: int = 20) -> int:
        return lb_autotune(self.h, steps)

    def set_seg_h(self, seg_h: int):
        lb_set_seg_h(self.h, seg_h)
        return self

    def monitor(self, ring=None, capacity: int = 0):
        lb_monitor(self.h, ring, capacity)
        return self

    def get_state(self):
        """[9][ny][nx] populations; for 16-bit storage the pair (rest plane
        float32 [ny][nx], raw deviation bits uint16 [8][ny][nx])."""
        if self.dev16:
            S = self.nx * self.ny
            buf = np.empty(S * 20, dtype=np.uint8)
            lb_get_state(self.h, buf)
            f0 = buf[:4 * S].view(np.float32).reshape(self.ny, self.nx).copy()
            d = buf[4 * S:].view(np.uint16).reshape(8, self.ny, self.nx).copy()
            return f0, d
        buf = np.empty((9, self.ny, self.nx), dtype=self.dtype)
        lb_get_state(self.h, buf)
        return buf

    def set_state(self, f, step: int = 0):
        if self.dev16:
            f0, d = f
            buf = np.concatenate([np.ascontiguousarray(f0, dtype=np.float32).view(np.uint8).ravel(),
                                  np.ascontiguousarray(d, dtype=np.uint16).view(np.uint8).ravel()])
            lb_set_state(self.h, buf, step)
            return self
        lb_set_state(self.h, np.ascontiguousarray(f, dtype=self.dtype), step)
        return self

    @property
    def t(self) -> int:
        return lb_get_step(self.h)

    def close(self):
        if self.h:
            lb_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """Owns one lb_batch: many independent lattices stepped together.
    ``batch[i]`` is a :class:`Solver`-like view of instance i (same methods,
    no ownership)."""

    def __init__(self, params: list, stream: int | None = None):
        ps = []
        for p in params:
            q = lb_params()
            C.memmove(C.byref(q), C.byref(p), C.sizeof(lb_params))
            q.stream = stream
            ps.append(q)
        self.params = ps
        self.b = lb_batch_create(ps)
        self.views = [_View(self, i) for i in range(len(ps))]

    def __len__(self):
        return len(self.views)

    def __getitem__(self, i):
        return self.views[i]

    def step(self, nsteps: int = 1):
        lb_batch_step(self.b, nsteps)
        return self

    def autotune(self, steps: int = 10) -> list[int]:
        return lb_batch_autotune(self.b, steps, len(self.views))

    def close(self):
        if self.b:
            lb_batch_destroy(self.b)
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class _View(Solver):
    """Instance i of a Batch (the batch owns the handle)."""

    def __init__(self, batch: Batch, i: int):  # noqa: super().__init__ is not called
        p = batch.params[i]
        self.nx, self.ny, self.precision = p.nx, p.ny, p.precision
        self.params = p
        self._batch, self._i = batch, i
        self.dtype = np.float64 if p.precision == LB_FP64 else np.float32
        self.dev16 = p.precision in (LB_BF16DEV, LB_FP16DEV)

    @property
    def h(self):
        return lb_batch_handle(self._batch.b, self._i)

    def close(self):
        pass

    def __del__(self):
        pass
