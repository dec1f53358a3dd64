"""Helpers shared by the GPU tests (no method arithmetic)."""
import numpy as np

import oracle
from paper_1307_6703_gb300 import Solver


def oracle_for(w, nthreads=0):
    return oracle.Oracle(oracle.Params(nthreads=nthreads, **w.physics()))


def solver_for(w, precision):
    return Solver(w.nx, w.ny, precision=precision, walls=w.walls, a=w.a, b=w.b, T=w.T,
                  kappa=w.kappa, tau=w.tau, A0=w.A0, lam=w.lam, u_bot=w.u_bot, u_top=w.u_top,
                  N=w.N, Q=w.Q)


def rel_err(a, b):
    return float(np.abs(np.asarray(a, np.float64) - b).max() / np.abs(b).max())


def dev16_solver(w, precision, rho_ref):
    return Solver(w.nx, w.ny, precision=precision, walls=w.walls, a=w.a, b=w.b, T=w.T,
                  kappa=w.kappa, tau=w.tau, A0=w.A0, lam=w.lam, u_bot=w.u_bot, u_top=w.u_top,
                  N=w.N, Q=w.Q, rho_ref=rho_ref)


def decode_dev(d, fmt):
    """Raw 16-bit deviation bits -> float64 values (exact)."""
    d = np.ascontiguousarray(d, dtype=np.uint16)
    if fmt == "bf16":
        return (d.astype(np.uint32) << 16).view(np.float32).astype(np.float64)
    return d.view(np.float16).astype(np.float64)


def decode_state(f0, d, fmt, rho_ref):
    """Stored 16-bit deviation state -> populations [9][ny][nx] in float64:
    f_0 as stored, f_i = r_i + d_i with the FP32-rounded references."""
    r = oracle.reference_pops(rho_ref)
    f = np.empty((9,) + f0.shape)
    f[0] = f0
    f[1:] = r[1:, None, None] + decode_dev(d, fmt)
    return f
