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
