"""The paper's physical regimes for the batched solver, and the observables
the paper reports for them.

This module states parameter sets (lattice units, see ``workloads``) and
measures solver output; it holds no arithmetic of the scheme itself.

* ``table1_cases``: droplets for the stencil scan of Table 1 (Sec. III):
  one droplet of radius 15 on 64 x 64 per temperature and (N, Q).
* ``couette_two_layer``: the sheared two-layer state of Sec. IV (liquid
  below a flat interface, vapour above, walls at -U_w / +U_w), whose
  x-averaged velocity is a broken line; ``broken_line_slopes`` fits it and
  ``broken_line_prediction`` gives the slopes that a uniform shear stress
  n nu du/dy across two bulk phases implies (the paper's formula, here for
  an interface at any height).
* ``table2_rows``: the 30 rows of Table 2 (interface-wave amplitudes), with
  the paper's units mapped to lattice units; ``interface_stats`` measures
  the liquid-vapour interfaces of a density field (how many cross each
  column, their amplitude A / L_y) and ``dominant_phase`` the phase of the
  interface profile's dominant x-mode, whose drift gives the wave speed.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from .workloads import TC

# The paper's vdW set in lattice units (a = 3/8, b = 1/3, kappa = 0.1 is its
# kappa = 0.3: kappa and T scale by 1/3, Sec. III with dt = 1).
A_VDW, B_VDW, KAPPA_LU = 3.0 / 8.0, 1.0 / 3.0, 0.1

# Table 1, OVC column: (N, Q) by reduced temperature.
TABLE1_OVC = {0.83: (0.3, 2.1), 0.85: (0.3, 2.3), 0.87: (0.3, 2.5), 0.89: (0.3, 2.6), 0.91: (0.3, 2.5),
              0.93: (0.3, 1.9), 0.95: (0.3, 2.0), 0.97: (0.3, 0.0), 0.98: (0.3, 3.9), 0.99: (0.5, 2.1)}
# Table 1, ODC column.
TABLE1_ODC = {0.83: (0.3, 2.1), 0.85: (0.3, 2.3), 0.87: (0.3, 2.5), 0.89: (0.3, 2.7), 0.91: (0.4, 1.7),
              0.93: (0.4, 1.9), 0.95: (0.4, 2.1), 0.97: (0.0, 0.0), 0.98: (0.3, 3.9), 0.99: (1.0, 1.0)}


@dataclass(frozen=True)
class Case:
    """One lattice of a batch: its parameters (lattice units) and a label."""
    label: str
    nx: int
    ny: int
    walls: bool
    T: float
    tau: float
    A0: float
    lam: float
    u_w: float
    N: float
    Q: float
    kappa: float = KAPPA_LU

    def lb_params(self, precision: int):
        from .lb import lb_params
        return lb_params(self.nx, self.ny, 1 if self.walls else 0, precision, A_VDW, B_VDW, self.T,
                         self.kappa, self.tau, self.A0, self.lam, -self.u_w, self.u_w, self.N, self.Q,
                         0.0, None)


# ------------------------------------------------------------------ Table 1
def table1_cases(reduced_T, Ns, Qs, L: int = 64) -> list[Case]:
    """Periodic L x L droplets, one per (T_r, N, Q)."""
    return [Case(f"T{tr}_N{N}_Q{Q}", L, L, False, tr * TC, 1.0, 0.0, 0.0, 0.0, N, Q)
            for tr in reduced_T for N in Ns for Q in Qs]


def droplet_errors(n, ux, uy, nL, nV):
    """Largest spurious speed, and the relative density error of the
    droplet's centre and the far corner against the coexistence densities."""
    L = n.shape[0]
    return (float(np.hypot(ux, uy).max()),
            float(abs(n[L // 2, L // 2] - nL) / nL + abs(n[0, 0] - nV) / nV))


# ------------------------------------------------------- broken-line profile
def couette_two_layer(ly: int, u_w: float, lx: int = 32, reduced_T: float = 0.95) -> Case:
    """Walls at -u_w (bottom) and +u_w (top); A0 = 0; OVC stencil."""
    N, Q = TABLE1_OVC[reduced_T]
    return Case(f"couette_{lx}x{ly}_u{u_w:g}", lx, ly, True, reduced_T * TC, 1.0, 0.0, 0.0, u_w, N, Q)


def two_layer_field(lx: int, ly: int, nL: float, nV: float, width: float = 3.0) -> np.ndarray:
    """Liquid below row ly/2, vapour above (tanh interface)."""
    y = np.arange(ly)[:, None] * np.ones((1, lx))
    return nV + (nL - nV) * 0.5 * (1.0 - np.tanh((y - ly / 2 + 0.5) / width))


def broken_line_slopes(n, ux, lo=(0.15, 0.38), hi=(0.62, 0.85)):
    """x-averaged profiles; least-squares slopes of <u_x>_x(y) in the lower
    and upper bulk (row fractions lo, hi), the mean densities there and the
    interface height (where <n>_x crosses the mid density, interpolated)."""
    ly = n.shape[0]
    u, nn = ux.mean(axis=1), n.mean(axis=1)
    y = np.arange(ly, dtype=float)
    a, b = slice(int(lo[0] * ly), int(lo[1] * ly)), slice(int(hi[0] * ly), int(hi[1] * ly))
    s_lo, s_hi = np.polyfit(y[a], u[a], 1)[0], np.polyfit(y[b], u[b], 1)[0]
    n_lo, n_hi = float(nn[a].mean()), float(nn[b].mean())
    mid = 0.5 * (n_lo + n_hi)
    k = int(np.where(np.diff(np.sign(nn - mid)) != 0)[0][0])
    y_i = k + (nn[k] - mid) / (nn[k] - nn[k + 1])
    return float(s_lo), float(s_hi), n_lo, n_hi, float(y_i)


def broken_line_prediction(u_w: float, ly: int, n_lo: float, n_hi: float, y_i: float):
    """Slopes of the two linear segments when the shear stress n nu du/dy
    is the same in both bulk phases (equal kinematic viscosity) and the
    velocity goes from -u_w on row 0 to +u_w on row ly - 1 without slip:
    s_lo h_lo + s_hi h_hi = 2 u_w and n_lo s_lo = n_hi s_hi, with h_lo = y_i
    and h_hi = ly - 1 - y_i.  For y_i = ly / 2 this is the paper's
    2 gamma n_u / (n_u + n_l) and 2 gamma n_l / (n_u + n_l), gamma = 2 u_w / L_y."""
    h_lo, h_hi = y_i, ly - 1 - y_i
    s_lo = 2.0 * u_w / (h_lo + h_hi * n_lo / n_hi)
    return s_lo, s_lo * n_lo / n_hi


# ------------------------------------------------------------------ Table 2
def table2_rows() -> list[dict]:
    """The rows of Table 2: T_r, lambda, tau, gamma (per step), A0, the
    paper's kappa, L_x x L_y, and the paper's A / L_y."""
    rows = []

    def add(tr, lams, tau, a0, kap, lxs, amps):
        for lx, amp in zip(lxs, amps):
            for lam in lams:
                rows.append(dict(T_r=tr, lam=lam, tau=tau, gamma=1e-3, A0=a0, kappa_paper=kap, lx=lx, ly=256,
                                 amp_paper=amp))
    add(0.95, (32, 64), 1, 1e-4, 0.3, (256, 512, 1024, 2048), (0.172, 0.316, 0.409, 0.417))
    add(0.95, (32, 64), 1, 1e-5, 0.3, (256, 512, 1024), (0.178, 0.335, 0.504))
    add(0.95, (32,), 1, 1e-4, 0.2, (256,), (0.172,))
    add(0.95, (32,), 1, 1e-4, 0.5, (256,), (0.172,))
    add(0.95, (32, 64), 2, 1e-4, 0.3, (256, 512), (0.112, 0.219))
    rows.append(dict(T_r=0.95, lam=32, tau=3, gamma=1e-3, A0=1e-4, kappa_paper=0.3, lx=256, ly=256, amp_paper=0.00782))
    rows.append(dict(T_r=0.95, lam=64, tau=3, gamma=1e-3, A0=1e-4, kappa_paper=0.3, lx=256, ly=256, amp_paper=0.0234))
    add(0.95, (32, 64), 3, 1e-4, 0.3, (512,), (0.166,))
    add(0.91, (32, 64), 1, 1e-4, 0.3, (256, 512, 1024), (0.255, 0.397, 0.496))
    return rows


def table2_case(row: dict) -> Case:
    """A Table 2 row in lattice units: walls at -/+ gamma L_y / 2 (the
    paper's gamma is per time step), kappa / 3, the row's Table 1 OVC
    stencil."""
    N, Q = TABLE1_OVC[row["T_r"]]
    u_w = row["gamma"] * row["ly"] / 2.0
    return Case(f"t2_T{row['T_r']}_l{row['lam']}_tau{row['tau']}_A{row['A0']:g}_k{row['kappa_paper']}_{row['lx']}",
                row["lx"], row["ly"], True, row["T_r"] * TC, float(row["tau"]), row["A0"], float(row["lam"]),
                u_w, N, Q, kappa=row["kappa_paper"] / 3.0)


def interface_stats(n: np.ndarray) -> dict:
    """Interfaces of a density field [ny][nx]: sites denser than the mid
    density are liquid; per column the number of liquid/vapour crossings
    along y (median over columns), the liquid height h(x) (liquid sites per
    column) and its range as the amplitude A / L_y."""
    mid = 0.5 * (float(n.max()) + float(n.min()))
    liq = n > mid
    cross = np.abs(np.diff(liq.astype(np.int8), axis=0)).sum(axis=0)
    h = liq.sum(axis=0).astype(float)
    return dict(crossings=int(np.median(cross)), amp=float((h.max() - h.min()) / n.shape[0]),
                liquid_fraction=float(liq.mean()), height=h)


def dominant_phase(h: np.ndarray, k: int | None = None):
    """(k, phase) of the dominant non-zero Fourier mode of a profile h(x)
    (or of mode k); the phase drift over time gives the wave speed
    -dphi/dt / (2 pi k / L_x)."""
    sp = np.fft.rfft(h - h.mean())
    if k is None:
        k = int(np.argmax(np.abs(sp[1:])) + 1)
    return k, float(np.angle(sp[k]))


def wave_speed(phases, dt: float, k: int, lx: int) -> float:
    """Speed (sites per step) of a mode-k wave from its phases sampled every
    dt steps (unwrapped least-squares drift)."""
    ph = np.unwrap(np.asarray(phases, dtype=float))
    slope = np.polyfit(np.arange(len(ph)) * dt, ph, 1)[0]
    return float(-slope / (2.0 * np.pi * k / lx))
