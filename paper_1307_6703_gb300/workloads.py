"""Synthetic workloads: parameter sets and seeded initial fields.

This module holds no arithmetic of the method; it only states the problems
(lattice-unit parameters) and draws seeded inputs.  Tests, the benchmark and
the smoke check use it for both the CUDA path and the oracle.

Parameter set.  The paper's van der Waals fluid in lattice units (dx = dt = 1,
T0 = 1/3): a = 3/8, b = 1/3 (critical point n_c = 1, T_c = 1/3),
kappa = 0.1 (the paper's 0.3), tau = 1, isotropic stencils from Table 1
(OVC column).  The lattice sizes, wall speeds and potential wavelengths are
those of the workloads below; temperatures and force amplitudes are the
paper's own (Sec. IV: T = 0.95 T_c, A0 = 1e-4) where larger values make the
scheme blow up from a noisy symmetric quench.
"""
from __future__ import annotations

from dataclasses import asdict, dataclass, replace

import numpy as np

TC = 1.0 / 3.0  # critical temperature of the paper's set in lattice units


@dataclass(frozen=True)
class Workload:
    name: str
    nx: int
    ny: int
    walls: bool
    T: float
    tau: float
    A0: float
    lam: float
    u_bot: float
    u_top: float
    N: float
    Q: float
    steps: int
    a: float = 3.0 / 8.0
    b: float = 1.0 / 3.0
    kappa: float = 0.1
    rho_mean: float = 1.0          # n_c
    noise: float = 0.01 / 3.5      # +-1 % of n_c... scaled from +-0.01 at rho_c = 3.5
    seed: int = 1

    def physics(self) -> dict:
        d = asdict(self)
        for k in ("name", "steps", "rho_mean", "noise", "seed"):
            d.pop(k)
        return d

    def with_(self, **kw) -> "Workload":
        return replace(self, **kw)


# Plain FP64 step, 64x32, static walls, T = 0.9 T_c, tau = 1, lambda = 32,
# A0 = 1e-3 (the paper's largest amplitude; 0.05 diverges), 2000 steps.
C1 = Workload("fp64_64x32_static_walls", 64, 32, True, 0.9 * TC, 1.0, 1e-3, 32.0, 0.0, 0.0,
              0.3, 2.6, 2000)

# Sheared zebra phase, FP32, 512x256, walls at -U_w / +U_w, lambda = 128,
# T = 0.95 T_c, tau = 1, A0 = 1e-4, 1000 steps.
def C2(u_w: float) -> Workload:
    return Workload(f"fp32_512x256_shear_{u_w:g}", 512, 256, True, 0.95 * TC, 1.0, 1e-4, 128.0,
                    -u_w, u_w, 0.3, 2.0, 1000)


# Headline lattice: 4096x1024, walls at -0.05 / +0.05, lambda = 512,
# T = 0.95 T_c, tau = 1, A0 = 1e-4.
C4 = Workload("fp32_4096x1024_shear_0.05", 4096, 1024, True, 0.95 * TC, 1.0, 1e-4, 512.0,
              -0.05, 0.05, 0.3, 2.0, 1000)


def noise_field(w: Workload, seed: int | None = None) -> np.ndarray:
    """Seeded noisy-uniform density rho_mean + noise * U(-1, 1), [ny][nx]."""
    rng = np.random.default_rng(w.seed if seed is None else seed)
    return w.rho_mean + w.noise * rng.uniform(-1.0, 1.0, size=(w.ny, w.nx))


def droplet_field(nx: int, ny: int, radius: float, n_in: float, n_out: float,
                  width: float = 3.0) -> np.ndarray:
    """Smooth disc of density n_in in a background n_out (tanh edge)."""
    yy, xx = np.mgrid[0:ny, 0:nx]
    r = np.hypot(xx - nx / 2 + 0.5, yy - ny / 2 + 0.5)
    return n_out + (n_in - n_out) * 0.5 * (1.0 - np.tanh((r - radius) / width))


def slab_field(nx: int, ny: int, n_in: float, n_out: float, width: float = 3.0) -> np.ndarray:
    """Liquid slab in the middle half of the rows (two flat interfaces)."""
    y = np.arange(ny)[:, None] * np.ones((1, nx))
    return n_out + (n_in - n_out) * 0.5 * (np.tanh((y - ny / 4) / width) - np.tanh((y - 3 * ny / 4) / width))


# Stencil parameters (N, Q) of Table 1 (OVC column) at the tabulated reduced
# temperatures used here.
_TABLE1_NQ = {0.85: (0.3, 2.3), 0.90: (0.3, 2.6), 0.95: (0.3, 2.0)}


def batch_workloads(count: int = 64, seed: int = 7) -> list[Workload]:
    """Seeded ensemble of independent sheared lattices for the batched
    solver: nx uniform over multiples of 32 in [128, 1024], ny over multiples
    of 16 in [64, 256]; wall speed U_w ~ U[0, 0.1] (walls at -U_w, +U_w);
    A0 ~ U[1e-4, 5e-4] (inside the paper's range); lambda 32 or 64 (the
    paper's wavelengths); T_r ~ U[0.92, 0.96] with (N, Q) of the nearest
    Table 1 row; tau = 1.  About 5.9 M sites for 64 lattices.  The oracle
    blows up from the noisy quench below T_r ~ 0.9 with the Table 1 stencils
    (Q >= 2) within a few hundred steps, with lambda of several hundred sites
    at A0 >= 2e-4 within ~1000 steps, and at lambda = 128, A0 ~ 8e-4 within
    ~1500 steps; inside this range it runs 4000 steps at the extremes."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        nx = 32 * int(rng.integers(4, 33))
        ny = 16 * int(rng.integers(4, 17))
        uw = float(rng.uniform(0.0, 0.1))
        a0 = float(rng.uniform(1e-4, 5e-4))
        lam = float((32, 64)[int(rng.integers(0, 2))])
        tr = float(rng.uniform(0.92, 0.96))
        nq = _TABLE1_NQ[min(_TABLE1_NQ, key=lambda t: abs(t - tr))]
        out.append(Workload(f"batch{i}_{nx}x{ny}", nx, ny, True, tr * TC, 1.0, a0, lam, -uw, uw,
                            nq[0], nq[1], 1000, seed=seed * 1000 + i))
    return out


# Warm-start network: seeded initial weights (random draws only; the network
# itself is defined in include/fno.h).  Both the CUDA network and its CPU
# reference are given these values.
N_FEATURES = 5


def network_groups(layers: int) -> list[str]:
    """Parameter groups in the order of the flat vector of include/fno.h."""
    return ["P", "p"] + sum([[f"W{l}", f"w{l}", f"Rr{l}", f"Ri{l}"] for l in range(layers)], []) + \
        ["Q1", "q1", "Q2", "q2"]


def network_weights(width: int, hidden: int, layers: int, mx: int, my: int, seed: int,
                    outputs: int = 1) -> dict:
    """Seeded initial weights: P, W_l, Q1, Q2 standard normal / sqrt(fan-in),
    biases zero, spectral weights Rr, Ri ~ U[0, 1] / width^2 with shape
    [modes_y][modes_x][width(in)][width(out)]."""
    rng = np.random.default_rng(seed)
    p = {"P": rng.standard_normal((width, N_FEATURES)) / np.sqrt(N_FEATURES),
         "p": np.zeros(width)}
    for l in range(layers):
        p[f"W{l}"] = rng.standard_normal((width, width)) / np.sqrt(width)
        p[f"w{l}"] = np.zeros(width)
        s = 1.0 / (width * width)
        p[f"Rr{l}"] = s * rng.uniform(0, 1, (my, mx, width, width))
        p[f"Ri{l}"] = s * rng.uniform(0, 1, (my, mx, width, width))
    p["Q1"] = rng.standard_normal((hidden, width)) / np.sqrt(width)
    p["q1"] = np.zeros(hidden)
    p["Q2"] = rng.standard_normal((outputs, hidden)) / np.sqrt(hidden)
    p["q2"] = np.zeros(outputs)
    return p


def network_pack(p: dict, layers: int) -> np.ndarray:
    """Flat FP32 parameter vector in the order of include/fno.h."""
    return np.concatenate([np.asarray(p[k], dtype=np.float64).ravel()
                           for k in network_groups(layers)]).astype(np.float32)
