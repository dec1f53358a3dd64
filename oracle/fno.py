"""FP64 CPU reference of the Fourier neural operator used as a learned warm
start for the lattice Boltzmann solver (not in the paper; a component of
this project).  TEST INFRASTRUCTURE ONLY: the test suite uses it to check
the CUDA network's forward pass and, by finite differences of its loss,
the CUDA backward pass.  It shares no code with the CUDA path.

The network (definitions written out plainly, no blocking or fusion):

  features  x[b, 0..4, y, x] from the parameters (U_w, A0, lambda, T_r):
            A0/1e-3 sin(2 pi x / lambda), A0/1e-3 cos(2 pi x / lambda),
            U_w/0.05 (2y/(ny-1) - 1), (T_r - 0.94)/0.02, 2y/(ny-1) - 1
  lift      v0 = P x + p                       (P: width x 5)
  layer l   z = W_l v + w_l + K_l v,  v' = gelu(z) (no gelu after the last)
            K_l v = IDFT_m( R_l[m] . DFT_m(v) ): the 2D DFT restricted to
            mx x-modes kx = 0..mx-1 and my y-modes ky = 0..my/2-1 and
            -my/2..-1, a complex width x width matrix per mode, and the
            real inverse transform of those modes (kx > 0 counted twice for
            the conjugate half, scale 1/(nx ny))
  project   h = gelu(Q1 v4 + q1),  out = Q2 h + q2     (Q1: hidden x width,
            Q2: outputs x hidden)
  loss      mean over b, output channel, y, x of (out - target)^2
gelu(z) = z Phi(z) with Phi the standard normal distribution function.

Parameters are a dict of float64 arrays keyed P, p, W{l}, w{l}, Rr{l}, Ri{l}
(Rr, Ri: [ky][kx][c_in][c_out]), Q1, q1, Q2, q2; the tests draw them with
the shared seeded generator and give the CUDA network the same values.
"""
from __future__ import annotations

import math

import numpy as np

N_FEATURES = 5


def features(params: np.ndarray, nx: int, ny: int) -> np.ndarray:
    """params[b] = (U_w, A0, lambda, T_r) -> x[b, 5, ny, nx] (float64)."""
    params = np.asarray(params, dtype=np.float64).reshape(-1, 4)
    B = params.shape[0]
    xs = np.arange(nx, dtype=np.float64)[None, :]
    ys = np.arange(ny, dtype=np.float64)[:, None]
    out = np.zeros((B, N_FEATURES, ny, nx))
    for b, (uw, a0, lam, tr) in enumerate(params):
        ph = 2.0 * math.pi * xs / lam
        yy = 2.0 * ys / (ny - 1) - 1.0
        out[b, 0] = (a0 / 1e-3) * np.sin(ph)
        out[b, 1] = (a0 / 1e-3) * np.cos(ph)
        out[b, 2] = (uw / 0.05) * yy
        out[b, 3] = (tr - 0.94) / 0.02
        out[b, 4] = yy
    return out


def gelu(z):
    erf = np.vectorize(math.erf)
    return z * 0.5 * (1.0 + erf(z / math.sqrt(2.0)))


def y_modes(my: int) -> np.ndarray:
    h = my // 2
    return np.array(list(range(h)) + list(range(-h, 0)))


def dft_modes(v: np.ndarray, mx: int, my: int) -> np.ndarray:
    """v[..., ny, nx] real -> V[..., my, mx] complex: sum over y, x of
    v exp(-2 pi i (ky y / ny + kx x / nx)) for the kept modes."""
    ny, nx = v.shape[-2:]
    kx = np.arange(mx)
    ky = y_modes(my)
    ex = np.exp(-2j * math.pi * np.outer(np.arange(nx), kx) / nx)   # [nx, mx]
    ey = np.exp(-2j * math.pi * np.outer(ky, np.arange(ny)) / ny)   # [my, ny]
    return np.einsum("ky,...yx,xm->...km", ey, v, ex)


def idft_modes(V: np.ndarray, ny: int, nx: int) -> np.ndarray:
    """Real inverse of dft_modes: (1/(nx ny)) sum over kept modes of
    c_kx Re(V exp(+2 pi i (ky y / ny + kx x / nx))), c_0 = 1, c_kx>0 = 2."""
    my, mx = V.shape[-2:]
    kx = np.arange(mx)
    ky = y_modes(my)
    ex = np.exp(2j * math.pi * np.outer(kx, np.arange(nx)) / nx)    # [mx, nx]
    ey = np.exp(2j * math.pi * np.outer(np.arange(ny), ky) / ny)    # [ny, my]
    c = np.where(kx == 0, 1.0, 2.0)
    out = np.einsum("yk,...km,m,mx->...yx", ey, V, c, ex)
    return out.real / (nx * ny)


def forward(p: dict, x: np.ndarray, layers: int, mx: int, my: int) -> np.ndarray:
    """x[b, 5, ny, nx] -> out[b, outputs, ny, nx]."""
    ny, nx = x.shape[-2:]
    v = np.einsum("oc,bcyx->boyx", p["P"], x) + p["p"][None, :, None, None]
    for l in range(layers):
        V = dft_modes(v, mx, my)                                     # [b, c, my, mx]
        R = p[f"Rr{l}"] + 1j * p[f"Ri{l}"]                           # [my, mx, c, o]
        Y = np.einsum("bckm,kmco->bokm", V, R)
        K = idft_modes(Y, ny, nx)
        z = np.einsum("oc,bcyx->boyx", p[f"W{l}"], v) + p[f"w{l}"][None, :, None, None] + K
        v = gelu(z) if l < layers - 1 else z
    h = gelu(np.einsum("hc,bcyx->bhyx", p["Q1"], v) + p["q1"][None, :, None, None])
    return np.einsum("oh,bhyx->boyx", p["Q2"], h) + p["q2"][None, :, None, None]


def loss(p: dict, x: np.ndarray, target: np.ndarray, layers: int, mx: int, my: int) -> float:
    d = forward(p, x, layers, mx, my) - target
    return float(np.mean(d * d))
