"""Pins of the CPU reference of the warm-start network (oracle/fno.py).

The truncated transforms are pinned to numpy's FFT, their round trip to the
identity on band-limited fields, gelu to the normal distribution function's
printed values, and the spectral layer with identity weights to the
projection onto the kept modes.  No GPU.
"""
import math

import numpy as np
import pytest

from oracle import fno
from paper_1307_6703_gb300.workloads import network_weights


def _band_limited(rng, ny, nx, mx, my):
    """Random real field made only of kept modes (|ky| < my/2, kx < mx)."""
    yy, xx = np.mgrid[0:ny, 0:nx]
    v = np.zeros((ny, nx))
    for kx in range(mx):
        for ky in range(-(my // 2) + 1, my // 2):
            a, b = rng.standard_normal(2)
            ph = 2 * math.pi * (kx * xx / nx + ky * yy / ny)
            v += a * np.cos(ph) + b * np.sin(ph)
    return v


@pytest.mark.parametrize("ny,nx", [(16, 64), (12, 40)])
def test_dft_modes_match_numpy_fft(ny, nx):
    rng = np.random.default_rng(1)
    v = rng.standard_normal((2, 3, ny, nx))
    mx, my = 7, 6
    V = fno.dft_modes(v, mx, my)
    F = np.fft.fft2(v)  # same sign convention: exp(-2 pi i k.r / n)
    ky = fno.y_modes(my)
    ref = F[..., ky % ny, :][..., :mx]
    assert np.allclose(V, ref, rtol=0, atol=1e-10 * np.abs(F).max())


def test_idft_inverts_dft_on_kept_modes():
    rng = np.random.default_rng(2)
    ny, nx, mx, my = 16, 64, 8, 8
    v = _band_limited(rng, ny, nx, mx, my)
    back = fno.idft_modes(fno.dft_modes(v, mx, my), ny, nx)
    assert np.max(np.abs(back - v)) <= 1e-11 * np.max(np.abs(v))


def test_gelu_values():
    """gelu(z) = z Phi(z): Phi(1) = 0.841344746068543 (standard normal table)."""
    g = fno.gelu(np.array([0.0, 1.0, -1.0, 8.0, -8.0]))
    assert g[0] == 0.0
    assert abs(g[1] - 0.841344746068543) < 1e-15
    assert abs(g[2] + (1 - 0.841344746068543)) < 1e-15
    assert abs(g[3] - 8.0) < 1e-12 and abs(g[4]) < 1e-12


def test_spectral_layer_with_identity_weights_projects():
    """With R = identity per mode and W = 0, w = 0, one linear layer maps a
    band-limited field (in every channel) to itself."""
    rng = np.random.default_rng(3)
    ny, nx, mx, my, width = 16, 32, 6, 6, 3
    p = network_weights(width, 4, 1, mx, my, seed=0)
    p["W0"][:] = 0.0
    p["Rr0"][:] = np.eye(width)[None, None]
    p["Ri0"][:] = 0.0
    v = np.stack([_band_limited(rng, ny, nx, mx, my) for _ in range(width)])[None]
    V = fno.dft_modes(v, mx, my)
    R = p["Rr0"] + 1j * p["Ri0"]
    K = fno.idft_modes(np.einsum("bckm,kmco->bokm", V, R), ny, nx)
    assert np.max(np.abs(K - v)) <= 1e-11 * np.max(np.abs(v))


def test_features_definition():
    x = fno.features(np.array([[0.05, 1e-3, 32.0, 0.96]]), 64, 9)
    assert x.shape == (1, 5, 9, 64)
    assert abs(x[0, 0, 0, 8] - 1.0) < 1e-15          # sin(pi/2) at x = lambda/4
    assert abs(x[0, 1, 0, 16] + 1.0) < 1e-15         # cos(pi) at x = lambda/2
    assert x[0, 2, 0, 0] == -1.0 and x[0, 2, 8, 0] == 1.0
    assert abs(x[0, 3, 3, 3] - 1.0) < 1e-12
    assert x[0, 4, 4, 7] == 0.0


def test_forward_is_affine_in_the_last_layer():
    """out is affine in (Q2, q2): doubling Q2 and q2 doubles out."""
    p = network_weights(4, 6, 2, 4, 4, seed=5, outputs=3)
    x = fno.features(np.array([[0.02, 5e-4, 32.0, 0.95]]), 32, 8)
    o1 = fno.forward(p, x, 2, 4, 4)
    p["Q2"] *= 2.0
    p["q2"] = p["q2"] * 2.0 + 0.0
    o2 = fno.forward(p, x, 2, 4, 4)
    assert np.allclose(o2, 2 * o1, rtol=1e-13, atol=1e-15)
