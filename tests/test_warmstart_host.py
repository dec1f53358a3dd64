"""Host logic of the learned warm start (no GPU): the periodic x-shift, the
change of a travelling pattern measured in its own frame, and the phase
alignment of travelling targets."""
import numpy as np

from paper_1307_6703_gb300.warmstart import comoving_change, phase_aligned, shift_x


def _wave(nx=256, ny=64, x0=40.3):
    x = np.arange(nx)
    y = np.arange(ny)[:, None]
    h = 30 + 6 * np.sin(2 * np.pi * (x - x0) / nx) + 2 * np.sin(6 * np.pi * (x - x0) / nx)
    n = 0.5 + 0.45 * (1 - np.tanh((y - h) / 3.0))
    return np.stack([n, 0.01 * np.sin(2 * np.pi * (x - x0) / nx) + 0 * y, 0.002 * (y - 32) + 0 * x])


def test_shift_x_is_an_exact_roll_for_whole_sites():
    f = _wave()
    assert np.allclose(shift_x(f, 5.0), np.roll(f, -5, axis=-1), atol=1e-12)
    assert np.allclose(shift_x(shift_x(f, 2.3), -2.3), f, atol=1e-12)


def test_comoving_change_finds_the_displacement():
    f = _wave()
    for d in (0.0, 3.25, -17.6, 100.5):
        ch, got = comoving_change(shift_x(f, -d), f)  # pattern moved by +d sites
        assert abs(got - d) < 0.05, (d, got)
        assert ch < 1e-3
    # a pattern that changes shape is not settled in any frame
    g = _wave()
    g[0] *= 1.01
    assert comoving_change(g, f)[0] > 1e-3


def test_phase_alignment_is_independent_of_the_phase():
    f = _wave()
    ref = phase_aligned(f)
    for d in (7.0, -33.4, 120.9):
        assert np.abs(phase_aligned(shift_x(f, d)) - ref).max() < 1e-9
