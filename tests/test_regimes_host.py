"""Host logic of the paper-regime measurements (no GPU): the broken-line
fit and prediction, the interface statistics and the phase drift of an
interface wave, on synthetic fields whose answers are known, and the
parameter mapping of Tables 1 and 2."""
import numpy as np

from paper_1307_6703_gb300 import regimes as R
from paper_1307_6703_gb300.workloads import TC


def test_broken_line_prediction_meets_the_walls_and_balances_the_stress():
    """Both segments start and end at the wall speeds, the shear stress
    n s is the same on both sides, and for the interface half-way the
    slopes are 2 gamma n_u / (n_u + n_l) and 2 gamma n_l / (n_u + n_l)."""
    u_w, ly, n_lo, n_hi = 0.02, 128, 1.47, 0.53
    for y_i in (40.0, 63.5, 90.25):
        s_lo, s_hi = R.broken_line_prediction(u_w, ly, n_lo, n_hi, y_i)
        u_top = -u_w + s_lo * y_i + s_hi * (ly - 1 - y_i)
        assert abs(u_top - u_w) < 1e-15
        assert abs(n_lo * s_lo - n_hi * s_hi) < 1e-15
    s_lo, s_hi = R.broken_line_prediction(u_w, ly, n_lo, n_hi, (ly - 1) / 2)
    gamma = 2 * u_w / (ly - 1)
    assert np.isclose(s_lo, 2 * gamma * n_hi / (n_lo + n_hi), rtol=1e-14)
    assert np.isclose(s_hi, 2 * gamma * n_lo / (n_lo + n_hi), rtol=1e-14)


def test_broken_line_slopes_recovers_a_synthetic_profile():
    """A tanh density step at row 63.5 and a velocity made of two straight
    segments: the fitted slopes, the bulk densities and the interface row
    come back."""
    ly, lx, u_w = 128, 16, 0.02
    n = R.two_layer_field(lx, ly, 1.47, 0.53, width=2.0)
    y_i = ly / 2 - 0.5
    s_lo, s_hi = R.broken_line_prediction(u_w, ly, 1.47, 0.53, y_i)
    y = np.arange(ly, dtype=float)
    u = np.where(y <= y_i, -u_w + s_lo * y, -u_w + s_lo * y_i + s_hi * (y - y_i))
    ux = np.repeat(u[:, None], lx, axis=1)
    f_lo, f_hi, m_lo, m_hi, yi = R.broken_line_slopes(n, ux)
    assert np.isclose(f_lo, s_lo, rtol=1e-10) and np.isclose(f_hi, s_hi, rtol=1e-10)
    assert abs(m_lo - 1.47) < 1e-6 and abs(m_hi - 0.53) < 1e-6
    assert abs(yi - y_i) < 0.02


def test_interface_stats_of_a_slab_and_of_a_wavy_interface():
    ly, lx = 64, 128
    y = np.arange(ly)[:, None] * np.ones((1, lx))
    slab = np.where((y >= 20) & (y < 44), 1.45, 0.58)
    st = R.interface_stats(slab)
    assert st["crossings"] == 2 and st["amp"] == 0.0 and abs(st["liquid_fraction"] - 24 / 64) < 1e-12
    x = np.arange(lx)[None, :]
    h = 32 + np.round(8 * np.sin(2 * np.pi * x / lx))
    wavy = np.where(y < h, 1.45, 0.58)
    st = R.interface_stats(wavy)
    assert st["crossings"] == 1 and abs(st["amp"] - 16 / 64) < 1e-12
    assert np.array_equal(st["height"], h[0])


def test_dominant_phase_and_wave_speed_of_a_travelling_profile():
    """h(x, t) = h0 + a sin(2 pi k (x - c t) / L): the dominant mode is k
    and its phase drift gives c, for either direction and across phase
    wraps."""
    lx, k = 512, 2
    x = np.arange(lx)
    for c in (0.05, -0.031, 0.4):
        dt = 200
        profiles = [40 + 9 * np.sin(2 * np.pi * k * (x - c * dt * j) / lx) + 0.5 * np.cos(2 * np.pi * 7 * x / lx)
                    for j in range(10)]
        kk, _ = R.dominant_phase(profiles[0])
        assert kk == k
        phases = [R.dominant_phase(h, k)[1] for h in profiles]
        assert abs(R.wave_speed(phases, dt, k, lx) - c) < 1e-9


def test_table_parameter_mapping():
    """Table 1 cases: one droplet per (T_r, N, Q); Table 2: the paper's 30
    rows, walls at -/+ gamma L_y / 2 and kappa / 3 in lattice units, the
    row's Table 1 stencil."""
    cases = R.table1_cases((0.89, 0.95), (0.2, 0.3), (1.0, 2.0, 3.0))
    assert len(cases) == 12 and all(c.nx == c.ny == 64 and not c.walls for c in cases)
    assert abs(cases[-1].T - 0.95 * TC) < 1e-15
    rows = R.table2_rows()
    assert len(rows) == 30
    assert {r["lx"] for r in rows} == {256, 512, 1024, 2048} and all(r["ly"] == 256 for r in rows)
    r = next(r for r in rows if r["T_r"] == 0.91 and r["lx"] == 1024 and r["lam"] == 64)
    c = R.table2_case(r)
    assert c.walls and c.u_w == r["gamma"] * 256 / 2 and abs(c.kappa - r["kappa_paper"] / 3) < 1e-15
    assert (c.N, c.Q) == R.TABLE1_OVC[0.91] and c.tau == r["tau"] and c.A0 == r["A0"]
