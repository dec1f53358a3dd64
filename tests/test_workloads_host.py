"""The seeded input recipes (no GPU): the named workloads carry the
parameters the design documents, and the generators are reproducible and
stay inside their stated ranges."""
import numpy as np

from paper_1307_6703_gb300.warmstart import sample_params
from paper_1307_6703_gb300.workloads import C1, C2, C4, TC, batch_workloads, droplet_field, noise_field, slab_field


def test_named_workloads():
    # (name, nx, ny, walls, T/T_c, tau, A0, lambda, U_w, (N, Q))
    for w, nx, ny, tr, a0, lam, uw, nq in ((C1, 64, 32, 0.9, 1e-3, 32.0, 0.0, (0.3, 2.6)),
                                           (C2(0.01), 512, 256, 0.95, 1e-4, 128.0, 0.01, (0.3, 2.0)),
                                           (C2(0.05), 512, 256, 0.95, 1e-4, 128.0, 0.05, (0.3, 2.0)),
                                           (C4, 4096, 1024, 0.95, 1e-4, 512.0, 0.05, (0.3, 2.0))):
        assert (w.nx, w.ny, w.walls, w.tau) == (nx, ny, True, 1.0)
        assert abs(w.T - tr * TC) < 1e-15 and w.A0 == a0 and w.lam == lam
        assert w.u_bot == -uw and w.u_top == uw and (w.N, w.Q) == nq
        assert (w.a, w.b, w.kappa) == (3.0 / 8.0, 1.0 / 3.0, 0.1)
    assert abs(TC - 8 * C4.a / (27 * C4.b)) < 1e-15      # T_c = 8a / (27 b)
    assert C4.name == "fp32_4096x1024_shear_0.05"


def test_noise_field_is_seeded_and_bounded():
    a, b = noise_field(C2(0.05)), noise_field(C2(0.05))
    assert np.array_equal(a, b) and a.shape == (256, 512)
    assert not np.array_equal(a, noise_field(C2(0.05), seed=2))
    w = C2(0.05)
    assert np.all(np.abs(a - w.rho_mean) <= w.noise) and abs(a.mean() - w.rho_mean) < 1e-4 * w.rho_mean
    assert abs(w.noise - 0.01 / 3.5) < 1e-18


def test_batch_ensemble_ranges():
    ws = batch_workloads()
    assert len(ws) == 64 and sum(w.nx * w.ny for w in ws) == 5960704
    assert [w.name for w in ws] == [w.name for w in batch_workloads()]
    for w in ws:
        assert w.nx % 32 == 0 and 128 <= w.nx <= 1024 and w.ny % 16 == 0 and 64 <= w.ny <= 256
        assert w.walls and w.u_bot == -w.u_top and 0.0 <= w.u_top <= 0.1
        assert 1e-4 <= w.A0 <= 5e-4 and w.lam in (32.0, 64.0) and 0.92 <= w.T / TC <= 0.96 and w.tau == 1.0


def test_warm_start_draws():
    for regime, lo, hi in (("steady", 0.0, 0.035), ("wave", 0.04, 0.06)):
        p = sample_params(200, seed=3, regime=regime)
        assert np.array_equal(p, sample_params(200, seed=3, regime=regime))
        assert np.all((p[:, 0] >= lo) & (p[:, 0] <= hi))
        assert np.all((p[:, 1] >= 3e-4) & (p[:, 1] <= 1e-3)) and set(p[:, 2]) == {32.0, 64.0}
        assert np.all((p[:, 3] >= 0.925) & (p[:, 3] <= 0.96))


def test_shaped_fields():
    d = droplet_field(64, 64, 15.0, 1.46, 0.58)
    assert d.shape == (64, 64) and abs(d[32, 32] - 1.46) < 1e-3 and abs(d[0, 0] - 0.58) < 1e-6
    s = slab_field(64, 64, 1.46, 0.58)
    assert abs(s[32, 0] - 1.46) < 1e-3 and abs(s[0, 0] - 0.58) < 1e-3 and np.allclose(s, s[:, :1])
