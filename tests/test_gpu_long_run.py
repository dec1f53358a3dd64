"""Long-run agreement with the oracle beyond the horizon where the noisy
quench amplifies rounding differences: the FP32 GPU run and the FP64 oracle
are compared on the statistics the physics fixes, not site by site, over
three seeds, with the spread across seeds printed.

The workload is the sheared zebra of the 512 x 256 configuration
(lambda = 128, A0 = 1e-4, T = 0.95 T_c, tau = 1; Sec. IV).  At U_w = 0.01 the
quench settles into a stationary state -- a liquid slab between two flat
interfaces parallel to the walls, modulated by the potential -- whose bulk
densities, x-averaged profile <n>_x(y), interface rows and x-wavelength are
compared with the oracle after 30,000 steps (by then they are within 1e-4
of their values at 80,000 steps on the GPU).  No interfacial wave travels:
the phase speed of the dominant x-mode is zero in both.  At U_w = 0.05 the
interfaces keep rearranging slowly for 200,000 steps without a travelling
wave either; that case is checked on the GPU alone (the oracle would need
hours).  A wave of one wavelength over L_x that an earlier version of this
test compared (256 x 128, U_w = 0.06, lambda = 32) turned out to be a
transient: over eight seeds its phase speed at 20,000 steps ranged from
-6e-3 to +4e-2 and every seed was static by 60,000 steps."""
import numpy as np
import pytest

from gpu_util import oracle_for

pytestmark = pytest.mark.gpu

from paper_1307_6703_gb300 import LB_FP32, Batch, lb_params  # noqa: E402
from paper_1307_6703_gb300.workloads import C2, noise_field  # noqa: E402

SEEDS = (1, 2, 3)


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    torch.cuda.set_device(0)
    yield
    torch.cuda.synchronize()


def _stats(series, every):
    """Statistics of the last density field of `series` (fields `every`
    steps apart): bulk densities, x-averaged profile, interface rows (where
    the profile crosses the mid density), and wavelength and phase speed of
    the dominant x-mode of the row with the largest x-variation."""
    n = series[-1]
    lo, hi = np.percentile(n, 5), np.percentile(n, 95)
    mid = 0.5 * (lo + hi)
    prof = n.mean(axis=1)
    cross = [int(y) for y in np.where(np.diff(np.sign(prof - mid)) != 0)[0]]
    y0 = int(np.argmax(n.var(axis=1)))
    sp = np.fft.rfft(n[y0] - n[y0].mean())
    k = int(np.argmax(np.abs(sp[1:])) + 1)
    ph = np.unwrap([np.angle(np.fft.rfft(f[y0] - f[y0].mean())[k]) for f in series])
    slope = np.polyfit(np.arange(len(ph)) * every, ph, 1)[0]
    return dict(n_liq=hi, n_vap=lo, profile=prof, interfaces=cross, wavelength=n.shape[1] / k,
                phase_speed=float(-slope / (2 * np.pi * k / n.shape[1])))


def _gpu_runs(w, steps, samples, every):
    b = Batch([lb_params(w.nx, w.ny, 1, LB_FP32, w.a, w.b, w.T, w.kappa, w.tau, w.A0, w.lam, w.u_bot,
                         w.u_top, w.N, w.Q, 0.0, None) for _ in SEEDS])
    for v, sd in zip(b, SEEDS):
        v.init_fields(noise_field(w, seed=sd))
    b.step(steps)
    series = [[v.moments()[0]] for v in b]
    for _ in range(samples):
        b.step(every)
        for i, v in enumerate(b):
            series[i].append(v.moments()[0])
    b.close()
    return [_stats(s, every) for s in series]


def _oracle_run(w, seed, steps, samples, every):
    o = oracle_for(w).init_fields(noise_field(w, seed=seed)).step(steps)
    series = [o.moments()[0]]
    for _ in range(samples):
        o.step(every)
        series.append(o.moments()[0])
    return _stats(series, every)


def _spread(rows, key):
    v = np.array([r[key] for r in rows], dtype=float)
    return f"{key} mean {v.mean():.6g} spread {v.max() - v.min():.2g}"


def test_config2_stationary_state_matches_oracle():
    w = C2(0.01)
    steps, samples, every = 30000, 4, 500
    gpu = _gpu_runs(w, steps, samples, every)
    ref = [_oracle_run(w, sd, steps, samples, every) for sd in SEEDS]
    for name, rows in (("gpu", gpu), ("oracle", ref)):
        print(name, "; ".join(_spread(rows, k) for k in ("n_liq", "n_vap", "wavelength", "phase_speed")),
              [r["interfaces"] for r in rows])
    for g, r in zip(gpu, ref):
        assert abs(g["n_liq"] - r["n_liq"]) <= 5e-3 * r["n_liq"]
        assert abs(g["n_vap"] - r["n_vap"]) <= 5e-3 * r["n_vap"]
        assert np.abs(g["profile"] - r["profile"]).max() <= 0.01 * r["profile"].max()
        assert len(g["interfaces"]) == len(r["interfaces"]) == 2
        assert all(abs(a - c) <= 1 for a, c in zip(g["interfaces"], r["interfaces"]))
        assert g["wavelength"] == r["wavelength"] == w.lam  # the potential's period, no L_x wave
        assert abs(g["phase_speed"]) < 1e-5 and abs(r["phase_speed"]) < 1e-5


def test_config2_strong_shear_has_no_travelling_wave():
    w = C2(0.05)
    gpu = _gpu_runs(w, 200000, 10, 1000)
    print("gpu", "; ".join(_spread(gpu, k) for k in ("n_liq", "n_vap", "wavelength", "phase_speed")),
          [r["interfaces"] for r in gpu])
    for g in gpu:
        assert g["wavelength"] == w.lam
        # against the wall speed: the transient wave above moved at ~10 % of it
        assert abs(g["phase_speed"]) < 1e-2 * w.u_top
        assert len(g["interfaces"]) == 2
