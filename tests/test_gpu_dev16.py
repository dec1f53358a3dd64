"""16-bit deviation storage (LB_BF16DEV, LB_FP16DEV) against the oracle's
model of the same format (FP64 step, then the format's rounding).

The GPU takes each rounding decision on its FP32 value and the oracle on its
FP64 value, so a stored deviation may differ by one unit in the last place
where the exact value lies within FP32 error of a rounding midpoint; every
other stored deviation must match exactly.  Over many steps the GPU's
distance from the exact-format oracle is held below the format's own error
(the distance between the exact-format and the full-precision oracle), and
mass is conserved to FP32 round-off.
"""
import numpy as np
import pytest

import oracle
from gpu_util import decode_dev, decode_state, dev16_solver, oracle_for, rel_err

pytestmark = pytest.mark.gpu

from paper_1307_6703_gb300 import LB_BF16DEV, LB_FP16DEV  # noqa: E402
from paper_1307_6703_gb300.workloads import C1, C2, C4, TC, noise_field, slab_field  # noqa: E402

FORMATS = [(LB_BF16DEV, "bf16"), (LB_FP16DEV, "fp16")]
RHO_REF = 1.0  # the vdW critical density 1/(3b) of the paper's set


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    torch.cuda.set_device(0)
    yield
    torch.cuda.synchronize()


def _ulp(x, fmt):
    p, emin = oracle.FORMATS[fmt]
    ax = np.abs(x)
    e = np.where(ax > 0, np.floor(np.log2(np.where(ax > 0, ax, 1.0))), emin)
    return 2.0 ** (np.maximum(e, emin) - p + 1)


def _round(x, fmt):
    return np.vectorize(lambda v: oracle.round_sig(float(v), fmt))(x)


def _check_rounding(dg, do, unrounded, fmt, eps):
    """dg: GPU deviations, do: oracle's rounded deviations, unrounded: the
    oracle's values before rounding, eps: bound of the GPU's FP32 error on
    the value it rounds.  Each GPU value must be the rounding of some value
    within eps of the oracle's unrounded one: rounding is monotonic, so it
    lies between round(u - eps) and round(u + eps).  Returns the fraction
    of decisions that differ."""
    mism = dg != do
    if mism.any():
        a, u = dg[mism], unrounded[mism]
        lo, hi = _round(u - eps, fmt), _round(u + eps, fmt)
        assert np.all((a >= lo) & (a <= hi)), \
            "a stored deviation is not a rounding of a value within FP32 error of the exact one"
    return float(mism.mean())


def _step_case(w, prec, fmt, n0, eps_rel=2e-6, steps_before=0):
    s = dev16_solver(w, prec, RHO_REF).init_fields(n0)
    if steps_before:
        s.step(steps_before)
    f0, d = s.get_state()
    F = decode_state(f0, d, fmt, RHO_REF)
    ref = oracle_for(w).set_state(F).step(1)
    q, unr = oracle.quantize(ref.f, fmt, RHO_REF, want_unrounded=True)
    s.step(1)
    g0, gd = s.get_state()
    s.close()
    r = oracle.reference_pops(RHO_REF)
    dg = decode_dev(gd, fmt)
    do = q[1:] - r[1:, None, None]
    eps = eps_rel * np.abs(F).max()
    frac = _check_rounding(dg, do, unr, fmt, eps)
    # the rest population carries the remainder of the rounded values
    slack = np.abs(dg - do).sum(axis=0) + eps
    assert np.all(np.abs(g0 - q[0]) <= slack)
    return frac


@pytest.mark.parametrize("prec,fmt", FORMATS)
def test_dev16_init_matches_oracle_format(prec, fmt):
    """lb_init mode 1 (FP32 equilibrium, then the format) = the oracle's
    equilibrium passed through the format, decision by decision."""
    w = C1.with_(nx=248, ny=67, walls=True, u_bot=-0.04, u_top=0.04)
    n0 = noise_field(w)
    s = dev16_solver(w, prec, RHO_REF).init_fields(n0)
    f0, d = s.get_state()
    s.close()
    ref = oracle_for(w).init_fields(n0)
    q, unr = oracle.quantize(ref.f, fmt, RHO_REF, want_unrounded=True)
    r = oracle.reference_pops(RHO_REF)
    frac = _check_rounding(decode_dev(d, fmt), q[1:] - r[1:, None, None], unr, fmt,
                           1e-7 * np.abs(ref.f).max())
    assert frac <= 1e-3
    # the rest population carries the remainder of the rounded values
    slack = np.abs(decode_dev(d, fmt) - (q[1:] - r[1:, None, None])).sum(axis=0) + 1e-6
    assert np.all(np.abs(f0 - q[0]) <= slack)


CASES = [
    # (nx, ny, walls, u_w): one and several strips, ragged strips and segments
    (8, 8, True, 0.02),
    (8, 8, False, 0.0),
    (248, 67, True, 0.04),
    (304, 130, False, 0.0),
    (304, 130, True, 0.05),
]


@pytest.mark.parametrize("prec,fmt", FORMATS)
@pytest.mark.parametrize("case", CASES, ids=lambda c: f"{c[0]}x{c[1]}{'w' if c[2] else 'p'}")
def test_dev16_one_step_parity(case, prec, fmt):
    nx, ny, walls, u_w = case
    w = C1.with_(nx=nx, ny=ny, walls=walls, u_bot=-u_w, u_top=u_w, lam=float(nx // 2))
    frac = _step_case(w, prec, fmt, noise_field(w), steps_before=5)
    assert frac <= 1e-2


@pytest.mark.parametrize("prec,fmt", FORMATS)
def test_dev16_full_size_one_step(prec, fmt):
    """4096x1024 (the benchmark lattice, same launch path), every site."""
    w = C4
    frac = _step_case(w, prec, fmt, noise_field(w))
    assert frac <= 1e-2


@pytest.mark.parametrize("prec,fmt", FORMATS)
def test_dev16_full_size_bench_launches(prec, fmt):
    """The benchmark's launch sequence with 16-bit storage on 4096x1024
    (autotuned tiling, a 5-step launch, then one persistent 20-step launch)
    against the full-precision oracle and the oracle that rounds its state
    to the format every step: the GPU's density error is within twice the
    format's own, and its distance from the exact-format run is a small
    fraction of that."""
    w = C4
    n0 = noise_field(w)
    s = dev16_solver(w, prec, RHO_REF).init_fields(n0)
    seg_h = s.autotune(20)
    s.step(5)
    s.step(20)
    n = s.moments()[0]
    rc, _ = s.reduce()
    s.close()
    exact = oracle_for(w).init_fields(n0).quantize(fmt, RHO_REF).step(25, storage=(fmt, RHO_REF))
    full = oracle_for(w).init_fields(n0).step(25)
    ne, nf = exact.moments()[0], full.moments()[0]
    gpu_err, fmt_err, gpu_exact = rel_err(n, nf), rel_err(ne, nf), rel_err(n, ne)
    print(f"4096x1024 {fmt}, seg_h {seg_h}, 5 + 20 steps: GPU vs full {gpu_err:.3e}, format vs full "
          f"{fmt_err:.3e}, GPU vs exact format {gpu_exact:.3e}")
    assert rc == 0
    assert gpu_err <= 2.0 * fmt_err + 1e-6


def test_dev16_largest_lattice_against_fp64():
    """The largest lattice whose padded planes the sweep indexes in 32 bits
    (16384 x 13000, 213 M sites), 16-bit storage with its 128-column
    window: three steps from the same noise against the FP64 path on every
    site (compared on the device), and the mass.  Bound: each step rounds
    every stored deviation to the format (half an ulp of deviations that
    stay below ~0.02 here: 8 links x 3 steps x 2^-9 x 0.02 ~ 1e-3 for bf16,
    8x less for fp16's 3 more bits); the measured errors are printed."""
    import torch
    from paper_1307_6703_gb300 import LB_DTYPE_F32, LB_DTYPE_F64, LB_FP64, lb_moments
    from gpu_util import solver_for
    w = C4.with_(nx=16384, ny=13000)
    pitch = ((w.nx + 8 + 31) // 32) * 32
    assert 9 * pitch * (w.ny + 8) < 2 ** 31
    s = solver_for(w, LB_FP64).init_noise(9, w.rho_mean, w.noise).step(3)
    n64 = torch.empty((w.ny, w.nx), dtype=torch.float64, device="cuda")
    lb_moments(s.h, n64, None, None, LB_DTYPE_F64, 1)
    rc, (m64, _, _) = s.reduce()
    s.close()
    assert rc == 0
    for prec, fmt, bound in ((LB_BF16DEV, "bf16", 1e-3), (LB_FP16DEV, "fp16", 1.25e-4)):
        s = dev16_solver(w, prec, RHO_REF).init_noise(9, w.rho_mean, w.noise).step(3)
        n = torch.empty((w.ny, w.nx), dtype=torch.float32, device="cuda")
        lb_moments(s.h, n, None, None, LB_DTYPE_F32, 1)
        torch.cuda.synchronize()
        rc, (m, _, _) = s.reduce()
        s.close()
        err = float(((n.double() - n64).abs().max() / n64.abs().max()).item())
        print(f"16384 x 13000 {fmt}: max rel density error after 3 steps {err:.2e}, mass {abs(m - m64) / m64:.1e}")
        assert rc == 0
        assert err <= bound
        assert abs(m - m64) / m64 <= 1e-6
    del n64


DAMPED = {
    # supercritical sheared fluid relaxing to Couette flow
    "couette": (dict(nx=128, ny=48, T=1.1 * TC, A0=0.0, lam=0.0, u_bot=-0.05, u_top=0.05),
                lambda w: 1.0 + 0.02 * np.sin(2 * np.pi * np.arange(w.nx) / w.nx)[None, :]
                * np.ones((w.ny, 1))),
    # flat liquid slab at rest between static walls (Maxwell coexistence)
    "slab": (dict(nx=64, ny=64, A0=0.0, lam=0.0, u_bot=0.0, u_top=0.0),
             lambda w: slab_field(w.nx, w.ny, 1.46, 0.58)),
}


@pytest.mark.parametrize("prec,fmt", FORMATS)
@pytest.mark.parametrize("case", sorted(DAMPED))
def test_dev16_multi_step_within_format_error(case, prec, fmt):
    """300 steps of a damped flow: the GPU's error against the full-precision
    oracle is at most twice the format's own error (the exact-format oracle
    against the full-precision oracle) -- FP32 arithmetic and the rounding
    decisions it moves add no more than the format itself."""
    kw, field = DAMPED[case]
    w = C2(0.0).with_(**kw)
    n0 = field(w)
    steps = 300
    s = dev16_solver(w, prec, RHO_REF).init_fields(n0).step(steps)
    n, ux, _ = s.moments()
    s.close()
    exact = oracle_for(w).init_fields(n0).quantize(fmt, RHO_REF).step(steps, storage=(fmt, RHO_REF))
    full = oracle_for(w).init_fields(n0).step(steps)
    ne, nf = exact.moments()[0], full.moments()[0]
    gpu_err, fmt_err, gpu_exact = rel_err(n, nf), rel_err(ne, nf), rel_err(n, ne)
    print(f"{case} {fmt}: GPU vs full {gpu_err:.3e}, format vs full {fmt_err:.3e}, "
          f"GPU vs exact format {gpu_exact:.3e}")
    assert gpu_err <= 2.0 * fmt_err + 1e-6


@pytest.mark.parametrize("prec,fmt", FORMATS)
def test_dev16_mass_conservation(prec, fmt):
    """1000 sheared steps: total mass to FP32 round-off, both through the
    step kernel's records and the exact sum over the stored state."""
    w = C2(0.05)
    s = dev16_solver(w, prec, RHO_REF).init_noise(w.seed, w.rho_mean, w.noise)
    rc, (m0, _, _) = s.reduce()
    assert rc == 0
    s.step(1000)
    rc, (m1, _, _) = s.reduce()
    assert rc == 0
    assert abs(m1 - m0) / m0 < 1e-6
    # exact FP64 sum over the decoded state (a restore invalidates the records)
    state = s.get_state()
    s.set_state(state, step=1000)
    rc, (m2, _, _) = s.reduce()
    assert rc == 0 and abs(m2 - m1) / m1 < 1e-6
    F = decode_state(*state, fmt, RHO_REF)
    assert abs(F.sum() - m2) / m2 < 1e-6
    s.close()


@pytest.mark.parametrize("prec,fmt", FORMATS)
def test_dev16_checkpoint_resume_is_bitwise(prec, fmt):
    w = C2(0.05).with_(nx=96, ny=48)
    a = dev16_solver(w, prec, RHO_REF).init_noise(5, w.rho_mean, w.noise).step(200)
    b = dev16_solver(w, prec, RHO_REF).init_noise(5, w.rho_mean, w.noise).step(100)
    state = b.get_state()
    b.close()
    c = dev16_solver(w, prec, RHO_REF).set_state(state, step=100).step(100)
    sa, sc = a.get_state(), c.get_state()
    assert np.array_equal(sa[0], sc[0]) and np.array_equal(sa[1], sc[1])
    a.close()
    c.close()


def test_dev16_default_reference_is_critical_density():
    """rho_ref = 0 selects 1/(3b): same trajectory as rho_ref = 1 for b = 1/3."""
    w = C2(0.05).with_(nx=64, ny=32)
    a = dev16_solver(w, LB_BF16DEV, 0.0).init_noise(1, w.rho_mean, w.noise).step(20)
    b = dev16_solver(w, LB_BF16DEV, 1.0).init_noise(1, w.rho_mean, w.noise).step(20)
    sa, sb = a.get_state(), b.get_state()
    assert np.array_equal(sa[0], sb[0]) and np.array_equal(sa[1], sb[1])
    a.close()
    b.close()


def test_storage_observables_against_fp64():
    """The headline physics (sheared quench, A0 = 1e-4, lambda = 512 scaled
    to 1024x256, lambda = 128) for 5000 steps in every storage, against the
    GPU FP64 path (itself bit-identical to the oracle): density profile
    <n>_x(y), dominant wavelength along x, mass drift."""
    from paper_1307_6703_gb300 import LB_FP32, LB_FP64
    from gpu_util import solver_for
    w = C4.with_(nx=1024, ny=256, lam=128.0)
    n0 = noise_field(w)
    res = {}
    for name, prec in (("fp64", LB_FP64), ("fp32", LB_FP32), ("bf16", LB_BF16DEV), ("fp16", LB_FP16DEV)):
        s = solver_for(w, prec) if prec in (LB_FP64, LB_FP32) else dev16_solver(w, prec, RHO_REF)
        s.init_fields(n0)
        m0 = s.reduce()[1][0]
        s.step(5000)
        rc, (m1, _, _) = s.reduce()
        n = s.moments()[0]
        s.close()
        spec = np.abs(np.fft.rfft(n[w.ny // 4] - n[w.ny // 4].mean()))
        res[name] = (n.mean(axis=1), w.nx / (np.argmax(spec[1:]) + 1), abs(m1 - m0) / m0, rc)
    prof64, lam64, drift64, _ = res["fp64"]
    assert lam64 == 128.0 and drift64 < 1e-12
    bounds = {"fp32": 1e-3, "fp16": 1e-2, "bf16": 5e-2}
    for name, bound in bounds.items():
        prof, lam, drift, rc = res[name]
        err = np.abs(prof - prof64).max() / np.abs(prof64).max()
        print(f"{name}: profile error {err:.2e}, wavelength {lam}, mass drift {drift:.2e}")
        assert rc == 0 and lam == lam64 and drift < 1e-5 and err < bound
