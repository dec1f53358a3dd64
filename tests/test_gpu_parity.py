"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

FP64 (parity mode, no fused multiply-add) must agree to 1e-12 relative and is
expected to agree bit for bit.  FP32 is held to 1e-5 max relative density
error where the dynamics do not amplify rounding, and on the unstable
512x256 quench to the drift FP32 rounding causes in the oracle itself (see
test_fp32_config_512x256_1000_steps).  Sizes span several
tiles with ragged tails, the degenerate 1x1 lattice and the wall/no-wall
cases; the full 4096x1024 lattice is checked step by step.
"""
import numpy as np
import pytest

from gpu_util import oracle_for, rel_err, solver_for

pytestmark = pytest.mark.gpu

from paper_1307_6703_gb300 import LB_ERR_UNSTABLE, LB_FP32, LB_FP64  # noqa: E402
from paper_1307_6703_gb300.workloads import C1, C2, C4, TC, noise_field  # noqa: E402

SMALL = [
    # (nx, ny, walls, u_w, steps)
    (1, 1, False, 0.0, 30),
    (3, 5, False, 0.0, 40),
    (5, 3, True, 0.03, 40),
    (33, 9, True, 0.02, 60),
    (37, 17, False, 0.0, 60),
    (70, 41, True, 0.05, 80),
]


def small_workload(nx, ny, walls, u_w, steps):
    return C1.with_(nx=nx, ny=ny, walls=walls, u_bot=-u_w, u_top=u_w, steps=steps,
                    lam=float(max(nx // 2, 1)), A0=1e-3 if nx > 1 else 0.0)


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    torch.cuda.set_device(0)
    yield
    torch.cuda.synchronize()


@pytest.mark.parametrize("case", SMALL, ids=lambda c: f"{c[0]}x{c[1]}{'w' if c[2] else 'p'}")
def test_fp64_small_lattices(case):
    w = small_workload(*case)
    n0 = noise_field(w)
    ref = oracle_for(w).init_fields(n0).step(w.steps)
    s = solver_for(w, LB_FP64).init_fields(n0).step(w.steps)
    f = s.get_state()
    assert rel_err(f, ref.f) <= 1e-12
    n, ux, uy = s.moments()
    rn, rux, ruy = ref.moments()
    assert rel_err(n, rn) <= 1e-12
    assert np.abs(ux - rux).max() <= 1e-12 * max(np.abs(rux).max(), 1e-3)
    assert np.abs(uy - ruy).max() <= 1e-12 * max(np.abs(ruy).max(), 1e-3)
    s.close()


@pytest.mark.parametrize("case", SMALL, ids=lambda c: f"{c[0]}x{c[1]}{'w' if c[2] else 'p'}")
def test_fp64_small_lattices_bitwise(case):
    """The FP64 parity mode evaluates the oracle's formulas in the same order
    without fused multiply-adds, so the populations agree bit for bit."""
    w = small_workload(*case)
    n0 = noise_field(w)
    ref = oracle_for(w).init_fields(n0).step(w.steps)
    s = solver_for(w, LB_FP64).init_fields(n0).step(w.steps)
    assert np.array_equal(s.get_state(), ref.f)
    s.close()


def test_fp64_noise_init_matches_oracle():
    """Device SplitMix64 initial condition (lb_init mode 0) = oracle's."""
    w = C1
    ref = oracle_for(w).init_noise(7, w.rho_mean, w.noise)
    s = solver_for(w, LB_FP64).init_noise(7, w.rho_mean, w.noise)
    assert np.array_equal(s.get_state(), ref.f)
    s.close()


def test_fp64_config_64x32_2000_steps():
    w = C1
    n0 = noise_field(w)
    ref = oracle_for(w).init_fields(n0).step(w.steps)
    s = solver_for(w, LB_FP64).init_fields(n0).step(w.steps)
    n, ux, uy = s.moments()
    rn, rux, ruy = ref.moments()
    assert rel_err(n, rn) <= 1e-12
    assert np.abs(ux - rux).max() <= 1e-12 * np.abs(rux).max()
    assert np.abs(uy - ruy).max() <= 1e-12 * np.abs(ruy).max()
    assert rel_err(s.get_state(), ref.f) <= 1e-12
    s.close()


# Lattices that take the FP32 strip-sweep kernel (nx % 4 == 0, nx, ny >= 8):
# one and several strips and segments, ragged strip widths and segment tails.
# At T = 0.9 T_c the quench amplifies FP32 rounding (max relative density
# error ~2e-6 at step 40, ~1.3e-5 at step 80 for both FP32 kernels), so these
# run 40 steps.
SWEEP = [
    (8, 8, True, 0.02, 40),
    (8, 8, False, 0.0, 40),
    (124, 9, False, 0.0, 40),
    (248, 67, True, 0.04, 40),
    (300, 130, True, 0.05, 40),
    (300, 130, False, 0.0, 40),
]


@pytest.mark.parametrize("case", SMALL + SWEEP, ids=lambda c: f"{c[0]}x{c[1]}{'w' if c[2] else 'p'}")
def test_fp32_small_lattices(case):
    w = small_workload(*case)
    n0 = noise_field(w)
    ref = oracle_for(w).init_fields(n0).step(w.steps)
    s = solver_for(w, LB_FP32).init_fields(n0).step(w.steps)
    n, _, _ = s.moments()
    rn, _, _ = ref.moments()
    assert rel_err(n, rn) <= 1e-5
    s.close()


def _fp32_storage_divergence(w, n0, steps):
    """How far the FP64 oracle drifts when its state is rounded to FP32
    after every step (no other change): the floor that FP32 storage alone
    imposes on this workload."""
    a = oracle_for(w).init_fields(n0)
    b = oracle_for(w).init_fields(n0)
    for _ in range(steps):
        a.step(1)
        b.step(1)
        b.f = b.f.astype(np.float32).astype(np.float64)
    na, nb = a.moments()[0], b.moments()[0]
    return float(np.abs(na - nb).max() / np.abs(na).max())


@pytest.mark.parametrize("u_w", [0.01, 0.05])
def test_fp32_config_512x256_1000_steps(u_w):
    """FP32 against the FP64 oracle on the sheared 512x256 quench.

    The noisy symmetric quench is linearly unstable (spinodal
    decomposition): perturbations of FP32 size are amplified ~1e3 between
    steps 100 and 500.  The max relative density error is held to 1e-5 at
    step 100, before the amplification, and at 1000 steps to a multiple of
    the drift that FP32 rounding produces in the oracle itself (its state
    rounded to FP32 after every step).  FP32 arithmetic rounds each
    population ~25 times per step, and the amplification carries that
    excess along: an ablation on this workload put FP32 kernels at 5-17x
    that floor at step 1000 (the paper's term order with IEEE division
    8.6x / 16.6x at U_w = 0.01 / 0.05; this kernel 7.0x / 12.8x, 4.7x /
    10.2x with IEEE division in place of the approximate reciprocal).  The
    bound, 20x, is 1.5x this kernel's largest measured ratio."""
    w = C2(u_w)
    n0 = noise_field(w)
    ref = oracle_for(w).init_fields(n0)
    s = solver_for(w, LB_FP32).init_fields(n0)
    curve = []
    done = 0
    for t in (100, 250, 500, 1000):
        ref.step(t - done)
        s.step(t - done)
        done = t
        n, _, _ = s.moments()
        rn, _, _ = ref.moments()
        curve.append((t, float(np.abs(n - rn).max() / np.abs(rn).max())))
    s.close()
    floor = _fp32_storage_divergence(w, n0, 1000)
    print(f"fp32 error curve (step, max rel density error): {curve}; "
          f"oracle FP32-storage divergence at 1000 steps: {floor:.3e}")
    assert curve[0][1] <= 1e-5, curve
    print(f"ratio to the FP32-storage floor at 1000 steps: {curve[-1][1] / floor:.1f}")
    assert curve[-1][1] <= 20.0 * floor, (curve, floor)


def _settled_droplet():
    """The paper's droplet (Figs. 3-4: R = 15, OVC, tau = 1, T = 0.95 T_c),
    64 x 64 periodic, settled 4000 steps in the oracle."""
    from oracle import maxwell
    w = C1.with_(nx=64, ny=64, walls=False, T=0.95 * TC, A0=0.0, lam=0.0, N=0.3, Q=2.0, u_bot=0.0, u_top=0.0)
    nL, nV = maxwell.coexistence(w.a, w.b, w.T)
    yy, xx = np.mgrid[0:64, 0:64]
    r = np.hypot(xx - 31.5, yy - 31.5)
    return w, oracle_for(w).init_fields(np.where(r < 15, nL, nV)).step(4000)


def _zebra_between_walls():
    """Zebra stripes between static walls (Fig. 7 regime: A0 = 1e-4,
    lambda = 32, T = 0.95 T_c), 128 x 64, settled 6000 steps in the oracle
    from stripes of the coexistence densities."""
    from oracle import maxwell
    w = C1.with_(nx=128, ny=64, walls=True, T=0.95 * TC, A0=1e-4, lam=32.0, N=0.3, Q=2.0,
                 u_bot=0.0, u_top=0.0)
    nL, nV = maxwell.coexistence(w.a, w.b, w.T)
    x = np.arange(128)[None, :] + np.zeros((64, 1))
    n0 = 0.5 * (nL + nV) - 0.5 * (nL - nV) * np.cos(2 * np.pi * x / 32)
    return w, oracle_for(w).init_fields(n0).step(6000)


def _supercritical_shear():
    """A single-phase fluid above the critical point (T = 1.1 T_c) between
    walls at -0.05 / +0.05, 256 x 128, from the noisy quench: the noise and
    the start of the Couette profile decay."""
    w = C2(0.05).with_(nx=256, ny=128, T=1.1 * TC)
    return w, oracle_for(w).init_fields(noise_field(w))


@pytest.mark.parametrize("make", [_settled_droplet, _zebra_between_walls, _supercritical_shear],
                         ids=["droplet", "zebra_between_walls", "supercritical_shear"])
def test_fp32_1000_steps_on_non_amplifying_states(make):
    """FP32 held to 1e-5 max relative density error, site by site, after
    1000 steps against the FP64 oracle, on states whose dynamics damp
    perturbations: a settled droplet, zebra stripes between walls and a
    supercritical sheared flow.  (A two-phase slab under shear is not one of
    them: its error grows from 1.4e-6 at step 250 to 9.5e-6 at step 1000.)  The FP32 run starts from the oracle's
    populations rounded to FP32; the curve is printed."""
    w, ref = make()
    s = solver_for(w, LB_FP32).init_fields(np.ones((w.ny, w.nx)))
    s.set_state(ref.f.astype(np.float32), 0)
    curve = []
    done = 0
    for t in (250, 500, 1000):
        ref.step(t - done)
        s.step(t - done)
        done = t
        n, _, _ = s.moments()
        rn, _, _ = ref.moments()
        curve.append((t, float(np.abs(n - rn).max() / np.abs(rn).max())))
    s.close()
    print(f"{make.__name__}: fp32 error curve (step, max rel density error): {curve}")
    assert all(e <= 1e-5 for _, e in curve), curve


def test_full_size_fp32_one_step():
    """4096x1024 (the benchmark lattice, same launch path): device noise
    init and one step against the oracle on every site."""
    w = C4
    ref = oracle_for(w).init_noise(w.seed, w.rho_mean, w.noise)
    s = solver_for(w, LB_FP32).init_noise(w.seed, w.rho_mean, w.noise)
    f0 = s.get_state()
    assert rel_err(f0, ref.f) <= 6e-8  # FP32 rounding of the FP64 equilibrium
    ref.step(1)
    s.step(1)
    assert rel_err(s.get_state(), ref.f) <= 1e-6
    n, ux, uy = s.moments()
    rn, rux, ruy = ref.moments()
    assert rel_err(n, rn) <= 1e-6
    s.close()


def test_full_size_bench_launches_against_oracle():
    """The benchmark's own launch sequence on 4096x1024: device noise init,
    the autotuner's tiling, a 5-step warm-up launch, then one persistent
    20-step launch; every site's populations and density against 25 oracle
    steps, at the FP32 tolerance of 1e-5."""
    w = C4
    s = solver_for(w, LB_FP32).init_noise(w.seed, w.rho_mean, w.noise)
    seg_h = s.autotune(20)
    s.step(5)
    s.step(20)
    ref = oracle_for(w).init_noise(w.seed, w.rho_mean, w.noise).step(25)
    e_f = rel_err(s.get_state(), ref.f)
    n, ux, uy = s.moments()
    rn, rux, ruy = ref.moments()
    e_n = rel_err(n, rn)
    e_u = max(float(np.abs(ux - rux).max()), float(np.abs(uy - ruy).max()))
    rc, _ = s.reduce()
    s.close()
    print(f"4096x1024, seg_h {seg_h}, 5 + 20 steps: populations {e_f:.2e}, density {e_n:.2e}, "
          f"velocity {e_u:.2e} (absolute)")
    assert rc == 0
    assert e_f <= 1e-5 and e_n <= 1e-5
    # u = (sum_i f_i c_i + F / 2) / n: six populations enter each component,
    # so at the population tolerance (1e-5 of max f ~ 0.5) and n ~ 0.5 the
    # velocity error is at most ~6e-5 in lattice units
    assert e_u <= 6e-5


def test_page_locked_and_pageable_host_arrays_agree():
    """lb_init reads page-locked host fields in place and stages pageable
    ones; lb_moments writes page-locked host arrays from the kernel and
    copies into pageable ones: both routes give the same bits."""
    import torch
    from paper_1307_6703_gb300 import LB_DTYPE_F32, lb_init, lb_moments
    w = C2(0.05)
    n0 = noise_field(w, seed=5)
    u0 = 0.01 * np.sin(2 * np.pi * np.arange(w.nx) / w.nx)[None, :] * np.ones((w.ny, 1))
    v0 = np.zeros_like(n0)
    pinned = [torch.from_numpy(a.copy()).pin_memory() for a in (n0, u0, v0)]
    out = []
    for fields in ((n0, u0, v0), tuple(p.numpy() for p in pinned), (n0, None, None),
                   (pinned[0].numpy(), None, None)):
        s = solver_for(w, LB_FP32)
        if fields[1] is None:
            lb_init(s.h, 1, 0, 0.0, 0.0, fields[0], None, None)
        else:
            lb_init(s.h, 1, 0, 0.0, 0.0, *fields)
        s.step(7)
        host = np.empty((3, w.ny, w.nx), np.float32)
        lb_moments(s.h, host[0], host[1], host[2], LB_DTYPE_F32, 0)
        locked = torch.empty((3, w.ny, w.nx), dtype=torch.float32).pin_memory()
        lb_moments(s.h, locked[0].data_ptr(), locked[1].data_ptr(), locked[2].data_ptr(), LB_DTYPE_F32, 0)
        assert np.array_equal(host, locked.numpy())
        out.append((s.get_state(), host))
        s.close()
    assert np.array_equal(out[0][0], out[1][0]) and np.array_equal(out[0][1], out[1][1])
    assert np.array_equal(out[2][0], out[3][0]) and np.array_equal(out[2][1], out[3][1])


def test_full_size_fp64_one_step_bitwise():
    w = C4
    ref = oracle_for(w).init_noise(3, w.rho_mean, w.noise).step(1)
    s = solver_for(w, LB_FP64).init_noise(3, w.rho_mean, w.noise).step(1)
    assert np.array_equal(s.get_state(), ref.f)
    s.close()


def test_full_size_fp32_mass_conservation():
    w = C4
    s = solver_for(w, LB_FP32).init_noise(w.seed, w.rho_mean, w.noise)
    rc, (m0, _, _) = s.reduce()
    assert rc == 0
    s.step(300)
    rc, (m1, jx, jy) = s.reduce()
    assert rc == 0
    assert abs(m1 - m0) / m0 < 2e-5
    s.close()


def test_checkpoint_resume_is_bitwise():
    w = C2(0.05).with_(nx=96, ny=48)
    a = solver_for(w, LB_FP32).init_noise(5, w.rho_mean, w.noise).step(200)
    b = solver_for(w, LB_FP32).init_noise(5, w.rho_mean, w.noise).step(100)
    state = b.get_state()
    b.close()
    c = solver_for(w, LB_FP32).set_state(state, step=100).step(100)
    assert c.t == 200
    assert np.array_equal(a.get_state(), c.get_state())
    a.close()
    c.close()


def test_instability_is_reported():
    """A poisoned initial field (NaN and a negative density) is caught by
    lb_reduce with LB_ERR_UNSTABLE; the context stays usable."""
    w = C1.with_(nx=32, ny=16)
    n0 = noise_field(w)
    n0[3, 5] = np.nan
    s = solver_for(w, LB_FP32).init_fields(n0).step(3)
    rc, _ = s.reduce()
    assert rc == LB_ERR_UNSTABLE
    n0 = noise_field(w)
    n0[2, 2] = -0.5
    s2 = solver_for(w, LB_FP32).init_fields(n0)
    rc, _ = s2.reduce()
    assert rc == LB_ERR_UNSTABLE
    ok = solver_for(w, LB_FP32).init_fields(noise_field(w)).step(3)
    assert ok.reduce()[0] == 0
    for x in (s, s2, ok):
        x.close()


@pytest.mark.parametrize("storage", ["fp32", "bf16dev"])
def test_reduce_async_matches_reduce(storage):
    """lb_reduce_async: one record per step into a pinned ring, read after
    one synchronisation -- the same sums as lb_reduce (same kernels, so bit
    for bit on the same state), mass conserved step by step, flags clear;
    a poisoned state raises its instability flag without stalling."""
    import torch
    from gpu_util import dev16_solver
    from paper_1307_6703_gb300 import LB_BF16DEV, lb_reduce_async
    w = C2(0.05).with_(nx=256, ny=128)
    s = (solver_for(w, LB_FP32) if storage == "fp32" else dev16_solver(w, LB_BF16DEV, 1.0))
    s.init_noise(2, w.rho_mean, w.noise)
    ring = torch.zeros((6, 5), dtype=torch.float64).pin_memory()
    lb_reduce_async(s.h, ring[0])
    for k in range(1, 6):
        s.step(7)
        lb_reduce_async(s.h, ring[k])
    torch.cuda.synchronize()
    r = ring.numpy().copy()
    rc, vals = s.reduce()
    assert rc == 0 and list(r[5, :3]) == vals
    assert np.all(np.abs(r[:, 0] - r[0, 0]) <= 1e-6 * r[0, 0])
    assert np.all(r[:, 3:] == 0.0)
    s.close()
    n0 = noise_field(C1.with_(nx=32, ny=16))
    n0[3, 5] = np.nan
    bad = solver_for(C1.with_(nx=32, ny=16), LB_FP32).init_fields(n0).step(3)
    out = torch.zeros(5, dtype=torch.float64).pin_memory()
    lb_reduce_async(bad.h, out)
    torch.cuda.synchronize()
    assert out[3].item() == 1.0 and out[4].item() == 0.0
    assert bad.reduce()[0] == LB_ERR_UNSTABLE
    bad.close()


@pytest.mark.parametrize("storage", ["fp32", "bf16dev"])
def test_monitor_ring_records_every_step(storage):
    """lb_monitor: with a pinned ring of 8 records, one lb_step(20) call
    leaves the records of steps 13..20 in host memory, each written by its
    step's kernel into slot (step mod 8): mass conserved, flags clear, the
    last equal to lb_reduce bit for bit; switched off, steps write nothing;
    a batch instance is refused."""
    import torch
    from gpu_util import dev16_solver
    from paper_1307_6703_gb300 import LB_BF16DEV, LB_ERR_ARG, Batch, LBError, lb_monitor, lb_params
    w = C2(0.05).with_(nx=256, ny=128)
    s = (solver_for(w, LB_FP32) if storage == "fp32" else dev16_solver(w, LB_BF16DEV, 1.0))
    s.init_noise(2, w.rho_mean, w.noise)
    ring = torch.full((8, 6), -1.0, dtype=torch.float64).pin_memory()
    s.monitor(ring)
    s.step(20)
    torch.cuda.synchronize()
    r = ring.numpy().copy()
    assert [int(r[i, 5]) for i in range(8)] == [16, 17, 18, 19, 20, 13, 14, 15]
    rc, vals = s.reduce()
    assert rc == 0 and list(r[20 % 8, :3]) == vals
    assert np.all(np.abs(r[:, 0] - vals[0]) <= 1e-6 * vals[0])
    assert np.all(r[:, 3:5] == 0.0)
    s.monitor(None)
    before = ring.clone()
    s.step(5)
    torch.cuda.synchronize()
    assert torch.equal(ring, before)
    s.close()
    b = Batch([lb_params(64, 32, 1, LB_FP32, w.a, w.b, w.T, w.kappa, w.tau, w.A0, 32.0, -0.01, 0.01,
                         w.N, w.Q, 0.0, None)])
    with pytest.raises(LBError) as e:
        lb_monitor(b.views[0].h, ring)
    assert e.value.code == LB_ERR_ARG
    b.close()


def test_concurrent_streams_match_solo_runs():
    """Two lattices stepped in interleaved calls on two streams (each step a
    dependent launch, the last of each call a records step with its own
    arrival counter) end bit for bit where each ends alone, sums included."""
    import torch
    from paper_1307_6703_gb300 import Solver
    w = C2(0.05).with_(nx=256, ny=128)

    def make(stream):
        return Solver(w.nx, w.ny, precision=LB_FP32, walls=w.walls, a=w.a, b=w.b, T=w.T, kappa=w.kappa,
                      tau=w.tau, A0=w.A0, lam=w.lam, u_bot=w.u_bot, u_top=w.u_top, N=w.N, Q=w.Q,
                      stream=stream)
    solo = []
    for seed in (3, 4):
        s = make(None).init_noise(seed, w.rho_mean, w.noise).step(60)
        solo.append((s.get_state(), s.reduce()))
        s.close()
    st = [torch.cuda.Stream(), torch.cuda.Stream()]
    both = [make(st[i].cuda_stream).init_noise(seed, w.rho_mean, w.noise) for i, seed in enumerate((3, 4))]
    for _ in range(6):
        for s in both:
            s.step(10)
    torch.cuda.synchronize()
    for s, (f, red) in zip(both, solo):
        assert np.array_equal(s.get_state(), f)
        assert s.reduce() == red
        s.close()


def test_moments_to_device_and_stream():
    """lb_moments writes device pointers (torch tensors) on a torch stream
    and agrees with the host path."""
    import torch
    from paper_1307_6703_gb300 import LB_DTYPE_F32, Solver, lb_moments
    w = C2(0.01).with_(nx=128, ny=64)
    st = torch.cuda.Stream()
    s = Solver(w.nx, w.ny, precision=LB_FP32, walls=True, a=w.a, b=w.b, T=w.T, kappa=w.kappa,
               tau=w.tau, A0=w.A0, lam=w.lam, u_bot=w.u_bot, u_top=w.u_top, N=w.N, Q=w.Q,
               stream=st.cuda_stream)
    s.init_noise(2, w.rho_mean, w.noise).step(20)
    n = torch.empty((w.ny, w.nx), device="cuda", dtype=torch.float32)
    u = torch.empty_like(n)
    v = torch.empty_like(n)
    lb_moments(s.h, n, u, v, LB_DTYPE_F32, 1)
    st.synchronize()
    hn, hu, hv = s.moments(dtype=np.float32)
    assert np.array_equal(n.cpu().numpy(), hn) and np.array_equal(u.cpu().numpy(), hu)
    s.close()


@pytest.mark.parametrize("prec", [LB_FP32, 2])
def test_autotune_keeps_the_trajectory(prec):
    """lb_autotune restores the state and step counter, and the sweep's
    results do not depend on the segment height it picks (same arithmetic
    per site, only the CTA that computes it changes): bitwise equal."""
    from gpu_util import dev16_solver
    w = C2(0.05).with_(nx=256, ny=200)
    make = (lambda: solver_for(w, prec)) if prec == LB_FP32 else (lambda: dev16_solver(w, prec, 1.0))
    a = make().init_noise(4, w.rho_mean, w.noise).step(10)
    b = make().init_noise(4, w.rho_mean, w.noise).step(10)
    seg = b.autotune(5)
    assert seg in (24, 32, 40, 48, 52, 56, 64, 72, 80, 96, 128, 192, 200)
    assert b.t == 10
    a.step(30)
    b.step(30)
    sa, sb = a.get_state(), b.get_state()
    if prec == LB_FP32:
        assert np.array_equal(sa, sb)
    else:
        assert np.array_equal(sa[0], sb[0]) and np.array_equal(sa[1], sb[1])
    # the per-CTA mass records sum FP32 per-thread partials over each
    # segment, so their rounding depends on the segment height
    ra, rb = a.reduce(), b.reduce()
    assert ra[0] == rb[0] == 0 and abs(ra[1][0] - rb[1][0]) <= 1e-7 * ra[1][0]
    a.close()
    b.close()


@pytest.mark.parametrize("seg", [8, 24, 64, 10 ** 6])
def test_set_seg_h_keeps_the_trajectory(seg):
    """lb_set_seg_h fixes the tiling without tuning (clamped to ny): the
    same state, bitwise, as the default tiling; seg_h < 1 is refused."""
    from paper_1307_6703_gb300 import LB_ERR_ARG, LBError
    w = C2(0.05).with_(nx=256, ny=200)
    a = solver_for(w, LB_FP32).init_noise(4, w.rho_mean, w.noise).step(20)
    b = solver_for(w, LB_FP32).init_noise(4, w.rho_mean, w.noise).set_seg_h(seg).step(20)
    assert np.array_equal(a.get_state(), b.get_state())
    with pytest.raises(LBError) as e:
        b.set_seg_h(0)
    assert e.value.code == LB_ERR_ARG
    a.close()
    b.close()


def test_zero_steps_is_a_no_op():
    w = C2(0.05).with_(nx=96, ny=40)
    s = solver_for(w, LB_FP32).init_noise(3, w.rho_mean, w.noise)
    before = s.get_state()
    s.step(0)
    assert s.t == 0 and np.array_equal(before, s.get_state())
    s.close()


@pytest.mark.parametrize("prec", [LB_FP64, LB_FP32])
def test_uniform_rest_state_is_a_fixed_point(prec):
    """Degenerate case: a uniform fluid at rest between walls at rest with no
    potential stays uniform and at rest (gradients, forces and the wall rule
    all vanish)."""
    w = C2(0.0).with_(nx=128, ny=48, A0=0.0, lam=0.0)
    s = solver_for(w, prec).init_fields(np.full((w.ny, w.nx), 0.8))
    s.step(200)
    n, ux, uy = s.moments()
    tol = 1e-14 if prec == LB_FP64 else 2e-6
    assert np.abs(n - 0.8).max() <= tol and np.abs(ux).max() <= tol and np.abs(uy).max() <= tol
    s.close()


def test_largest_sweep_lattice_matches_fp64():
    """The largest lattice whose padded planes the sweep kernel indexes in
    32 bits (9 * pitch * (ny + 8) < 2^31: 16384 x 13000, 213 M sites): three
    FP32 sweep steps against the FP64 path (bit-identical to the oracle) on
    every site, compared on the device."""
    import torch
    from paper_1307_6703_gb300 import LB_DTYPE_F32, LB_DTYPE_F64, lb_moments
    w = C4.with_(nx=16384, ny=13000)
    pitch = ((w.nx + 8 + 31) // 32) * 32
    assert 9 * pitch * (w.ny + 8) < 2 ** 31
    out = {}
    for prec, dt, code in ((LB_FP64, torch.float64, LB_DTYPE_F64), (LB_FP32, torch.float32, LB_DTYPE_F32)):
        s = solver_for(w, prec).init_noise(9, w.rho_mean, w.noise).step(3)
        n = torch.empty((w.ny, w.nx), dtype=dt, device="cuda")
        lb_moments(s.h, n, None, None, code, 1)
        torch.cuda.synchronize()
        rc, (m, _, _) = s.reduce()
        assert rc == 0
        out[prec] = (n, m)
        s.close()
    n64, m64 = out[LB_FP64]
    n32, m32 = out[LB_FP32]
    err = float(((n32.double() - n64).abs().max() / n64.abs().max()).item())
    assert err <= 1e-6, err
    assert abs(m32 - m64) / m64 <= 1e-6
