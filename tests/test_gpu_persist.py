"""The multi-step sweeps (lb_step and lb_batch_step with nsteps >= 2: one
cooperative launch per chunk of steps, (step, item) tickets and per-item
completion counters in place of a grid-wide barrier between steps) against
one launch per step (lb_step(1) / lb_batch_step(1) repeated) and against the
FP64 oracle.

Both launch forms run the same per-site arithmetic on the same items; they
are different kernels, compiled separately, so they are compared to FP32
rounding (and reported bit for bit when they agree exactly).  Batches cover
one and many lattices, one and several strips and segments, walls and
periodic rows (whose tiles depend on the opposite edge through the ghost
images), tilings with more items than resident CTAs (each CTA then works
through several items per step) and odd step counts.
"""
import numpy as np
import pytest

from gpu_util import dev16_solver, oracle_for, rel_err, solver_for

pytestmark = pytest.mark.gpu

from paper_1307_6703_gb300 import LB_BF16DEV, LB_FP16DEV, LB_FP32, Batch  # noqa: E402
from paper_1307_6703_gb300.workloads import C2, batch_workloads, noise_field  # noqa: E402

CASES = [
    # (nx, ny, walls, seg_h, steps)
    (8, 8, True, None, 7),
    (96, 40, False, 8, 9),
    (256, 200, True, 24, 12),
    (256, 200, False, 24, 12),
    (600, 130, True, 16, 11),
]


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    torch.cuda.set_device(0)
    yield
    torch.cuda.synchronize()


def _solver(w, prec):
    return solver_for(w, prec) if prec == LB_FP32 else dev16_solver(w, prec, 1.0)


def _state_diff(prec, a, b):
    """(difference, bitwise): FP32 max relative difference of the
    populations; 16-bit storage: rest planes within FP32 rounding and
    deviation codes at most one unit apart (a rounding decision moved)."""
    if prec == LB_FP32:
        return rel_err(a, b.astype(np.float64)), np.array_equal(a, b)
    d = np.abs(a[1].astype(np.int32) - b[1].astype(np.int32))
    return max(rel_err(a[0], b[0].astype(np.float64)), float(d.max() > 1)), \
        np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])


def _pair(ws, prec, seg=None):
    """Two batches of the same lattices from the same initial fields."""
    out = []
    for _ in range(2):
        alone = [_solver(w, prec) for w in ws]
        b = Batch([s.params for s in alone])
        for s in alone:
            s.close()
        for v, w in zip(b, ws):
            v.init_fields(noise_field(w))
            if seg:
                v.set_seg_h(seg)
        out.append(b)
    return out


@pytest.mark.parametrize("prec", [LB_FP32, LB_BF16DEV, LB_FP16DEV])
@pytest.mark.parametrize("case", CASES, ids=lambda c: f"{c[0]}x{c[1]}{'w' if c[2] else 'p'}s{c[3]}")
def test_multistep_matches_single_steps(case, prec):
    nx, ny, walls, seg, steps = case
    w = C2(0.05).with_(nx=nx, ny=ny, walls=walls, u_bot=-0.05 if walls else 0.0,
                       u_top=0.05 if walls else 0.0, lam=float(nx // 2))
    a, b = _pair([w], prec, seg)
    for _ in range(steps):
        a.step(1)
    b.step(steps)
    va, vb = a[0], b[0]
    assert va.t == vb.t == steps
    err, same = _state_diff(prec, va.get_state(), vb.get_state())
    print(f"{nx}x{ny} prec {prec}: max rel diff {err:.2e}, bitwise {same}")
    assert err <= 2e-6
    ra, rb = va.reduce(), vb.reduce()
    assert ra[0] == rb[0] == 0
    assert abs(ra[1][0] - rb[1][0]) <= 1e-7 * ra[1][0]
    a.close()
    b.close()


@pytest.mark.parametrize("prec", [LB_FP32, LB_BF16DEV, LB_FP16DEV])
@pytest.mark.parametrize("case", CASES, ids=lambda c: f"{c[0]}x{c[1]}{'w' if c[2] else 'p'}s{c[3]}")
def test_single_lattice_multistep_matches_single_steps(case, prec):
    nx, ny, walls, seg, steps = case
    w = C2(0.05).with_(nx=nx, ny=ny, walls=walls, u_bot=-0.05 if walls else 0.0,
                       u_top=0.05 if walls else 0.0, lam=float(nx // 2))
    a = _solver(w, prec).init_fields(noise_field(w))
    b = _solver(w, prec).init_fields(noise_field(w))
    if seg:
        a.set_seg_h(seg)
        b.set_seg_h(seg)
    for _ in range(steps):
        a.step(1)
    b.step(steps)
    assert a.t == b.t == steps
    err, same = _state_diff(prec, a.get_state(), b.get_state())
    print(f"single {nx}x{ny} prec {prec}: max rel diff {err:.2e}, bitwise {same}")
    assert err <= 2e-6
    ra, rb = a.reduce(), b.reduce()
    assert ra[0] == rb[0] == 0
    assert abs(ra[1][0] - rb[1][0]) <= 1e-7 * ra[1][0]
    a.close()
    b.close()


def test_single_lattice_multistep_full_size():
    """The 4096 x 1024 workload at the tilings the autotuner tries (48- and
    24-row segments: 792 and 1548 tiles, more than one wave of CTAs): 12
    steps in one launch against 12 launches, and the fused sums of the last
    step against a fresh reduction of the same state."""
    from paper_1307_6703_gb300.workloads import C4
    for seg in (48, 24):
        a = solver_for(C4, LB_FP32).init_noise(7, C4.rho_mean, C4.noise).set_seg_h(seg)
        b = solver_for(C4, LB_FP32).init_noise(7, C4.rho_mean, C4.noise).set_seg_h(seg)
        for _ in range(12):
            a.step(1)
        b.step(12)
        err, same = _state_diff(LB_FP32, a.get_state(), b.get_state())
        print(f"4096x1024 seg {seg}: max rel diff {err:.2e}, bitwise {same}")
        assert err <= 2e-6
        ra, rb = a.reduce(), b.reduce()
        assert ra[0] == rb[0] == 0 and abs(ra[1][0] - rb[1][0]) <= 1e-7 * ra[1][0]
        a.close()
        b.close()


@pytest.mark.parametrize("prec", [LB_FP32, LB_BF16DEV])
def test_multistep_ensemble_matches_single_steps(prec):
    """The 64-lattice ensemble of uneven sizes, 21 steps in one multi-step
    launch (odd, so it ends on the other buffer parity) against 21 single
    batch steps."""
    ws = batch_workloads(64, seed=11)
    a, b = _pair(ws, prec)
    for _ in range(21):
        a.step(1)
    b.step(21)
    worst, all_same = 0.0, True
    for va, vb in zip(a, b):
        err, same = _state_diff(prec, va.get_state(), vb.get_state())
        worst, all_same = max(worst, err), all_same and same
        assert va.reduce()[0] == 0
    print(f"ensemble prec {prec}: max rel diff {worst:.2e}, bitwise {all_same}")
    assert worst <= 2e-6
    a.close()
    b.close()


def test_multistep_against_oracle_with_many_items_per_cta():
    """8-row and 5-row segments on 1024 x 512: 576 and 927 items, the
    latter more than one wave of resident CTAs, so CTAs work through
    several items per step in step order; 30 steps against the oracle."""
    w = C2(0.05).with_(nx=1024, ny=512, lam=256.0)
    n0 = noise_field(w)
    ref = oracle_for(w).init_fields(n0).step(30)
    for seg in (8, 5):
        s = solver_for(w, LB_FP32)
        b = Batch([s.params])
        s.close()
        v = b[0]
        v.init_fields(n0)
        v.set_seg_h(seg)
        b.step(30)
        assert rel_err(v.get_state(), ref.f) <= 1e-5
        rc, (m, _, _) = v.reduce()
        assert rc == 0 and abs(m - ref.mass()) <= 1e-6 * ref.mass()
        b.close()


def test_multistep_after_retiling_and_restore():
    """Counters restart when the work list is rebuilt (a lattice re-tiled
    or restored alone in between): a run interrupted by both ends where an
    uninterrupted run ends."""
    w = C2(0.05).with_(nx=512, ny=256, lam=128.0)
    ws = [w, w.with_(nx=256, ny=128, lam=64.0)]
    a, b = _pair(ws, LB_FP32)
    a.step(40)
    b.step(10)
    b[0].set_seg_h(32)
    b.step(11)
    b[1].set_state(b[1].get_state(), 21)
    b.step(19)
    for va, vb in zip(a, b):
        assert va.t == vb.t == 40
        err, _ = _state_diff(LB_FP32, va.get_state(), vb.get_state())
        assert err <= 2e-6
    a.close()
    b.close()


@pytest.mark.parametrize("steps", [2, 63, 64, 65, 150])
def test_monitor_across_multistep_launches(steps):
    """While monitoring, a multi-step launch covers at most 64 steps, each
    with its own record slot and arrival counter: every step's record lands
    in the host ring, and the last equals lb_reduce bit for bit."""
    import torch
    w = C2(0.05).with_(nx=256, ny=128)
    s = solver_for(w, LB_FP32).init_noise(2, w.rho_mean, w.noise)
    cap = 200
    ring = torch.full((cap, 6), -1.0, dtype=torch.float64).pin_memory()
    s.monitor(ring)
    s.step(steps)
    torch.cuda.synchronize()
    r = ring.numpy().copy()
    got = sorted(int(v) for v in r[:, 5] if v >= 0)
    assert got == list(range(1, steps + 1))
    rc, vals = s.reduce()
    assert rc == 0 and list(r[steps % cap, :3]) == vals
    assert np.all(np.abs(r[r[:, 5] >= 0, 0] - vals[0]) <= 1e-6 * vals[0])
    assert np.all(r[r[:, 5] >= 0, 3:5] == 0.0)
    s.close()


@pytest.mark.parametrize("cap,steps", [(5, 23), (1, 7)])
def test_monitor_ring_smaller_than_the_run(cap, steps):
    """A ring of fewer records than steps: each record holds the latest
    step of its residue (s mod cap), the last equal to lb_reduce bit for
    bit."""
    import torch
    w = C2(0.05).with_(nx=256, ny=128)
    s = solver_for(w, LB_FP32).init_noise(3, w.rho_mean, w.noise)
    ring = torch.full((cap, 6), -1.0, dtype=torch.float64).pin_memory()
    s.monitor(ring)
    s.step(steps)
    torch.cuda.synchronize()
    r = ring.numpy().copy()
    latest = {s_ % cap: s_ for s_ in range(1, steps + 1)}
    assert [int(r[k, 5]) for k in range(cap)] == [latest[k] for k in range(cap)]
    rc, vals = s.reduce()
    assert rc == 0 and list(r[steps % cap, :3]) == vals
    assert np.all(r[:, 3:5] == 0.0)
    s.close()
