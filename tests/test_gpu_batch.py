"""Batched solver (lb_batch_*): many independent lattices in one launch per
step.  Every instance must follow the trajectory it follows alone, through
plain launches, the two-step CUDA graph, odd step counts, instances stepped
or restored individually in between, and the autotuner.  The batched and the
single-lattice kernels evaluate the same formulas but are compiled
separately, and the compiler is free to fuse a multiply and an add
differently in each, so the two agree to FP32 rounding rather than bit for
bit; each batched instance is also checked against the oracle."""
import numpy as np
import pytest

from gpu_util import dev16_solver, oracle_for, rel_err, solver_for

pytestmark = pytest.mark.gpu

from paper_1307_6703_gb300 import LB_BF16DEV, LB_FP16DEV, LB_FP32, Batch  # noqa: E402
from paper_1307_6703_gb300.workloads import batch_workloads, noise_field  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    torch.cuda.set_device(0)
    yield
    torch.cuda.synchronize()


def _ensemble(count, prec):
    ws = batch_workloads(count, seed=11)
    if prec != LB_FP32:  # 16-bit storage: nx a multiple of 8 (all multiples of 32 here)
        pass
    return ws


def _make(ws, prec):
    alone = [solver_for(w, prec) if prec == LB_FP32 else dev16_solver(w, prec, 1.0) for w in ws]
    batch = Batch([s.params for s in alone])
    for s, v, w in zip(alone, batch, ws):
        n0 = noise_field(w)
        s.init_fields(n0)
        v.init_fields(n0)
    return alone, batch


def _same(a, b, steps=10):
    """FP32: relative difference of the populations at FP32-rounding level
    (2e-6 after ~10 steps, as the FP32 parity tests allow).  16-bit storage:
    a rounding decision moved by an FP32 ulp changes a stored deviation by
    one 16-bit unit (2.4e-4 at |d| ~ 0.05), so few deviations may differ and
    those by about one unit."""
    sa, sb = a.get_state(), b.get_state()
    if isinstance(sa, tuple):
        from gpu_util import decode_dev
        da, db = decode_dev(sa[1], "bf16"), decode_dev(sb[1], "bf16")
        frac = float(np.mean(da != db))
        return frac <= 1e-2 and np.abs(da - db).max() <= 2e-3 and np.abs(sa[0] - sb[0]).max() <= 2e-3
    return rel_err(sa, sb.astype(np.float64)) <= 2e-6 * max(1.0, steps / 10)


@pytest.mark.parametrize("prec", [LB_FP32, LB_BF16DEV, LB_FP16DEV], ids=["fp32", "bf16dev", "fp16dev"])
def test_batch_matches_instances_alone(prec):
    ws = _ensemble(7, prec)
    alone, batch = _make(ws, prec)
    # plain step, graph pairs, odd counts
    for k in (1, 4, 3, 2):
        batch.step(k)
        for s in alone:
            s.step(k)
    for s, v in zip(alone, batch):
        assert v.t == s.t == 10
        assert _same(s, v)
        rs, rv = s.reduce(), v.reduce()
        assert rs[0] == rv[0] == 0 and abs(rs[1][0] - rv[1][0]) <= 1e-7 * rs[1][0]
    for s in alone:
        s.close()
    batch.close()


def test_batch_instance_touched_in_between():
    """An instance stepped alone, or restored from a checkpoint, between
    batch steps: the batch picks up its new buffer parity."""
    ws = _ensemble(4, LB_FP32)
    alone, batch = _make(ws, LB_FP32)
    batch.step(3)
    batch[1].step(1)          # instance 1 alone
    state = batch[2].get_state()
    batch[2].set_state(state, step=3)  # restore instance 2 (same state)
    batch.step(2)
    steps = [5, 6, 5, 5]
    for s, n in zip(alone, steps):
        s.step(n)
    for s, v in zip(alone, batch):
        assert _same(s, v)
    for s in alone:
        s.close()
    batch.close()


def test_batch_instance_against_oracle():
    """One instance of a stepped batch against the FP64 oracle."""
    ws = _ensemble(3, LB_FP32)
    ws = [w.with_(nx=min(w.nx, 256), ny=min(w.ny, 96)) for w in ws]
    batch = Batch([solver_for(w, LB_FP32).params for w in ws])
    n0s = [noise_field(w) for w in ws]
    for v, n0 in zip(batch, n0s):
        v.init_fields(n0)
    batch.step(40)
    for v, w, n0 in zip(batch, ws, n0s):
        ref = oracle_for(w).init_fields(n0).step(40)
        n, _, _ = v.moments()
        assert rel_err(n, ref.moments()[0]) <= 1e-5
    batch.close()


def test_batch_autotune_keeps_trajectories():
    ws = _ensemble(6, LB_FP32)
    alone, batch = _make(ws, LB_FP32)
    batch.step(5)
    segs = batch.autotune(3)
    assert len(segs) == 6 and all(1 <= s_ <= w.ny for s_, w in zip(segs, ws))
    batch.step(7)
    for s in alone:
        s.step(12)
    for s, v in zip(alone, batch):
        assert v.t == 12 and _same(s, v, 12)
    for s in alone:
        s.close()
    batch.close()


def test_batch_ensemble_is_stable():
    """The 64-lattice ensemble of the batch benchmark stays physical for
    3000 steps (every instance's lb_reduce returns LB_OK)."""
    from paper_1307_6703_gb300.workloads import batch_workloads
    ws = batch_workloads(64, seed=7)
    batch = Batch([solver_params(w) for w in ws])
    for v, w in zip(batch, ws):
        v.init_fields(noise_field(w))
    batch.step(3000)
    bad = [i for i, v in enumerate(batch) if v.reduce()[0] != 0]
    batch.close()
    assert bad == []


def solver_params(w):
    from paper_1307_6703_gb300 import lb_params
    return lb_params(w.nx, w.ny, int(w.walls), LB_FP32, w.a, w.b, w.T, w.kappa, w.tau, w.A0, w.lam,
                     w.u_bot, w.u_top, w.N, w.Q, 0.0, None)
