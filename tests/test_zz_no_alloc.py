"""lb_reduce_noalloc: the mass / momentum / stability reduction for callers
that cannot allocate device memory (for example a solver embedded in a host
application that owns the whole device memory budget).  Called through the
C ABI on caller-owned device buffers, twice in a row, and compared with the
handle-based lb_reduce within the tolerance of the FP64 parity tests.

This file is collected last on purpose: it must pass on its own in a fresh
process and after every other test."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _state_on_device(torch, w, precision, steps, seed):
    from gpu_util import solver_for
    s = solver_for(w, precision).init_noise(seed, w.rho_mean, w.noise).step(steps)
    rc, ref = s.reduce()
    assert rc == 0
    f = torch.from_numpy(s.get_state()).cuda()
    s.close()
    return f, ref


@pytest.mark.parametrize("prec_name", ["fp64", "fp32"])
def test_noalloc_reduce_matches_lb_reduce_twice(prec_name):
    import torch
    from paper_1307_6703_gb300 import LB_FP32, LB_FP64, lb_reduce_noalloc
    from paper_1307_6703_gb300.workloads import C2

    torch.cuda.set_device(0)
    prec = LB_FP64 if prec_name == "fp64" else LB_FP32
    w = C2(0.05).with_(nx=300, ny=130)
    out = torch.zeros(3, dtype=torch.float64, device="cuda")
    flag = torch.full((1,), 7, dtype=torch.int32, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    for call, (steps, seed) in enumerate(((40, 3), (90, 4))):
        f, ref = _state_on_device(torch, w, prec, steps, seed)
        lb_reduce_noalloc(f, prec, w.nx, w.ny, w.b, out, flag, stream)
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        assert int(flag.item()) == 0, call
        # FP64 states: both sums are FP64 throughout.  FP32 states: lb_reduce
        # reads the per-CTA records of the FP32 step kernel, whose site sums
        # are formed in FP32 (relative accuracy ~1e-7 per site).
        rtol = 1e-12 if prec == LB_FP64 else 2e-6
        assert abs(got[0] - ref[0]) <= rtol * abs(ref[0]), (call, got, ref)
        scale = max(abs(ref[0]) * rtol, 1e-9)
        assert abs(got[1] - ref[1]) <= scale and abs(got[2] - ref[2]) <= scale, (call, got, ref)


def test_noalloc_reduce_flags_bad_state_and_rejects_oversize():
    import torch
    from paper_1307_6703_gb300 import LB_FP32, LBError, lb_reduce_noalloc
    from paper_1307_6703_gb300.workloads import C2

    torch.cuda.set_device(0)
    w = C2(0.01).with_(nx=64, ny=32)
    f, _ = _state_on_device(torch, w, LB_FP32, 10, 1)
    f[0, 5, 7] = float("nan")
    out = torch.zeros(3, dtype=torch.float64, device="cuda")
    flag = torch.zeros(1, dtype=torch.int32, device="cuda")
    lb_reduce_noalloc(f, LB_FP32, w.nx, w.ny, w.b, out, flag, None)
    torch.cuda.synchronize()
    assert int(flag.item()) == 1
    with pytest.raises(LBError):
        lb_reduce_noalloc(f, LB_FP32, w.nx, 16385, w.b, out, flag, None)
