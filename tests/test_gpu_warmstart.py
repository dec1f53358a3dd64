"""Learned warm start, end to end on the GPU: training data from the solver
(noisy quenches run to their steady striped states at 256x64 and 512x128),
the network trained by its own CUDA forward/backward/Adam kernels, and the
plain solver as arbiter -- steps until the density and velocity stop changing
(max change < 1e-4 per 1000 steps), from the predicted fields against from a
noisy uniform state, on held-out parameter draws at 512x128.  The network
must shorten the run on average; the state reached is the solver's own
either way."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    torch.cuda.set_device(0)
    yield
    torch.cuda.synchronize()


def _initial_params():
    from paper_1307_6703_gb300.workloads import network_pack, network_weights
    return network_pack(network_weights(32, 64, 4, 16, 8, seed=0, outputs=3), 4)


def test_warm_start_shortens_the_run_to_steady_state():
    from paper_1307_6703_gb300 import warmstart as ws
    from paper_1307_6703_gb300.fno import Fno
    ptr = ws.sample_params(512, seed=1)
    n1, d1, _ = ws.generate(ptr[:384], 256, 64, 25000, seed=1)
    n2, d2, _ = ws.generate(ptr[384:], 512, 128, 30000, seed=2)
    k1, k2 = d1 <= ws.STEADY_TOL, d2 <= ws.STEADY_TOL
    assert k1.mean() > 0.9 and k2.mean() > 0.6  # the training states are steady
    net = Fno(width=32, hidden=64, layers=4, modes_x=16, modes_y=8, outputs=3, batch_max=16,
              nx_max=512, ny_max=128, gemm_bf16=True)
    net.set_params(_initial_params())
    hist = ws.train(net, [(ptr[:384][k1], n1[k1]), (ptr[384:][k2], n2[k2])], steps=3000, lr=2e-3)
    assert hist[-1][1] < 0.2 * hist[0][1] and hist[-1][1] < 1e-2
    pte = ws.sample_params(16, seed=99)
    pred = ws.predict(net, pte, 512, 128)
    # the device-side rescale and mass projection against the same steps in
    # numpy on the network's raw output
    import torch
    raw = torch.empty((16, 3, 128, 512), dtype=torch.float32, device="cuda")
    net.forward(torch.tensor(pte, dtype=torch.float32, device="cuda"), 512, 128, raw)
    ref = raw.cpu().numpy().astype(np.float64)
    for j, sc in enumerate(ws.SCALES):
        ref[:, j] *= sc
    ref[:, 0] += 1.0
    ref[:, 0] += 1.0 - ref[:, 0].mean(axis=(1, 2), keepdims=True)
    got = pred.cpu().numpy()
    assert np.abs(got - ref).max() <= 1e-13
    assert np.allclose(got[:, 0].mean(axis=(1, 2)), 1.0, atol=1e-12)
    s_noise = ws.steps_to_steady(pte, 512, 128, None, seed=7)
    s_pred = ws.steps_to_steady(pte, 512, 128, pred, seed=7)
    net.close()
    print(f"steps to steady state, noisy start: mean {s_noise.mean():.0f} {s_noise.tolist()}; "
          f"warm start: mean {s_pred.mean():.0f} {s_pred.tolist()}")
    assert s_pred.mean() <= 0.9 * s_noise.mean()
