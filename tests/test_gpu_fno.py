"""The warm-start network's CUDA forward and backward passes against the
FP64 CPU reference (oracle/fno.py): outputs and loss directly, gradients
against central finite differences of the reference loss, for sampled
entries of every parameter group.  With FP32 GEMMs the agreement is FP32
rounding; with BF16 GEMM inputs (8 significant bits) it is the BF16
rounding of the activations."""
import numpy as np
import pytest

from oracle import fno as ref
from paper_1307_6703_gb300.workloads import network_weights

pytestmark = pytest.mark.gpu

CFG = dict(width=8, hidden=16, layers=2, modes_x=8, modes_y=4, outputs=3)
NX, NY = 64, 16
PARAMS = np.array([[0.03, 6e-4, 32.0, 0.95], [0.0, 3e-4, 64.0, 0.93]])


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    torch.cuda.set_device(0)
    yield
    torch.cuda.synchronize()


def pack(p, layers):
    """Flat parameter vector in the order include/fno.h documents."""
    parts = [p["P"], p["p"]]
    for l in range(layers):
        parts += [p[f"W{l}"], p[f"w{l}"], p[f"Rr{l}"], p[f"Ri{l}"]]
    parts += [p["Q1"], p["q1"], p["Q2"], p["q2"]]
    return np.concatenate([np.asarray(a, dtype=np.float64).ravel() for a in parts])


def unpack(flat, p, layers):
    out, at = {}, 0
    names = ["P", "p"] + sum([[f"W{l}", f"w{l}", f"Rr{l}", f"Ri{l}"] for l in range(layers)], []) + ["Q1", "q1", "Q2", "q2"]
    for n in names:
        sz = p[n].size
        out[n] = np.asarray(flat[at:at + sz], dtype=np.float64).reshape(p[n].shape)
        at += sz
    return out


def _reference_params(seed):
    p = network_weights(CFG["width"], CFG["hidden"], CFG["layers"], CFG["modes_x"], CFG["modes_y"], seed,
                        outputs=CFG["outputs"])
    rng = np.random.default_rng(seed + 1)
    for k in list(p):  # exercise the biases and scale the spectral weights up
        if k in ("p", "q1", "q2") or k.startswith("w"):
            p[k] = 0.1 * rng.standard_normal(p[k].shape)
        if k.startswith("R"):
            p[k] = p[k] * 20.0
    return p


def _gpu_run(p, target, bf16):
    import torch
    from paper_1307_6703_gb300.fno import Fno
    net = Fno(**CFG, batch_max=2, nx_max=NX, ny_max=NY, gemm_bf16=bf16)
    net.set_params(pack(p, CFG["layers"]).astype(np.float32))
    prm = torch.tensor(PARAMS, dtype=torch.float32, device="cuda")
    out = torch.empty((2, CFG["outputs"], NY, NX), dtype=torch.float32, device="cuda")
    net.forward(prm, NX, NY, out)
    loss = net.backward(torch.tensor(target, dtype=torch.float32, device="cuda"))
    grads = unpack(net.get_grads(), p, CFG["layers"])
    o = out.cpu().numpy().astype(np.float64)
    net.close()
    return o, loss, grads


def _fd_checks(p, x, target, grads, rng, per_group=4):
    """(analytic, finite-difference) pairs for sampled entries of each group."""
    L = CFG["layers"]
    pairs = {}
    for name, g in grads.items():
        idx = rng.choice(g.size, size=min(per_group, g.size), replace=False)
        got = []
        for i in idx:
            h = 1e-6
            pp = {k: v.copy() for k, v in p.items()}
            pp[name].ravel()[i] += h
            lp = ref.loss(pp, x, target, L, CFG["modes_x"], CFG["modes_y"])
            pp[name].ravel()[i] -= 2 * h
            lm = ref.loss(pp, x, target, L, CFG["modes_x"], CFG["modes_y"])
            got.append((g.ravel()[i], (lp - lm) / (2 * h)))
        pairs[name] = np.array(got)
    return pairs


@pytest.mark.parametrize("bf16", [False, True], ids=["fp32-gemm", "bf16-gemm"])
def test_network_forward_and_gradients(bf16):
    p = _reference_params(3)
    x = ref.features(PARAMS, NX, NY)
    rng = np.random.default_rng(4)
    target = rng.standard_normal((2, CFG["outputs"], NY, NX)) * 0.5
    out, loss, grads = _gpu_run(p, target, bf16)
    o_ref = ref.forward(p, x, CFG["layers"], CFG["modes_x"], CFG["modes_y"])
    l_ref = ref.loss(p, x, target, CFG["layers"], CFG["modes_x"], CFG["modes_y"])
    tol_out, tol_g = (2e-5, 2e-3) if not bf16 else (3e-2, 8e-2)
    assert np.abs(out - o_ref).max() <= tol_out * max(np.abs(o_ref).max(), 1.0)
    assert abs(loss - l_ref) <= tol_out * l_ref
    pairs = _fd_checks(p, x, target, grads, rng)
    allg = np.concatenate([v for v in pairs.values()])
    scale = np.abs(allg[:, 1]).max()
    for name, v in pairs.items():
        err = np.abs(v[:, 0] - v[:, 1])
        gscale = max(np.abs(v[:, 1]).max(), 1e-3 * scale)
        assert np.all(err <= tol_g * gscale + 1e-7), (name, v)
    cos = float(allg[:, 0] @ allg[:, 1] / (np.linalg.norm(allg[:, 0]) * np.linalg.norm(allg[:, 1])))
    assert cos >= (0.99999 if not bf16 else 0.99)


def test_adam_step_matches_the_update_rule():
    """One Adam step from zero moments moves every parameter by
    -lr * g / (|g| + eps') (bias-corrected first step)."""
    import torch
    from paper_1307_6703_gb300.fno import Fno
    p = _reference_params(5)
    net = Fno(**CFG, batch_max=2, nx_max=NX, ny_max=NY, gemm_bf16=False)
    flat = pack(p, CFG["layers"]).astype(np.float32)
    net.set_params(flat)
    prm = torch.tensor(PARAMS, dtype=torch.float32, device="cuda")
    out = torch.empty((2, CFG["outputs"], NY, NX), dtype=torch.float32, device="cuda")
    net.forward(prm, NX, NY, out)
    net.backward(torch.zeros((2, CFG["outputs"], NY, NX), dtype=torch.float32, device="cuda"))
    g = net.get_grads().astype(np.float64)
    net.adam(1e-3, 0.9, 0.999, 1e-8)
    new = net.get_params().astype(np.float64)
    expect = flat - 1e-3 * g / (np.abs(g) + 1e-8)
    assert np.abs(new - expect).max() <= 1e-6
    net.close()


def test_fields_from_the_network_output():
    """fno_fields against the same steps in numpy: rescale the three output
    channels, then shift each density to the mean rho_mean (FP64, each
    operation rounded once); batches outside 1..8192 are refused."""
    import torch
    from paper_1307_6703_gb300.fno import Fno, fno_fields
    from paper_1307_6703_gb300.lb import LBError
    net = Fno(**CFG, batch_max=2, nx_max=NX, ny_max=NY, gemm_bf16=False)
    rng = np.random.default_rng(11)
    B, scales, rho_mean = 3, (0.5, 0.05, 0.05), 0.93
    raw = rng.standard_normal((B, CFG["outputs"], NY, NX)).astype(np.float32)
    out = torch.tensor(raw, device="cuda")
    fields = torch.empty((B, 3, NY, NX), dtype=torch.float64, device="cuda")
    net.fields(out, NX, NY, scales, rho_mean, fields)
    torch.cuda.synchronize()
    ref = raw[:, :3].astype(np.float64)
    for j, sc in enumerate(scales):
        ref[:, j] *= sc
    ref[:, 0] += 1.0
    ref[:, 0] += rho_mean - ref[:, 0].mean(axis=(1, 2), keepdims=True)
    got = fields.cpu().numpy()
    assert np.abs(got - ref).max() <= 1e-13
    assert np.allclose(got[:, 0].mean(axis=(1, 2)), rho_mean, atol=1e-13)
    for bad in (0, 8193):
        with pytest.raises(LBError):
            fno_fields(net.h, out, bad, NX, NY, scales, rho_mean, fields)
    net.close()
