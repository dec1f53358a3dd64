"""Learned warm start: training data from the solver itself, the training
loop of the network (include/fno.h), and the measurement of steps to the
steady state that decides whether the network helps.

Every step of the physics runs in the lattice Boltzmann library and every
step of the network in its CUDA kernels; this module only moves buffers and
loops.  The plain solver from a noisy uniform state is both the fallback and
the arbiter: a predicted field is only an initial condition, and the state
it leads to is the solver's.

Steady state (the criterion used throughout): the maximum change of the
density and of the velocity over 1000 steps is below STEADY_TOL, measured
every `block` steps, in the frame that moves with the pattern: the fields
are compared after the periodic shift along x that best overlays them, so
a travelling interface wave that keeps its shape counts as settled.  The
training targets of travelling states are phase-aligned: shifted along x
so that the dominant x-mode of the column masses has zero phase.

The network predicts density and velocity (three output channels, scaled
as (n - 1)/0.5, u_x/0.05, u_y/0.05).  A predicted density is shifted to the
total mass of the noisy state it replaces before the solver starts from it:
the solver conserves mass, so a prediction with the wrong mass would lead
it to a different steady state.
"""
from __future__ import annotations

import math

import numpy as np

from .lb import LB_FP32, Batch, lb_params
from .workloads import TC, Workload

STEADY_TOL = 1e-4          # max |delta n|, |delta u| per 1000 steps
SCALES = (0.5, 0.05, 0.05) # network outputs (n - 1) / 0.5, u_x / 0.05, u_y / 0.05
_NQ = {0.90: (0.3, 2.6), 0.95: (0.3, 2.0)}   # Table 1 rows used in this range


def sample_params(n: int, seed: int, regime: str = "steady") -> np.ndarray:
    """Seeded draws (U_w, A0, lambda, T_r): A0 ~ U[3e-4, 1e-3], lambda 32 or
    64, T_r ~ U[0.925, 0.96], and U_w ~ U[0, 0.035] in the "steady" regime,
    where the solver settles into a static striped state (at 2048 x 512 draws
    with U_w >= 0.04 had not settled after 1.5 M steps), U_w ~ U[0.04, 0.06]
    in the "wave" regime, where the interfaces keep moving."""
    rng = np.random.default_rng(seed)
    out = np.empty((n, 4))
    out[:, 0] = rng.uniform(0.0, 0.035, n) if regime == "steady" else rng.uniform(0.04, 0.06, n)
    out[:, 1] = rng.uniform(3e-4, 1e-3, n)
    out[:, 2] = np.where(rng.integers(0, 2, n) == 0, 32.0, 64.0)
    out[:, 3] = rng.uniform(0.925, 0.96, n)
    return out


def workload(p, nx: int, ny: int, seed: int = 0) -> Workload:
    uw, a0, lam, tr = (float(v) for v in p)
    nq = _NQ[min(_NQ, key=lambda t: abs(t - tr))]
    return Workload(f"ws_{nx}x{ny}", nx, ny, True, tr * TC, 1.0, a0, lam, -uw, uw, nq[0], nq[1], 0,
                    seed=seed)


def _batch(ws, stream=None) -> Batch:
    return Batch([lb_params(w.nx, w.ny, 1, LB_FP32, w.a, w.b, w.T, w.kappa, w.tau, w.A0, w.lam,
                            w.u_bot, w.u_top, w.N, w.Q, 0.0, None) for w in ws], stream=stream)


def _noise(w: Workload) -> np.ndarray:
    rng = np.random.default_rng(w.seed)
    return w.rho_mean + w.noise * rng.uniform(-1.0, 1.0, size=(w.ny, w.nx))


def _fields(b):
    return [np.stack(v.moments(np.float32)) for v in b]   # [3][ny][nx]: n, u_x, u_y


def shift_x(f: np.ndarray, d: float) -> np.ndarray:
    """Fields [..][nx] moved by d sites towards -x (out(x) = f(x + d)),
    periodic, by the Fourier shift theorem."""
    nx = f.shape[-1]
    k = np.arange(nx // 2 + 1)
    return np.fft.irfft(np.fft.rfft(f, axis=-1) * np.exp(2j * np.pi * k * d / nx), n=nx, axis=-1)


def comoving_change(cur: np.ndarray, prev: np.ndarray):
    """Largest change between two field sets [3][ny][nx] (n, u_x, u_y) in
    the frame of the pattern: the displacement d along x that maximises the
    overlap of the two densities (periodic cross-correlation, refined to a
    fraction of a site by a parabola through its peak), then the change
    after moving `cur` back by d; the smaller of that and the plain change,
    with d."""
    plain = float(np.abs(cur - prev).max())
    nx = cur.shape[-1]
    a = cur[0] - cur[0].mean()
    b = prev[0] - prev[0].mean()
    corr = np.fft.irfft((np.fft.rfft(a, axis=1) * np.conj(np.fft.rfft(b, axis=1))).sum(axis=0), n=nx)
    j = int(np.argmax(corr))
    cm, c0, cp = corr[(j - 1) % nx], corr[j], corr[(j + 1) % nx]
    den = cm - 2.0 * c0 + cp
    d = j + (0.5 * (cm - cp) / den if den < 0.0 else 0.0)
    if d > nx / 2:
        d -= nx
    moved = float(np.abs(shift_x(cur, d) - prev).max())
    return min(plain, moved), float(d)


def phase_aligned(f: np.ndarray) -> np.ndarray:
    """Fields [3][ny][nx] shifted along x so that the dominant non-zero
    x-mode of the column masses sum_y n has zero phase."""
    m = f[0].sum(axis=0)
    sp = np.fft.rfft(m - m.mean())
    k = int(np.argmax(np.abs(sp[1:])) + 1)
    return shift_x(f, -np.angle(sp[k]) * f.shape[-1] / (2.0 * np.pi * k))


def generate(params: np.ndarray, nx: int, ny: int, steps: int, seed: int):
    """Run the solver from noisy uniform states for `steps` steps; returns
    the final fields [n][3][ny][nx] (density, u_x, u_y; float32), each
    lattice's change of them over its last 1000 steps in the pattern's
    frame, and whether the pattern moved (by more than a quarter site over
    those steps while its plain change exceeded the tolerance).  The fields
    of moving patterns are phase-aligned."""
    ws = [workload(p, nx, ny, seed * 100003 + i) for i, p in enumerate(params)]
    b = _batch(ws)
    for v, w in zip(b, ws):
        v.init_fields(_noise(w))
    b.step(max(steps - 1000, 0))
    prev = _fields(b)
    b.step(1000)
    cur = _fields(b)
    b.close()
    delta, moving = [], []
    for i, (c, q) in enumerate(zip(cur, prev)):
        ch, d = comoving_change(c, q)
        mv = abs(d) > 0.25 and float(np.abs(c - q).max()) > STEADY_TOL
        delta.append(ch)
        moving.append(mv)
        if mv:
            cur[i] = phase_aligned(c).astype(np.float32)
    return np.stack(cur), np.array(delta), np.array(moving)


def steps_to_steady(params: np.ndarray, nx: int, ny: int, init=None, seed: int = 0,
                    block: int = 500, max_steps: int = 40000) -> np.ndarray:
    """Steps until each lattice is steady (STEADY_TOL), from the given
    initial fields [n][3][ny][nx] (density, u_x, u_y) or, with init=None,
    from noisy uniform states at rest.  max_steps + block where it never
    settles."""
    ws = [workload(p, nx, ny, seed * 100003 + i) for i, p in enumerate(params)]
    b = _batch(ws)
    for i, (v, w) in enumerate(zip(b, ws)):
        if init is None:
            v.init_fields(_noise(w))
        else:
            f = init[i] if hasattr(init, "data_ptr") else np.asarray(init[i], dtype=np.float64)
            v.init_fields(f[0], f[1], f[2])
    prev = _fields(b)
    done = np.full(len(ws), max_steps + block)
    t = 0
    while t < max_steps and (done > max_steps).any():
        b.step(block)
        t += block
        cur = _fields(b)
        for i in range(len(ws)):
            if done[i] > max_steps and comoving_change(cur[i], prev[i])[0] * (1000.0 / block) < STEADY_TOL:
                done[i] = t
        prev = cur
    b.close()
    return done


def train(net, datasets, steps: int, lr: float = 2e-3, batch: int = 16, seed: int = 0, log=None):
    """Adam with a cosine schedule over `steps` steps.  datasets: list of
    (params [n][4], fields [n][3][ny][nx]); each step draws one batch from
    one dataset (alternating), so several lattice sizes train the same
    network.  Returns the loss history."""
    import torch
    rng = np.random.default_rng(seed)
    dev = []
    for prm, n in datasets:
        t = np.asarray(n, dtype=np.float32).copy()
        t[:, 0] -= 1.0
        for j, sc in enumerate(SCALES):
            t[:, j] /= sc
        dev.append((torch.tensor(prm, dtype=torch.float32, device="cuda"),
                    torch.tensor(t, dtype=torch.float32, device="cuda")))
    out = {}
    hist = []
    for k in range(steps):
        prm, tgt = dev[k % len(dev)]
        idx = torch.as_tensor(rng.choice(prm.shape[0], size=min(batch, prm.shape[0]), replace=False),
                              device="cuda")
        p_b, t_b = prm[idx].contiguous(), tgt[idx].contiguous()
        ny, nx = t_b.shape[2], t_b.shape[3]
        key = tuple(t_b.shape)
        if key not in out:
            out[key] = torch.empty(key, dtype=torch.float32, device="cuda")
        net.forward(p_b, nx, ny, out[key])
        loss = net.backward(t_b, want_loss=(k % 50 == 0 or k == steps - 1))
        net.adam(lr * 0.5 * (1.0 + math.cos(math.pi * k / steps)))
        if loss is not None:
            hist.append((k, loss))
            if log:
                log(f"step {k} loss {loss:.4e}")
    return hist


def predict(net, params: np.ndarray, nx: int, ny: int, rho_mean: float = 1.0):
    """Initial fields [n][3][ny][nx] (density, u_x, u_y; float64, on the
    device) for the solver: the network's prediction rescaled and with each
    density shifted to the mean rho_mean, the mass of the noisy uniform
    state it replaces (fno_fields).  Ready for lb_init when it returns."""
    import torch
    prm = torch.tensor(np.asarray(params, dtype=np.float32), device="cuda")
    out = torch.empty((prm.shape[0], net.outputs, ny, nx), dtype=torch.float32, device="cuda")
    net.forward(prm, nx, ny, out)
    fields = torch.empty((prm.shape[0], 3, ny, nx), dtype=torch.float64, device="cuda")
    net.fields(out, nx, ny, SCALES, rho_mean, fields)
    torch.cuda.synchronize()
    return fields
