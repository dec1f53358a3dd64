"""Pins of the oracle's 16-bit deviation storage format (not in the paper).

The format stores d_i = f_i - r_i (i = 1..8) rounded to bfloat16 or IEEE
half and lets the rest population carry the remainder of the site density.
The rounding is pinned against library conversions (numpy's binary16, torch's
bfloat16), hand-worked ties, and the exact invariants of the format: the site
density is unchanged, every stored deviation is a representable number, and
the rounding error is at most half a unit in the last place.  No GPU.
"""
import math

import numpy as np
import pytest
import torch


def _ulp(x: float, p: int, emin: int) -> float:
    e = max(math.frexp(x)[1] - 1, emin) if x != 0.0 else emin
    return 2.0 ** (e - p + 1)


def test_round_fp16_matches_numpy(oracle_mod):
    """binary16 rounding of doubles = numpy's correctly rounded conversion,
    over normal and subnormal magnitudes and both signs."""
    rng = np.random.default_rng(31)
    mags = 10.0 ** rng.uniform(-8.0, 2.0, 4000)
    xs = mags * rng.choice([-1.0, 1.0], mags.size)
    for x in xs:
        assert oracle_mod.round_sig(x, "fp16") == float(np.float16(x)), x


def test_round_bf16_matches_torch(oracle_mod):
    """bfloat16 rounding = torch's float32 -> bfloat16 conversion (round to
    nearest even) on float32-exact inputs."""
    rng = np.random.default_rng(32)
    xs = (10.0 ** rng.uniform(-6.0, 2.0, 4000) * rng.choice([-1.0, 1.0], 4000)).astype(np.float32)
    ref = torch.from_numpy(xs).to(torch.bfloat16).to(torch.float64).numpy()
    for x, r in zip(xs, ref):
        assert oracle_mod.round_sig(float(x), "bf16") == r, x


@pytest.mark.parametrize("fmt,p", [("bf16", 8), ("fp16", 11)])
def test_round_ties_to_even(oracle_mod, fmt, p):
    """Hand-worked midpoints: 1 + u/2 -> 1 (even), 1 + 3u/2 -> 1 + 2u,
    and values just off the midpoint go to the nearer neighbour."""
    u = 2.0 ** (1 - p)
    assert oracle_mod.round_sig(1.0 + u / 2, fmt) == 1.0
    assert oracle_mod.round_sig(1.0 + 3 * u / 2, fmt) == 1.0 + 2 * u
    assert oracle_mod.round_sig(1.0 + u / 2 + 1e-12, fmt) == 1.0 + u
    assert oracle_mod.round_sig(-(1.0 + u / 2 - 1e-12), fmt) == -1.0
    assert oracle_mod.round_sig(0.0, fmt) == 0.0


def _random_state(rng, shape=(6, 7)):
    """Populations near equilibrium at densities 0.5 .. 1.6 (liquid/vapour)."""
    from oracle import feq
    ny, nx = shape
    f = np.zeros((9, ny, nx))
    for y in range(ny):
        for x in range(nx):
            n = rng.uniform(0.5, 1.6)
            ux, uy = rng.uniform(-0.05, 0.05, 2)
            f[:, y, x] = feq(n, ux, uy, 0.3) * (1.0 + 1e-3 * rng.standard_normal(9))
    return f


@pytest.mark.parametrize("fmt", ["bf16", "fp16"])
def test_quantize_invariants(oracle_mod, fmt):
    """Site density unchanged; stored deviations representable; rounding
    error at most half an ulp; unrounded deviations are f_i - r_i."""
    rng = np.random.default_rng(33)
    p, emin = oracle_mod.FORMATS[fmt]
    for rho_ref in (1.0, 3.5, 0.75):
        f = _random_state(rng)
        q, dev = oracle_mod.quantize(f, fmt, rho_ref, want_unrounded=True)
        r = oracle_mod.reference_pops(rho_ref)
        assert r[1] == float(np.float32(rho_ref / 9.0)) and r[5] == float(np.float32(rho_ref / 36.0))
        n0, n1 = f.sum(axis=0), q.sum(axis=0)
        assert np.max(np.abs(n1 - n0) / n0) <= 4e-16
        for i in range(1, 9):
            d = dev[i - 1]
            assert np.array_equal(d, f[i] - r[i])
            dq = q[i] - r[i]
            for a, b in zip(d.ravel(), dq.ravel()):
                assert abs(b - a) <= 0.5 * _ulp(abs(a), p, emin) * (1 + 1e-12)
                if fmt == "fp16":
                    assert float(np.float16(b)) == b
                else:
                    assert float(torch.tensor(b, dtype=torch.float32).to(torch.bfloat16)) == b


@pytest.mark.parametrize("fmt", ["bf16", "fp16"])
def test_quantize_rest_state_at_reference_density(oracle_mod, fmt):
    """At n = rho_ref, u = 0, T = T0 the populations are w_i rho_ref, so the
    deviations are only the FP32 rounding of the references: the stored
    state equals the equilibrium to ~1e-8 (a swapped axis/diagonal reference
    or a wrong weight would leave errors of order 1e-4)."""
    from oracle import feq
    for rho_ref in (1.0, 3.5):
        fe = feq(rho_ref, 0.0, 0.0, 1.0 / 3.0).reshape(9, 1, 1)
        q = oracle_mod.quantize(fe, fmt, rho_ref)
        assert np.max(np.abs(q - fe)) <= 2e-8 * rho_ref
        assert abs(q.sum() - fe.sum()) <= 1e-15 * rho_ref


def test_quantized_step_conserves_mass(oracle_mod):
    """A sheared, walled run through the bfloat16 format: total mass equal to
    the initial mass to round-off (the remainder keeps each site's density)."""
    from oracle import Oracle, Params
    p = Params(nx=24, ny=12, walls=True, a=3 / 8, b=1 / 3, kappa=0.1, T=0.9 / 3, tau=1.0,
               A0=1e-3, lam=24, u_bot=-0.02, u_top=0.02, N=0.3, Q=2.6)
    rng = np.random.default_rng(34)
    o = Oracle(p).init_fields(1.0 + 0.01 * rng.standard_normal((12, 24)))
    o.quantize("bf16", 1.0)
    m0 = o.mass()
    o.step(50, storage=("bf16", 1.0))
    assert abs(o.mass() - m0) <= 1e-13 * m0
