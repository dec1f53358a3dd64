"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Every check here is independent of the oracle's own code: exact moment
identities of the Hermite projections, exactness of the stencils on
polynomials, the closed-form moments of the wall rule, exact conservation
laws, closed-form hydrodynamics (sound dispersion and damping, Couette flow),
the Laplace law, and numbers printed in the paper (tests/golden).  No GPU.
"""
import json
import math
import os

import numpy as np
import pytest

GOLD = os.path.join(os.path.dirname(__file__), "golden")
T0 = 1.0 / 3.0
CX = np.array([0, 1, 0, -1, 0, 1, -1, -1, 1], dtype=float)
CY = np.array([0, 0, 1, 0, -1, 1, 1, -1, -1], dtype=float)

# The paper's parameter set in lattice units (dx = dt = 1, T0 = 1/3):
# a = 9/8 / 3, b = 1/3, kappa = 0.3 / 3, T = T_reduced / 3.
PAPER = dict(a=3.0 / 8.0, b=1.0 / 3.0, kappa=0.1)
TC_PAPER = 1.0 / 3.0


def golden(name):
    with open(os.path.join(GOLD, name)) as fh:
        return json.load(fh)


# --------------------------------------------------------------- identities

def test_feq_moments(oracle_mod):
    """Sec. II: sum f^eq = n, sum f^eq c = n u, sum f^eq cc = n T I + n u u."""
    rng = np.random.default_rng(11)
    for _ in range(200):
        n = rng.uniform(0.2, 7.0)
        ux, uy = rng.uniform(-0.2, 0.2, 2)
        T = rng.uniform(0.1, 0.7)
        f = oracle_mod.feq(n, ux, uy, T)
        assert abs(f.sum() - n) <= 1e-14 * n
        assert abs((f * CX).sum() - n * ux) <= 2e-15 * n
        assert abs((f * CY).sum() - n * uy) <= 2e-15 * n
        assert abs((f * CX * CX).sum() - (n * T + n * ux * ux)) <= 2e-15 * n
        assert abs((f * CY * CY).sum() - (n * T + n * uy * uy)) <= 2e-15 * n
        assert abs((f * CX * CY).sum() - n * ux * uy) <= 2e-15 * n


def test_forcing_moments(oracle_mod):
    """Eq. (forceterm): sum F_i = A = 0, sum F_i c = B, sum F_i cc = C (the
    Hermite projection reproduces its coefficients), and B = (1 - 1/2tau) F."""
    rng = np.random.default_rng(12)
    for _ in range(200):
        tau = rng.uniform(0.55, 3.0)
        T = rng.uniform(0.1, 0.7)
        ux, uy, Fx, Fy, dnx, dny, divJ = rng.uniform(-0.3, 0.3, 7)
        Fi = oracle_mod.forcing(tau, T, ux, uy, Fx, Fy, dnx, dny, divJ)
        g = 1.0 - 1.0 / (2.0 * tau)
        assert abs(Fi.sum()) < 1e-15
        assert abs((Fi * CX).sum() - g * Fx) < 1e-15
        assert abs((Fi * CY).sum() - g * Fy) < 1e-15
        # The second moment is symmetric and traceful; its trace and the
        # velocity-independent part are fixed by the paper's C.
        Sxx = (Fi * CX * CX).sum()
        Syy = (Fi * CY * CY).sum()
        Sxy = (Fi * CX * CY).sum()
        # With u = 0 the only surviving term is (T0 - T) delta div(n u*).
        Fi0 = oracle_mod.forcing(tau, T, 0.0, 0.0, Fx, Fy, dnx, dny, divJ)
        assert abs((Fi0 * CX * CX).sum() - g * (T0 - T) * divJ) < 1e-15
        assert abs((Fi0 * CX * CY).sum()) < 1e-15
        assert abs(Sxy - Sxy.real) == 0 and np.isfinite([Sxx, Syy]).all()


def test_forcing_second_moment_is_guo_stress(oracle_mod):
    """u F + F u enters the second moment with the factor (1 - 1/2tau)."""
    tau, T = 0.9, 0.4
    ux, uy, Fx, Fy = 0.05, -0.03, 0.02, 0.07
    Fi = oracle_mod.forcing(tau, T, ux, uy, Fx, Fy, 0.0, 0.0, 0.0)
    g = 1.0 - 1.0 / (2.0 * tau)
    assert abs((Fi * CX * CX).sum() - g * 2 * ux * Fx) < 1e-16
    assert abs((Fi * CY * CY).sum() - g * 2 * uy * Fy) < 1e-16
    assert abs((Fi * CX * CY).sum() - g * (ux * Fy + Fx * uy)) < 1e-16


@pytest.mark.parametrize("NQ", [(0.5, 1.0), (0.3, 2.0), (0.4, 2.1), (0.0, 0.0), (1.0, 3.9)])
def test_stencils_exact_on_polynomials(oracle_mod, NQ):
    """Eqs. (xstencil, laplstencil) with 2N + 4M = 1, Q + 2R = 1 are exact
    on linear (derivative) and quadratic (Laplacian) fields; d_y(y) = +1."""
    N, Q = NQ
    rng = np.random.default_rng(3)
    for _ in range(50):
        a, b, c, d, e, f0 = rng.uniform(-1, 1, 6)
        x0, y0 = rng.uniform(-5, 5, 2)
        xs, ys = x0 + CX, y0 + CY
        lin = a * xs + b * ys + c
        dx, dy, lap = oracle_mod.stencils(N, Q, lin)
        assert abs(dx - a) < 1e-13 and abs(dy - b) < 1e-13 and abs(lap) < 1e-13
        quad = d * xs * xs + e * ys * ys + f0 * xs * ys
        dx, dy, lap = oracle_mod.stencils(N, Q, quad)
        assert abs(lap - 2 * (d + e)) < 1e-12
        assert abs(dx - (2 * d * x0 + f0 * y0)) < 1e-12
        assert abs(dy - (2 * e * y0 + f0 * x0)) < 1e-12
    dx, dy, lap = oracle_mod.stencils(N, Q, CY.copy())  # phi = y
    assert dy == pytest.approx(1.0, abs=1e-15) and dx == 0.0


def test_standard_choice_is_central_difference(oracle_mod):
    """N = 1/2, M = 0, Q = 1, R = 0 is the standard central scheme (SC)."""
    phi = np.random.default_rng(4).uniform(0, 1, 9)
    dx, dy, lap = oracle_mod.stencils(0.5, 1.0, phi)
    assert dx == pytest.approx(0.5 * (phi[1] - phi[3]), abs=1e-16)
    assert dy == pytest.approx(0.5 * (phi[2] - phi[4]), abs=1e-16)
    assert lap == pytest.approx(phi[1] + phi[2] + phi[3] + phi[4] - 4 * phi[0], abs=1e-15)


@pytest.mark.parametrize("top", [False, True])
def test_wall_rule_moments(oracle_mod, top):
    """Sec. II moving walls: after the rule, sum f = n-hat (mass), and
    n u* = sum f c + F/2 equals (n-hat U, 0): the fluid moves with the wall
    and does not cross it."""
    rng = np.random.default_rng(5 + top)
    for _ in range(100):
        f = rng.uniform(0.01, 0.5, 9)
        g = rng.uniform(0.01, 0.5, 9)
        U, Fx, Fy = rng.uniform(-0.1, 0.1, 3)
        out, nh = oracle_mod.wall(top, U, Fx, Fy, f, g)
        assert abs(out.sum() - nh) < 1e-14
        assert abs((out * CX).sum() + 0.5 * Fx - nh * U) < 1e-15
        assert abs((out * CY).sum() + 0.5 * Fy) < 1e-15
        # Only the unknown links and the rest population were rebuilt.
        known = [1, 3, 4, 7, 8] if not top else [1, 3, 2, 5, 6]
        assert np.array_equal(out[known], f[known])


def test_splitmix64_published_outputs(oracle_mod):
    gold = golden("splitmix64.json")
    seq = [int(s) for s in gold["seed_1234567"]]
    # orc_noise_field maps output k to amp*(2U-1), U = (out >> 11) * 2^-53.
    field = oracle_mod.noise_field(len(seq), 1, 1234567, 0.0, 1.0)[0]
    expect = [((z >> 11) * 2.0 ** -53) * 2.0 - 1.0 for z in seq]
    assert np.array_equal(field, np.array(expect))
    z0 = int(gold["seed_0_first"], 16)
    assert oracle_mod.noise_field(1, 1, 0, 0.0, 1.0)[0, 0] == ((z0 >> 11) * 2.0 ** -53) * 2.0 - 1.0


def test_maxwell_matches_paper():
    from oracle import maxwell
    g = golden("paper_values.json")["maxwell_T095"]
    nL, nV = maxwell.coexistence(9.0 / 8.0, 1.0 / 3.0, g["T_reduced"])
    assert round(nL, 6) == g["n_L"] and round(nV, 6) == g["n_V"]
    # The same densities in lattice units (p scaled by 1/3).
    nL2, nV2 = maxwell.coexistence(3.0 / 8.0, 1.0 / 3.0, g["T_reduced"] / 3.0)
    assert abs(nL2 - nL) < 1e-12 and abs(nV2 - nV) < 1e-12


# ------------------------------------------------------- whole-step physics

def _noisy(oracle_mod, **kw):
    p = oracle_mod.Params(**kw)
    return oracle_mod.Oracle(p)


@pytest.mark.parametrize("walls", [True, False])
def test_mass_conservation(oracle_mod, walls):
    """Collision conserves mass (A = 0) and every population that leaves
    through a wall is counted in n-hat, so total mass is exact up to
    rounding, also with moving walls and the periodic force."""
    o = _noisy(oracle_mod, nx=64, ny=32, walls=walls, T=0.9 * TC_PAPER, tau=1.0,
               A0=1e-3, lam=32, u_bot=-0.03, u_top=0.03, N=0.3, Q=2.6, **PAPER)
    o.init_noise(7, 1.0, 0.01 / 3.5)
    m0 = o.mass()
    o.step(2000)
    # rounding only: a few ulp per site and step (sites x steps x eps ~ 1e-12)
    assert abs(o.mass() - m0) / m0 < 1e-12


def test_uniform_translation_is_fixed_point(oracle_mod):
    """A uniform state moving with velocity U is stationary (Galilean
    invariance of the equilibrium, no spurious force on a uniform field)."""
    p = oracle_mod.Params(nx=8, ny=6, walls=False, T=0.95 * TC_PAPER, tau=0.9,
                          N=0.3, Q=2.0, **PAPER)
    o = oracle_mod.Oracle(p).init_fields(np.full((6, 8), 1.3), np.full((6, 8), 0.07),
                                         np.full((6, 8), -0.02))
    o.step(200)
    n, ux, uy = o.moments()
    assert np.abs(n - 1.3).max() < 1e-13
    assert np.abs(ux - 0.07).max() < 1e-14 and np.abs(uy + 0.02).max() < 1e-14


def _fit_sound(oracle_mod, a, b, T, kappa, tau, n0, L=128, steps=2500):
    from scipy.optimize import curve_fit
    from oracle import maxwell
    p = oracle_mod.Params(nx=L, ny=1, walls=False, a=a, b=b, T=T, kappa=kappa,
                          tau=tau, N=0.3, Q=2.0)
    k = 2 * math.pi / L
    x = np.arange(L)
    o = oracle_mod.Oracle(p).init_fields((n0 * (1 + 1e-5 * np.cos(k * x)))[None, :])
    ts, ys = [], []
    for _ in range(steps):
        n, _, _ = o.moments()
        ts.append(o.t)
        ys.append((np.sum((n[0] - n0) * np.cos(k * x)) * 2 / L))
        o.step(1)
    ts, ys = np.array(ts, float), np.array(ys)
    # Linearised Navier-Stokes of Eq. (nav) with the force of Eq. (force2):
    # omega^2 = (dp^w/dn + kappa n0 k^2) k^2, amplitude decay nu k^2 with
    # nu = eta / n = T0 (tau - 1/2)  (eta = n (tau - dt/2) in the paper's units).
    w0 = math.sqrt(maxwell.dpressure(n0, a, b, T) + kappa * n0 * k * k) * k
    g0 = T0 * (tau - 0.5) * k * k

    def model(t, A, w, g, ph):
        return A * np.cos(w * t + ph) * np.exp(-g * t)

    popt, _ = curve_fit(model, ts, ys, p0=[ys[0], w0, g0, 0.0])
    return popt[1] / w0, popt[2] / g0


@pytest.mark.parametrize("case", [
    # T above T0 (the temperature term of f^eq and the (T0 - T) terms of C
    # are large): vdW constants a = 9/49, b = 2/21 at 1.2 T_c.
    dict(a=9 / 49, b=2 / 21, T=1.2 * 4 / 7, kappa=0.049, tau=1.0, n0=3.5),
    dict(a=9 / 49, b=2 / 21, T=1.2 * 4 / 7, kappa=0.049, tau=0.8, n0=3.5),
    # T below T0: the paper's set at 1.1 T_c, two relaxation times.
    dict(a=3 / 8, b=1 / 3, T=1.1 / 3, kappa=0.1, tau=1.0, n0=1.0),
    dict(a=3 / 8, b=1 / 3, T=1.1 / 3, kappa=0.1, tau=2.0, n0=1.0),
])
def test_sound_dispersion_and_damping(oracle_mod, case):
    """Sound speed from the vdW equation of state (Eq. eqstate) plus the
    kappa term, and viscous damping with bulk = shear viscosity
    eta = n T0 (tau - 1/2).  A dropped or mis-signed (T0 - T) term of C, a
    wrong EOS or a wrong viscosity shifts these by several percent."""
    rw, rg = _fit_sound(oracle_mod, **case)
    assert abs(rw - 1) < 3e-3, rw
    assert abs(rg - 1) < 1e-2, rg


def test_couette_profile_is_exact(oracle_mod):
    """Homogeneous fluid between walls moving at -U and +U relaxes to the
    linear Couette profile u* = (U (2y/(Ny-1) - 1), 0) (Sec. IV)."""
    ny, U = 17, 0.02
    p = oracle_mod.Params(nx=4, ny=ny, walls=True, T=1.1 * TC_PAPER, tau=1.0,
                          u_bot=-U, u_top=U, N=0.3, Q=2.0, **PAPER)
    o = oracle_mod.Oracle(p).init_fields(np.full((ny, 4), 1.0))
    o.step(8000)
    n, ux, uy = o.moments()
    y = np.arange(ny)
    assert np.abs(ux - (-U + 2 * U * y / (ny - 1))[:, None]).max() < 1e-12
    assert np.abs(uy).max() < 1e-12
    assert np.abs(n - 1.0).max() < 1e-12


def _flat_interface(oracle_mod, tau=1.0, ny=128, steps=20000, Tr=0.95, ux=None):
    from oracle import maxwell
    T = Tr * TC_PAPER
    nL, nV = maxwell.coexistence(PAPER["a"], PAPER["b"], T)
    p = oracle_mod.Params(nx=1, ny=ny, walls=False, T=T, tau=tau, N=0.3, Q=2.0, **PAPER)
    y = np.arange(ny)
    n0 = nV + (nL - nV) * 0.5 * (np.tanh((y - ny / 4) / 3) - np.tanh((y - 3 * ny / 4) / 3))
    o = oracle_mod.Oracle(p).init_fields(n0[:, None])
    o.step(steps)
    return o


def _discrete_balance_solve(n_init, T, Fext=None):
    """Static 1D states of the scheme without running it.

    At a steady state at rest (u* = 0, so C = 0 and n u* = 0) with variation
    along one lattice axis only, the moments of propagation plus collision
    (Eqs. evoleq, newvel, forceterm, coeff) reduce to two site-by-site
    balances, whatever tau is:
      momentum: D_c(n T) = F + (1/4) lap F,    mass: lap(n T) = D_c F,
    with D_c the central difference, lap the 3-point Laplacian and F the
    force of Eq. (force2) plus F_ext (the stencils of Eqs. xstencil and
    laplstencil reduce to D_c and lap on such fields for any N, Q).  The
    (1/4) lap F term is the lattice's own trapezoidal treatment of the force
    (F/2 in Eq. newvel): the scheme balances the force against the pressure
    over a link, (F_y + F_(y+1))/2 = T (n_(y+1) - n_y).  These equations and
    the mass fix n(y); they are solved here by least squares from the same
    initial profile, with no lattice Boltzmann step."""
    from scipy.optimize import least_squares
    a, b, kappa = PAPER["a"], PAPER["b"], PAPER["kappa"]
    n_init = np.asarray(n_init, dtype=np.float64)
    Fext = np.zeros_like(n_init) if Fext is None else Fext
    mass = n_init.sum()
    dc = lambda f: 0.5 * (np.roll(f, -1) - np.roll(f, 1))
    lap = lambda f: np.roll(f, -1) + np.roll(f, 1) - 2.0 * f

    def resid(n):
        pw = n * T / (1.0 - b * n) - a * n * n
        F = dc(n * T - pw) + kappa * n * dc(lap(n)) + Fext
        return np.concatenate([dc(n * T) - F - 0.25 * lap(F), lap(n * T) - dc(F), [n.sum() - mass]])

    sol = least_squares(resid, n_init, xtol=1e-15, ftol=1e-15, gtol=1e-15, max_nfev=4000)
    assert np.abs(sol.fun).max() < 1e-13
    return sol.x


def test_flat_interface_is_the_schemes_discrete_balance(oracle_mod):
    """The oracle's flat interface (20,000 steps, periodic 1 x 128) has the
    bulk densities of the static state of the discrete moment balances,
    solved without any lattice Boltzmann step, to 1e-12 relative; its
    density and force fields satisfy the momentum balance to rounding.  A dropped F/2,
    a wrong forcing coefficient or a wrong propagation would move the state
    far beyond that."""
    from oracle import maxwell
    o = _flat_interface(oracle_mod)
    n, ux, uy, Fx, Fy = o.moments(forces=True)
    n, F = n[:, 0], Fy[:, 0]
    T = 0.95 * TC_PAPER
    dc = lambda f: 0.5 * (np.roll(f, -1) - np.roll(f, 1))
    lap = lambda f: np.roll(f, -1) + np.roll(f, 1) - 2.0 * f
    assert np.abs(dc(n * T) - F - 0.25 * lap(F)).max() < 1e-14
    assert np.abs(uy).max() < 1e-12
    ny = len(n)
    y = np.arange(ny)
    nL, nV = maxwell.coexistence(PAPER["a"], PAPER["b"], T)
    n_init = nV + (nL - nV) * 0.5 * (np.tanh((y - ny / 4) / 3) - np.tanh((y - 3 * ny / 4) / 3))
    nb = _discrete_balance_solve(n_init, T)
    # bulk densities (the interfaces may sit a few 1e-6 sites apart: the
    # balances fix the profile up to a translation)
    assert abs(n.max() - nb.max()) <= 1e-12 * nL and abs(n.min() - nb.min()) <= 1e-12 * nL
    # Mechanical equilibrium holds exactly, p^w(n_L) = p^w(n_V); the bulk
    # densities sit below Maxwell's (n_L -0.62 %, n_V -2.99 %) because of the
    # (1/4) lap F term, which no reading of the printed equations removes
    # (see the design notes' table of readings).
    dp = maxwell.pressure(n[64], PAPER["a"], PAPER["b"], T) - maxwell.pressure(n[0], PAPER["a"], PAPER["b"], T)
    assert abs(dp) < 1e-8
    assert abs(n[64] / nL - 1 + 0.00624) < 5e-4 and abs(n[0] / nV - 1 + 0.02989) < 5e-4


def test_phase_diagram_independent_of_tau(oracle_mod):
    """Sec. III: the equilibrium densities do not depend on tau (the paper
    reports < 1 %); for the static flat interface they agree to rounding."""
    a = _flat_interface(oracle_mod, tau=1.0).moments()[0][:, 0]
    b = _flat_interface(oracle_mod, tau=2.0, steps=40000).moments()[0][:, 0]
    assert np.abs(a - b).max() < 1e-9


def test_galilean_boost_of_flat_interface(oracle_mod):
    """A flat interface translated along itself with velocity U stays
    unchanged (up to O(U^2)) and moves with U: the uF + Fu and (T0 - T) u dn
    parts of C remove the spurious stresses."""
    rest = _flat_interface(oracle_mod)
    n_rest = rest.moments()[0]
    for U in (0.02, 0.04):
        o = oracle_mod.Oracle(rest.p).init_fields(n_rest, np.full_like(n_rest, U), None)
        r = oracle_mod.Oracle(rest.p).init_fields(n_rest)
        o.step(4000)
        r.step(4000)
        n, ux, uy = o.moments()
        nr, _, uyr = r.moments()
        # Same density profile and transverse flow as the interface at rest
        # (both started from the equilibrium populations of the same profile).
        assert np.abs(n - nr).max() < 1e-10
        assert np.abs(uy - uyr).max() < 1e-13
        # Moves with the boost; the residual slip is proportional to U.
        assert np.abs(ux - U).max() < 1e-3 * U


def test_interface_profile_width(oracle_mod):
    """Eq. (interface): tanh profile of width sqrt(2 kappa / (1/T - 1)) in
    reduced units (an approximate solution; 15 % tolerance)."""
    from scipy.optimize import curve_fit
    from oracle import maxwell
    o = _flat_interface(oracle_mod)
    n = o.moments()[0][:, 0]
    nL, nV = n[64], n[0]
    y = np.arange(128)

    def prof(yy, y0, xi):
        return nV + (nL - nV) * 0.5 * (1 + np.tanh((yy - y0) / xi))

    popt, _ = curve_fit(prof, y[5:60], n[5:60], p0=[32, 3])
    xi = maxwell.interface_width(0.3, 0.95)
    assert abs(popt[1] / xi - 1) < 0.15


def test_droplet_matches_paper(oracle_mod):
    """Figs. 3-4: droplet R = 15, kappa = 0.3, tau = 1, OVC, T = 0.95:
    bulk n_L = 1.462721, n_V = 0.580015 and maximum spurious velocity 0.002
    (Fig. 12 caption)."""
    from oracle import maxwell
    g = golden("paper_values.json")
    d = g["droplet_T095"]
    T = d["T_reduced"] * TC_PAPER
    nL, nV = maxwell.coexistence(PAPER["a"], PAPER["b"], T)
    L = 64
    p = oracle_mod.Params(nx=L, ny=L, walls=False, T=T, tau=d["tau"], N=d["N"], Q=d["Q"], **PAPER)
    yy, xx = np.mgrid[0:L, 0:L]
    r = np.hypot(xx - L / 2 + 0.5, yy - L / 2 + 0.5)
    o = oracle_mod.Oracle(p).init_fields(np.where(r < d["R"], nL, nV))
    o.step(6000)
    n, ux, uy = o.moments()
    assert abs(n[L // 2, L // 2] / d["n_L"] - 1) < 0.005
    assert abs(n[0, 0] / d["n_V"] - 1) < 0.005
    umax = np.hypot(ux, uy).max()
    # printed to one digit: 0.002 stands for [0.0015, 0.0025)
    u_paper = g["spurious_velocity_T095"]["u_max"]
    assert 0.75 * u_paper <= umax < 1.25 * u_paper


def test_laplace_law(oracle_mod):
    """p^w(n_in) - p^w(n_out) = sigma / R for droplets, sigma = kappa int n'^2
    from the flat interface (square-gradient free energy of Sec. II)."""
    from oracle import maxwell
    T = 0.95 * TC_PAPER
    flat = _flat_interface(oracle_mod).moments()[0][:, 0]
    dn = 0.5 * (np.roll(flat, -1) - np.roll(flat, 1))
    sigma = PAPER["kappa"] * np.sum(dn ** 2) / 2.0
    nL, nV = maxwell.coexistence(PAPER["a"], PAPER["b"], T)
    L = 96
    for R in (16, 22):
        p = oracle_mod.Params(nx=L, ny=L, walls=False, T=T, tau=1.0, N=0.3, Q=2.0, **PAPER)
        yy, xx = np.mgrid[0:L, 0:L]
        r = np.hypot(xx - L / 2 + 0.5, yy - L / 2 + 0.5)
        o = oracle_mod.Oracle(p).init_fields(nV + (nL - nV) * 0.5 * (1 - np.tanh((r - R) / 3)))
        o.step(10000)
        n = o.moments()[0]
        nin, nout = n[L // 2, L // 2], n[0, 0]
        Req = math.sqrt((n.sum() - nout * L * L) / (nin - nout) / math.pi)
        dp = maxwell.pressure(nin, PAPER["a"], PAPER["b"], T) - maxwell.pressure(nout, PAPER["a"], PAPER["b"], T)
        assert abs(dp * Req / sigma - 1) < 0.05, (R, dp * Req / sigma)


def test_zebra_phase_at_rest(oracle_mod):
    """Fig. 7 (top): zebra phase with A0 = 1e-4, lambda = 32, tau = 1,
    kappa = 0.3, T = 0.95.  The oracle's stripes equal the static state of
    the discrete moment balances with the periodic force (solved without
    any lattice Boltzmann step) to 1e-9 relative.  The paper prints bulk
    values 1.459906 / 0.580089; this scheme's own fixed point sits 0.76 % /
    3.06 % below them, as the flat interface sits below Maxwell, and no
    reading of the printed equations closes that gap (design notes, table
    of readings), so the printed values bound the result only loosely."""
    z = golden("paper_values.json")["zebra_T095"]
    T = z["T_reduced"] * TC_PAPER
    p = oracle_mod.Params(nx=32, ny=1, walls=False, T=T, tau=z["tau"],
                          A0=z["A0"], lam=z["lambda"], N=0.3, Q=2.0, **PAPER)
    o = oracle_mod.Oracle(p).init_noise(1, 1.0, 0.003)
    o.step(60000)
    n, ux, _ = o.moments()
    n = n[0]
    x = np.arange(32)
    n_init = n.mean() + 0.44 * np.cos(2 * np.pi * (x - 16) / 32)
    nb = _discrete_balance_solve(n_init, T, z["A0"] * np.sin(2 * np.pi * x / z["lambda"]))
    assert np.abs(n - nb).max() <= 1e-9 * n.max()  # the force fixes the stripes' position
    assert abs(n.max() / z["n_L"] - 1 + 0.0076) < 1e-3
    assert abs(n.min() / z["n_V"] - 1 + 0.0306) < 1e-3
    # One liquid and one vapour stripe per wavelength, the liquid where the
    # force converges (x = lambda / 2).
    assert np.argmax(n) == 16 and np.argmin(n) == 0


def test_table1_stencil_optima(oracle_mod):
    """Table 1 at T = 0.95 (droplet R = 15, kappa = 0.3, tau = 1): over
    N in {0.2, 0.3, 0.4} at the table's Q values the largest spurious
    velocity is smallest at N = 0.3, the OVC row's N, and the density error
    |n_L^th - n_L| + |n_V^th - n_V| is smallest at N = 0.4, the ODC row's N.
    (A full scan, N in [0, 1] by 0.1 and Q in [0, 4] by 0.1, finds the same
    two N; along Q both measures vary by a few percent only, so Q itself is
    not pinned.)  The standard central scheme (0.5, 1.0) has larger spurious
    velocities than OVC (Fig. 2)."""
    from oracle import maxwell
    T = 0.95 * TC_PAPER
    nL, nV = maxwell.coexistence(PAPER["a"], PAPER["b"], T)
    L = 64
    yy, xx = np.mgrid[0:L, 0:L]
    r = np.hypot(xx - L / 2 + 0.5, yy - L / 2 + 0.5)

    def droplet(N, Q):
        p = oracle_mod.Params(nx=L, ny=L, walls=False, T=T, tau=1.0, N=N, Q=Q, **PAPER)
        o = oracle_mod.Oracle(p).init_fields(np.where(r < 15, nL, nV)).step(2000)
        n, ux, uy = o.moments()
        return float(np.hypot(ux, uy).max()), abs(n[L // 2, L // 2] - nL) + abs(n[0, 0] - nV)

    for Q in (2.0, 2.1):
        res = {N: droplet(N, Q) for N in (0.2, 0.3, 0.4)}
        assert min(res, key=lambda N: res[N][0]) == 0.3, res
        assert min(res, key=lambda N: res[N][1]) == 0.4, res
    assert droplet(0.5, 1.0)[0] > 2.0 * droplet(0.3, 2.0)[0]


def test_workload_parameter_readings():
    """The literal vdW constants a = 9/49, b = 2/21 (n_c = 3.5, T_c = 4/7)
    with kappa = 0.049, A0 = 0.05 diverge in this scheme within a few hundred
    steps of a noisy quench at 0.9 T_c; the paper's own parameter set at the
    same lattice, temperature ratio and the paper's force amplitude stays
    finite.  This is why the workloads use the paper's set."""
    import oracle
    from paper_1307_6703_gb300.workloads import C1, noise_field

    lit = oracle.Params(nx=64, ny=32, walls=True, a=9 / 49, b=2 / 21, T=0.9 * 4 / 7,
                        kappa=0.049, tau=1.0, A0=0.05, lam=32, N=0.3, Q=2.6)
    o = oracle.Oracle(lit).init_noise(1, 3.5, 0.01)
    blew_up = False
    for _ in range(6):
        o.step(100)
        if not np.isfinite(o.f).all():
            blew_up = True
            break
    assert blew_up

    w = C1
    o = oracle.Oracle(oracle.Params(**w.physics())).init_fields(noise_field(w))
    o.step(w.steps)
    n, ux, uy = o.moments()
    assert np.isfinite(o.f).all() and n.min() > 0 and n.max() < 1 / w.b
