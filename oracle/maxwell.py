"""Equal-area (Maxwell) construction for the van der Waals fluid.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Eq. (eqstate) of the paper: p^w = n T / (1 - b n) - a n^2, derived from the
bulk free energy psi = n T ln(n / (1 - b n)) - a n^2 (the paper writes the
b = 1/3, a = 9/8 case, whose critical point is n_c = T_c = 1).  Coexisting
densities n_V < n_L satisfy p(n_L) = p(n_V) and mu(n_L) = mu(n_V) with
mu = d psi / d n = T ln(n / (1 - b n)) + T / (1 - b n) - 2 a n.  The paper
compares its droplet densities with these values (caption of Fig. 4).
"""
from __future__ import annotations

import math

from scipy.optimize import brentq


def critical_point(a: float, b: float) -> tuple[float, float]:
    """(n_c, T_c) of p = nT/(1-bn) - a n^2: n_c = 1/(3b), T_c = 8a/(27b)."""
    return 1.0 / (3.0 * b), 8.0 * a / (27.0 * b)


def pressure(n, a, b, T):
    return n * T / (1.0 - b * n) - a * n * n


def dpressure(n, a, b, T):
    """c_s^2 = dp/dn = T / (1 - b n)^2 - 2 a n."""
    return T / (1.0 - b * n) ** 2 - 2.0 * a * n


def chem(n, a, b, T):
    return T * math.log(n / (1.0 - b * n)) + T / (1.0 - b * n) - 2.0 * a * n


def dchem(n, a, b, T):
    return dpressure(n, a, b, T) / n


def spinodals(a, b, T):
    nc, Tc = critical_point(a, b)
    if T >= Tc:
        raise ValueError("no spinodal above the critical temperature")
    lo = brentq(lambda n: dpressure(n, a, b, T), 1e-12, nc)
    hi = brentq(lambda n: dpressure(n, a, b, T), nc, (1.0 - 1e-12) / b)
    return lo, hi


def coexistence(a: float, b: float, T: float) -> tuple[float, float]:
    """Return (n_L, n_V) at temperature T < T_c, to ~1e-13 relative."""
    s1, s2 = spinodals(a, b, T)
    p_hi = pressure(s1, a, b, T)
    p_lo = max(pressure(s2, a, b, T), 0.0) + 1e-15

    def vap(P):
        return brentq(lambda n: pressure(n, a, b, T) - P, 1e-14, s1, xtol=1e-15, rtol=1e-15)

    def liq(P):
        return brentq(lambda n: pressure(n, a, b, T) - P, s2, (1.0 - 1e-14) / b,
                      xtol=1e-15, rtol=1e-15)

    def g(P):
        return chem(liq(P), a, b, T) - chem(vap(P), a, b, T)

    P = brentq(g, p_lo + 1e-14 * abs(p_hi), p_hi - 1e-14 * abs(p_hi), xtol=1e-16, rtol=1e-15)
    nL, nV = liq(P), vap(P)
    # Newton polish on the 2x2 system p(nL)=p(nV), mu(nL)=mu(nV).
    for _ in range(8):
        r1 = pressure(nL, a, b, T) - pressure(nV, a, b, T)
        r2 = chem(nL, a, b, T) - chem(nV, a, b, T)
        j11, j12 = dpressure(nL, a, b, T), -dpressure(nV, a, b, T)
        j21, j22 = dchem(nL, a, b, T), -dchem(nV, a, b, T)
        det = j11 * j22 - j12 * j21
        dL = (r1 * j22 - r2 * j12) / det
        dV = (j11 * r2 - j21 * r1) / det
        nL, nV = nL - dL, nV - dV
        if abs(dL) + abs(dV) < 1e-15:
            break
    return nL, nV


def interface_width(kappa: float, T_reduced: float) -> float:
    """Width xi of the approximate tanh profile, Eq. (interface):
    n(x) = n_V + (n_L - n_V)/2 [1 + tanh(x / xi)], xi = sqrt(2 kappa / (1/T - 1)),
    with kappa and T in the paper's reduced units."""
    return math.sqrt(2.0 * kappa / (1.0 / T_reduced - 1.0))
