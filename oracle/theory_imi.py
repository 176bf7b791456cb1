"""Thin-film surface-plasmon theory on the electron line (test infrastructure).

This file belongs to the oracle: only tests, the smoke check and the bench's
CPU-baseline leg may import it.  Nothing in the CUDA path uses it.

Sec. IV of the paper compares the PIC peaks with the intersections of the
electron line (omega = k*v) and the two dispersion branches of a metal film
(Fig. 2, Table 1).  The film equations come from the paper's ref. [10], which
is not reproduced in the text; they are the standard insulator-metal-insulator
(IMI) results for a film of thickness d in vacuum with a lossless Drude
permittivity eps(omega) = 1 - wp^2/omega^2 (Eq. 1 with gamma -> 0):

    kd = sqrt(k^2 - omega^2/c^2),  km = sqrt(k^2 - eps*omega^2/c^2)
    upper branch:  tanh(km d / 2) = -eps kd / km
    lower branch:  coth(km d / 2) = -eps kd / km

On the electron line k = omega/(beta c).  As d -> infinity both branches go to
eps(omega) = -gamma_L^2, i.e. omega = wp / sqrt(1 + gamma_L^2), the single
entry the paper lists for 150 nm.
"""
from __future__ import annotations

import math

import numpy as np
from scipy.optimize import brentq

C0 = 299792458.0
MEC2_KEV = 510.99895


def beta_of(kev: float) -> float:
    g = 1.0 + kev / MEC2_KEV
    return math.sqrt(1.0 - 1.0 / (g * g))


def _residual(omega: float, wp: float, d: float, beta: float, branch: str) -> float:
    eps = 1.0 - (wp / omega) ** 2
    k = omega / (beta * C0)
    kd = math.sqrt(k * k - (omega / C0) ** 2)
    km = math.sqrt(k * k - eps * (omega / C0) ** 2)
    x = 0.5 * km * d
    # Both branches written without division by tanh/coth singularities:
    # upper: km*tanh(x) + eps*kd = 0 ; lower: km + eps*kd*tanh(x) = 0
    if branch == "upper":
        return km * math.tanh(x) + eps * kd
    return km + eps * kd * math.tanh(x)


def thick_film_omega(wp: float, kev: float) -> float:
    """omega where eps(omega) = -gamma_L^2 (single-interface limit)."""
    g = 1.0 + kev / MEC2_KEV
    return wp / math.sqrt(1.0 + g * g)


def film_modes(wp: float, d: float, kev: float, n_scan: int = 4000):
    """Return (omega_minus, omega_plus) in rad/s: the electron-line crossings
    of the lower (coth) and upper (tanh) film branches.  The metal needs
    eps < 0, so the scan runs over 0 < omega < wp."""
    beta = beta_of(kev)
    grid = np.linspace(1e-3 * wp, wp * (1 - 1e-9), n_scan)
    out = {}
    for branch in ("lower", "upper"):
        vals = np.array([_residual(w, wp, d, beta, branch) for w in grid])
        roots = []
        for a in range(n_scan - 1):
            if vals[a] == 0.0 or vals[a] * vals[a + 1] < 0:
                roots.append(brentq(_residual, grid[a], grid[a + 1],
                                    args=(wp, d, beta, branch), xtol=1e-6, rtol=1e-15))
        out[branch] = roots
    lo = out["lower"][0] if out["lower"] else float("nan")
    hi = out["upper"][0] if out["upper"] else float("nan")
    return lo, hi


def film_modes_thz(wp: float, d: float, kev: float):
    lo, hi = film_modes(wp, d, kev)
    return lo / (2 * math.pi) / 1e12, hi / (2 * math.pi) / 1e12


def branch_omega(wp: float, d: float, k: float, branch: str, n_scan: int = 4000) -> float:
    """omega (rad/s) of a bound film mode of real wavenumber k (rad/m) on the
    given branch ("upper" or "lower"): the same two equations as above with k
    independent of omega, on 0 < omega < min(wp, c k) (below the light line,
    eps < 0).  nan if the branch has no mode at this k."""
    top = min(wp, C0 * k) * (1 - 1e-12)

    def res(omega):
        eps = 1.0 - (wp / omega) ** 2
        kd = math.sqrt(max(k * k - (omega / C0) ** 2, 0.0))
        km = math.sqrt(k * k - eps * (omega / C0) ** 2)
        x = 0.5 * km * d
        if branch == "upper":
            return km * math.tanh(x) + eps * kd
        return km + eps * kd * math.tanh(x)

    grid = np.linspace(1e-3 * top, top, n_scan)
    vals = [res(w) for w in grid]
    for a in range(n_scan - 1):
        if vals[a] == 0.0 or vals[a] * vals[a + 1] < 0:
            return brentq(res, grid[a], grid[a + 1], xtol=1e-6, rtol=1e-15)
    return float("nan")


def single_interface_omega(wp: float, k: float) -> float:
    """Closed form of the lossless Drude surface plasmon on one metal-vacuum
    interface, k^2 = (omega/c)^2 eps/(1+eps): omega^2 = wp^2/2 + (ck)^2 -
    sqrt(wp^4/4 + (ck)^4)."""
    ck = C0 * k
    return math.sqrt(0.5 * wp * wp + ck * ck - math.sqrt(0.25 * wp ** 4 + ck ** 4))

