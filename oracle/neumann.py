"""Closed-form Neumann solution of the two-phase Stefan problem (Sec. 2).

Test infrastructure only (see ``oracle/__init__.py``).  With equal phase
properties (rho = k = alpha = 1, as in the paper's enthalpy model):

* Eq. (3): lambda solves  exp(-l^2)/erf(l) + theta0 exp(-l^2)/erfc(l) = l sqrt(pi)/Ste,
  found here by bisection;
* Eq. (2): the interface is x_f = 2 lambda sqrt(t); the liquid is
  theta_l = 1 - erf(x/2sqrt t)/erf(lambda), the solid
  theta_s = theta0 - theta0 erfc(x/2sqrt t)/erfc(lambda).

Lattice mapping (Sec. 5, end): tau - 1/2 = 3 dt/dx^2, so after ``steps``
steps on ``n`` nodes spanning [0, L] (dx = L/(n-1)) the time is
steps * (tau - 1/2) dx^2 / 3.
"""
from __future__ import annotations

import math

import numpy as np
from scipy.special import erf, erfc


def stefan_residual(lam, ste, theta0, k=1.0, alpha=1.0, rho=1.0):
    """Left minus right side of Eq. (3)."""
    sa = math.sqrt(alpha)
    return (math.exp(-lam * lam) / math.erf(lam)
            + theta0 * k / sa * math.exp(-lam * lam / alpha) / math.erfc(lam / sa)
            - rho * lam * math.sqrt(math.pi) / ste)


def stefan_lambda(ste, theta0, k=1.0, alpha=1.0, rho=1.0, tol=1e-15):
    """Root of Eq. (3) by bisection.  The residual is +inf at 0+ and
    decreasing through zero for theta0 <= 0."""
    lo, hi = 1e-12, 1.0
    while stefan_residual(hi, ste, theta0, k, alpha, rho) > 0.0:
        hi *= 2.0
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if stefan_residual(mid, ste, theta0, k, alpha, rho) > 0.0:
            lo = mid
        else:
            hi = mid
        if hi - lo <= tol * hi:
            break
    return 0.5 * (lo + hi)


def front(t, lam):
    """Interface position x_f = 2 lambda sqrt(t)."""
    return 2.0 * lam * np.sqrt(t)


def profile(x, t, ste, theta0, lam=None):
    """Temperature of Eq. (2) at positions ``x`` and time ``t`` > 0."""
    if lam is None:
        lam = stefan_lambda(ste, theta0)
    x = np.asarray(x, dtype=np.float64)
    eta = x / (2.0 * np.sqrt(t))
    liquid = 1.0 - erf(eta) / math.erf(lam)
    solid = theta0 - theta0 * erfc(eta) / math.erfc(lam)
    return np.where(x <= front(t, lam), liquid, solid)


def lattice_time(steps, n, tau, length=1.0):
    """Physical (dimensionless) time after ``steps`` steps on ``n`` nodes over [0, length]."""
    dx = length / (n - 1)
    return steps * (tau - 0.5) * dx * dx / 3.0
