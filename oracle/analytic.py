"""Closed-form solutions used to pin the oracle.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

* One-dimensional consolidation (Terzaghi; the paper names it as a standard
  poromechanics check in Sec. 1).  Column of height H drained at the top, no flow
  at the bottom, uniaxial strain, a step load F at t = 0:
     p0  = alpha M F / (K_v + alpha^2 M)              (undrained response)
     c_v = (k/mu) M K_v / (K_v + alpha^2 M),  K_v = lambda + 2 mu
     p(z,t) = (4 p0 / pi) sum_m (-1)^m / (2m+1) cos((2m+1) pi z / 2H)
                         exp(-(2m+1)^2 pi^2 c_v t / 4H^2),
  z measured from the impermeable bottom.  Derived from Eq. fluid_content,
  Eq. darcy_matrix and Eq. stress restricted to one dimension.
* Line source on a planar fault (Theis; Sec. 4.2):
     p(r,t) = dp* E1(r^2 / (4 D t)),  dp* = Q mu / (4 pi w k_par),
     D = w k_par M_F / (mu w)   (fracture storage w / M_F, Sec. 3.2.3).
* Circular frictional rupture, zero Poisson ratio, rigid-plastic limit
  (Sec. 4.2, after Saez et al. 2022): the rupture radius is R = lambda L with
  L = sqrt(4 D t) and lambda the root of
     T = int_0^1 E1(lambda^2 s^2) s / sqrt(1 - s^2) ds,
     T = (1 - tau0 / (f sigma'_0)) / (dp* / sigma'_0).
  This follows from requiring a zero stress-intensity factor at r = R for the
  axisymmetric stress drop f p(r) - f sigma'_0 (1 - tau0 / (f sigma'_0)) of a
  penny-shaped crack (Sneddon's weight r / sqrt(R^2 - r^2)).  For T -> 0,
  lambda -> 1 / sqrt(2 T).
"""
from __future__ import annotations

import math

import numpy as np
from scipy import integrate, optimize, special


def terzaghi_params(E, nu, alpha, M, k, mu, F):
    lam = E * nu / ((1 + nu) * (1 - 2 * nu))
    G = E / (2 * (1 + nu))
    Kv = lam + 2 * G
    p0 = alpha * M * F / (Kv + alpha * alpha * M)
    cv = (k / mu) * M * Kv / (Kv + alpha * alpha * M)
    return p0, cv


def terzaghi_pressure(z, t, H, p0, cv, terms=400):
    z = np.asarray(z, float)
    out = np.zeros_like(z)
    for m in range(terms):
        a = (2 * m + 1) * math.pi / (2 * H)
        out += ((-1) ** m / (2 * m + 1)) * np.cos(a * z) * math.exp(-a * a * cv * t)
    return 4.0 * p0 / math.pi * out


def theis_dpstar(Q, mu, wk_par):
    return Q * mu / (4.0 * math.pi * wk_par)


def fault_diffusivity(wk_par, MF, mu, w):
    return wk_par * MF / (mu * w)


def theis_pressure(r, t, Q, mu, wk_par, MF, w):
    D = fault_diffusivity(wk_par, MF, mu, w)
    return theis_dpstar(Q, mu, wk_par) * special.exp1(np.asarray(r, float) ** 2 / (4 * D * t))


def T_of_lambda(lam):
    """T(lambda) = int_0^1 E1(lambda^2 s^2) s / sqrt(1 - s^2) ds, with s = sin(theta)."""
    f = lambda th: special.exp1((lam * math.sin(th)) ** 2) * math.sin(th)
    val, _ = integrate.quad(f, 0.0, math.pi / 2, limit=400)
    return val


def lambda_of_T(T):
    """Root of T_of_lambda(lambda) = T (T_of_lambda decreases monotonically)."""
    lo, hi = 1e-4, 1e3
    return optimize.brentq(lambda l: T_of_lambda(l) - T, lo, hi, xtol=1e-14, rtol=1e-13)


def stress_injection_parameter(tau0, f, sig0, Q, mu, wk_par):
    return (1.0 - tau0 / (f * sig0)) / (theis_dpstar(Q, mu, wk_par) / sig0)
