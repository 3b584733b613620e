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
* Cryer's sphere (Sec. 4.1): a sphere of radius R, drained at its surface,
  under a suddenly applied uniform compressive surface traction sigma0.  With
  spherical symmetry the displacement is irrotational, so equilibrium makes
  K_v eps - alpha p = g(t) uniform in space (K_v = lambda + 2G); the surface
  traction fixes g in terms of the volume mean <p>, and the fluid balance
  becomes
     dp/dt = c lap(p) - beta d<p>/dt,    c = (k/mu) / S,  S = 1/M + alpha^2/K_v,
     beta = 4 G alpha^2 / (3 K K_v S)    (K = lambda + 2G/3),
  with the undrained start p0 = alpha sigma0 / (K S (1 + beta)).  Laplace
  transform and residues give the centre pressure
     p(0,t)/p0 = sum_i -2 eta (1 - xi_i / sin xi_i) / (xi_i h'(xi_i))
                 exp(-xi_i^2 c t / R^2),
     xi h'(xi) = (xi cot xi + xi^2 / sin^2 xi - 2) / xi^2,
  over the positive roots of (1 - eta xi^2) tan xi = xi, eta = (1 + beta)/(3 beta).
  The reduced equation is also solved by radial finite volumes (the pin).

Pinned by: tests/test_oracle_analytic.py (lambda(T) limits for small and large
T, the consolidation series at t = 0 and late times, the scale dp*) and
tests/test_golden.py (T of the printed cases); Cryer's series against the
radial finite volumes in tests/test_oracle_tet.py.
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


def cryer_params(E, nu, alpha, M, k, mu, sigma0):
    """Coefficients of Cryer's problem (see the module docstring)."""
    lam = E * nu / ((1 + nu) * (1 - 2 * nu))
    G = E / (2 * (1 + nu))
    Kv = lam + 2 * G
    K = lam + 2 * G / 3
    S = 1.0 / M + alpha * alpha / Kv
    beta = 4 * G * alpha * alpha / (3 * K * Kv * S)
    return dict(c=(k / mu) / S, beta=beta, eta=(1 + beta) / (3 * beta),
                p0=alpha * sigma0 / (K * S * (1 + beta)))


def cryer_roots(eta, n):
    """First n positive roots of (1 - eta xi^2) sin xi - xi cos xi = 0."""
    f = lambda x: (1 - eta * x * x) * math.sin(x) - x * math.cos(x)
    roots = []
    grid = np.linspace(1e-3, (n + 2) * math.pi, 200 * (n + 2))
    vals = [f(x) for x in grid]
    for a, b, fa, fb in zip(grid[:-1], grid[1:], vals[:-1], vals[1:]):
        if fa == 0.0:
            roots.append(a)
        elif fa * fb < 0:
            roots.append(optimize.brentq(f, a, b, xtol=1e-15, rtol=1e-15))
        if len(roots) == n:
            break
    return np.array(roots)


def cryer_center_pressure(t, R, prm, n_terms=400):
    """p(0, t) / p0 for t > 0 (series above)."""
    xi = cryer_roots(prm["eta"], n_terms)
    s, c = np.sin(xi), np.cos(xi)
    xh = (xi * c / s + xi * xi / (s * s) - 2.0) / (xi * xi)       # xi h'(xi)
    amp = -2.0 * prm["eta"] * (1.0 - xi / s) / xh
    t = np.atleast_1d(np.asarray(t, float))
    return np.array([np.sum(amp * np.exp(-xi * xi * prm["c"] * ti / (R * R))) for ti in t])


def cryer_radial_fv(t_end, R, prm, J=400, steps=4000):
    """The reduced radial equation by finite volumes (nodes r_j = j R / J,
    p_J = 0) and backward Euler from the uniform start p0: returns the times
    and p(0, t) / p0."""
    h = R / J
    r = np.arange(J + 1) * h
    rp = np.minimum(r + h / 2, R)
    rm = np.maximum(r - h / 2, 0.0)
    V = (rp ** 3 - rm ** 3) / 3.0                       # control volumes (times 4 pi)
    A = np.zeros((J + 1, J + 1))
    for j in range(J):
        if j + 1 <= J:
            g = rp[j] ** 2 / h
            A[j, j] -= g
            A[j, j + 1] += g
        if j >= 1:
            g = rm[j] ** 2 / h
            A[j, j] -= g
            A[j, j - 1] += g
    L = A / V[:, None]                                  # div grad on the control volumes
    w = 3.0 * V / R ** 3                                # <p> = w . p
    dt = t_end / steps
    c, beta = prm["c"], prm["beta"]
    n = J                                               # unknowns p_0 .. p_{J-1}
    Mtx = np.eye(n) - dt * c * L[:n, :n] + beta * np.outer(np.ones(n), w[:n])
    lu = __import__("scipy.linalg", fromlist=["lu_factor"]).lu_factor(Mtx)
    from scipy.linalg import lu_solve
    p = np.ones(n)
    out_t, out_p = [0.0], [1.0]
    for k in range(1, steps + 1):
        rhs = p + beta * np.dot(w[:n], p)
        p = lu_solve(lu, rhs)
        out_t.append(k * dt)
        out_p.append(p[0])
    return np.array(out_t), np.array(out_p)
