"""Pins for the oracle of the paper's own discretisation (P1 tetrahedra,
Sec. 3.1) and Cryer's sphere (Sec. 4.1): element identities that hold
exactly for linear fields, Cryer's closed-form centre pressure against a
brute-force radial solve of the same reduced equations, and the 3-D octant
run against that closed form within the paper's 4 % bound."""
import numpy as np
import pytest

import workloads as W
from oracle import analytic as A, tet

E, NU, ALPHA, M, K, MU = 20e9, 0.25, 0.8, 50e9, 1e-15, 1e-3


def random_tet(seed):
    rng = np.random.default_rng(seed)
    X = rng.normal(size=(4, 3))
    G, V = tet.tet_gradients(X[None])
    assert V[0] > 1e-3
    return X


def test_tet_element_identities():
    X = random_tet(3)
    Ke, Ae, Me, Le = (m[0] for m in tet.tet_element_matrices(X[None], E, NU, ALPHA, 1.0 / M, K / MU))
    G, V = tet.tet_gradients(X[None])
    V = V[0]
    assert np.allclose(Ke, Ke.T, rtol=1e-12, atol=1e-3 * np.abs(Ke).max() * 1e-9)
    w = np.linalg.eigvalsh(Ke)
    assert np.sum(np.abs(w) < 1e-9 * w.max()) == 6             # rigid-body modes
    # linear displacement u = H x: Biot work A^T u = alpha (V/4) tr(H) per pressure dof
    H = np.random.default_rng(4).normal(size=(3, 3))
    u = (X @ H.T).reshape(-1)                                    # local dofs 3a + c
    assert np.allclose(Ae.T @ u, ALPHA * V / 4 * np.trace(H), rtol=1e-12)
    # storage integrates 1/M over the volume; Darcy energy of a linear pressure field
    assert np.sum(Me) == pytest.approx(V / M, rel=1e-12)
    g = np.array([0.3, -1.2, 0.7])
    p = X @ g
    assert p @ Le @ p == pytest.approx(K / MU * V * g @ g, rel=1e-12)
    assert np.allclose(Le @ np.ones(4), 0.0, atol=1e-12 * np.abs(Le).max())


def test_cryer_series_matches_radial_finite_volumes():
    """The residue series of Cryer's centre pressure against backward-Euler
    finite volumes of the reduced radial equation: the gap shrinks as the
    radial grid is refined (200, 400, 800 cells), as the finite-volume error
    does."""
    prm = A.cryer_params(E, NU, ALPHA, M, K, MU, 1e6)
    ts = np.array([0.002, 0.01, 0.05, 0.1, 0.2, 0.4])
    T = ts / prm["c"]
    cf = A.cryer_center_pressure(T, 1.0, prm)
    gaps = []
    for J in (200, 400, 800):
        tt, pp = A.cryer_radial_fv(T[-1], 1.0, prm, J=J, steps=8000)
        gaps.append(np.max(np.abs(np.interp(T, tt, pp) - cf)))
    assert gaps[2] < 1.5e-3 and gaps[2] < 0.7 * gaps[1] < 0.7 * 0.7 * gaps[0], gaps
    assert 1.15 < cf.max() < 1.25                                 # Mandel-Cryer rise


def test_cryer_octant_centre_pressure():
    """P1 tetrahedra on an octant of the ball (10 cells per radius, 80 steps):
    the centre pressure follows Cryer's solution within 4 % of its peak (the
    paper's bound, Sec. 4.1), starts at Skempton's undrained value and rises
    above it before it decays."""
    prob = W.cryer_octant(n=10, steps=80)
    _, ts, pc, _, _ = tet.run(prob)
    prm = A.cryer_params(prob.E, prob.nu, prob.alpha, prob.M, prob.k, prob.mu_f, prob.sigma0)
    an = A.cryer_center_pressure(ts, 1.0, prm)
    num = pc / prm["p0"]
    assert np.max(np.abs(num - an)) / an.max() < 0.04
    assert num[0] == pytest.approx(an[0], rel=0.02)
    assert num.max() > 1.1 and num[-1] < 0.05
