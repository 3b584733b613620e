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


def test_tet_element_energy_and_storage_quadrature():
    """Values, not only structure: the strain energy of a linear displacement
    equals V (lambda tr(eps)^2 + 2 mu eps:eps) with eps = sym(H) (isotropic
    Hooke's law, Sec. 2.1), and the storage energy of a linear pressure equals
    (1/M) times its square integrated by the degree-2 exact four-point rule on
    the tetrahedron (Keast), which shares nothing with the closed-form matrix."""
    X = random_tet(7)
    Ke, _, Me, _ = (m[0] for m in tet.tet_element_matrices(X[None], E, NU, ALPHA, 1.0 / M, K / MU))
    _, V = tet.tet_gradients(X[None])
    V = V[0]
    lam = E * NU / ((1 + NU) * (1 - 2 * NU))
    mu = E / (2 * (1 + NU))
    H = np.random.default_rng(8).normal(size=(3, 3))
    eps = 0.5 * (H + H.T)
    u = (X @ H.T).reshape(-1)
    assert u @ Ke @ u == pytest.approx(V * (lam * np.trace(eps) ** 2 + 2 * mu * np.sum(eps * eps)),
                                       rel=1e-11)
    a, b = 0.5854101966249685, 0.1381966011250105
    p = np.random.default_rng(9).normal(size=4)
    quad = 0.0
    for q in range(4):
        bary = np.full(4, b)
        bary[q] = a
        quad += V / 4 * (bary @ p) ** 2
    assert p @ Me @ p == pytest.approx(quad / M, rel=1e-12)


def test_tet_assembled_patch_identities():
    """Assembly on the Cryer octant (4 cells per radius, curved surface):
    a linear displacement leaves no force at nodes off the boundary (constant
    stress is divergence free), a linear pressure leaves no Darcy flux there,
    A_pu^T of a linear displacement is alpha tr(H) times each node's lumped
    volume, the storage rows sum to that volume / M, and the surface load's
    resultant is -sigma0 times the area that the mesh's symmetry face
    x = 0 covers (the closed polyhedral surface has zero net area vector)."""
    prob = W.cryer_octant(4, steps=2)
    m = tet.TetModel(prob)
    x = prob.nodes
    tol = 1e-9
    interior = ((x > tol).all(axis=1)) & (np.linalg.norm(x, axis=1) < 1.0 - 1e-3)
    interior &= ~np.isin(np.arange(m.N), prob.load_tris.reshape(-1))
    assert interior.sum() >= 8
    H = np.random.default_rng(10).normal(size=(3, 3))
    u = (x @ H.T).T.reshape(-1)                                   # field-major
    f = (m.Kb @ u).reshape(3, m.N)
    scale = np.abs(m.Kb).max() * np.abs(u).max()
    assert np.abs(f[:, interior]).max() < 1e-11 * scale
    g = np.array([0.4, -0.9, 1.3])
    p = x @ g
    assert np.abs((m.C @ p)[interior]).max() < 1e-11 * np.abs(m.C).max() * np.abs(p).max()
    _, V = tet.tet_gradients(x[prob.tets])
    vol = np.zeros(m.N)
    np.add.at(vol, prob.tets, np.repeat(V[:, None] / 4, 4, axis=1))
    assert np.allclose(m.Apu.T @ u, ALPHA * np.trace(H) * vol, rtol=1e-11, atol=0)
    assert np.allclose(np.asarray(m.S.sum(axis=1)).ravel(), vol / M, rtol=1e-12)
    faces = np.concatenate([prob.tets[:, [0, 1, 2]], prob.tets[:, [0, 1, 3]], prob.tets[:, [0, 2, 3]],
                            prob.tets[:, [1, 2, 3]]])
    on_x0 = faces[(x[faces, 0] == 0.0).all(axis=1)]
    a = x[on_x0]
    area_x0 = 0.5 * np.linalg.norm(np.cross(a[:, 1] - a[:, 0], a[:, 2] - a[:, 0]), axis=1).sum()
    fx = m.fu.reshape(3, m.N)[0].sum()
    assert fx == pytest.approx(-prob.sigma0 * area_x0, rel=1e-12)
    assert area_x0 == pytest.approx(np.pi / 4, rel=0.05)          # quarter disc of radius 1


def terzaghi_tet_error(nz, steps=400, tstar=0.2):
    H, F = 1.0, 1e6
    p0, cv = A.terzaghi_params(E, NU, ALPHA, M, K, MU, F)
    t_end = tstar * H * H / cv
    prob = W.column_terzaghi_tet(nz=nz, H=H, load=F, steps=steps, dt=t_end / steps)
    _, _, _, _, p = tet.run(prob)
    axis = (prob.nodes[:, 0] == 0) & (prob.nodes[:, 1] == 0)
    err = np.abs(p[axis] - A.terzaghi_pressure(prob.nodes[axis, 2], t_end, H, p0, cv)).max() / p0
    level = np.round(prob.nodes[:, 2] * nz / H).astype(int)
    spread = max(np.ptp(p[level == lv]) for lv in range(nz + 1)) / p0
    return err, spread


def test_terzaghi_on_tetrahedra_converges_at_second_order():
    """1-D consolidation (the series of the structured pin) on a column of
    Kuhn tetrahedra: the pressure along the column converges to the series at
    second order (8 -> 16 cells), and the pressure difference between the four
    nodes of a level, which the Kuhn cut introduces, vanishes at the same rate."""
    e8, s8 = terzaghi_tet_error(8)
    e16, s16 = terzaghi_tet_error(16)
    assert e16 < 0.005 and e8 / e16 > 2.5
    assert s8 / s16 > 2.5
