"""Pins for the oracle of the fault on P1 tetrahedra (Sec. 3.1.1-3.1.2):
interface elements on the fault triangles of a tetrahedralised faulted box.
Each check holds exactly (or within the paper's bound) and fails for a
plausible slip in the geometry, the assembly or the fault-flow terms."""
import math

import numpy as np
import pytest
import scipy.linalg as sla
from scipy import special

import workloads as W
from oracle import analytic, solve, tetfault as TF


def lame(E, nu):
    return E * nu / ((1 + nu) * (1 - 2 * nu)), E / (2 * (1 + nu))


def test_fault_geometry_of_a_sheared_plane():
    """Pair areas sum to the area of the sheared plane, interior pairs carry
    hx hy sqrt(1 + sx^2 + sy^2) (six triangles of area / 3 each), the normal
    is (-sx, -sy, 1) normalised and the frame is orthonormal with t1 in the
    plane spanned by n and the reference direction."""
    sx, sy = 0.3, -0.2
    prob = W.tetrahedralize(W.tiny_faulted(4, 3, 2, shear=(sx, sy), h=(0.5, 0.4, 0.5)))
    fg = TF.triangle_fault_geometry(prob.nodes, prob.pairs, prob.fault_tris, prob.t1_ref)
    J = math.sqrt(1 + sx * sx + sy * sy)
    assert fg["area"].sum() == pytest.approx(2.0 * 1.2 * J, rel=1e-13)
    i = np.arange(prob.pairs.shape[0]) % 5
    j = np.arange(prob.pairs.shape[0]) // 5
    inner = (i > 0) & (i < 4) & (j > 0) & (j < 3)
    assert np.allclose(fg["area"][inner], 0.5 * 0.4 * J, rtol=1e-13)
    assert np.allclose(fg["n"], np.array([-sx, -sy, 1.0]) / J, atol=1e-14)
    for a, b in (("n", "t1"), ("n", "t2"), ("t1", "t2")):
        assert np.abs(np.sum(fg[a] * fg[b], axis=1)).max() < 1e-14
    assert np.allclose(np.cross(fg["n"], fg["t1"]), fg["t2"], atol=1e-14)
    ex = np.array([1.0, 0.0, 0.0])
    assert np.all(fg["t1"] @ ex > 0)
    assert np.abs(np.einsum("pi,pi->p", np.cross(fg["n"], ex[None, :]), fg["t1"])).max() < 1e-14


def test_triangle_laplacian_kernel_and_linear_energy():
    """Constants are in the kernel of each triangle's Laplacian and a linear
    in-plane field q = g . x gives q^T L_t q = a_t |P g|^2 with P the in-plane
    projector (exact gradient energy)."""
    prob = W.tetrahedralize(W.tiny_faulted(3, 3, 2, shear=(0.4, 0.1)))
    fg = TF.triangle_fault_geometry(prob.nodes, prob.pairs, prob.fault_tris, prob.t1_ref)
    Lt = fg["Lt"]
    assert np.abs(Lt @ np.ones(3)).max() < 1e-13 * np.abs(Lt).max()
    g = np.array([0.7, -1.1, 0.4])
    X = prob.nodes[prob.pairs[prob.fault_tris, 0]]
    q = X @ g
    n = fg["n"][0]
    Pg = g - (g @ n) * n
    e = np.einsum("ta,tab,tb->t", q, Lt, q)
    assert np.allclose(e, fg["at"] * (Pg @ Pg), rtol=1e-12)


def test_rigid_modes_open_and_stuck_fault():
    """Without constraints the two blocks move rigidly on their own: the bulk
    stiffness has 12 zero modes; adding the stuck-fault tangent of every pair
    (contact k_n n n^T plus stick k_s P_t) joins them, leaving 6."""
    prob = W.tetrahedralize(W.tiny_faulted(2, 2, 2, shear=(0.2, 0.0)))
    m = TF.TetFaultModel(prob)
    K = m.Kb.toarray()
    w = sla.eigvalsh(K)
    assert np.sum(np.abs(w) < 1e-9 * w.max()) == 12
    fg, fp, N = m.fg, prob.fault, m.N
    Kc = np.zeros_like(K)
    for i, (a, b) in enumerate(prob.pairs):
        n = fg["n"][i]
        D = fp.kn * np.outer(n, n) + fp.ks * (np.eye(3) - np.outer(n, n))
        for (r, sr) in ((b, 1.0), (a, -1.0)):
            for (c, sc) in ((b, 1.0), (a, -1.0)):
                Kc[np.ix_([r, N + r, 2 * N + r], [c, N + c, 2 * N + c])] += sr * sc * fg["area"][i] * D
    w = sla.eigvalsh(K + Kc)
    assert np.sum(np.abs(w) < 1e-9 * w.max()) == 6


def test_constant_stress_loads_the_lips_with_the_interface_traction():
    """A linear displacement u = H x, continuous across the fault, gives a
    constant stress sigma; the bulk forces at interior pairs are the nodal
    loads of the traction on each lip's face: -A_i sigma n on the plus lip,
    +A_i sigma n on the minus lip.  Ties the assembly, the pair areas and the
    pair normals together."""
    prob = W.tetrahedralize(W.tiny_faulted(4, 4, 2, shear=(0.25, 0.0), h=(0.5, 0.5, 0.5)))
    m = TF.TetFaultModel(prob)
    H = np.random.default_rng(12).normal(size=(3, 3))
    u = (prob.nodes @ H.T).T.reshape(-1)
    f = (m.Kb @ u).reshape(3, m.N)
    lam, mu = lame(prob.E[0], prob.nu)
    eps = 0.5 * (H + H.T)
    sig = lam * np.trace(eps) * np.eye(3) + 2 * mu * eps
    i = np.arange(prob.pairs.shape[0]) % 5
    j = np.arange(prob.pairs.shape[0]) // 5
    inner = (i > 0) & (i < 4) & (j > 0) & (j < 4)
    t = (sig @ m.fg["n"].T).T * m.fg["area"][:, None]
    ref = np.abs(t[inner]).max()
    mi, pl = prob.pairs[inner, 0], prob.pairs[inner, 1]
    assert np.abs(f[:, pl].T + t[inner]).max() < 1e-10 * ref
    assert np.abs(f[:, mi].T - t[inner]).max() < 1e-10 * ref
    assert np.abs(m.jump(u)).max() < 1e-15 * np.abs(u).max() + 1e-300


def test_lip_pressure_force_and_aperture_volume():
    """A^f_pu with <p> = 1 on every pair pushes the lips apart with total force
    (fault area) n on the plus lip; its transpose maps a uniform opening
    [[u]] = d n to the aperture volume d A_i per pair (Sec. 3.2.3)."""
    prob = W.tetrahedralize(W.tiny_faulted(3, 2, 2, shear=(0.3, 0.1), k_perp=1e-18))
    m = TF.TetFaultModel(prob)
    N, fg = m.N, m.fg
    p = np.zeros(N)
    p[prob.pairs.ravel()] = 1.0
    F = (m.Apu_f @ p).reshape(3, N)
    total = fg["area"].sum()
    n = fg["n"][0]
    assert np.allclose(F[:, prob.pairs[:, 1]].sum(axis=1), total * n, rtol=1e-13)
    assert np.allclose(F[:, prob.pairs[:, 0]].sum(axis=1), -total * n, rtol=1e-13)
    d = 1e-4
    u = np.zeros((3, N))
    u[:, prob.pairs[:, 1]] = (d * fg["n"]).T
    v = m.Apu_f.T @ u.reshape(-1)
    assert np.allclose(v[prob.pairs[:, 0]] + v[prob.pairs[:, 1]], d * fg["area"], rtol=1e-12)
    assert np.allclose(v[prob.pairs[:, 0]], v[prob.pairs[:, 1]], rtol=1e-12)


def test_line_source_fault_pressure_on_triangles():
    """Impermeable, uncoupled matrix on tetrahedra (Sec. 4.2): after 50 steps
    the pressure front, where p = dp* E1(1), lies within the paper's 8 % of
    L = sqrt(4Dt) on both axes, and the pressure at radii of 3 to 8 cells is
    within 6 % of dp* of dp* E1(r^2/4Dt)."""
    base = W.theis_plate(n=32, steps=50)
    prob = W.tetrahedralize(base)
    model, res = TF.run(prob, solver="sparse")
    fp = prob.fault
    t = sum(prob.dts)
    pairs = prob.pairs
    Q = prob.fp.sum()
    dps = analytic.theis_dpstar(Q, prob.mu_f, fp.wk_par)
    xy = prob.nodes[pairs[:, 0], :2]
    r = np.linalg.norm(xy, axis=1)
    p = res[-1].p[pairs[:, 0]]
    D = analytic.fault_diffusivity(fp.wk_par, fp.MF, prob.mu_f, fp.w0)
    L = math.sqrt(4 * D * t)
    assert 4 * base.h[0] < L < 10.0
    level = special.exp1(1.0)
    for ax in (0, 1):
        ray = (np.abs(xy[:, 1 - ax]) < 1e-9) & (xy[:, ax] > 0)
        o = np.argsort(xy[ray, ax])
        rr, pp = xy[ray, ax][o], p[ray][o] / dps
        k = np.nonzero(pp < level)[0][0]
        front = rr[k - 1] + (pp[k - 1] - level) / (pp[k - 1] - pp[k]) * (rr[k] - rr[k - 1])
        assert abs(front / L - 1) < 0.08
    h = base.h[0]
    sel = (r >= 3 * h - 1e-9) & (r <= 8 * h + 1e-9)
    pan = analytic.theis_pressure(r[sel], t, Q, prob.mu_f, fp.wk_par, fp.MF, fp.w0)
    assert pan.max() > 0.5 * dps
    assert (np.abs(p[sel] - pan) / dps).max() < 0.06


@pytest.mark.parametrize("k_perp", [0.0, 1e-18])
def test_newton_step_direct_equals_prevost(k_perp):
    """The Newton step on tetrahedra reaches the same state with the dense
    monolithic LU and with Prevost's partitioned CG (Sec. 3.3.2), with slip."""
    prob = W.tetrahedralize(W.tiny_faulted(3, 3, 2, k_perp=k_perp, Q=2e-4, steps=3))
    out = {}
    for solver in ("lu", "prevost"):
        _, res = TF.run(prob, solver=solver, rtol=1e-12)
        out[solver] = res
    for a, b in zip(out["lu"], out["prevost"]):
        assert np.array_equal(a.flags, b.flags)
        assert np.abs(a.u - b.u).max() < 1e-9 * np.abs(a.u).max()
        assert np.abs(a.p - b.p).max() < 1e-9 * np.abs(a.p).max()
    assert (out["lu"][-1].flags == 2).sum() >= 3


def test_tetrahedral_fault_small_has_all_three_states():
    """The unit-cube faulted case on tetrahedra, five steps: the final state
    holds open, sticking and slipping pairs, and no pair sits within 1e-8 of
    a contact or friction tie (the comparisons stay decidable)."""
    prob = W.tetrahedralize(W.fault_small(8))
    _, res = TF.run(prob)
    fl = res[-1].flags
    assert (fl == 0).sum() >= 1 and (fl == 1).sum() >= 4 and (fl == 2).sum() >= 4
    fp = prob.fault
    contact = fl != 0
    margin_F = np.abs(res[-1].F[contact]) / (fp.f * np.abs(res[-1].tn[contact]))
    assert margin_F.min() > 1e-8
