"""Pins for the oracle's element and assembly layer (no GPU).

Each check compares against a fact fixed by mechanics or calculus, not against
a re-typed formula: rigid-body null spaces, exact energies of linear fields,
patch tests (linear fields reproduced exactly in the interior), areas and
volumes of the affine cells, and symmetry.
"""
import numpy as np
import pytest

import workloads as W
from oracle import fem, solve


def cell(h=(1.0, 1.0, 1.0), shear=(0.0, 0.0)):
    m = fem.Mesh(1, 1, 1, (0.3, -0.2, 0.1), h, shear, None)
    return m.coords()[m.connectivity()][0], m


def rigid_modes(X):
    modes = []
    for c in range(3):
        v = np.zeros((8, 3)); v[:, c] = 1.0; modes.append(v.ravel())
    for axis in range(3):
        w = np.zeros(3); w[axis] = 1.0
        modes.append(np.cross(w, X).ravel())
    return np.array(modes).T                    # element dofs 3a + c


@pytest.mark.parametrize("shear", [(0.0, 0.0), (1.7320508075688772, 0.0), (0.4, -0.3)])
@pytest.mark.parametrize("h", [(1.0, 1.0, 1.0), (0.5, 0.25, 2.0)])
def test_stiffness_symmetry_and_rigid_nullspace(h, shear):
    X, _ = cell(h, shear)
    K, _, _, _ = fem.element_matrices(X[None], 20e9, 0.25, 0.8, 1 / 50e9, 1e-12)
    K = K[0]
    assert np.allclose(K, K.T, rtol=0, atol=1e-6 * np.abs(K).max())
    R = rigid_modes(X)
    assert np.abs(K @ R).max() < 1e-9 * np.abs(K).max()
    ev = np.linalg.eigvalsh(K)
    assert np.sum(ev > 1e-8 * ev.max()) == 18          # 24 dofs - 6 rigid modes


@pytest.mark.parametrize("shear", [(0.0, 0.0), (1.7320508075688772, 0.0)])
def test_energies_of_linear_fields(shear):
    """For u = A x, p = const or linear: exact integrals over the cell volume V."""
    h = (0.5, 0.25, 2.0)
    X, _ = cell(h, shear)
    E, nu, alpha, M, cond = 20e9, 0.25, 0.8, 50e9, 3e-12
    K, Apu, S, C = [a[0] for a in fem.element_matrices(X[None], E, nu, alpha, 1 / M, cond)]
    V = h[0] * h[1] * h[2]                                # affine shear keeps the volume
    rng = np.random.default_rng(0)
    A = rng.normal(size=(3, 3))
    u = (X @ A.T).ravel()
    eps = 0.5 * (A + A.T)
    lam = E * nu / ((1 + nu) * (1 - 2 * nu)); mu = E / (2 * (1 + nu))
    energy = V * (lam * np.trace(eps) ** 2 + 2 * mu * np.sum(eps * eps))
    assert u @ K @ u == pytest.approx(energy, rel=1e-12)
    p0 = 3.7e6
    assert u @ Apu @ np.full(8, p0) == pytest.approx(alpha * p0 * np.trace(A) * V, rel=1e-12)
    one = np.ones(8)
    assert one @ S @ one == pytest.approx(V / M, rel=1e-12)
    g = rng.normal(size=3)
    pl = X @ g
    assert pl @ C @ pl == pytest.approx(cond * (g @ g) * V, rel=1e-12)
    assert np.abs(C @ one).max() < 1e-12 * np.abs(C).max()
    # consistent mass of a linear field: int (g.x)^2 over the parallelepiped,
    # by the exact centroid/second-moment formula of an affine cube
    Jm = np.array([[h[0], 0, 0], [0, h[1], 0], [shear[0] * h[0], shear[1] * h[1], h[2]]])
    c = X.mean(axis=0)
    second = V * ((g @ c) ** 2 + (g @ Jm @ Jm.T @ g) / 12.0)
    assert pl @ S @ pl == pytest.approx(second / M, rel=1e-12)


def test_patch_test_global_elasticity_and_flow():
    """Linear u and linear p are reproduced exactly at interior nodes when the
    boundary nodes carry the exact values (bulk without fault, sheared grid)."""
    prob = W.tiny_faulted(3, 3, 3, shear=(0.5, 0.2))
    prob.kf = None
    prob.fault = None
    N = (prob.nx + 1) * (prob.ny + 1) * (prob.nz + 1)
    prob.fixed = np.zeros((4, N), np.uint8)
    prob.fu = np.zeros((3, N)); prob.fp = np.zeros(N)
    model = fem.Model(prob)
    X = model.mesh.coords()
    ii = np.arange(N)
    nb = model.mesh.nb
    i = ii % (prob.nx + 1); j = (ii % nb) // (prob.nx + 1); k = ii // nb
    interior = (i > 0) & (i < prob.nx) & (j > 0) & (j < prob.ny) & (k > 0) & (k < prob.nz)
    rng = np.random.default_rng(1)
    A = rng.normal(size=(3, 3)) * 1e-4
    uex = (X @ A.T).T.reshape(-1)                       # (3N,)
    I = np.concatenate([interior] * 3)
    Kb = model.Kb.tocsr()
    rhs = -Kb[I][:, ~I] @ uex[~I]
    from scipy.sparse.linalg import spsolve
    uI = spsolve(Kb[I][:, I].tocsc(), rhs)
    assert np.abs(uI - uex[I]).max() < 1e-10 * np.abs(uex).max()
    g = rng.normal(size=3) * 1e5
    pex = X @ g
    C = model.C.tocsr()
    pI = spsolve(C[interior][:, interior].tocsc(), -C[interior][:, ~interior] @ pex[~interior])
    assert np.abs(pI - pex[interior]).max() < 1e-10 * np.abs(pex).max()
    # Biot: a constant pressure loads only boundary nodes (div of a constant)
    f = model.Apu @ np.full(N, 1e6)
    assert np.abs(f[I]).max() < 1e-9 * np.abs(f).max()


def test_global_nullspace_with_fault_open_and_closed():
    """Free stiffness of a faulted box: 6 rigid modes when the lips are tied by
    the stick tangent, 12 when every pair is open (two free blocks)."""
    prob = W.tiny_faulted(2, 2, 2)
    N = prob.n_nodes
    prob.fixed = np.zeros((4, N), np.uint8)
    model = fem.Model(prob)
    st = solve.initial_state(model)
    r, force, Kcoh = solve.fault_terms(model, st.u, st.dlie)
    assert np.all(r["state"] == 1)
    assert np.abs(force).max() < 1e-6                    # in-situ state is balanced
    for Kc, nzero in ((Kcoh, 6), (None, 12)):
        Kt = (model.Kb + Kc).toarray() if Kc is not None else model.Kb.toarray()
        ev = np.linalg.eigvalsh(0.5 * (Kt + Kt.T))
        assert np.sum(np.abs(ev) < 1e-9 * ev.max()) == nzero
        assert np.allclose(Kt, Kt.T, atol=1e-6 * np.abs(Kt).max())


@pytest.mark.parametrize("shear", [(0.0, 0.0), (1.7320508075688772, 0.0), (0.3, 0.4)])
def test_fault_geometry(shear):
    m = fem.Mesh(3, 4, 2, (0, 0, 0), (0.5, 0.25, 1.0), shear, 1)
    fg = fem.fault_geometry(m)
    total = 3 * 0.5 * 4 * 0.25 * np.sqrt(1 + shear[0] ** 2 + shear[1] ** 2)
    assert fg["area"].sum() == pytest.approx(total, rel=1e-13)
    nexp = np.array([-shear[0], -shear[1], 1.0]) / np.sqrt(1 + shear[0] ** 2 + shear[1] ** 2)
    assert np.allclose(fg["n"], nexp[None], atol=1e-14)
    assert np.allclose(np.sum(fg["t1"] * fg["n"], 1), 0, atol=1e-14)
    assert np.allclose(np.linalg.norm(fg["t2"], axis=1), 1, atol=1e-14)
    # Laplacian: constants in the kernel; linear field energy = |grad|^2 * area
    Lq = fg["Lq"]
    assert np.abs(Lq.sum(axis=2)).max() < 1e-12
    X = m.coords()[m.pairs()[:, 0]]
    g = np.array([1.3, -0.7, 0.0])
    gt = g - (g @ nexp) * nexp                          # surface gradient of g.x
    pl = X @ g
    quads = fg["quads"]
    e = np.einsum("qa,qab,qb->", pl[quads], Lq, pl[quads])
    assert e == pytest.approx((gt @ gt) * total, rel=1e-12)


def test_fault_coupling_identities():
    """A uniform fault pressure p0 pushes the lips apart with total force
    p0 * area * n on the upper lip (and the opposite on the lower lip), and a
    uniform opening d n gives a fluid-volume change d * area (App. B)."""
    prob = W.tiny_faulted(3, 2, 2, shear=(0.6, 0.0))
    prob.alpha = 0.0                                    # bulk Biot term off
    model = fem.Model(prob)
    fg = model.fg
    N = model.N
    p = np.zeros(N)
    p[fg["pairs"][:, 0]] = 2e6
    f = (model.Apu @ p).reshape(3, N)
    area = fg["area"].sum()
    n = fg["n"][0]
    assert np.allclose(f[:, fg["pairs"][:, 1]].sum(axis=1), 2e6 * area * n, rtol=1e-12)
    assert np.allclose(f[:, fg["pairs"][:, 0]].sum(axis=1), -2e6 * area * n, rtol=1e-12)
    u = np.zeros((3, N))
    u[:, fg["pairs"][:, 1]] = 1e-5 * n[:, None]
    q = model.Apu.T @ u.reshape(-1)
    assert q.sum() == pytest.approx(1e-5 * area, rel=1e-12)


@pytest.mark.parametrize("shear", [(0.0, 0.0), (1.7320508075688772, 0.0), (0.4, -0.3)])
def test_transverse_fracture_flow_of_a_uniform_lip_jump(shear):
    """Transverse fracture flow (Sec. 3.2.3): with p = dp on every node above
    the fault (the plus lip included) and 0 below, the bulk blocks are
    constant on each side and <p> is uniform, so only the transverse term
    k_perp / (mu w0) [[p]] carries flux.  Each plus-lip row must hold
    A_i k_perp dp / (mu w0), with A_i the nodal share of the sheared quads
    (hx hy sqrt(1 + sx^2 + sy^2) per quad, a quarter per corner), each
    minus-lip row its negative, every other row zero, and the plus-lip total
    must equal the fault plane's area times k_perp dp / (mu w0)."""
    nx, ny, nz = 3, 4, 2
    h = (0.5, 0.25, 0.4)
    prob = W.tiny_faulted(nx, ny, nz, shear=shear, k_perp=3e-13, h=h)
    model = fem.Model(prob)
    m = model.mesh
    fp = prob.fault
    dp = 2.5e5
    kk = np.arange(m.N) // m.nb
    p = np.where(kk >= m.kf + 1, dp, 0.0)
    flux = model.C @ p
    coef = fp.k_perp * dp / (prob.mu_f * fp.w0)
    quad_area = h[0] * h[1] * np.sqrt(1.0 + shear[0] ** 2 + shear[1] ** 2)
    i = np.arange(m.nb) % (m.nx + 1)
    j = np.arange(m.nb) // (m.nx + 1)
    share = (np.where((i == 0) | (i == m.nx), 0.5, 1.0) * np.where((j == 0) | (j == m.ny), 0.5, 1.0))
    Ai = quad_area * share
    plus = m.kf + 1
    minus = m.kf
    assert flux[plus * m.nb:(plus + 1) * m.nb] == pytest.approx(Ai * coef, rel=1e-12)
    assert flux[minus * m.nb:(minus + 1) * m.nb] == pytest.approx(-Ai * coef, rel=1e-12)
    rest = np.ones(m.N, bool)
    rest[minus * m.nb:(plus + 1) * m.nb] = False
    assert np.abs(flux[rest]).max() <= 1e-12 * coef * quad_area
    total = nx * h[0] * ny * h[1] * np.sqrt(1.0 + shear[0] ** 2 + shear[1] ** 2)
    assert flux[plus * m.nb:(plus + 1) * m.nb].sum() == pytest.approx(total * coef, rel=1e-12)
