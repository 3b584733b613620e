"""Oracle of the paper's own discretisation: P1 tetrahedra for displacement
and pressure (Sec. 3.1: linear shape functions on tetrahedra for both fields),
without fault elements.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Element operators of a tetrahedron with volume V and constant shape-function
gradients G (4 x 3), all integrals exact:
  K_e  = V B^T D B                       (Eq. stress; B the strain-displacement matrix)
  A_e  = alpha (V/4) B^T m 1^T            (Biot coupling, m = [1 1 1 0 0 0], App. A)
  M_e  = (1/M) (V/20) (1 + delta_ij)      (storage, consistent mass)
  L_e  = (k/mu) V G G^T                   (Darcy)
Global vectors are field-major like the structured oracle: u = [ux | uy | uz],
p.  The time step is the backward-Euler monolithic system of Sec. 3.3 without
fault terms, solved directly (sparse LU plus two steps of iterative refinement):
  K u - A p = f,   A^T (u - u_n) + S (p - p_n) + dt C p = 0.

Pinned by: tests/test_oracle_tet.py (symmetry and rigid modes; exact strain
energy, Biot work, storage energy against an independent quadrature and Darcy
energy of linear fields; assembled patch identities and the surface-load
resultant on the Cryer octant; 1-D consolidation on a tetrahedral column at
second order; Cryer's centre pressure within the paper's 4 %).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from .fem import elasticity_D

VOIGT_M = np.array([1.0, 1.0, 1.0, 0.0, 0.0, 0.0])


def tet_gradients(X):
    """X (ne, 4, 3) -> gradients G (ne, 4, 3) and volumes V (ne,)."""
    ne = X.shape[0]
    A = np.ones((ne, 4, 4))
    A[:, :, 1:] = X
    inv = np.linalg.inv(A)              # rows: coefficients (1, x, y, z) of N_a in column a
    G = np.transpose(inv[:, 1:, :], (0, 2, 1))
    V = np.abs(np.linalg.det(A)) / 6.0
    return G, V


def tet_B(G):
    """Strain-displacement matrix for element-local dofs 3a + c: (ne, 6, 12)."""
    ne = G.shape[0]
    B = np.zeros((ne, 6, 12))
    for a in range(4):
        gx, gy, gz = G[:, a, 0], G[:, a, 1], G[:, a, 2]
        c = 3 * a
        B[:, 0, c + 0] = gx
        B[:, 1, c + 1] = gy
        B[:, 2, c + 2] = gz
        B[:, 3, c + 1] = gz
        B[:, 3, c + 2] = gy
        B[:, 4, c + 0] = gz
        B[:, 4, c + 2] = gx
        B[:, 5, c + 0] = gy
        B[:, 5, c + 1] = gx
    return B


def tet_element_matrices(X, E, nu, alpha, invM, cond):
    """K (ne,12,12), A (ne,12,4), Ms (ne,4,4), L (ne,4,4) for P1 tetrahedra;
    E and cond (= k / mu) scalar or one per element."""
    G, V = tet_gradients(X)
    B = tet_B(G)
    ne = X.shape[0]
    D = elasticity_D(np.broadcast_to(np.asarray(E, float), (ne,)).copy(), nu)
    cond = np.broadcast_to(np.asarray(cond, float), (ne,))[:, None, None]
    K = V[:, None, None] * np.einsum("eia,eij,ejb->eab", B, D, B)
    Bm = np.einsum("eia,i->ea", B, VOIGT_M)
    A = alpha * (V / 4.0)[:, None, None] * Bm[:, :, None] * np.ones(4)[None, None, :]
    Ms = invM * (V / 20.0)[:, None, None] * (np.ones((4, 4)) + np.eye(4))[None]
    L = cond * V[:, None, None] * np.einsum("eac,ebc->eab", G, G)
    return K, A, Ms, L


class TetModel:
    """Assembled operators of a TetProblem (workloads.TetProblem)."""

    def __init__(self, prob):
        self.prob = prob
        N = prob.nodes.shape[0]
        self.N = N
        X = prob.nodes[prob.tets]
        K, A, Ms, L = tet_element_matrices(X, prob.E, prob.nu, prob.alpha, 1.0 / prob.M, prob.k / prob.mu_f)
        T = prob.tets
        udof = np.stack([c * N + T for c in range(3)], axis=2).reshape(T.shape[0], 12)   # local 3a + c
        self.Kb = self._asm(K, udof, udof, 3 * N, 3 * N)
        self.Apu = self._asm(A, udof, T, 3 * N, N)
        self.S = self._asm(Ms, T, T, N, N)
        self.C = self._asm(L, T, T, N, N)
        self.free_u = prob.fixed[0:3].reshape(-1) == 0
        self.free_p = prob.fixed[3] == 0
        # compressive normal traction: -sigma0 n over each surface triangle, A/3 per vertex
        f = np.zeros(3 * N)
        tri = prob.load_tris
        x0, x1, x2 = (prob.nodes[tri[:, q]] for q in range(3))
        an = 0.5 * np.cross(x1 - x0, x2 - x0)          # area times outward normal
        for q in range(3):
            for c in range(3):
                np.add.at(f, c * N + tri[:, q], -prob.sigma0 * an[:, c] / 3.0)
        self.fu = f

    @staticmethod
    def _asm(Ke, rows, cols, nr, nc):
        ne, a, b = Ke.shape
        r = np.repeat(rows, b, axis=1).reshape(-1)
        c = np.tile(cols, (1, a)).reshape(-1)
        return sp.coo_matrix((Ke.reshape(-1), (r, c)), shape=(nr, nc)).tocsr()

    def step(self, u, p, dt):
        """One backward-Euler step of the linear problem (constrained dofs 0)."""
        N = self.N
        fu, fp = self.free_u, self.free_p
        J = sp.bmat([[self.Kb, -self.Apu], [self.Apu.T, self.S + dt * self.C]]).tocsr()
        rhs = np.concatenate([self.fu, self.Apu.T @ u + self.S @ p])
        free = np.concatenate([fu, fp])
        Jf = J[free][:, free].tocsc()
        lu = spla.splu(Jf)
        xf = lu.solve(rhs[free])
        # two steps of iterative refinement: force and flow rows differ by many
        # orders of magnitude, and the direct solve alone leaves errors of
        # ~1e-7 in p although its residual is ~1e-14
        for _ in range(2):
            xf += lu.solve(rhs[free] - Jf @ xf)
        x = np.zeros(4 * N)
        x[free] = xf
        return x[:3 * N], x[3 * N:]


def run(prob, nsteps=None):
    """Times and the pressure at the centre node (the origin) over the steps."""
    m = TetModel(prob)
    u = np.zeros(3 * m.N)
    p = np.zeros(m.N)
    centre = int(np.argmin(np.linalg.norm(prob.nodes, axis=1)))
    t, out_t, out_p = 0.0, [], []
    for dt in prob.dts[: (nsteps or len(prob.dts))]:
        u, p = m.step(u, p, dt)
        t += dt
        out_t.append(t)
        out_p.append(p[centre])
    return m, np.array(out_t), np.array(out_p), u, p
