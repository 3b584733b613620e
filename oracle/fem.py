"""Discretisation for the oracle: structured Q1 mesh with a duplicated fault plane,
element matrices by Gauss quadrature, fault geometry and sparse assembly.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Paper: Sec. 3.1 (shared mesh, nodal unknowns, interface elements with duplicated
nodes, element normal = average of the facet normals), Sec. 3.2.1-3.2.3 (weak
forms), App. A (A_pu, A_up for solid elements), App. B (A^f_up, A^f_pu for
interface elements).  The paper's tetrahedra/triangles are replaced by trilinear
hexahedra (Q1) and bilinear fault quadrilaterals on a structured, possibly
affinely sheared grid (Sec. 3.1 states other standard elements may be used).

Global DOF layout inside the oracle: u component-major, dof = c * N + n; p dof = n.

Pinned by: tests/test_oracle_element.py (symmetry and the 6 rigid-body modes of
the element stiffness on box and sheared cells; exact strain, Biot, storage and
Darcy energies of linear fields; global patch tests for elasticity and flow;
null space 6 / 12 with the fault stuck / open; fault area, normals and frame;
uniform lip pressure force and aperture volume) and, through the solvers, the
consolidation and line-source tests of tests/test_oracle_solvers.py.
"""
from __future__ import annotations

import math

import numpy as np
import scipy.sparse as sp

# ---------------------------------------------------------------------------
# Reference Q1 hexahedron
# ---------------------------------------------------------------------------

# local node a = ax + 2 ay + 4 az; reference coordinates in {-1, +1}^3
LOCAL = np.array([[(a >> 0) & 1, (a >> 1) & 1, (a >> 2) & 1] for a in range(8)])
XI_NODE = 2.0 * LOCAL - 1.0
GAUSS_1D = np.array([-1.0, 1.0]) / math.sqrt(3.0)
GAUSS_PTS = np.array([[GAUSS_1D[i], GAUSS_1D[j], GAUSS_1D[k]]
                      for k in range(2) for j in range(2) for i in range(2)])
GAUSS_W = np.ones(8)


def q1_shape(xi):
    """Trilinear shape functions N_a and their reference gradients at point xi."""
    xi = np.asarray(xi, float)
    f = 0.5 * (1.0 + XI_NODE * xi[None, :])            # (8, 3) 1-D factors
    N = f[:, 0] * f[:, 1] * f[:, 2]
    dN = np.empty((8, 3))
    dN[:, 0] = 0.5 * XI_NODE[:, 0] * f[:, 1] * f[:, 2]
    dN[:, 1] = 0.5 * XI_NODE[:, 1] * f[:, 0] * f[:, 2]
    dN[:, 2] = 0.5 * XI_NODE[:, 2] * f[:, 0] * f[:, 1]
    return N, dN


def lame(E, nu):
    lam = E * nu / ((1.0 + nu) * (1.0 - 2.0 * nu))
    mu = E / (2.0 * (1.0 + nu))
    return lam, mu


def elasticity_D(E, nu):
    """Isotropic stiffness in Voigt order [xx, yy, zz, yz, xz, xy] with
    engineering shear strains (Eq. stress, small strain Eq. strain)."""
    lam, mu = lame(np.asarray(E, float), nu)
    ne = lam.size
    D = np.zeros((ne, 6, 6))
    for i in range(3):
        for j in range(3):
            D[:, i, j] = lam
        D[:, i, i] += 2.0 * mu
    for i in range(3, 6):
        D[:, i, i] = mu
    return D


def strain_B(G):
    """Strain-displacement matrix for element-local dofs 3a + c.
    G: (ne, 8, 3) physical shape-function gradients -> (ne, 6, 24)."""
    ne = G.shape[0]
    B = np.zeros((ne, 6, 24))
    for a in range(8):
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


VOIGT_I = np.array([1.0, 1.0, 1.0, 0.0, 0.0, 0.0])


def element_matrices(X, E, nu, alpha, invM, cond):
    """Element operators of the Q1 hexahedra, exact 2x2x2 Gauss quadrature.

    X: (ne, 8, 3) node coordinates; E, cond = k / mu_f per element.
    Returns
      K   (ne, 24, 24)  int B^T D B                      (Sec. 3.2.1, first term)
      Apu (ne, 24, 8)   int alpha B^T {I} N_p            (App. A, Eq. Apdp)
      S   (ne, 8, 8)    int (1/M) N_p^T N_p              (Sec. 3.2.2, storage)
      C   (ne, 8, 8)    int (k/mu) grad N^T grad N       (Sec. 3.2.2, Darcy)
    A_up of App. A (Eq. Adpd) is Apu transposed, element by element.
    """
    X = np.asarray(X, float)
    ne = X.shape[0]
    E = np.broadcast_to(np.asarray(E, float), (ne,))
    cond = np.broadcast_to(np.asarray(cond, float), (ne,))
    D = elasticity_D(E, nu)
    K = np.zeros((ne, 24, 24))
    Apu = np.zeros((ne, 24, 8))
    S = np.zeros((ne, 8, 8))
    C = np.zeros((ne, 8, 8))
    for q in range(8):
        N, dN = q1_shape(GAUSS_PTS[q])
        J = np.einsum("ead,ak->edk", X, dN)            # dX_d / dxi_k
        detJ = np.linalg.det(J)
        if np.any(detJ <= 0):
            raise ValueError("inverted element")
        Jinv = np.linalg.inv(J)                        # dxi_k / dX_d
        G = np.einsum("ak,ekd->ead", dN, Jinv)         # dN_a / dX_d
        B = strain_B(G)
        w = GAUSS_W[q] * detJ
        K += w[:, None, None] * np.einsum("eia,eij,ejb->eab", B, D, B)
        Bm = np.einsum("eia,i->ea", B, VOIGT_I)        # B^T {I}: divergence row
        Apu += (w * alpha)[:, None, None] * Bm[:, :, None] * N[None, None, :]
        S += (w * invM)[:, None, None] * np.outer(N, N)[None]
        C += (w * cond)[:, None, None] * np.einsum("ead,ebd->eab", G, G)
    return K, Apu, S, C


# ---------------------------------------------------------------------------
# Structured mesh with an optional duplicated fault plane
# ---------------------------------------------------------------------------

class Mesh:
    """Structured grid; node numbering and lip duplication as in ``workloads``.

    Physical position of original node (i, j, k):
      x = ox + i hx,  y = oy + j hy,  z = oz + k hz + sx * (i hx) + sy * (j hy).
    """

    def __init__(self, nx, ny, nz, origin, h, shear, kf):
        self.nx, self.ny, self.nz = int(nx), int(ny), int(nz)
        self.origin = np.asarray(origin, float)
        self.h = np.asarray(h, float)
        self.shear = np.asarray(shear, float)
        self.kf = kf
        self.nplanes = self.nz + 1 + (0 if kf is None else 1)
        self.nb = (self.nx + 1) * (self.ny + 1)
        self.N = self.nb * self.nplanes
        self.n_el = self.nx * self.ny * self.nz

    def node(self, i, j, kk):
        return np.asarray(i) + (self.nx + 1) * (np.asarray(j) + (self.ny + 1) * np.asarray(kk))

    def orig_plane(self, kk):
        kk = np.asarray(kk)
        if self.kf is None:
            return kk
        return np.where(kk > self.kf, kk - 1, kk)

    def coords(self):
        kk, j, i = np.meshgrid(np.arange(self.nplanes), np.arange(self.ny + 1),
                               np.arange(self.nx + 1), indexing="ij")
        i, j, kk = i.ravel(), j.ravel(), kk.ravel()
        k = self.orig_plane(kk)
        x = self.origin[0] + i * self.h[0]
        y = self.origin[1] + j * self.h[1]
        z = (self.origin[2] + k * self.h[2] + self.shear[0] * i * self.h[0]
             + self.shear[1] * j * self.h[1])
        return np.stack([x, y, z], axis=1)

    def element_ijk(self, e):
        e = np.asarray(e)
        ei = e % self.nx
        ej = (e // self.nx) % self.ny
        ek = e // (self.nx * self.ny)
        return ei, ej, ek

    def connectivity(self, elems=None):
        """(ne, 8) node ids, local node a = ax + 2 ay + 4 az."""
        if elems is None:
            elems = np.arange(self.n_el)
        ei, ej, ek = self.element_ijk(elems)
        kb = ek + (0 if self.kf is None else (ek >= self.kf).astype(int))
        conn = np.empty((len(elems), 8), dtype=np.int64)
        for a in range(8):
            ax, ay, az = LOCAL[a]
            conn[:, a] = self.node(ei + ax, ej + ay, kb + az)
        return conn

    # -- fault ---------------------------------------------------------------
    def pairs(self):
        """(n_pairs, 2) node ids (minus, plus); pair id = i + (nx+1) j."""
        if self.kf is None:
            return np.zeros((0, 2), dtype=np.int64)
        pid = np.arange(self.nb)
        return np.stack([pid + self.nb * self.kf, pid + self.nb * (self.kf + 1)], axis=1)

    def fault_quads(self):
        """(nq, 4) pair ids of the bilinear fault quads, local b = bx + 2 by."""
        qi, qj = np.meshgrid(np.arange(self.nx), np.arange(self.ny), indexing="xy")
        qi, qj = qi.ravel(), qj.ravel()
        out = np.empty((qi.size, 4), dtype=np.int64)
        for b in range(4):
            bx, by = b & 1, (b >> 1) & 1
            out[:, b] = (qi + bx) + (self.nx + 1) * (qj + by)
        return out


# ---------------------------------------------------------------------------
# Interface (fault) geometry and fracture-flow element matrices
# ---------------------------------------------------------------------------

XI2_NODE = np.array([[-1.0, -1.0], [1.0, -1.0], [-1.0, 1.0], [1.0, 1.0]])


def q1_shape_2d(xi):
    f = 0.5 * (1.0 + XI2_NODE * np.asarray(xi, float)[None, :])
    N = f[:, 0] * f[:, 1]
    dN = np.stack([0.5 * XI2_NODE[:, 0] * f[:, 1], 0.5 * XI2_NODE[:, 1] * f[:, 0]], axis=1)
    return N, dN


def fault_geometry(mesh: Mesh):
    """Per-pair tributary area, unit normal (minus -> plus) and tangents, and the
    per-quad longitudinal Laplacian  int grad_G N^T grad_G N dGamma.

    Interface tractions, fault storage and the A^f couplings use nodal (2x2
    Lobatto) quadrature on each quad, so each node pair carries one
    integration point with weight A_i.  The pair normal is the normalised sum
    of the normals of the quads around it (Sec. 3.1.1: element normal = average
    of the facet normals; the facets coincide in the reference state).  t1 is
    the unit projection of the grid's i-direction onto the fault; t2 = n x t1.
    The Laplacian uses 2x2 Gauss points (exact for parallelogram quads).
    """
    X = mesh.coords()
    pairs = mesh.pairs()
    quads = mesh.fault_quads()
    Xq = X[pairs[quads, 0]]                                  # (nq, 4, 3) minus lip
    npairs = pairs.shape[0]
    area = np.zeros(npairs)
    nsum = np.zeros((npairs, 3))
    esum = np.zeros((npairs, 3))
    Lq = np.zeros((quads.shape[0], 4, 4))
    for b in range(4):                                       # nodal quadrature
        _, dN = q1_shape_2d(XI2_NODE[b])
        Js = np.einsum("qbd,bk->qdk", Xq, dN)                # (nq, 3, 2)
        cr = np.cross(Js[:, :, 0], Js[:, :, 1])
        jac = np.linalg.norm(cr, axis=1)
        np.add.at(area, quads[:, b], jac)
        np.add.at(nsum, quads[:, b], cr)
        np.add.at(esum, quads[:, b], Js[:, :, 0])
    for g in range(4):                                       # Gauss for the Laplacian
        xi = np.array([GAUSS_1D[g & 1], GAUSS_1D[g >> 1]])
        _, dN = q1_shape_2d(xi)
        Js = np.einsum("qbd,bk->qdk", Xq, dN)
        Gm = np.einsum("qdk,qdl->qkl", Js, Js)               # surface metric
        jac = np.sqrt(np.linalg.det(Gm))
        Ginv = np.linalg.inv(Gm)
        Lq += jac[:, None, None] * np.einsum("ak,qkl,bl->qab", dN, Ginv, dN)
    n = nsum / np.linalg.norm(nsum, axis=1)[:, None]
    e1 = esum - np.sum(esum * n, axis=1)[:, None] * n
    t1 = e1 / np.linalg.norm(e1, axis=1)[:, None]
    t2 = np.cross(n, t1)
    return dict(pairs=pairs, quads=quads, area=area, n=n, t1=t1, t2=t2, Lq=Lq)


# ---------------------------------------------------------------------------
# Global assembly
# ---------------------------------------------------------------------------

class Model:
    """All assembled operators of one problem (workloads.Problem)."""

    def __init__(self, prob, elements=None):
        """elements: optional subset of element ids to assemble (the rows of nodes
        whose adjacent elements are all in the subset are then exact); the fault
        terms are always assembled in full."""
        self.prob = prob
        m = Mesh(prob.nx, prob.ny, prob.nz, prob.origin, prob.h, prob.shear, prob.kf)
        self.mesh = m
        N = m.N
        self.N = N
        X = m.coords()
        elems = np.arange(m.n_el) if elements is None else np.asarray(elements, dtype=np.int64)
        conn = m.connectivity(elems)
        self.conn = conn
        E = np.broadcast_to(np.asarray(prob.E, float), (m.n_el,))[elems]
        cond = np.broadcast_to(np.asarray(prob.k, float), (m.n_el,))[elems] / prob.mu_f
        Ke, Ae, Se, Ce = element_matrices(X[conn], E, prob.nu, prob.alpha, 1.0 / prob.M, cond)
        nel_sub = elems.size

        # pressure dof map: tied lips (k_perp infinite) share the minus node's dof
        fp = prob.fault
        self.tied = fp is not None and not (fp.k_perp > 0)
        pdof = np.arange(N)
        if prob.kf is not None:
            pairs = m.pairs()
            if self.tied:
                pdof[pairs[:, 1]] = pairs[:, 0]
        self.pdof = pdof

        # element dof maps
        udof = np.empty((nel_sub, 24), dtype=np.int64)
        for a in range(8):
            for c in range(3):
                udof[:, 3 * a + c] = c * N + conn[:, a]
        pd = pdof[conn]

        def coo(rows, cols, vals, shape):
            return sp.coo_matrix((vals.ravel(), (rows.ravel(), cols.ravel())), shape=shape).tocsr()

        rr = lambda a, b: np.broadcast_to(a[:, :, None], (a.shape[0], a.shape[1], b.shape[1]))
        cc = lambda a, b: np.broadcast_to(b[:, None, :], (a.shape[0], a.shape[1], b.shape[1]))
        self.Kb = coo(rr(udof, udof), cc(udof, udof), Ke, (3 * N, 3 * N))
        Apu = coo(rr(udof, pd), cc(udof, pd), Ae, (3 * N, N))
        S = coo(rr(pd, pd), cc(pd, pd), Se, (N, N))
        C = coo(rr(pd, pd), cc(pd, pd), Ce, (N, N))

        self.fg = None
        if prob.kf is not None:
            fg = fault_geometry(m)
            self.fg = fg
            pairs = fg["pairs"]
            A = fg["area"]
            nrm = fg["n"]
            mi, pl = pairs[:, 0], pairs[:, 1]
            # A^f_pu: force +/- A_i <p> n on the two lips (App. B, Eq. afpdp read as
            # the transpose of Eq. afdpd); <p> = (p+ + p-)/2, Eq. operators.
            rows, cols, vals = [], [], []
            for c in range(3):
                for lip, sgn in ((pl, 1.0), (mi, -1.0)):
                    for side in (pl, mi):
                        rows.append(c * N + lip)
                        cols.append(pdof[side])
                        vals.append(sgn * 0.5 * A * nrm[:, c])
            Apu = Apu + coo(np.concatenate(rows), np.concatenate(cols), np.concatenate(vals),
                            (3 * N, N))
            # storage of the fracture: int <r> w S_F <p>, S_F = 1/M_F, lumped (Sec. 3.2.3)
            st = A * fp.w0 / fp.MF
            rows, cols, vals = [], [], []
            for s1 in (pl, mi):
                for s2 in (pl, mi):
                    rows.append(pdof[s1]); cols.append(pdof[s2]); vals.append(0.25 * st)
            S = S + coo(np.concatenate(rows), np.concatenate(cols), np.concatenate(vals), (N, N))
            # longitudinal flow: int (w k_par / mu) grad<r> . grad<p>   (Sec. 3.2.3)
            quads = fg["quads"]
            Lq = fg["Lq"] * (fp.wk_par / prob.mu_f)
            rows, cols, vals = [], [], []
            for s1 in (pl, mi):
                for s2 in (pl, mi):
                    r_ = pdof[s1][quads]
                    c_ = pdof[s2][quads]
                    rows.append(rr(r_, c_)); cols.append(cc(r_, c_)); vals.append(0.25 * Lq)
            C = C + coo(np.concatenate([x.ravel() for x in rows]),
                        np.concatenate([x.ravel() for x in cols]),
                        np.concatenate([x.ravel() for x in vals]), (N, N))
            # transverse flow: int [[r]] (k_perp / (mu w)) [[p]]   (Sec. 3.2.3)
            if not self.tied:
                tr = A * fp.k_perp / (prob.mu_f * fp.w0)
                rows = np.concatenate([pl, pl, mi, mi])
                cols = np.concatenate([pl, mi, pl, mi])
                vals = np.concatenate([tr, -tr, -tr, tr])
                C = C + coo(rows, cols, vals, (N, N))
        self.Apu = Apu
        self.S = S
        self.C = C

        # constraints: homogeneous Dirichlet, plus the slave (upper-lip) pressure
        # dofs of tied pairs, which carry no equation of their own
        fixed = np.asarray(prob.fixed, bool).copy()
        if self.tied and prob.kf is not None:
            fixed[3, m.pairs()[:, 1]] = True
        self.fixed = fixed
        self.free_u = ~fixed[0:3].reshape(-1)
        self.free_p = ~fixed[3]
        fu = np.asarray(prob.fu, float).reshape(-1).copy()
        fpv = np.zeros(N)
        np.add.at(fpv, pdof, np.asarray(prob.fp, float))
        self.fu = fu
        self.fpv = fpv
        self.dK = self.Kb.diagonal()

    # -- helpers ------------------------------------------------------------
    def A22(self, dt):
        return (self.S + dt * self.C).tocsr()

    def expand_p(self, p):
        """Copy master pressures onto the slave (upper-lip) nodes of tied pairs."""
        return p[self.pdof]

    def jump(self, u):
        """[[u]] = u+ - u- per pair, (n_pairs, 3); u as (3N,) component-major."""
        N = self.N
        pairs = self.fg["pairs"]
        U = u.reshape(3, N)
        return (U[:, pairs[:, 1]] - U[:, pairs[:, 0]]).T


def elements_touching(mesh: Mesh, nodes):
    """Element ids adjacent to the given nodes (and, for tied pairs, to the
    partner lip), for sampled row checks."""
    nodes = np.asarray(nodes, dtype=np.int64)
    nb = mesh.nb
    kk = nodes // nb
    rem = nodes % nb
    j = rem // (mesh.nx + 1)
    i = rem % (mesh.nx + 1)
    if mesh.kf is not None:
        lip = (kk == mesh.kf) | (kk == mesh.kf + 1)
        partner = np.where(kk == mesh.kf, kk + 1, kk - 1)
        i = np.concatenate([i, i[lip]])
        j = np.concatenate([j, j[lip]])
        kk = np.concatenate([kk, partner[lip]])
    out = set()
    for di in (-1, 0):
        for dj in (-1, 0):
            for dk in (-1, 0):
                ei, ej = i + di, j + dj
                kb = kk + dk                       # element's lower extended plane
                if mesh.kf is not None:
                    ok_gap = kb != mesh.kf         # no element spans the fault gap
                    ek = np.where(kb > mesh.kf, kb - 1, kb)
                else:
                    ok_gap = np.ones_like(kb, dtype=bool)
                    ek = kb
                ok = (ei >= 0) & (ei < mesh.nx) & (ej >= 0) & (ej < mesh.ny) & \
                     (ek >= 0) & (ek < mesh.nz) & (kb >= 0) & (kb + 1 < mesh.nplanes) & ok_gap
                e = ei + mesh.nx * (ej + mesh.ny * ek)
                out.update(e[ok].tolist())
    return np.array(sorted(out), dtype=np.int64)
