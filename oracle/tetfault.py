"""Oracle of the paper's own discretisation with a fault: P1 tetrahedra for
displacement and pressure and zero-thickness interface elements on the
triangles of the fault surface (Sec. 3.1.1-3.1.2), on meshes with one planar
fault of duplicated nodes (workloads.FaultedTetProblem).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

The interface terms are those of the structured oracle (fem.Model) with the
bilinear fault quads replaced by linear triangles:
  - tractions, fault storage and the A^f couplings use nodal quadrature on
    each triangle (weight area / 3 at each vertex; exact for linear fields),
    so each node pair carries one integration point of weight A_i, the same
    reading as for the quads;
  - the pair normal is the normalised area-weighted sum of the normals of
    the triangles around the pair (Sec. 3.1.1: the element normal averages
    the facet normals); t1 is the unit projection of the problem's reference
    direction onto the plane normal to n, t2 = n x t1;
  - the longitudinal Laplacian of a triangle is (w k_par / mu) a_t G_t G_t^T
    with G_t the constant surface gradients of its shape functions (exact).
The contact / Coulomb return map, the Newton loop and the linear solvers are
those of law.py and solve.py, applied unchanged to this model.

Pinned by: tests/test_oracle_tetfault.py (fault area, normal and frame of a
sheared plane; Laplacian kernel and linear-field energy; rigid modes 12 / 6
for an open / stuck fault; nodal forces of a constant stress at the lips
against -/+ A_i sigma n; uniform lip pressure force and aperture volume;
line-source pressure front within the paper's 8 % and profile within 6 % of
dp*; dense LU = Prevost CG on the Newton step).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from . import solve
from .tet import tet_element_matrices


def triangle_fault_geometry(nodes, pairs, tris, t1_ref):
    """Per pair: tributary area, unit normal (minus -> plus), tangents; per
    triangle: area and the unit-coefficient Laplacian a_t G_t G_t^T (T, 3, 3).
    Sec. 3.1.1 (interface element geometry, averaged facet normals) and Sec.
    3.2.3 (longitudinal fracture flow), on linear triangles."""
    X = nodes[pairs[tris, 0]]                                   # (T, 3, 3) minus lip
    e1 = X[:, 1] - X[:, 0]
    e2 = X[:, 2] - X[:, 0]
    cr = np.cross(e1, e2)                                       # 2 a_t n_t
    at = 0.5 * np.linalg.norm(cr, axis=1)
    P = pairs.shape[0]
    area = np.zeros(P)
    nsum = np.zeros((P, 3))
    for b in range(3):
        np.add.at(area, tris[:, b], at / 3.0)
        np.add.at(nsum, tris[:, b], cr / 6.0)                   # (a_t / 3) n_t
    if np.any(area <= 0.0):
        raise ValueError("a fault pair lies on no fault triangle")
    n = nsum / np.linalg.norm(nsum, axis=1)[:, None]
    d = np.asarray(t1_ref, float)
    e = d[None, :] - (n @ d)[:, None] * n
    t1 = e / np.linalg.norm(e, axis=1)[:, None]
    t2 = np.cross(n, t1)
    Js = np.stack([e1, e2], axis=2)                             # (T, 3, 2)
    Gm = np.einsum("tdk,tdl->tkl", Js, Js)
    dN = np.array([[-1.0, -1.0], [1.0, 0.0], [0.0, 1.0]])
    Lt = at[:, None, None] * np.einsum("ak,tkl,bl->tab", dN, np.linalg.inv(Gm), dN)
    return dict(pairs=pairs, tris=tris, area=area, n=n, t1=t1, t2=t2, at=at, Lt=Lt)


def _coo(rows, cols, vals, shape):
    return sp.coo_matrix((np.ravel(vals), (np.ravel(rows), np.ravel(cols))), shape=shape).tocsr()


class TetFaultModel:
    """Assembled operators of a FaultedTetProblem, with the attributes the
    Newton loop of solve.py reads (N, prob, fg, Kb, Apu, S, C, free_u, free_p,
    fu, fpv, dK, A22, jump, expand_p): the bulk P1 operators of Sec. 3.2 and
    App. A, and the fault blocks of Sec. 3.2.3 and App. B (A^f_pu read as the
    transpose of A^f_up, storage w/M_F, tied or transverse lip pressures)."""

    def __init__(self, prob):
        self.prob = prob
        N = prob.nodes.shape[0]
        self.N = N
        fp = prob.fault
        pairs = np.asarray(prob.pairs, np.int64)
        T = np.asarray(prob.tets, np.int64)
        self.tied = not (fp.k_perp > 0)
        pdof = np.arange(N)
        if self.tied:
            pdof[pairs[:, 1]] = pairs[:, 0]
        self.pdof = pdof
        K, A, Ms, L = tet_element_matrices(prob.nodes[T], prob.E, prob.nu, prob.alpha, 1.0 / prob.M,
                                           np.asarray(prob.k, float) / prob.mu_f)
        udof = np.stack([c * N + T for c in range(3)], axis=2).reshape(T.shape[0], 12)
        pd = pdof[T]
        rr = lambda a, b: np.broadcast_to(a[:, :, None], (a.shape[0], a.shape[1], b.shape[1]))
        cc = lambda a, b: np.broadcast_to(b[:, None, :], (a.shape[0], a.shape[1], b.shape[1]))
        self.Kb = _coo(rr(udof, udof), cc(udof, udof), K, (3 * N, 3 * N))
        Apu = _coo(rr(udof, pd), cc(udof, pd), A, (3 * N, N))
        S = _coo(rr(pd, pd), cc(pd, pd), Ms, (N, N))
        C = _coo(rr(pd, pd), cc(pd, pd), L, (N, N))

        fg = triangle_fault_geometry(prob.nodes, pairs, np.asarray(prob.fault_tris, np.int64),
                                     prob.t1_ref)
        self.fg = fg
        Ai, nrm = fg["area"], fg["n"]
        mi, pl = pairs[:, 0], pairs[:, 1]
        # A^f_pu: force +/- A_i <p> n on the two lips, <p> = (p+ + p-) / 2
        rows, cols, vals = [], [], []
        for c in range(3):
            for lip, sgn in ((pl, 1.0), (mi, -1.0)):
                for side in (pl, mi):
                    rows.append(c * N + lip)
                    cols.append(pdof[side])
                    vals.append(sgn * 0.5 * Ai * nrm[:, c])
        self.Apu_f = _coo(np.concatenate(rows), np.concatenate(cols), np.concatenate(vals), (3 * N, N))
        # fracture storage A_i w / M_F on <p> (lumped)
        st = Ai * fp.w0 / fp.MF
        rows, cols, vals = [], [], []
        for s1 in (pl, mi):
            for s2 in (pl, mi):
                rows.append(pdof[s1]); cols.append(pdof[s2]); vals.append(0.25 * st)
        S_f = _coo(np.concatenate(rows), np.concatenate(cols), np.concatenate(vals), (N, N))
        # longitudinal flow (w k_par / mu) on <p> over the fault triangles
        tris = fg["tris"]
        Lt = fg["Lt"] * (fp.wk_par / prob.mu_f)
        rows, cols, vals = [], [], []
        for s1 in (pl, mi):
            for s2 in (pl, mi):
                r_ = pdof[s1][tris]
                c_ = pdof[s2][tris]
                rows.append(rr(r_, c_).ravel()); cols.append(cc(r_, c_).ravel())
                vals.append((0.25 * Lt).ravel())
        C_f = _coo(np.concatenate(rows), np.concatenate(cols), np.concatenate(vals), (N, N))
        if not self.tied:
            tr = Ai * fp.k_perp / (prob.mu_f * fp.w0)
            C_f = C_f + _coo(np.concatenate([pl, pl, mi, mi]), np.concatenate([pl, mi, pl, mi]),
                             np.concatenate([tr, -tr, -tr, tr]), (N, N))
        self.S_f, self.C_f = S_f, C_f
        self.Apu = (Apu + self.Apu_f).tocsr()
        self.S = (S + S_f).tocsr()
        self.C = (C + C_f).tocsr()

        fixed = np.asarray(prob.fixed, bool).copy()
        if self.tied:
            fixed[3, pl] = True
        self.fixed = fixed
        self.free_u = ~fixed[0:3].reshape(-1)
        self.free_p = ~fixed[3]
        self.fu = np.asarray(prob.fu, float).reshape(-1).copy()
        fpv = np.zeros(N)
        np.add.at(fpv, pdof, np.asarray(prob.fp, float))
        self.fpv = fpv
        self.dK = self.Kb.diagonal()

    def A22(self, dt):
        return (self.S + dt * self.C).tocsr()

    def expand_p(self, p):
        return p[self.pdof]

    def jump(self, u):
        U = u.reshape(3, self.N)
        pairs = self.fg["pairs"]
        return (U[:, pairs[:, 1]] - U[:, pairs[:, 0]]).T


def run(prob, nsteps=None, model=None, **kw):
    """Time loop of a FaultedTetProblem through solve.implicit_step; returns
    (model, [StepResult])."""
    model = TetFaultModel(prob) if model is None else model
    st = solve.initial_state(model)
    dts = prob.dts if nsteps is None else prob.dts[:nsteps]
    return model, [solve.implicit_step(model, st, dt, **kw) for dt in dts]
