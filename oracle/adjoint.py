"""Adjoint of one converged implicit step, for the oracle.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

For the converged step F(x; theta) = 0 (Sec. 3.3.1: r_m, r_f of Eq.
nonlinear_system with x = (u, p) the totals at the end of the step and the
previous state fixed), and an objective J(x),

    dJ/dtheta = - lambda^T dF/dtheta,   (dF/dx)^T lambda = (dJ/dx)^T  (free dofs),

with dF/dx the consistent Jacobian at the converged state and the fault states
frozen (stick / slip / open as found by the last return map).  The consistent
fault tangent of a slipping pair is nonsymmetric:
    dT/d[[u]] = k_n n n^T - f k_n tau n^T + k_s (f t'_n / |t^tr|)(P_t - tau tau^T),
the symmetric Newton tangent minus f k_n tau n^T (checked against finite
differences in tests/test_oracle_law.py).

Parameters theta: log k_e per element (enters C), the friction coefficient per
pair (enters the slip traction, dT/df = t'_n tau), and log Q, a common scaling
of the fluid sources (enters -dt f^p).

Pinned by: central finite differences of complete oracle steps
(tests/test_oracle_adjoint.py).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from .fem import Model, element_matrices
from .law import SLIP, return_map


def consistent_fault_terms(model: Model, u, dlie_prev, f=None):
    """Return map at u plus the consistent (nonsymmetric) cohesive Jacobian."""
    N = model.N
    fg = model.fg
    fp = model.prob.fault
    P = fg["pairs"].shape[0]
    fr = np.broadcast_to(np.asarray(fp.f if f is None else f, float), (P,))
    r = return_map(model.jump(u), fg["n"], fg["t1"], fg["t2"], fp.kn, fp.ks, fr, fp.tn0,
                   fp.tau0, dlie_prev)
    D = r["D"].copy()
    slip = r["state"] == SLIP
    tau = np.zeros((P, 3))
    nt = np.linalg.norm(r["ttr"], axis=1)
    tt = np.zeros((P, 2))
    tt[slip] = r["ttr"][slip] / nt[slip, None]
    tau = tt[:, 0:1] * fg["t1"] + tt[:, 1:2] * fg["t2"]
    D[slip] -= (fr[slip] * fp.kn)[:, None, None] * np.einsum("pi,pj->pij", tau[slip], fg["n"][slip])
    A = fg["area"]
    mi, pl = fg["pairs"][:, 0], fg["pairs"][:, 1]
    rows, cols, vals = [], [], []
    for a in range(3):
        for b in range(3):
            d = A * D[:, a, b]
            for (ra, sa) in ((pl, 1.0), (mi, -1.0)):
                for (cb, sb) in ((pl, 1.0), (mi, -1.0)):
                    rows.append(a * N + ra)
                    cols.append(b * N + cb)
                    vals.append(sa * sb * d)
    Kc = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                       shape=(3 * N, 3 * N)).tocsr()
    return r, Kc, tau, fr


def adjoint_of_last_step(model: Model, u, p, dlie_prev, dt, dJ_du=None, dJ_dp=None,
                         dJ_dslip=None, f=None):
    """Adjoint of the step ending at (u, p) (totals) from a previous state whose
    inelastic slip was dlie_prev.  See the module docstring."""
    N = model.N
    fu, fpf = model.free_u, model.free_p
    g_u = np.zeros(3 * N) if dJ_du is None else np.asarray(dJ_du, float).copy()
    g_p = np.zeros(N) if dJ_dp is None else np.asarray(dJ_dp, float).copy()
    P = 0 if model.fg is None else model.fg["pairs"].shape[0]
    if model.fg is not None:
        r, Kc, tau, fr = consistent_fault_terms(model, u, dlie_prev, f=f)
        if dJ_dslip is not None:
            fg = model.fg
            dsl = np.asarray(dJ_dslip, float)
            gvec = dsl[:, 0:1] * fg["t1"] + dsl[:, 1:2] * fg["t2"]   # d slip / d [[u]]
            for c in range(3):
                np.add.at(g_u, c * N + fg["pairs"][:, 1], gvec[:, c])
                np.add.at(g_u, c * N + fg["pairs"][:, 0], -gvec[:, c])
    else:
        Kc = sp.csr_matrix((3 * N, 3 * N))
        r = None
    # pressure gradient on slave dofs belongs to the master
    if model.tied and model.fg is not None:
        pairs = model.fg["pairs"]
        g_p[pairs[:, 0]] += g_p[pairs[:, 1]]
        g_p[pairs[:, 1]] = 0.0
    Jc = sp.bmat([[model.Kb + Kc, -model.Apu], [model.Apu.T, model.A22(dt)]]).tocsr()
    free = np.concatenate([fu, fpf])
    Jf = Jc[free][:, free]
    rhs = np.concatenate([g_u, g_p])[free]
    s = 1.0 / np.sqrt(np.abs(Jf.diagonal()))
    lam_f = s * spla.spsolve((sp.diags(s) @ Jf.T @ sp.diags(s)).tocsc(), s * rhs)
    lam = np.zeros(4 * N)
    lam[free] = lam_f
    lam_u, lam_p = lam[:3 * N], lam[3 * N:]
    # d F_f / d log k_e = dt (k_e/mu) L_e p_e  (element by element)
    m = model.mesh
    conn = m.connectivity()
    X = m.coords()
    prob = model.prob
    kap = np.broadcast_to(np.asarray(prob.k, float), (m.n_el,)) / prob.mu_f
    _, _, _, Ce = element_matrices(X[conn], np.broadcast_to(np.asarray(prob.E, float), (m.n_el,)),
                                   prob.nu, prob.alpha, 1.0 / prob.M, kap)
    pd = model.pdof[conn]
    pe = p[pd]
    le = lam_p[pd]
    g_logk = -dt * np.einsum("ea,eab,eb->e", le, Ce, pe)
    # d F_m / d f_i at slipping pairs: +- A_i t'_n tau on the lips
    g_f = np.zeros(P)
    if r is not None:
        fg = model.fg
        slip = r["state"] == SLIP
        jl = (lam_u.reshape(3, N)[:, fg["pairs"][:, 1]] - lam_u.reshape(3, N)[:, fg["pairs"][:, 0]]).T
        g_f[slip] = -(fg["area"] * r["tn"])[slip] * np.sum(tau[slip] * jl[slip], axis=1)
    # d F_f / d log Q = -dt f^p
    g_logQ = dt * float(lam_p @ model.fpv)
    return dict(g_logk=g_logk, g_f=g_f, g_logQ=g_logQ, lam_u=lam_u, lam_p=lam_p)
