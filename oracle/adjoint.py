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
                         dJ_dslip=None, f=None, extra_u=None, extra_p=None):
    """Adjoint of the step ending at (u, p) (totals) from a previous state whose
    inelastic slip was dlie_prev.  See the module docstring.  extra_u / extra_p
    are added to the right-hand side (history terms of a multi-step adjoint)."""
    N = model.N
    fu, fpf = model.free_u, model.free_p
    g_u = np.zeros(3 * N) if dJ_du is None else np.asarray(dJ_du, float).copy()
    g_p = np.zeros(N) if dJ_dp is None else np.asarray(dJ_dp, float).copy()
    if extra_u is not None:
        g_u += extra_u
    if extra_p is not None:
        g_p += extra_p
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


# ---------------------------------------------------------------------------
# Several steps: the inelastic slip h_n = delta_ie after step n is history.
# Step n: F_n(x_n; x_{n-1}, h_{n-1}, theta) = 0 and h_n = H_n(x_n, h_{n-1}, theta),
# H_n = h_{n-1} for stick/open pairs and h_{n-1} + (F/k_s) tau for slipping ones
# (Eq. plastic_slip_increment with Eq. corrector).  With the Lagrangian
#   L = J - sum_n lambda_n^T F_n - sum_n mu_n^T (h_n - H_n)
# the reverse sweep is, for n = K .. 1 (lambda_{K+1} = 0, mu_K = 0 when J does
# not depend on h_K):
#   mu_n = -(dF_{n+1}/dh_n)^T lambda_{n+1} + (dH_{n+1}/dh_n)^T mu_{n+1}
#   (dF_n/dx_n)^T lambda_n = dJ/dx_n - (dF_{n+1}/dx_n)^T lambda_{n+1} + (dH_n/dx_n)^T mu_n
#   dJ/dtheta = sum_n [ -lambda_n^T dF_n/dtheta + mu_n^T dH_n/dtheta ]
# where -(dF_{n+1}/dx_n)^T lambda_{n+1} = [A_pu lambda_p ; S lambda_p]_{n+1}
# (the flow residual holds -A_up u_n - S p_n).  Per pair, in the fault frame
# (tau = t^tr/|t^tr|, r = f t'_n/|t^tr|, F the trial yield value):
#   dT_s/dh: stick -k_s I, slip -k_s r (I - tau tau^T), open 0
#   dH/dh  : stick/open I, slip (1 - F/|t^tr|)(I - tau tau^T)
#   dH/dg_s: slip tau tau^T + (F/|t^tr|)(I - tau tau^T),  dH/d delta_n: slip (f k_n/k_s) tau
#   dH/df  : slip -(t'_n/k_s) tau
# ---------------------------------------------------------------------------

def frozen_pairs(model: Model, u, h_prev, f=None):
    fg = model.fg
    fp = model.prob.fault
    P = fg["pairs"].shape[0]
    fr = np.broadcast_to(np.asarray(fp.f if f is None else f, float), (P,))
    r = return_map(model.jump(u), fg["n"], fg["t1"], fg["t2"], fp.kn, fp.ks, fr, fp.tn0,
                   fp.tau0, h_prev)
    nt = np.sqrt(np.sum(r["ttr"] ** 2, axis=1))
    tau = np.zeros((P, 2))
    sl = r["state"] == SLIP
    tau[sl] = r["ttr"][sl] / nt[sl, None]
    return dict(state=r["state"], tn=r["tn"], nt=nt, F=r["F"], tau=tau, f=fr, dlie=r["dlie"])


def _lip_jump(model, lam_u):
    N = model.N
    pairs = model.fg["pairs"]
    L = lam_u.reshape(3, N)
    return (L[:, pairs[:, 1]] - L[:, pairs[:, 0]]).T            # (P, 3)


def history_mu(model: Model, fz_next, lam_u_next, mu_next):
    """mu_n from step n+1's frozen pair data and adjoints."""
    fg = model.fg
    fp = model.prob.fault
    A = fg["area"]
    dl = _lip_jump(model, lam_u_next)
    dls = np.stack([np.sum(fg["t1"] * dl, 1), np.sum(fg["t2"] * dl, 1)], axis=1)   # (P, 2)
    P = dls.shape[0]
    mu = np.zeros((P, 2))
    st = fz_next["state"]
    stick = st == 1
    slip = st == SLIP
    mu[stick] = (A[stick] * fp.ks)[:, None] * dls[stick] + mu_next[stick]
    t = fz_next["tau"][slip]
    proj = lambda v: v - np.sum(t * v, axis=1)[:, None] * t                    # (I - tau tau^T) v
    rr = fz_next["f"][slip] * fz_next["tn"][slip] / fz_next["nt"][slip]
    mu[slip] = (A[slip] * fp.ks * rr)[:, None] * proj(dls[slip]) \
        + (1.0 - fz_next["F"][slip] / fz_next["nt"][slip])[:, None] * proj(mu_next[slip])
    open_ = st == 0
    mu[open_] = mu_next[open_]
    return mu


def history_rhs_u(model: Model, fz, mu):
    """(dH_n/dx_n)^T mu_n as a (3N,) vector on the lips, and mu^T dH/df per pair."""
    N = model.N
    fg = model.fg
    fp = model.prob.fault
    P = mu.shape[0]
    slip = fz["state"] == SLIP
    t = fz["tau"]
    ratio = np.zeros(P)
    ratio[slip] = fz["F"][slip] / fz["nt"][slip]
    # dH/dg_s^T mu = tau (tau.mu) + ratio (mu - tau (tau.mu));  dH/d dn^T mu = (f kn/ks) tau.mu
    tm = np.sum(t * mu, axis=1)
    gs = t * tm[:, None] + ratio[:, None] * (mu - t * tm[:, None])
    gn = fz["f"] * fp.kn / fp.ks * tm
    vec = gs[:, 0:1] * fg["t1"] + gs[:, 1:2] * fg["t2"] + gn[:, None] * fg["n"]
    vec[~slip] = 0.0
    out = np.zeros(3 * N)
    for c in range(3):
        np.add.at(out, c * N + fg["pairs"][:, 1], vec[:, c])
        np.add.at(out, c * N + fg["pairs"][:, 0], -vec[:, c])
    gf = np.where(slip, -(fz["tn"] / fp.ks) * tm, 0.0)
    return out, gf


def adjoint_multistep(model: Model, traj, dts, dJ_du=None, dJ_dp=None, dJ_dslip=None, f=None):
    """Reverse sweep over a trajectory.

    traj[n] (n = 0 .. K-1) holds the state after step n+1: u (3N,), p (N,) master
    dofs, and h_prev (P, 2) the inelastic slip before that step.  The objective
    depends on the final state only (dJ_* as in adjoint_of_last_step).
    Returns dict(g_logk, g_f, g_logQ)."""
    K = len(traj)
    N = model.N
    P = model.fg["pairs"].shape[0]
    g_logk = np.zeros(model.mesh.n_el)
    g_f = np.zeros(P)
    g_logQ = 0.0
    lam_next = None
    mu_next = np.zeros((P, 2))
    fz_next = None
    for n in range(K - 1, -1, -1):
        s = traj[n]
        fz = frozen_pairs(model, s["u"], s["h_prev"], f=f)
        if n == K - 1:
            mu = np.zeros((P, 2))
            ex_u = np.zeros(3 * N)
            ex_p = np.zeros(N)
        else:
            mu = history_mu(model, fz_next, lam_next[:3 * N], mu_next)
            lp = lam_next[3 * N:]
            ex_u = model.Apu @ lp
            ex_p = model.S @ lp
        hu, gf_h = history_rhs_u(model, fz, mu)
        ex_u = ex_u + hu
        last = n == K - 1
        g = adjoint_of_last_step(model, s["u"], s["p"], s["h_prev"], dts[n],
                                 dJ_du=dJ_du if last else None, dJ_dp=dJ_dp if last else None,
                                 dJ_dslip=dJ_dslip if last else None, f=f,
                                 extra_u=ex_u, extra_p=ex_p)
        g_logk += g["g_logk"]
        g_f += g["g_f"] + gf_h
        g_logQ += g["g_logQ"]
        lam_next = np.concatenate([g["lam_u"], g["lam_p"]])
        mu_next = mu
        fz_next = fz
    return dict(g_logk=g_logk, g_f=g_f, g_logQ=g_logQ)
