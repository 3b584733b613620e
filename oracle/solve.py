"""Newton / time stepping and linear solvers for the oracle.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Paper Sec. 3.3:
  Eq. nonlinear_system  r_m = K(u) du - A_pu dp - f^u + K(u_n) u_n - A_pu p_n,
                        r_f = A_up du + (S + C dt) dp - (f^p - C p_n) dt,
    which for the linear bulk and the nonlinear fault reads
      r_m = K_b u + F_coh(u) - A_pu p - f^u,  r_f = A_up du + S dp + dt C p - dt f^p.
  Eq. linear_system     [K_T  -A_pu; A_up  S + C dt] [du; dp] = [-r_m; -r_f].
  Eqs. prevost_system / schur_system: A11 = K_T, A12 = -A_pu, A21 = A_up,
    A22 = S + C dt;  (A22 - A21 A11^-1 A12) x2 = b2 - A21 A11^-1 b1, solved by
    CG preconditioned with A22^-1;  x1 = A11^-1 (b1 - A12 x2).
A_up = A_pu^T (App. A Eq. Adpd is the transpose of Eq. Apdp; App. B likewise).

Newton stopping rule (the paper gives none): iteration i >= 1 stops when the
fault states equal those of iteration i - 1 and the Jacobi-scaled residual
  rhat = sqrt( sum b1^2 / diag(K_b) + sum b2^2 / diag(A22) )   (free dofs)
satisfies rhat <= rtol * max(rhat_0, 1e-3 * shat), where
  shat = sqrt( sum diag(K_b) u^2 + sum diag(A22) p^2 + sum F0^2 / diag(K_b) )
is the same scaling applied to the current total state and to F0, the nodal
force of the in-situ fault tractions (+/- A_i (-t'_n0 n + tau0) on the lips);
all terms have units of energy.  The shat term only sets a floor near the
rounding level of the residual evaluation when a step changes little.

Pinned by: tests/test_oracle_solvers.py (dense LU = sparse direct = Prevost CG
on faulted boxes, tied and untied; Newton paths equal across the linear
solvers; the unit-cube case reaches open, stick and slip without near-ties;
1-D consolidation against the series at second order; line-source pressure
front within the paper's 8 %).
"""
from __future__ import annotations

import dataclasses

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from .fem import Model
from .law import return_map


@dataclasses.dataclass
class State:
    u: np.ndarray        # (3N,) component-major total displacement since t = 0
    p: np.ndarray        # (N,) pressure, master dofs (tied slaves hold 0)
    dlie: np.ndarray     # (P, 2) inelastic slip
    flags: np.ndarray    # (P,) fault state at the last accepted step
    t: float = 0.0


def initial_state(model: Model) -> State:
    P = 0 if model.fg is None else model.fg["pairs"].shape[0]
    return State(u=np.zeros(3 * model.N), p=np.zeros(model.N), dlie=np.zeros((P, 2)),
                 flags=np.ones(P, dtype=np.int64))


def fault_terms(model: Model, u, dlie_prev, f=None):
    """Return map at every pair plus its nodal force vector and tangent matrix.

    force: A_i T on the upper lip, -A_i T on the lower lip (nodal quadrature).
    Kcoh:  A_i D on (+,+) and (-,-), -A_i D on (+,-) and (-,+).
    """
    N = model.N
    if model.fg is None:
        return None, np.zeros(3 * N), sp.csr_matrix((3 * N, 3 * N))
    fg = model.fg
    fp = model.prob.fault
    r = return_map(model.jump(u), fg["n"], fg["t1"], fg["t2"], fp.kn, fp.ks,
                   fp.f if f is None else f, fp.tn0, fp.tau0, dlie_prev)
    A = fg["area"]
    mi, pl = fg["pairs"][:, 0], fg["pairs"][:, 1]
    force = np.zeros(3 * N)
    for c in range(3):
        force[c * N + pl] += A * r["T"][:, c]
        force[c * N + mi] -= A * r["T"][:, c]
    rows, cols, vals = [], [], []
    for a in range(3):
        for b in range(3):
            d = A * r["D"][:, a, b]
            for (ra, sa) in ((pl, 1.0), (mi, -1.0)):
                for (cb, sb) in ((pl, 1.0), (mi, -1.0)):
                    rows.append(a * N + ra)
                    cols.append(b * N + cb)
                    vals.append(sa * sb * d)
    Kcoh = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                         shape=(3 * N, 3 * N)).tocsr()
    return r, force, Kcoh


def residuals(model: Model, st: State, du, dp, dt, force):
    """b1 = -r_m, b2 = -r_f of Eq. nonlinear_system; constrained dofs zeroed."""
    u = st.u + du
    p = st.p + dp
    b1 = model.fu - model.Kb @ u - force + model.Apu @ p
    b2 = dt * (model.fpv - model.C @ p) - model.S @ dp - model.Apu.T @ du
    b1[~model.free_u] = 0.0
    b2[~model.free_p] = 0.0
    return b1, b2


def insitu_floor(model: Model):
    """sum over free lip dofs of F0^2 / diag(K_b), F0 = +/- A_i (-t'_n0 n + tau0)."""
    if model.fg is None:
        return 0.0
    fg = model.fg
    fp = model.prob.fault
    P = fg["n"].shape[0]
    tn0 = np.broadcast_to(np.asarray(fp.tn0, float), (P,))[:, None]
    tau0 = np.broadcast_to(np.asarray(fp.tau0, float), (P, 2))
    F0 = (-tn0 * fg["n"] + tau0[:, 0:1] * fg["t1"] + tau0[:, 1:2] * fg["t2"]) * fg["area"][:, None]
    N = model.N
    tot = 0.0
    for lip in (fg["pairs"][:, 0], fg["pairs"][:, 1]):
        for c in range(3):
            d = c * N + lip
            ok = model.free_u[d]
            tot += float(np.sum(F0[ok, c] ** 2 / model.dK[d[ok]]))
    return tot


def scaled_norm(model: Model, b1, b2, dA):
    fu, fp = model.free_u, model.free_p
    return float(np.sqrt(np.sum(b1[fu] ** 2 / model.dK[fu]) + np.sum(b2[fp] ** 2 / dA[fp])))


def jacobian_blocks(model: Model, Kcoh, dt):
    fu, fp = model.free_u, model.free_p
    KT = (model.Kb + Kcoh).tocsr()[fu][:, fu]
    Apu = model.Apu.tocsr()[fu][:, fp]
    A22 = model.A22(dt)[fp][:, fp]
    return KT, Apu, A22


def solve_monolithic(KT, Apu, A22, b1, b2, dense=True):
    """Eq. linear_system solved directly (dense LU with partial pivoting, or a
    sparse direct factorisation)."""
    J = sp.bmat([[KT, -Apu], [Apu.T, A22]]).tocsc()
    rhs = np.concatenate([b1, b2])
    # symmetric Jacobi scaling: the mechanical and flow blocks differ by ~20
    # orders of magnitude; scaling changes nothing mathematically
    s = 1.0 / np.sqrt(np.abs(J.diagonal()))
    Js = (sp.diags(s) @ J @ sp.diags(s)).tocsc()
    if dense:
        x = s * sla.solve(Js.toarray(), s * rhs)
    else:
        x = s * spla.spsolve(Js, s * rhs)
    n1 = KT.shape[0]
    return x[:n1], x[n1:]


def solve_prevost(KT, Apu, A22, b1, b2, rtol=1e-13, maxit=1000):
    """Prevost's partitioned CG (Sec. 3.3.2, Eq. schur_system) with exact inner
    solves by sparse LU.  Schur operator S~ x = A22 x + A_pu^T K^-1 A_pu x,
    preconditioner A22^-1, x2_0 = 0.  Returns (x1, x2, iterations)."""
    K_lu = spla.splu(KT.tocsc())
    A_lu = spla.splu(A22.tocsc())
    y1 = K_lu.solve(b1)
    r = b2 - Apu.T @ y1                       # b2 - A21 A11^-1 b1
    x2 = np.zeros_like(b2)
    r0 = np.linalg.norm(r)
    z = A_lu.solve(r)
    pdir = z.copy()
    rz = r @ z
    it = 0
    while np.linalg.norm(r) > rtol * r0 and r0 > 0 and it < maxit:
        q = A22 @ pdir + Apu.T @ K_lu.solve(Apu @ pdir)
        alpha = rz / (pdir @ q)
        x2 += alpha * pdir
        r -= alpha * q
        z = A_lu.solve(r)
        rz_new = r @ z
        pdir = z + (rz_new / rz) * pdir
        rz = rz_new
        it += 1
    x1 = K_lu.solve(b1 + Apu @ x2)            # A11^-1 (b1 - A12 x2)
    return x1, x2, it


@dataclasses.dataclass
class StepResult:
    u: np.ndarray           # (3, N)
    p: np.ndarray           # (N,) with tied slave values filled in
    slip: np.ndarray        # (P, 2) P_t [[u]] in the fault frame
    dlie: np.ndarray        # (P, 2)
    flags: np.ndarray       # (P,)
    newton: int
    rhat: float
    rhat0: float
    F: np.ndarray           # (P,) yield values at the converged state
    tn: np.ndarray          # (P,) effective normal traction
    dn: np.ndarray          # (P,) n.[[u]]


def implicit_step(model: Model, st: State, dt: float, rtol=1e-12, maxit=50, solver="auto",
                  f=None, inner_rtol=1e-14):
    """One backward-Euler step: Newton on Eq. nonlinear_system (Sec. 3.3.1)."""
    fu, fp = model.free_u, model.free_p
    du = np.zeros(3 * model.N)
    dp = np.zeros(model.N)
    dA = model.A22(dt).diagonal()
    prev_state = None
    rhat0 = None
    f0sq = insitu_floor(model)
    for it in range(maxit + 1):
        r, force, Kcoh = fault_terms(model, st.u + du, st.dlie, f=f)
        b1, b2 = residuals(model, st, du, dp, dt, force)
        rhat = scaled_norm(model, b1, b2, dA)
        if rhat0 is None:
            rhat0 = rhat
        ut, pt = st.u + du, st.p + dp
        shat = float(np.sqrt(np.sum(model.dK[fu] * ut[fu] ** 2) + np.sum(dA[fp] * pt[fp] ** 2)
                             + f0sq))
        states = None if r is None else r["state"]
        if states is None:
            same = True
        else:
            same = prev_state is not None and np.array_equal(states, prev_state)
        if it > 0 and same and rhat <= rtol * max(rhat0, 1e-3 * shat):
            break
        if it == maxit:
            raise RuntimeError(f"Newton did not converge: rhat/rhat0={rhat / max(rhat0, 1e-300):.3e}")
        KT, Apu, A22 = jacobian_blocks(model, Kcoh, dt)
        if solver == "auto":
            solver = "lu" if KT.shape[0] + A22.shape[0] <= 6000 else "sparse"
        if solver == "lu":
            x1, x2 = solve_monolithic(KT, Apu, A22, b1[fu], b2[fp], dense=True)
        elif solver == "sparse":
            x1, x2 = solve_monolithic(KT, Apu, A22, b1[fu], b2[fp], dense=False)
        elif solver == "prevost":
            x1, x2, _ = solve_prevost(KT, Apu, A22, b1[fu], b2[fp], rtol=inner_rtol)
        else:
            raise ValueError(solver)
        du[fu] += x1
        dp[fp] += x2
        prev_state = states
    st.u = st.u + du
    st.p = st.p + dp
    st.t += dt
    P = 0 if r is None else r["state"].size
    if r is not None:
        st.dlie = r["dlie"].copy()
        st.flags = r["state"].copy()
    N = model.N
    return StepResult(u=st.u.reshape(3, N).copy(), p=model.expand_p(st.p).copy(),
                      slip=(np.zeros((0, 2)) if r is None else r["gs"].copy()),
                      dlie=st.dlie.copy(), flags=st.flags.copy(), newton=it, rhat=rhat,
                      rhat0=rhat0, F=(np.zeros(P) if r is None else r["F"].copy()),
                      tn=(np.zeros(P) if r is None else r["tn"].copy()),
                      dn=(np.zeros(P) if r is None else r["dn"].copy()))


def run(prob, nsteps=None, model=None, **kw):
    """Run the time loop of a workloads.Problem; returns (model, [StepResult])."""
    model = Model(prob) if model is None else model
    st = initial_state(model)
    out = []
    dts = prob.dts if nsteps is None else prob.dts[:nsteps]
    for dt in dts:
        out.append(implicit_step(model, st, dt, **kw))
    return model, out


# ---------------------------------------------------------------------------
# Single operator applications (for the GPU apply parity tests)
# ---------------------------------------------------------------------------

def apply(model: Model, which: str, u=None, p=None, dt=1.0, Kcoh=None):
    """Constrained operator products y = P_f A P_f x on free dofs.

    which: 'Kb' (bulk elasticity), 'KT' (K_b + fault tangent, needs Kcoh),
    'A22' (S + dt C), 'Apu', 'Aup' (= Apu^T), 'J' (Eq. linear_system matrix).
    u: (3N,) component-major, p: (N,) master dofs.  Returns (yu, yp).
    """
    fu, fp = model.free_u, model.free_p
    N = model.N
    uz = None if u is None else np.where(fu, u, 0.0)
    pz = None if p is None else np.where(fp, p, 0.0)
    yu = np.zeros(3 * N)
    yp = np.zeros(N)
    if which == "Kb":
        yu = model.Kb @ uz
    elif which == "KT":
        yu = (model.Kb + Kcoh) @ uz
    elif which == "A22":
        yp = model.A22(dt) @ pz
    elif which == "Apu":
        yu = model.Apu @ pz
    elif which == "Aup":
        yp = model.Apu.T @ uz
    elif which == "J":
        yu = (model.Kb + Kcoh) @ uz - model.Apu @ pz
        yp = model.Apu.T @ uz + model.A22(dt) @ pz
    else:
        raise ValueError(which)
    yu = np.where(fu, yu, 0.0)
    yp = np.where(fp, yp, 0.0)
    return yu, yp
