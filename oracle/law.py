"""Cohesive-fault constitutive law for the oracle: penalty contact, Mohr-Coulomb
yield, elastic-predictor / plastic-corrector return map.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Paper Sec. 2.2.1:
  Eq. normal_traction   t'_n = k_n |delta_n| for delta_n <= 0, zero (no tension)
                        when the lips separate;
  Eq. yield_function    F = |t'_s| - f t'_n <= 0;
  Eq. slip_split        delta_s = delta_el + delta_ie,  t'_s = k_s delta_el;
  Eq. plastic_slip_increment / kuhn-tucker
                        d delta_ie = d lambda tau, tau = t'_s / |t'_s|;
  Eq. corrector         d lambda = (|t'^tr_s| - f t'_n) / k_s.
In-situ state (Sec. 2.1, incremental form; Sec. 4.2 initial tractions): the
displacement u is measured from the pre-injection equilibrium, in which the
lips carry t'_n0 and tau0.  Hence the total normal opening is
delta_n = n.[[u]] - t'_n0 / k_n and the total slip is P_t [[u]] + tau0 / k_s
with delta_ie = 0 initially.

Tie rules: delta_n <= 0 is contact (t'_n >= 0); F <= 0 or |t^tr| = 0 is STICK.

Tangent (symmetric reading, used by both Newton solvers so their paths agree):
  STICK  k_n n n^T + k_s P_t
  SLIP   k_n n n^T + k_s (f t'_n / |t^tr|) (P_t - tau tau^T)
  OPEN   0
Pinned by: closed-form single-pair cases in tests/test_oracle_law.py.
"""
from __future__ import annotations

import numpy as np

OPEN, STICK, SLIP = 0, 1, 2


def return_map(jump, n, t1, t2, kn, ks, f, tn0, tau0, dlie_prev):
    """Evaluate the fault law at every node pair.

    jump      (P, 3) displacement jump [[u]] = u+ - u- in global axes
    n,t1,t2   (P, 3) local frame
    f         scalar or (P,) friction coefficient
    tn0, tau0 in-situ effective normal traction (scalar or (P,)) and shear
              traction in the frame (t1, t2) ((2,) or (P, 2)); depth-dependent
              in-situ stress gives one value per pair
    dlie_prev (P, 2) inelastic slip at the last accepted step, frame (t1, t2)
    Returns dict with
      state (P,) int, tn (P,), ts (P, 2), dlie (P, 2), dlam (P,),
      T (P, 3)  incremental conjugate traction  -(t'_n - t'_n0) n + (t_s - tau0)
      D (P, 3, 3) tangent of T with respect to [[u]]
      F (P,) trial yield value, ttr (P, 2) trial shear traction.
    """
    jump = np.asarray(jump, float)
    P = jump.shape[0]
    f = np.broadcast_to(np.asarray(f, float), (P,))
    tn0 = np.broadcast_to(np.asarray(tn0, float), (P,))
    tau0 = np.broadcast_to(np.asarray(tau0, float), (P, 2))
    dn = np.sum(n * jump, axis=1)
    gs = np.stack([np.sum(t1 * jump, axis=1), np.sum(t2 * jump, axis=1)], axis=1)
    tn_c = tn0 - kn * dn                      # contact traction if the lips touch
    contact = tn_c >= 0.0
    ttr = tau0 + ks * (gs - dlie_prev)
    nt = np.sqrt(np.sum(ttr * ttr, axis=1))
    tn = np.where(contact, tn_c, 0.0)
    F = nt - f * tn
    slip = contact & (F > 0.0) & (nt > 0.0)
    stick = contact & ~slip
    state = np.where(contact, np.where(slip, SLIP, STICK), OPEN)

    ts = np.zeros((P, 2))
    dlie = dlie_prev.copy()
    dlam = np.zeros(P)
    ts[stick] = ttr[stick]
    tau = np.zeros((P, 2))
    tau[slip] = ttr[slip] / nt[slip, None]
    dlam[slip] = F[slip] / ks
    ts[slip] = (f[slip] * tn[slip])[:, None] * tau[slip]
    dlie[slip] = dlie_prev[slip] + dlam[slip, None] * tau[slip]

    # incremental traction T = -(t'_n - t'_n0) n + (t_s - tau0), written without
    # subtracting the in-situ values where the algebra allows it:
    #   contact: -(t'_n - t'_n0) = k_n n.[[u]];  open: = t'_n0
    #   stick:   t_s - tau0 = k_s (g_s - delta_ie);  slip: f t'_n tau - tau0;  open: -tau0
    Tn = np.where(contact, kn * dn, tn0)
    Ts = np.zeros((P, 2))
    Ts[stick] = ks * (gs[stick] - dlie_prev[stick])
    Ts[slip] = ts[slip] - tau0[slip]
    Ts[state == OPEN] = -tau0[state == OPEN]
    T = Tn[:, None] * n + Ts[:, 0:1] * t1 + Ts[:, 1:2] * t2

    nn = np.einsum("pi,pj->pij", n, n)
    Pt = np.einsum("pi,pj->pij", t1, t1) + np.einsum("pi,pj->pij", t2, t2)
    taug = tau[:, 0:1] * t1 + tau[:, 1:2] * t2
    tt = np.einsum("pi,pj->pij", taug, taug)
    D = np.zeros((P, 3, 3))
    D[stick] = kn * nn[stick] + ks * Pt[stick]
    ratio = np.zeros(P)
    ratio[slip] = f[slip] * tn[slip] / nt[slip]
    D[slip] = kn * nn[slip] + ks * ratio[slip, None, None] * (Pt[slip] - tt[slip])
    return dict(state=state, tn=tn, ts=ts, dlie=dlie, dlam=dlam, T=T, D=D, F=F, ttr=ttr,
                dn=dn, gs=gs)
