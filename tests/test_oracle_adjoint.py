"""Pins for the oracle's single-step adjoint: gradients of a slip + pressure
objective w.r.t. element log-permeability, the friction coefficient and the
log source scaling, against central finite differences of complete oracle
steps (tolerance 1e-5 relative; the active set does not change under the
perturbations)."""
import copy
import math

import numpy as np
import pytest

import workloads as W
from oracle import adjoint, fem, solve

S0, P0 = 1e-6, 1e6


def setup_case():
    prob = W.fault_small(n=6, Q=5e-5, steps=3)
    model = fem.Model(prob)
    st = solve.initial_state(model)
    for dt in prob.dts[:2]:
        solve.implicit_step(model, st, dt, rtol=1e-13)
    rng = np.random.default_rng(5)
    P = model.fg["pairs"].shape[0]
    obs_pairs = rng.choice(P, 12, replace=False)
    obs_nodes = rng.choice(model.N, 8, replace=False)
    obs_nodes = obs_nodes[model.free_p[obs_nodes] | (model.pdof[obs_nodes] != obs_nodes)]
    return prob, model, st, obs_pairs, obs_nodes


def objective(res, obs_pairs, obs_nodes):
    return float(np.sum(res.slip[obs_pairs] ** 2) / S0 ** 2 + np.sum(res.p[obs_nodes]) / P0)


def run_last(model, st0, dt, f=None):
    st = copy.deepcopy(st0)
    return solve.implicit_step(model, st, dt, rtol=1e-13, f=f)


@pytest.fixture(scope="module")
def case():
    prob, model, st0, obs_pairs, obs_nodes = setup_case()
    dt = prob.dts[2]
    res = run_last(model, st0, dt)
    assert (res.flags == 2).sum() >= 5
    P = res.slip.shape[0]
    dJ_dslip = np.zeros((P, 2))
    dJ_dslip[obs_pairs] = 2 * res.slip[obs_pairs] / S0 ** 2
    dJ_dp = np.zeros(model.N)
    np.add.at(dJ_dp, obs_nodes, 1.0 / P0)
    g = adjoint.adjoint_of_last_step(model, res.u.reshape(-1), st0_p(model, res.p),
                                     st0.dlie, dt, dJ_dp=dJ_dp, dJ_dslip=dJ_dslip)
    return dict(prob=prob, model=model, st0=st0, dt=dt, res=res, g=g, obs_pairs=obs_pairs,
                obs_nodes=obs_nodes)


def st0_p(model, p_expanded):
    """Master-dof pressure vector (slave entries zero) from an expanded field."""
    p = p_expanded.copy()
    if model.tied:
        p[model.fg["pairs"][:, 1]] = 0.0
    return p


def test_gradient_log_source_scaling(case):
    h = 1e-4
    model, st0, dt = case["model"], case["st0"], case["dt"]
    fp0 = model.fpv.copy()
    J = []
    for sgn in (1, -1):
        model.fpv = fp0 * math.exp(sgn * h)
        r = run_last(model, st0, dt)
        assert np.array_equal(r.flags, case["res"].flags)
        J.append(objective(r, case["obs_pairs"], case["obs_nodes"]))
    model.fpv = fp0
    fd = (J[0] - J[1]) / (2 * h)
    assert case["g"]["g_logQ"] == pytest.approx(fd, rel=1e-5)


def test_gradient_friction(case):
    h = 1e-6
    model, st0, dt = case["model"], case["st0"], case["dt"]
    f0 = case["prob"].fault.f
    J = []
    for sgn in (1, -1):
        r = run_last(model, st0, dt, f=f0 + sgn * h)
        assert np.array_equal(r.flags, case["res"].flags)
        J.append(objective(r, case["obs_pairs"], case["obs_nodes"]))
    fd = (J[0] - J[1]) / (2 * h)
    assert case["g"]["g_f"].sum() == pytest.approx(fd, rel=1e-5)
    assert np.abs(case["g"]["g_f"]).max() > 0


def test_gradient_element_permeability(case):
    h = 1e-4
    prob, st0, dt = case["prob"], case["st0"], case["dt"]
    g = case["g"]["g_logk"]
    # elements around the injection point carry the largest sensitivities
    for e in np.argsort(-np.abs(g))[:3]:
        J = []
        for sgn in (1, -1):
            p2 = copy.deepcopy(prob)
            p2.k = np.array(prob.k, float).copy()
            p2.k[e] *= math.exp(sgn * h)
            m2 = fem.Model(p2)
            r = run_last(m2, st0, dt)
            J.append(objective(r, case["obs_pairs"], case["obs_nodes"]))
        fd = (J[0] - J[1]) / (2 * h)
        assert g[e] == pytest.approx(fd, rel=1e-5, abs=1e-9 * np.abs(g).max())


# ---------------------------------------------------------------------------
# several steps (inelastic slip carried as history), random directions
# ---------------------------------------------------------------------------

def run_traj(prob, steps, k=None, f=None, qscale=1.0):
    p2 = copy.deepcopy(prob)
    if k is not None:
        p2.k = k
    model = fem.Model(p2)
    model.fpv = model.fpv * qscale
    st = solve.initial_state(model)
    traj = []
    for dt in prob.dts[:steps]:
        h_prev = st.dlie.copy()
        r = solve.implicit_step(model, st, dt, rtol=1e-13, f=f)
        pm = st.p.copy()
        traj.append(dict(u=st.u.copy(), p=pm, h_prev=h_prev, res=r))
    return model, traj


def test_multistep_adjoint_directional_derivatives():
    prob = W.fault_small(n=6, Q=5e-5, steps=4)
    K = 4
    model, traj = run_traj(prob, K)
    final = traj[-1]["res"]
    assert (final.flags == 2).sum() >= 5
    rng = np.random.default_rng(9)
    P = final.slip.shape[0]
    obs_pairs = rng.choice(P, 12, replace=False)
    obs_nodes = rng.choice(model.N, 8, replace=False)
    dJ_dslip = np.zeros((P, 2))
    dJ_dslip[obs_pairs] = 2 * final.slip[obs_pairs] / S0 ** 2
    dJ_dp = np.zeros(model.N)
    np.add.at(dJ_dp, obs_nodes, 1.0 / P0)
    g = adjoint.adjoint_multistep(model, traj, prob.dts[:K], dJ_dp=dJ_dp, dJ_dslip=dJ_dslip)
    k0 = np.asarray(prob.k, float)
    f0 = prob.fault.f
    for d in range(2):
        vk = rng.normal(size=k0.size)
        vf = rng.normal()
        vq = rng.normal()
        pred = g["g_logk"] @ vk + g["g_f"].sum() * vf + g["g_logQ"] * vq
        h = 1e-5
        J = []
        for sgn in (1, -1):
            _, tr = run_traj(prob, K, k=k0 * np.exp(sgn * h * vk), f=f0 + sgn * h * vf,
                             qscale=math.exp(sgn * h * vq))
            assert np.array_equal(tr[-1]["res"].flags, final.flags)
            J.append(objective(tr[-1]["res"], obs_pairs, obs_nodes))
        fd = (J[0] - J[1]) / (2 * h)
        assert pred == pytest.approx(fd, rel=1e-5)


def test_multistep_adjoint_aquifer_caprock_pressure():
    """Faulted-aquifer case (20x6x8 cells; layers, per-pair in-situ tractions,
    sheared grid, a slipping pair): the multi-step adjoint gradient of the
    hanging-wall caprock pressure after three steps w.r.t. log Q equals the
    central difference of complete oracle runs."""
    prob = W.faulted_aquifer(nv=20, ny=6, nz=8, steps=3, Q=0.5)
    K = 3
    nb = (prob.nx + 1) * (prob.ny + 1)
    node = np.arange(prob.n_nodes)
    height = (node % (prob.nx + 1)) * prob.h[0]
    cap = np.where((height >= 1000) & (height <= 1200) & (node // nb < prob.kf))[0]

    def run(p):
        m = fem.Model(p)
        st = solve.initial_state(m)
        traj = []
        for dt in p.dts[:K]:
            h_prev = st.dlie.copy()
            res = solve.implicit_step(m, st, dt, rtol=1e-10)
            traj.append(dict(u=st.u.copy(), p=st.p.copy(), h_prev=h_prev))
        return m, st, traj, res

    model, st, traj, res = run(prob)
    assert (res.flags == 2).sum() >= 1
    g_p = np.zeros(model.N)
    g_p[cap] = 1.0 / P0
    g = adjoint.adjoint_multistep(model, traj, prob.dts[:K], dJ_dp=g_p)
    h = 1e-4
    Js = []
    for sgn in (1, -1):
        p2 = copy.deepcopy(prob)
        p2.fp = prob.fp * math.exp(sgn * h)
        _, st2, _, r2 = run(p2)
        assert np.array_equal(r2.flags, res.flags)
        Js.append(float(np.sum(st2.p[cap]) / P0))
    assert g["g_logQ"] == pytest.approx((Js[0] - Js[1]) / (2 * h), rel=1e-5)
