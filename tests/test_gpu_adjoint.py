"""Adjoint of the converged implicit step on the GPU: gradients w.r.t. element
log-permeability, friction (per pair) and log source scaling match the oracle's
assembled adjoint (consistent tangent, frozen fault states), central finite
differences of GPU steps, and the torch.autograd wrapper."""
import copy
import math

import numpy as np
import pytest

import workloads as W
from oracle import adjoint as oadj, fem, solve as osolve

from gpu_common import cuda, need_gpu, rel, solver_for, torch

pytestmark = pytest.mark.gpu
S0, P0 = 1e-6, 1e6


def scenario():
    prob = W.fault_small(n=6, Q=5e-5, steps=3)
    rng = np.random.default_rng(5)
    P = prob.n_pairs
    obs_pairs = rng.choice(P, 12, replace=False)
    obs_nodes = rng.choice(prob.n_nodes, 8, replace=False)
    return prob, obs_pairs, obs_nodes


def J_of(slip, p, obs_pairs, obs_nodes):
    """slip (P, 2), p (N,)"""
    return float(np.sum(slip[obs_pairs] ** 2) / S0 ** 2 + np.sum(p[obs_nodes]) / P0)


def dJ(slip, obs_pairs, obs_nodes, N):
    g_s = np.zeros_like(slip)
    g_s[obs_pairs] = 2 * slip[obs_pairs] / S0 ** 2
    g_p = np.zeros(N)
    np.add.at(g_p, obs_nodes, 1.0 / P0)
    return g_s, g_p


@pytest.fixture(scope="module")
def gpu_case():
    need_gpu()
    prob, obs_pairs, obs_nodes = scenario()
    s = solver_for(prob)
    for dt in prob.dts[:2]:
        s.step(dt, newton_rtol=1e-12)
    st2 = s.get_state()
    s.step(prob.dts[2], newton_rtol=1e-12)
    st3 = s.get_state()
    g_s, g_p = dJ(st3["slip"].T, obs_pairs, obs_nodes, s.N)
    gk, gf, gq, rep = s.adjoint(dJ_dp=cuda(g_p), dJ_dslip=cuda(g_s.T), rtol=1e-11)
    return dict(prob=prob, s=s, st2=st2, st3=st3, gk=gk.cpu().numpy(), gf=gf.cpu().numpy(), gq=gq,
                rep=rep, obs_pairs=obs_pairs, obs_nodes=obs_nodes, g_s=g_s, g_p=g_p)


def test_adjoint_matches_oracle(gpu_case):
    c = gpu_case
    prob = c["prob"]
    model = fem.Model(prob)
    st = osolve.initial_state(model)
    for dt in prob.dts[:2]:
        osolve.implicit_step(model, st, dt, rtol=1e-13)
    dlie_prev = st.dlie.copy()
    res = osolve.implicit_step(model, st, prob.dts[2], rtol=1e-13)
    assert np.array_equal(res.flags, c["st3"]["flags"].astype(np.int64))
    assert (res.flags == 2).sum() >= 5
    g_s, g_p = dJ(res.slip, c["obs_pairs"], c["obs_nodes"], model.N)
    p_master = res.p.copy()
    p_master[model.fg["pairs"][:, 1]] = 0.0
    g = oadj.adjoint_of_last_step(model, res.u.reshape(-1), p_master, dlie_prev, prob.dts[2],
                                  dJ_dp=g_p, dJ_dslip=g_s)
    assert c["rep"]["rel_residual"] < 1e-9
    assert rel(c["gk"], g["g_logk"]) < 1e-6
    assert rel(c["gf"], g["g_f"]) < 1e-6
    assert c["gq"] == pytest.approx(g["g_logQ"], rel=1e-6)


def test_adjoint_log_source_scaling_vs_finite_differences(gpu_case):
    c = gpu_case
    prob, s = c["prob"], c["s"]
    h = 1e-4
    Js = []
    for sgn in (1, -1):
        s.set_state(u=c["st2"]["u"], p=c["st2"]["p"], dlie=c["st2"]["dlie"], flags=c["st2"]["flags"])
        s.loads(prob.fu, prob.fp * math.exp(sgn * h))
        s.step(prob.dts[2], newton_rtol=1e-12)
        st = s.get_state()
        Js.append(J_of(st["slip"].T, st["p"], c["obs_pairs"], c["obs_nodes"]))
    s.loads(prob.fu, prob.fp)
    fd = (Js[0] - Js[1]) / (2 * h)
    assert c["gq"] == pytest.approx(fd, rel=1e-5)


def test_adjoint_friction_vs_finite_differences(gpu_case):
    c = gpu_case
    prob, s = c["prob"], c["s"]
    h = 1e-6
    Js = []
    for sgn in (1, -1):
        s.set_state(u=c["st2"]["u"], p=c["st2"]["p"], dlie=c["st2"]["dlie"], flags=c["st2"]["flags"])
        s.set_friction(np.array([prob.fault.f + sgn * h]))
        s.step(prob.dts[2], newton_rtol=1e-12)
        st = s.get_state()
        Js.append(J_of(st["slip"].T, st["p"], c["obs_pairs"], c["obs_nodes"]))
    s.set_friction(np.array([prob.fault.f]))
    fd = (Js[0] - Js[1]) / (2 * h)
    assert c["gf"].sum() == pytest.approx(fd, rel=1e-5)


def test_autograd_function_gradients():
    need_gpu()
    import paper_2410_17133_gb300 as gm
    prob, obs_pairs, obs_nodes = scenario()
    s = solver_for(prob)
    for dt in prob.dts[:2]:
        s.step(dt, newton_rtol=1e-12)
    Fn = gm.implicit_step_fn()
    logk = torch.tensor(np.log(np.asarray(prob.k, float)), device="cuda", requires_grad=True)
    f = torch.tensor(prob.fault.f, dtype=torch.float64, device="cuda", requires_grad=True)
    logQ = torch.tensor(0.0, dtype=torch.float64, device="cuda", requires_grad=True)
    slip, p = Fn.apply(logk, f, logQ, s, prob.dts[2], (prob.fu, prob.fp), {"newton_rtol": 1e-12})
    op = torch.as_tensor(obs_pairs, device="cuda")
    on = torch.as_tensor(obs_nodes, device="cuda")
    J = (slip[:, op] ** 2).sum() / S0 ** 2 + p[on].sum() / P0
    J.backward()
    st3 = s.get_state()
    g_s, g_p = dJ(st3["slip"].T, obs_pairs, obs_nodes, s.N)
    gk, gf, gq, _ = s.adjoint(dJ_dp=cuda(g_p), dJ_dslip=cuda(g_s.T), rtol=1e-11)
    assert rel(logk.grad.cpu().numpy(), gk.cpu().numpy()) < 1e-8
    assert f.grad.item() == pytest.approx(gf.sum().item(), rel=1e-8)
    assert logQ.grad.item() == pytest.approx(gq, rel=1e-8)


def test_multistep_adjoint_matches_oracle_and_fd():
    """Four steps with slipping pairs, checkpoints every 2 steps: gradients of an
    objective of the final state equal the oracle's multi-step adjoint, and a
    random-direction derivative equals central finite differences of GPU runs."""
    need_gpu()
    import paper_2410_17133_gb300 as gm
    from oracle import adjoint as oadj
    prob = W.fault_small(n=6, Q=5e-5, steps=4)
    K = 4
    rng = np.random.default_rng(9)
    obs_pairs = rng.choice(prob.n_pairs, 12, replace=False)
    obs_nodes = rng.choice(prob.n_nodes, 8, replace=False)
    kw = {"newton_rtol": 1e-12}

    def objective_grad(st):
        g_s, g_p = dJ(st["slip"].T, obs_pairs, obs_nodes, prob.n_nodes)
        return None, cuda(g_p), cuda(g_s.T)

    s = solver_for(prob)
    final, gk, gf, gq = gm.run_with_adjoint(s, prob.dts[:K], objective_grad, checkpoint_every=2,
                                            step_kw=kw, rtol=1e-11)
    assert (final["flags"] == 2).sum() >= 5
    # oracle
    model = fem.Model(prob)
    st = osolve.initial_state(model)
    traj = []
    for dt in prob.dts[:K]:
        h_prev = st.dlie.copy()
        osolve.implicit_step(model, st, dt, rtol=1e-13)
        traj.append(dict(u=st.u.copy(), p=st.p.copy(), h_prev=h_prev))
    res_slip = model.jump(st.u)
    g_s_o = np.zeros((prob.n_pairs, 2))
    gsl = np.stack([np.sum(model.fg["t1"] * res_slip, 1), np.sum(model.fg["t2"] * res_slip, 1)], 1)
    g_s_o[obs_pairs] = 2 * gsl[obs_pairs] / S0 ** 2
    g_p_o = np.zeros(model.N)
    np.add.at(g_p_o, obs_nodes, 1.0 / P0)
    go = oadj.adjoint_multistep(model, traj, prob.dts[:K], dJ_dp=g_p_o, dJ_dslip=g_s_o)
    assert rel(gk.cpu().numpy(), go["g_logk"]) < 1e-6
    assert rel(gf.cpu().numpy(), go["g_f"]) < 1e-6
    assert gq == pytest.approx(go["g_logQ"], rel=1e-6)
    # finite differences on the GPU along one random direction
    k0 = np.asarray(prob.k, float)
    vk, vf, vq = rng.normal(size=k0.size), rng.normal(), rng.normal()
    pred = gk.cpu().numpy() @ vk + gf.sum().item() * vf + gq * vq
    h = 1e-5
    Js = []
    for sgn in (1, -1):
        s2 = solver_for(prob)
        s2.set_permeability(k0 * np.exp(sgn * h * vk))
        s2.set_friction(np.array([prob.fault.f + sgn * h * vf]))
        s2.loads(prob.fu, prob.fp * math.exp(sgn * h * vq))
        for dt in prob.dts[:K]:
            s2.step(dt, newton_rtol=1e-12)
        stt = s2.get_state()
        Js.append(J_of(stt["slip"].T, stt["p"], obs_pairs, obs_nodes))
    fd = (Js[0] - Js[1]) / (2 * h)
    assert pred == pytest.approx(fd, rel=1e-5)



def test_aquifer_caprock_pressure_gradient():
    """Gradient of the caprock pressure (hanging-wall nodes 1000-1200 m high)
    after three steps of the small faulted-aquifer case (layers over six
    decades of permeability, per-pair in-situ tractions, sheared grid, a
    slipping pair), checkpoints every 2 steps: equal to the oracle's
    multi-step adjoint, and to central differences of GPU runs along log Q and
    a random log-permeability direction (1e-5).  The friction derivative is
    much smaller than the source derivative here, so its difference quotient
    carries the noise of the Newton tolerance (1e-10, the FP64 floor of this
    case): checked to 1e-4."""
    need_gpu()
    import paper_2410_17133_gb300 as gm
    from oracle import adjoint as oadj
    prob = W.faulted_aquifer(nv=20, ny=6, nz=8, steps=3, Q=0.5)
    K = 3
    nb = (prob.nx + 1) * (prob.ny + 1)
    node = np.arange(prob.n_nodes)
    height = (node % (prob.nx + 1)) * prob.h[0]
    cap = np.where((height >= 1000) & (height <= 1200) & (node // nb < prob.kf))[0]
    kw = {"newton_rtol": 1e-10}
    g_p = np.zeros(prob.n_nodes)
    g_p[cap] = 1.0 / P0

    def objective_grad(st):
        return None, cuda(g_p), None

    s = solver_for(prob)
    final, gk, gf, gq = gm.run_with_adjoint(s, prob.dts[:K], objective_grad, checkpoint_every=2,
                                            step_kw=kw, rtol=1e-11)
    assert (final["flags"] == 2).sum() >= 1
    model = fem.Model(prob)
    st = osolve.initial_state(model)
    traj = []
    for dt in prob.dts[:K]:
        h_prev = st.dlie.copy()
        osolve.implicit_step(model, st, dt, rtol=1e-10)
        traj.append(dict(u=st.u.copy(), p=st.p.copy(), h_prev=h_prev))
    go = oadj.adjoint_multistep(model, traj, prob.dts[:K], dJ_dp=g_p)
    assert rel(gk.cpu().numpy(), go["g_logk"]) < 1e-6
    assert rel(gf.cpu().numpy(), go["g_f"]) < 1e-6
    assert gq == pytest.approx(go["g_logQ"], rel=1e-6)

    k0 = np.asarray(prob.k, float)
    vk = np.random.default_rng(12).normal(size=k0.size)

    def J(k=None, f=None, qs=1.0):
        s2 = solver_for(prob)
        if k is not None:
            s2.set_permeability(k)
        if f is not None:
            s2.set_friction(np.array([f]))
        if qs != 1.0:
            s2.loads(prob.fu, prob.fp * qs)
        for dt in prob.dts[:K]:
            s2.step(dt, **kw)
        stt = s2.get_state()
        assert np.array_equal(stt["flags"], final["flags"])
        return float(np.sum(stt["p"][cap]) / P0)

    h = 1e-4
    fd_q = (J(qs=math.exp(h)) - J(qs=math.exp(-h))) / (2 * h)
    assert gq == pytest.approx(fd_q, rel=1e-5)
    h = 1e-3
    fd_k = (J(k=k0 * np.exp(h * vk)) - J(k=k0 * np.exp(-h * vk))) / (2 * h)
    assert float(gk.cpu().numpy() @ vk) == pytest.approx(fd_k, rel=1e-5)
    fd_f = (J(f=prob.fault.f + h) - J(f=prob.fault.f - h)) / (2 * h)
    assert float(gf.sum().item()) == pytest.approx(fd_f, rel=1e-4)
