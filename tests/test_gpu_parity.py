"""GPU path vs the CPU oracle, element by element, on seeded inputs.

Sizes span several 15x15 node tiles with ragged edges, plane chunks that start
at either fault lip, the box and both sheared cell classes, tied and double-node
pressures, and a fault-free grid.  FP64 operator applies must agree to 1e-12
(relative L2), solves to their tolerances, implicit steps to 1e-9 with
identical fault states (the 1e-9 bound is the FP64 parity target)."""
import numpy as np
import pytest

import workloads as W
from oracle import fem, solve as osolve

from gpu_common import cuda, need_gpu, rel, solver_for, torch

pytestmark = pytest.mark.gpu

CASES = {
    "box_tied_8": lambda: W.fault_small(),
    "ragged_tied": lambda: W.tiny_faulted(17, 16, 6, seed=5, h=(0.4, 0.3, 0.5)),
    "chunk_at_upper_lip": lambda: W.tiny_faulted(16, 3, 6, seed=6),
    "sheared_x_untied": lambda: W.tiny_faulted(9, 7, 6, shear=(1.7320508075688772, 0.0), k_perp=1e-13, seed=7),
    "sheared_xy_tied": lambda: W.tiny_faulted(6, 5, 4, shear=(0.4, -0.3), seed=8),
    "no_fault": lambda: _nofault(),
}


def _nofault():
    p = W.tiny_faulted(18, 5, 7, seed=9)
    p.kf = None
    p.fault = None
    N = p.n_nodes
    p.fixed = np.zeros((4, N), np.uint8)
    p.fixed[0:3, : (p.nx + 1) * (p.ny + 1)] = 1
    p.fixed[3, -3:] = 1
    p.fu = np.zeros((3, N)); p.fp = np.zeros(N)
    p.fp[N // 2] = 3e-5
    p.fu[2, -1] = -1e5
    p.dts = [1.0, 2.0, 4.0]
    return p


def setup(name, dt=1.7):
    need_gpu()
    prob = CASES[name]()
    model = fem.Model(prob)
    s = solver_for(prob)
    s.timestep(dt)
    return prob, model, s


def lip_state(prob, model, s, seed):
    """Seeded displacement with lip jumps; the fault state is evaluated on both sides."""
    u = W.random_vectors(model.N, seed, scale_u=1e-5)[0]
    if prob.kf is not None:
        u += W.random_displacement_jump(prob, seed + 1, scale=5e-6)
    st = osolve.initial_state(model)
    r, force, Kcoh = osolve.fault_terms(model, u.reshape(-1), st.dlie)
    g = s.fault_update(cuda(u)) if prob.kf is not None else None
    return u, r, Kcoh, g


@pytest.mark.parametrize("name", list(CASES))
def test_return_map(name):
    prob, model, s = setup(name)
    if prob.kf is None:
        pytest.skip("no fault")
    u, r, _, g = lip_state(prob, model, s, 11)
    assert np.array_equal(g["flags"].cpu().numpy().astype(np.int64), r["state"])
    assert len(set(r["state"].tolist())) >= 2          # the seeded jumps exercise several states
    assert rel(g["tn"].cpu().numpy(), r["tn"]) < 1e-13
    assert rel(g["ts"].cpu().numpy().T, r["ts"]) < 1e-13
    assert rel(g["dlie"].cpu().numpy().T, r["dlie"]) < 1e-13
    assert rel(g["T"].cpu().numpy().T, r["T"]) < 1e-12


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("op", ["KB", "KT", "A22", "APU", "AUP", "J"])
def test_apply_fp64(name, op):
    dt = 1.7
    prob, model, s = setup(name, dt)
    u, r, Kcoh, _ = lip_state(prob, model, s, 21)
    x_u, x_p = W.random_vectors(model.N, 22)
    if op == "KT" and prob.kf is None:
        Kcoh = None
        op_o = "Kb"
    else:
        op_o = {"KB": "Kb", "KT": "KT", "A22": "A22", "APU": "Apu", "AUP": "Aup", "J": "J"}[op]
    yu_o, yp_o = osolve.apply(model, op_o, x_u.reshape(-1), x_p, dt=dt, Kcoh=Kcoh)
    if op in ("KB", "KT"):
        y = s.apply(op, cuda(x_u)).cpu().numpy()
        assert rel(y.reshape(-1), yu_o) < 1e-12
    elif op == "A22":
        y = s.apply(op, cuda(x_p)).cpu().numpy()
        assert rel(y, yp_o) < 1e-12
    elif op == "APU":
        y = s.apply(op, cuda(x_p)).cpu().numpy()
        assert rel(y.reshape(-1), yu_o) < 1e-12
    elif op == "AUP":
        y = s.apply(op, cuda(x_u)).cpu().numpy()
        assert rel(y, yp_o) < 1e-12
    else:
        x = np.concatenate([x_u, x_p[None]], axis=0)
        y = s.apply(op, cuda(x)).cpu().numpy()
        assert rel(y[:3].reshape(-1), yu_o) < 1e-12
        assert rel(y[3], yp_o) < 1e-12


@pytest.mark.parametrize("name", ["box_tied_8", "ragged_tied", "sheared_x_untied"])
@pytest.mark.parametrize("op", ["KT", "A22", "J"])
def test_apply_fp32(name, op):
    dt = 1.7
    prob, model, s = setup(name, dt)
    u, r, Kcoh, _ = lip_state(prob, model, s, 31)
    x_u, x_p = W.random_vectors(model.N, 32)
    op_o = {"KT": "KT", "A22": "A22", "J": "J"}[op]
    yu_o, yp_o = osolve.apply(model, op_o, x_u.reshape(-1), x_p, dt=dt, Kcoh=Kcoh)
    if op == "KT":
        y = s.apply(op, cuda(x_u, torch.float32)).cpu().numpy()
        assert rel(y.reshape(-1), yu_o) < 2e-5
    elif op == "A22":
        y = s.apply(op, cuda(x_p, torch.float32)).cpu().numpy()
        assert rel(y, yp_o) < 2e-5
    else:
        x = np.concatenate([x_u, x_p[None]], axis=0)
        y = s.apply(op, cuda(x, torch.float32)).cpu().numpy()
        assert rel(y[:3].reshape(-1), yu_o) < 2e-5


@pytest.mark.parametrize("zchunk", [0, 2, 3, 5])
@pytest.mark.parametrize("name", list(CASES))
def test_apply_fp32_kernel_all_cells_and_chunks(name, zchunk, monkeypatch):
    """The FP32 bulk kernel (K_b, K_T and S + dt C applies) on every cell class,
    tied and double-node lips and the fault-free grid, with the plane-chunk
    length forced (GM_BULK_ZCHUNK) so that chunks start at, below and above
    either lip: against the oracle evaluated on the same FP32 inputs, within
    FP32 rounding (5e-6 relative L2)."""
    dt = 1.7
    if zchunk:
        monkeypatch.setenv("GM_BULK_ZCHUNK", str(zchunk))
    else:
        monkeypatch.delenv("GM_BULK_ZCHUNK", raising=False)
    prob, model, s = setup(name, dt)
    u, r, Kcoh, _ = lip_state(prob, model, s, 51)
    x_u, x_p = W.random_vectors(model.N, 52)
    x_u = x_u.astype(np.float32).astype(np.float64)
    x_p = x_p.astype(np.float32).astype(np.float64)
    for op in ("KB", "KT", "A22"):
        if op == "KT" and prob.kf is None:
            continue
        op_o = {"KB": "Kb", "KT": "KT", "A22": "A22"}[op]
        yu_o, yp_o = osolve.apply(model, op_o, x_u.reshape(-1), x_p, dt=dt, Kcoh=Kcoh)
        if op == "A22":
            y = s.apply(op, cuda(x_p, torch.float32)).cpu().numpy()
            assert rel(y, yp_o) < 5e-6, (op, rel(y, yp_o))
        else:
            y = s.apply(op, cuda(x_u, torch.float32)).cpu().numpy()
            assert rel(y.reshape(-1), yu_o) < 5e-6, (op, rel(y.reshape(-1), yu_o))


@pytest.mark.parametrize("name", ["box_tied_8", "ragged_tied", "sheared_x_untied", "no_fault"])
def test_residual(name):
    dt = 1.3
    prob, model, s = setup(name, dt)
    du, dp = W.random_vectors(model.N, 41, scale_u=1e-6, scale_p=1e5)
    # a state satisfies the homogeneous constraints: zero at constrained dofs
    du = np.where(model.free_u.reshape(3, -1), du, 0.0)
    dp = np.where(model.free_p, dp, 0.0)
    st = osolve.initial_state(model)
    _, force, _ = osolve.fault_terms(model, du.reshape(-1), st.dlie)
    b1, b2 = osolve.residuals(model, st, du.reshape(-1), dp, dt, force)
    rh = osolve.scaled_norm(model, b1, b2, model.A22(dt).diagonal())
    b, rhat = s.residual(cuda(du), cuda(dp))
    b = b.cpu().numpy()
    assert rel(b[:3].reshape(-1), b1) < 1e-12
    assert rel(b[3], b2) < 1e-12
    assert abs(rhat - rh) <= 1e-12 * rh


@pytest.mark.parametrize("name", ["box_tied_8", "sheared_x_untied", "no_fault"])
@pytest.mark.parametrize("op", ["KT", "A22"])
def test_pcg(name, op):
    dt = 0.9
    prob, model, s = setup(name, dt)
    u, r, Kcoh, _ = lip_state(prob, model, s, 51)
    if Kcoh is None or prob.kf is None:
        Kcoh = model.Kb * 0
    KT, Apu, A22 = osolve.jacobian_blocks(model, Kcoh, dt)
    bu, bp = W.random_vectors(model.N, 52, scale_u=1e3, scale_p=1e-9)
    from scipy.sparse.linalg import spsolve
    if op == "KT":
        b = np.where(model.free_u, bu.reshape(-1), 0.0)
        x_o = np.zeros(3 * model.N)
        x_o[model.free_u] = spsolve(KT.tocsc(), b[model.free_u])
        x, rep = s.pcg("KT", cuda(b.reshape(3, -1)), rtol=1e-13, maxit=20000)
        assert rel(x.cpu().numpy().reshape(-1), x_o) < 1e-9
    else:
        b = np.where(model.free_p, bp, 0.0)
        x_o = np.zeros(model.N)
        x_o[model.free_p] = spsolve(A22.tocsc(), b[model.free_p])
        x, rep = s.pcg("A22", cuda(b), rtol=1e-13, maxit=20000)
        assert rel(x.cpu().numpy(), x_o) < 1e-9
    assert rep["iterations"] > 0 and rep["rel_residual"] <= 1e-13


@pytest.mark.parametrize("name", ["box_tied_8", "sheared_x_untied", "chunk_at_upper_lip"])
def test_prevost_vs_direct(name):
    dt = 2.0
    prob, model, s = setup(name, dt)
    u, r, Kcoh, _ = lip_state(prob, model, s, 61)
    KT, Apu, A22 = osolve.jacobian_blocks(model, Kcoh, dt)
    bu, bp = W.random_vectors(model.N, 62, scale_u=1e3, scale_p=1e-9)
    b1 = np.where(model.free_u, bu.reshape(-1), 0.0)
    b2 = np.where(model.free_p, bp, 0.0)
    x1, x2 = osolve.solve_monolithic(KT, Apu, A22, b1[model.free_u], b2[model.free_p], dense=False)
    b = np.concatenate([b1.reshape(3, -1), b2[None]], axis=0)
    x, rep = s.prevost(cuda(b), outer_rtol=1e-12, inner_rtol=1e-14)
    x = x.cpu().numpy()
    assert rel(x[:3].reshape(-1)[model.free_u], x1) < 1e-8
    assert rel(x[3][model.free_p], x2) < 1e-8
    assert rep["iterations"] >= 1


@pytest.mark.parametrize("name,steps,sp", [("box_tied_8", 5, 0), ("sheared_x_untied", 2, 0),
                                           ("ragged_tied", 2, 0), ("no_fault", 3, 0),
                                           ("box_tied_8", 5, 1), ("sheared_x_untied", 2, 1)])
def test_implicit_steps(name, steps, sp):
    """sp = 1 uses the fixed-stress Schur preconditioner: same converged result."""
    prob = CASES[name]()
    if name == "ragged_tied":
        prob.fp = prob.fp * 20
    need_gpu()
    s = solver_for(prob)
    model, ref = osolve.run(prob, nsteps=steps, rtol=1e-12)
    for k in range(steps):
        rep = s.step(prob.dts[k], newton_rtol=1e-12, schur_precond=sp)
        st = s.get_state()
        r = ref[k]
        assert rel(st["u"], r.u) < 1e-9, (k, rel(st["u"], r.u))
        assert rel(st["p"], r.p) < 1e-9, (k, rel(st["p"], r.p))
        if prob.kf is not None:
            assert np.array_equal(st["flags"].astype(np.int64), r.flags), k
            assert rel(st["slip"].T, r.slip) < 1e-9
            assert rel(st["dlie"].T, r.dlie) < 1e-9 or np.abs(r.dlie).max() == 0
    if name == "box_tied_8":
        fl = st["flags"]
        assert (fl == 0).sum() >= 1 and (fl == 2).sum() >= 4 and (fl == 1).sum() >= 4


def test_state_roundtrip():
    need_gpu()
    prob = W.fault_small(steps=1)
    s = solver_for(prob)
    s.step(prob.dts[0])
    a = s.get_state()
    s2 = solver_for(prob)
    s2.set_state(u=a["u"], p=a["p"], dlie=a["dlie"], flags=a["flags"])
    b = s2.get_state()
    for k in ("u", "p", "dlie", "flags", "slip"):
        assert np.array_equal(a[k], b[k]), k


@pytest.mark.parametrize("name,steps,kind", [("box_tied_8", 5, 1), ("sheared_x_untied", 2, 1),
                                             ("box_tied_8", 5, 0)])
def test_implicit_steps_fp32_refined(name, steps, kind):
    """FP32 operators and preconditioners inside the FP64 Newton / refinement loop:
    fields within 1e-8 of the FP64 oracle and identical fault states, with the
    block-Jacobi (kind 0) and the default multigrid (kind 1) K_T preconditioner."""
    prob = CASES[name]()
    need_gpu()
    s = solver_for(prob)
    s.set_preconditioner(kind)
    model, ref = osolve.run(prob, nsteps=steps, rtol=1e-12)
    for k in range(steps):
        s.step(prob.dts[k], newton_rtol=1e-12, precision=1)
        st = s.get_state()
        r = ref[k]
        assert rel(st["u"], r.u) < 1e-8, (k, rel(st["u"], r.u))
        assert rel(st["p"], r.p) < 1e-8, (k, rel(st["p"], r.p))
        assert np.array_equal(st["flags"].astype(np.int64), r.flags), k


def insitu_varying_case():
    """fault_small on 6^3 with in-situ tractions that vary over the fault, as
    depth-dependent stress makes them: t'_n0 from 8 to 12 MPa along x, tau0_1
    from 4.9 to 5.9 MPa along y, a small tau0_2 that changes sign."""
    import dataclasses
    prob = W.fault_small(n=6, Q=5e-5, steps=3)
    n = prob.nx
    i = np.arange(prob.n_pairs) % (n + 1) / n
    j = np.arange(prob.n_pairs) // (n + 1) / n
    tn0 = 10e6 * (0.8 + 0.4 * i)
    tau0 = np.stack([5.4e6 * (0.9 + 0.2 * j), 0.3e6 * (i - 0.5)], 1)
    prob.fault = dataclasses.replace(prob.fault, tn0=tn0, tau0=tau0)
    return prob


@pytest.mark.parametrize("precision", [0, 1])
def test_implicit_steps_per_pair_insitu(precision):
    """gm_set_insitu: per-pair in-situ tractions give the oracle's steps (FP64
    1e-9, FP32-refined 1e-8) with identical fault states; clearing them
    restores the uniform-traction solver."""
    need_gpu()
    prob = insitu_varying_case()
    s = solver_for(prob)
    model, ref = osolve.run(prob, nsteps=3, rtol=1e-12)
    tol = 1e-9 if precision == 0 else 1e-8
    for k in range(3):
        s.step(prob.dts[k], newton_rtol=1e-12, precision=precision)
        st = s.get_state()
        r = ref[k]
        assert np.array_equal(st["flags"].astype(np.int64), r.flags), k
        assert rel(st["u"], r.u) < tol, (k, rel(st["u"], r.u))
        assert rel(st["p"], r.p) < tol
        assert rel(st["slip"].T, r.slip) < tol
    assert (r.flags == 2).sum() >= 10 and (r.flags == 1).sum() >= 10
    # back to the uniform values of the fault parameters
    s.set_insitu(None, None)
    uni = W.fault_small(n=6, Q=5e-5, steps=3)
    s2 = solver_for(uni)
    s.set_state(u=np.zeros((3, s.N)), p=np.zeros(s.N), dlie=np.zeros((2, s.P)),
                flags=np.ones(s.P, np.int8))
    for k in range(2):
        s.step(uni.dts[k], newton_rtol=1e-12, precision=precision)
        s2.step(uni.dts[k], newton_rtol=1e-12, precision=precision)
    a, b = s.get_state(), s2.get_state()
    assert rel(a["u"], b["u"]) < 1e-12 and np.array_equal(a["flags"], b["flags"])


@pytest.mark.parametrize("precision", [0, 1])
def test_faulted_aquifer_small_steps(precision):
    """The faulted-aquifer workload (layers, log-normal aquifer, sheared grid,
    depth-dependent in-situ tractions per pair, line source) on 20x6x8 cells
    with Q raised to 0.5 m^3/s so pairs slip: three implicit steps equal the
    oracle's.  Newton stops at 1e-10: with permeabilities over six decades the
    FP64 residual evaluation floors near 1e-12 of the initial residual."""
    need_gpu()
    prob = W.faulted_aquifer(nv=20, ny=6, nz=8, steps=3, Q=0.5)
    s = solver_for(prob)
    model, ref = osolve.run(prob, nsteps=3, rtol=1e-10)
    for k in range(3):
        s.step(prob.dts[k], newton_rtol=1e-10, precision=precision)
        st = s.get_state()
        r = ref[k]
        assert np.array_equal(st["flags"].astype(np.int64), r.flags), k
        assert rel(st["u"], r.u) < 1e-8, (k, rel(st["u"], r.u))
        assert rel(st["p"], r.p) < 1e-8, (k, rel(st["p"], r.p))
        assert rel(st["slip"].T, r.slip) < 1e-8, (k, rel(st["slip"].T, r.slip))
    assert (r.flags == 2).sum() >= 2


MG_CASES = {
    "box_tied_8": (lambda: W.fault_small(), 5, 1e-12),
    "sheared_8_untied": (lambda: W.tiny_faulted(8, 8, 8, shear=(1.7320508075688772, 0.0), k_perp=1e-13, seed=7),
                         2, 1e-12),
    "aquifer_small": (lambda: W.faulted_aquifer(nv=20, ny=6, nz=8, steps=3, Q=0.5), 3, 1e-10),
    "odd_cells_fallback": (lambda: W.tiny_faulted(9, 7, 6, shear=(1.7320508075688772, 0.0), k_perp=1e-13, seed=7),
                           2, 1e-12),
}


@pytest.mark.parametrize("name", list(MG_CASES))
def test_implicit_steps_fp32_multigrid(name):
    """gm_set_preconditioner(1): the FP32 K_T solves preconditioned by the
    multigrid V-cycle give the oracle's steps within 1e-8 and its fault
    states (grids with odd cell counts fall back to block Jacobi)."""
    need_gpu()
    make, steps, rtol = MG_CASES[name]
    prob = make()
    s = solver_for(prob)
    s.set_preconditioner(1)
    model, ref = osolve.run(prob, nsteps=steps, rtol=rtol)
    for k in range(steps):
        s.step(prob.dts[k], newton_rtol=rtol, precision=1)
        st = s.get_state()
        r = ref[k]
        assert np.array_equal(st["flags"].astype(np.int64), r.flags), k
        assert rel(st["u"], r.u) < 1e-8, (k, rel(st["u"], r.u))
        assert rel(st["p"], r.p) < 1e-8, (k, rel(st["p"], r.p))


def test_multigrid_cuts_inner_iterations():
    """On the 32^3 slip-front grid the V-cycle preconditioner reaches the same
    converged steps as block Jacobi with at most a third of the K_T iterations."""
    need_gpu()
    prob = W.slip_front(n=32)
    out = {}
    for kind in (0, 1):
        s = solver_for(prob)
        s.set_preconditioner(kind)
        its = 0
        for k in range(3):
            its += s.step(prob.dts[k], newton_rtol=1e-10, precision=1)["inner_k"]
        out[kind] = (its, s.get_state())
    (i0, a), (i1, b) = out[0], out[1]
    assert rel(b["u"], a["u"]) < 1e-7 and rel(b["p"], a["p"]) < 1e-7
    assert np.array_equal(a["flags"], b["flags"])
    assert i1 * 3 <= i0, (i0, i1)
