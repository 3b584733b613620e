"""GPU parity of the fault on P1 tetrahedra (interface elements on the fault
triangles, Sec. 3.1.1-3.1.2; Newton and Prevost's partitioned CG, Sec.
3.3.1-3.3.2) with the oracle's TetFaultModel: the fault-aware operators
within 1e-12 of the assembled matrices, tied and untied lip pressures; and
implicit steps with contact and Coulomb slip: u, p, slip and inelastic slip
within 1e-9 of the oracle's, fault states equal."""
import numpy as np
import pytest

import workloads as W
from oracle import solve, tetfault as TF

from gpu_common import cuda, need_gpu, torch

pytestmark = pytest.mark.gpu

K_PERP = {"tied": 0.0, "untied": 1e-18}


def rel(a, b):
    return float(np.abs(np.asarray(a) - np.asarray(b)).max() / max(np.abs(b).max(), 1e-300))


@pytest.mark.parametrize("case", sorted(K_PERP))
def test_fault_operators_match_assembled(case):
    need_gpu()
    import paper_2410_17133_gb300 as gm
    prob = W.tetrahedralize(W.tiny_faulted(3, 2, 2, shear=(0.3, 0.1), k_perp=K_PERP[case], Q=2e-4))
    m = TF.TetFaultModel(prob)
    s = gm.TetFaultSolver.from_problem(prob)
    rng = np.random.default_rng(3)
    u = rng.normal(size=3 * m.N)
    p = rng.normal(size=m.N)
    for gw, ow, xu, xp, dt in (("KT", "Kb", u, None, 0.0), ("APU", "Apu", None, p, 0.0),
                               ("AUP", "Aup", u, None, 0.0), ("A22", "A22", None, p, 0.7)):
        yu, yp = solve.apply(m, ow, u=xu, p=xp, dt=dt)
        x = cuda(xu.reshape(3, -1)) if xu is not None else cuda(xp)
        y = s.fault_apply(gw, x, dt=dt).cpu().numpy().reshape(-1)
        ref = yu if gw in ("KT", "APU") else yp
        assert rel(y, ref) <= 1e-12, gw


STEP_CASES = {
    "tiny-tied": (lambda: W.tetrahedralize(W.tiny_faulted(3, 3, 2, Q=2e-4, steps=3)), 3),
    "tiny-untied": (lambda: W.tetrahedralize(W.tiny_faulted(3, 3, 2, k_perp=1e-18, Q=2e-4, steps=3)), 3),
    "fault8": (lambda: W.tetrahedralize(W.fault_small(8)), 2),
}


@pytest.mark.parametrize("precision", [0, 1], ids=["fp64", "fp32_refined"])
@pytest.mark.parametrize("case", sorted(STEP_CASES))
def test_fault_steps_match_oracle(case, precision):
    """FP64, and FP32-refined (FP32 inner K_T solves inside the FP64 Newton
    loop, which refines them to the same Newton tolerance): the oracle's
    steps within 1e-9 and its fault states."""
    need_gpu()
    import paper_2410_17133_gb300 as gm
    make, nsteps = STEP_CASES[case]
    prob = make()
    _, res = TF.run(prob, nsteps=nsteps, solver="lu")
    s = gm.TetFaultSolver.from_problem(prob)
    u = torch.zeros((3, s.N), dtype=torch.float64, device="cuda")
    p = torch.zeros(s.N, dtype=torch.float64, device="cuda")
    for k, dt in enumerate(prob.dts[:nsteps]):
        rep = s.fault_step(dt, u, p, precision=precision)
        print(case, precision, k, rep["newton"], rep["outer"], rep["inner_k"])
        st = s.fault_state()
        o = res[k]
        assert np.array_equal(st["flags"], o.flags), f"step {k}"
        assert rel(u.cpu().numpy(), o.u) < 1e-9, f"step {k}"
        assert rel(p.cpu().numpy(), o.p) < 1e-9, f"step {k}"
        assert rel(st["slip"], o.slip) < 1e-9, f"step {k}"
        if np.abs(o.dlie).max() > 0:
            assert rel(st["dlie"], o.dlie) < 1e-9, f"step {k}"
        assert rep["n_slip"] == int((o.flags == 2).sum())
    assert (res[nsteps - 1].flags == 2).sum() >= 1


def test_fault_input_errors_are_reported():
    """Invalid fault descriptions and out-of-order calls return status codes
    (GM_EINVAL = -1, GM_ESTATE = -7) through the binding as GMError, before any
    device work: a node in two pairs, a triangle naming a pair out of range,
    t1_ref normal to the fault, a step before the fault is set, dt = 0, and
    fault descriptions whose triangle order or lip order would flip the pair
    normal: one triangle reversed (an edge then runs the same way in two
    triangles), every triangle reversed (normal from plus to minus), and the
    lips of every pair swapped."""
    need_gpu()
    import paper_2410_17133_gb300 as gm
    prob = W.tetrahedralize(W.tiny_faulted(2, 2, 2))
    s = gm.TetFaultSolver()
    s.mesh(prob.nodes, prob.tets)
    s.materials(prob.E[0], prob.nu, prob.alpha, prob.M, prob.k[0], prob.mu_f)
    u = torch.zeros((3, s.N), dtype=torch.float64, device="cuda")
    p = torch.zeros(s.N, dtype=torch.float64, device="cuda")
    with pytest.raises(gm.GMError) as e:
        s.fault_step(1.0, u, p)
    assert e.value.code == -7
    bad = prob.pairs.copy()
    bad[1] = bad[0]
    with pytest.raises(gm.GMError) as e:
        s.fault(bad, prob.fault_tris, prob.t1_ref, prob.fault)
    assert e.value.code == -1
    tris = prob.fault_tris.copy()
    tris[0, 0] = prob.pairs.shape[0]
    with pytest.raises(gm.GMError) as e:
        s.fault(prob.pairs, tris, prob.t1_ref, prob.fault)
    assert e.value.code == -1
    with pytest.raises(gm.GMError) as e:
        s.fault(prob.pairs, prob.fault_tris, (0.0, 0.0, 1.0), prob.fault)
    assert e.value.code == -1
    one = prob.fault_tris.copy()
    one[0] = one[0, ::-1]
    with pytest.raises(gm.GMError) as e:
        s.fault(prob.pairs, one, prob.t1_ref, prob.fault)
    assert e.value.code == -1 and "ordered inconsistently" in str(e.value)
    with pytest.raises(gm.GMError) as e:
        s.fault(prob.pairs, prob.fault_tris[:, ::-1].copy(), prob.t1_ref, prob.fault)
    assert e.value.code == -1 and "side" in str(e.value)
    with pytest.raises(gm.GMError) as e:
        s.fault(prob.pairs[:, ::-1].copy(), prob.fault_tris, prob.t1_ref, prob.fault)
    assert e.value.code == -1 and "side" in str(e.value)
    s.fault(prob.pairs, prob.fault_tris, prob.t1_ref, prob.fault)
    with pytest.raises(gm.GMError) as e:
        s.fault_step(0.0, u, p)
    assert e.value.code == -1
