"""Operators of P1 tetrahedra on an unstructured mesh (include/gm_tet.h)
against the oracle's assembled matrices (oracle/tet.py) on the Cryer octant
mesh: K, A_pu, A_up, S + dt C and the coupled Jacobian, FP64 to 1e-12 and
FP32 to 2e-5, and bitwise repeatable."""
import numpy as np
import pytest

import workloads as W
from oracle import tet

from gpu_common import cuda, need_gpu, rel, torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def case():
    need_gpu()
    import paper_2410_17133_gb300 as gm
    prob = W.cryer_octant(n=8, steps=2)
    model = tet.TetModel(prob)
    s = gm.TetSolver.from_problem(prob)
    rng = np.random.default_rng(21)
    xu = rng.normal(size=(3, model.N)) * 1e-4
    xp = rng.normal(size=model.N) * 1e6
    return prob, model, s, xu, xp


@pytest.mark.parametrize("dtype,tol", [(torch.float64, 1e-12), (torch.float32, 2e-5)])
def test_tet_operators_match_oracle(case, dtype, tol):
    prob, m, s, xu, xp = case
    dt = 0.3 * prob.dts[1]
    ref = {
        "KB": (xu, (m.Kb @ xu.reshape(-1)).reshape(3, -1)),
        "APU": (xp, (m.Apu @ xp).reshape(3, -1)),
        "AUP": (xu, m.Apu.T @ xu.reshape(-1)),
        "A22": (xp, m.S @ xp + dt * (m.C @ xp)),
    }
    for op, (x, y_ref) in ref.items():
        y = s.apply(op, cuda(x, dtype), dt=dt).double().cpu().numpy()
        assert rel(y, y_ref) < tol, (op, rel(y, y_ref))
    x4 = np.concatenate([xu, xp[None]], 0)
    yj = s.apply("J", cuda(x4, dtype), dt=dt).double().cpu().numpy()
    yu_ref = m.Kb @ xu.reshape(-1) - m.Apu @ xp
    yp_ref = m.Apu.T @ xu.reshape(-1) + m.S @ xp + dt * (m.C @ xp)
    assert rel(yj[:3].reshape(-1), yu_ref) < tol
    assert rel(yj[3], yp_ref) < tol


def test_tet_apply_is_repeatable(case):
    prob, m, s, xu, xp = case
    x = cuda(xu)
    a = s.apply("KB", x).cpu().numpy()
    b = s.apply("KB", x).cpu().numpy()
    assert np.array_equal(a, b)


def test_tet_steps_match_oracle_cryer():
    """Cryer's sphere on the GPU (octant, 6 cells per radius, the first 20
    steps of the geometric schedule): each step by the library's partitioned
    CG (gm_tet_step) equals the oracle's direct solve of the monolithic system
    within 1e-9 in u and p, and the centre pressure shows the undrained start
    and the Mandel-Cryer rise."""
    need_gpu()
    import paper_2410_17133_gb300 as gm
    prob = W.cryer_octant(n=6, steps=40)
    K = 20
    m, ts, pc, u_ref, p_ref = tet.run(prob, nsteps=K)
    s = gm.TetSolver.from_problem(prob)
    u = torch.zeros((3, m.N), dtype=torch.float64, device="cuda")
    p = torch.zeros(m.N, dtype=torch.float64, device="cuda")
    mu_, mp_ = np.zeros(3 * m.N), np.zeros(m.N)
    centre = int(np.argmin(np.linalg.norm(prob.nodes, axis=1)))
    pg = []
    for k in range(K):
        s.step(prob.dts[k], u, p, rtol=1e-12)
        mu_, mp_ = m.step(mu_, mp_, prob.dts[k])
        assert rel(u.cpu().numpy().reshape(-1), mu_) < 1e-9, k
        assert rel(p.cpu().numpy(), mp_) < 1e-9, k
        pg.append(p[centre].item())
    assert np.allclose(pg, pc, rtol=1e-9)
    from oracle import analytic as A
    prm = A.cryer_params(prob.E, prob.nu, prob.alpha, prob.M, prob.k, prob.mu_f, prob.sigma0)
    assert 0.85 < pg[0] / prm["p0"] < 1.1 and max(pg) / prm["p0"] > 1.05
