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
