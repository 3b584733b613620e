"""The slip-front set-up (Sec. 4.2, Table 1) stepped on the GPU and by the CPU
oracle side by side: the critically stressed fault at the three shear-to-
strength ratios 0.9, 0.95 and 0.99, with the injection rate set from the
stress-injection parameter T, on the 40 m cube at 12^3 hexes (the largest grid
the oracle steps in a few seconds per step), six geometric steps that take the
fault from sticking to slipping (and, at the lower ratios, opening) pairs.

Fields must agree with the oracle to 1e-9 (FP64 path) and 1e-8 (FP32
operators and preconditioners inside the FP64 Newton refinement), and every
pair's stick / slip / open state must be identical after every step."""
import numpy as np
import pytest

import workloads as W
from oracle import solve as osolve

from gpu_common import need_gpu, rel, solver_for

pytestmark = pytest.mark.gpu

N = 12
STEPS = 6
DT0 = 40.0
_REF = {}


def problem(ratio, T):
    return W.slip_front(n=N, ratio=ratio, T=T, dt0=DT0, steps=STEPS)


def reference(ratio, T):
    key = (ratio, T)
    if key not in _REF:
        _REF[key] = osolve.run(problem(ratio, T), nsteps=STEPS, rtol=1e-12)[1]
    return _REF[key]


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("ratio,T", [(0.9, 0.1), (0.95, 0.1), (0.99, 0.1)])
def test_slip_front_steps_match_oracle(ratio, T, precision):
    need_gpu()
    prob = problem(ratio, T)
    ref = reference(ratio, T)
    s = solver_for(prob)
    tol = 1e-9 if precision == 0 else 1e-8
    slipped = 0
    for k in range(STEPS):
        s.step(prob.dts[k], newton_rtol=1e-12, precision=precision)
        st = s.get_state()
        r = ref[k]
        assert rel(st["u"], r.u) < tol, (k, rel(st["u"], r.u))
        assert rel(st["p"], r.p) < tol, (k, rel(st["p"], r.p))
        assert np.array_equal(st["flags"].astype(np.int64), r.flags), k
        assert rel(st["slip"].T, r.slip) < tol or np.abs(r.slip).max() == 0
        slipped = max(slipped, int((r.flags == 2).sum()))
    assert slipped >= 1
