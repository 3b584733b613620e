"""Sec. 5's stress-rotation study on the faulted aquifer at half size
(64 x 128 x 128 hexes, 1.09 M nodes): for each rotation beta of the horizontal
principal stresses about the vertical, FP32-refined steps from the
in-situ state until the first fault pair slips (run_until_slip), and the
injected volume Q t at that onset.  Only the angles whose printed stress
gradients leave the fault below failure before injection are run (outside
6-48.5 and 131.5-174 degrees, see the workload's notes).  The paper finds the
fault most stable with the larger horizontal stress across it (beta = 90); the
volume to the onset must therefore grow from beta = 60 to 90 and fall again to
120, and beta and 180 - beta (the same Coulomb ratio) must agree within the
step size.  Steps of one day, up to 400 days of injection.  About 10
minutes on a GB300, so it runs only when GM_ROTATION_SWEEP=1; the table of the
last run is recorded with the results."""
import os

import numpy as np
import pytest

import workloads as W

from gpu_common import need_gpu, solver_for

pytestmark = pytest.mark.gpu

BETAS = [0.0, 60.0, 75.0, 90.0, 105.0, 120.0, 180.0]


@pytest.mark.skipif(os.environ.get("GM_ROTATION_SWEEP") != "1", reason="long run: set GM_ROTATION_SWEEP=1")
def test_injected_volume_to_slip_onset_against_beta():
    need_gpu()
    import paper_2410_17133_gb300 as gm
    dt, nmax = 86400.0, 400
    vol = {}
    for beta in BETAS:
        prob = W.faulted_aquifer(64, 128, 128, steps=nmax, dt=dt, beta_deg=beta)
        Q = float(np.sum(prob.fp))
        s = solver_for(prob)
        n, t, v, st = gm.run_until_slip(s, prob.dts, Q, step_kw=dict(newton_rtol=1e-10, precision=1,
                                                                       schur_precond=1))
        slipped = bool(np.any(np.asarray(st["flags"]) == gm.SLIP))
        vol[beta] = v if slipped else float("inf")
        print(f"beta {beta:5.1f} deg: onset after {n} steps, t = {t / 86400:.2f} d, "
              f"injected volume {v:.4g} m^3" + ("" if slipped else " (no slip within the run)"))
        del s
    assert vol[90.0] >= vol[75.0] >= vol[60.0]
    assert vol[90.0] >= vol[105.0] >= vol[120.0]
    for b in (0.0, 60.0, 75.0):
        a, c = vol[b], vol[180.0 - b]
        assert a == c or abs(a - c) <= dt * float(np.sum(W.faulted_aquifer(64, 128, 128, steps=1).fp)) + 1e-9
