"""The full faulted-aquifer workload (Sec. 5 restated on 128 x 256 x 256 hexes,
8.55 M nodes, 34 M DoF): 100 FP32-refined implicit steps of 12 h, then the
checkpointed adjoint of the caprock pressure (hanging-wall nodes 1000-1200 m
high) with respect to log Q, checked against a central difference of two more
100-step GPU runs.  About 15 minutes on a GB300, so it runs only when
GM_FULL_AQUIFER=1; the timings of the last run are recorded with the results."""
import math
import os
import time

import numpy as np
import pytest

import workloads as W

from gpu_common import need_gpu, solver_for, torch

pytestmark = pytest.mark.gpu

P0 = 1e6


@pytest.mark.skipif(os.environ.get("GM_FULL_AQUIFER") != "1", reason="long run: set GM_FULL_AQUIFER=1")
def test_full_aquifer_100_steps_and_caprock_gradient():
    need_gpu()
    import paper_2410_17133_gb300 as gm
    prob = W.faulted_aquifer()
    nb = (prob.nx + 1) * (prob.ny + 1)
    node = np.arange(prob.n_nodes)
    height = (node % (prob.nx + 1)) * prob.h[0]
    cap = np.where((height >= 1000) & (height <= 1200) & (node // nb < prob.kf))[0]
    g_p = np.zeros(prob.n_nodes)
    g_p[cap] = 1.0 / P0
    kw = dict(newton_rtol=1e-10, precision=1, schur_precond=1)
    s = solver_for(prob)
    s.set_adjoint_options(gm.F32, 1e-3, 1)
    t0 = time.perf_counter()
    final, _, _, gq = gm.run_with_adjoint(s, prob.dts, lambda st: (None, torch.as_tensor(
        g_p, device="cuda"), None), checkpoint_every=5, step_kw=kw, rtol=1e-10)
    t_adj = time.perf_counter() - t0
    nslip = int((final["flags"] == 2).sum())

    def caprock(qscale):
        s2 = solver_for(prob)
        s2.loads(prob.fu, prob.fp * qscale)
        t = time.perf_counter()
        for dt in prob.dts:
            s2.step(dt, **kw)
        return float(np.sum(s2.get_state()["p"][cap]) / P0), time.perf_counter() - t

    h = 1e-4
    jp, t_fwd = caprock(math.exp(h))
    jm, _ = caprock(math.exp(-h))
    fd = (jp - jm) / (2 * h)
    print(f"full aquifer: {prob.n_nodes} nodes, {len(prob.dts)} steps; forward run {t_fwd:.1f} s "
          f"({t_fwd / len(prob.dts):.2f} s per step); forward + checkpointed recompute + adjoint sweep "
          f"{t_adj:.1f} s; slipping pairs at the end {nslip}; caprock log Q: adjoint {gq:.12e} fd {fd:.12e}")
    assert gq == pytest.approx(fd, rel=1e-5)
