"""Gradient workload at full size: 64^3 hexes, log-normal permeability, 20
implicit steps (FP32 operators inside FP64 Newton refinement), objective
= squared slip at 256 random fault pairs + pressure at 64 random bulk nodes
after the last step.  The checkpointed multi-step adjoint (checkpoints every
5 steps) is checked against central finite differences of full GPU runs along
random log-permeability directions (numpy default_rng(45)) and along the
friction and log-source parameters.  Each finite-difference run must keep the
contact/friction state history of the base run, else the difference quotient
crosses a kink and the check is void.  GM_ADJOINT_FD_DIRECTIONS sets the
number of permeability directions (default 16, the count the gradient
workload asks for).  The half-size faulted aquifer
carries a caprock-pressure gradient checked the same way along log Q."""
import math
import os

import numpy as np
import pytest

import workloads as W

from gpu_common import need_gpu, solver_for, torch

pytestmark = pytest.mark.gpu
S0, P0 = 1e-6, 1e6
STEP = dict(newton_rtol=1e-12, precision=1, schur_precond=1)


def objective(st, pairs, nodes):
    return float(np.sum(st["slip"][:, pairs] ** 2) / S0 ** 2 + np.sum(st["p"][nodes]) / P0)


def forward(prob, k=None, f=None, qscale=1.0):
    s = solver_for(prob)
    if k is not None:
        s.set_permeability(k)
    if f is not None:
        s.set_friction(np.array([f]))
    if qscale != 1.0:
        s.loads(prob.fu, prob.fp * qscale)
    flags = []
    for dt in prob.dts:
        s.step(dt, **STEP)
        flags.append(s.get_state()["flags"].copy())
    return s.get_state(), np.stack(flags)


@pytest.fixture(scope="module")
def base():
    need_gpu()
    import paper_2410_17133_gb300 as gm
    prob = W.adjoint_lognormal()
    pairs, nodes = W.adjoint_objective(prob)
    s = solver_for(prob)
    s.set_adjoint_options(gm.F32, 1e-3, 1)

    def og(st):
        g_s = np.zeros_like(st["slip"])
        g_s[:, pairs] = 2 * st["slip"][:, pairs] / S0 ** 2
        g_p = np.zeros(s.N)
        np.add.at(g_p, nodes, 1.0 / P0)
        return None, torch.as_tensor(g_p, device="cuda"), torch.as_tensor(g_s, device="cuda")

    final, gk, gf, gq = gm.run_with_adjoint(s, prob.dts, og, checkpoint_every=5, step_kw=STEP,
                                            rtol=1e-10)
    _, flags = forward(prob)
    return dict(prob=prob, pairs=pairs, nodes=nodes, final=final, flags=flags,
                gk=gk.cpu().numpy(), gf=float(gf.sum().item()), gq=gq)


def central_difference(b, h, **perturb):
    Js = []
    for sgn in (1, -1):
        kw = {name: fn(sgn * h) for name, fn in perturb.items()}
        st, fl = forward(b["prob"], **kw)
        assert np.array_equal(fl, b["flags"]), "perturbed run left the base contact path"
        Js.append(objective(st, b["pairs"], b["nodes"]))
    return (Js[0] - Js[1]) / (2 * h)


def test_workload_has_slipping_pairs(base):
    assert (base["flags"][-1] == 2).sum() >= 20
    assert np.array_equal(base["final"]["flags"], base["flags"][-1])


def test_log_permeability_directions(base):
    prob = base["prob"]
    k0 = np.asarray(prob.k, float)
    rng = np.random.default_rng(45)
    nd = int(os.environ.get("GM_ADJOINT_FD_DIRECTIONS", "16"))
    worst = 0.0
    for d in range(nd):
        v = rng.normal(size=k0.size)
        pred = float(base["gk"] @ v)
        fd = central_difference(base, 1e-4, k=lambda e: k0 * np.exp(e * v))
        err = abs(pred - fd) / abs(fd)
        worst = max(worst, err)
        print(f"log-k direction {d}: adjoint {pred:.12e} fd {fd:.12e} rel {err:.2e}")
        assert err < 1e-5, f"direction {d}"
    print(f"log-k directions: {nd}, worst relative difference {worst:.2e}")


def test_friction_and_source_directions(base):
    prob = base["prob"]
    fd_f = central_difference(base, 1e-5, f=lambda e: prob.fault.f + e)
    fd_q = central_difference(base, 1e-5, qscale=lambda e: math.exp(e))
    print(f"friction: adjoint {base['gf']:.12e} fd {fd_f:.12e}; "
          f"log source: adjoint {base['gq']:.12e} fd {fd_q:.12e}")
    assert base["gf"] == pytest.approx(fd_f, rel=1e-5)
    assert base["gq"] == pytest.approx(fd_q, rel=1e-5)


def test_half_size_aquifer_caprock_gradient():
    """Faulted aquifer at half size (64x128x128 cells, 1.09 M nodes), 20 steps
    of 12 h, FP32 operators inside Newton to 1e-10: the checkpointed adjoint of
    the caprock pressure (hanging-wall nodes 1000-1200 m high) with respect to
    log Q equals the central difference of two GPU runs (h = 1e-4) to 1e-6."""
    need_gpu()
    import paper_2410_17133_gb300 as gm
    prob = W.faulted_aquifer(64, 128, 128, steps=20)
    nb = (prob.nx + 1) * (prob.ny + 1)
    node = np.arange(prob.n_nodes)
    height = (node % (prob.nx + 1)) * prob.h[0]
    cap = np.where((height >= 1000) & (height <= 1200) & (node // nb < prob.kf))[0]
    g_p = np.zeros(prob.n_nodes)
    g_p[cap] = 1.0 / P0
    kw = dict(newton_rtol=1e-10, precision=1, schur_precond=1)
    s = solver_for(prob)
    s.set_adjoint_options(gm.F32, 1e-3, 1)
    _, _, _, gq = gm.run_with_adjoint(s, prob.dts, lambda st: (None, torch.as_tensor(
        g_p, device="cuda"), None), checkpoint_every=5, step_kw=kw, rtol=1e-10)

    def caprock(qscale):
        s2 = solver_for(prob)
        s2.loads(prob.fu, prob.fp * qscale)
        for dt in prob.dts:
            s2.step(dt, **kw)
        return float(np.sum(s2.get_state()["p"][cap]) / P0)

    h = 1e-4
    fd = (caprock(math.exp(h)) - caprock(math.exp(-h))) / (2 * h)
    print(f"caprock log Q: adjoint {gq:.12e} fd {fd:.12e}")
    assert gq == pytest.approx(fd, rel=1e-6)
