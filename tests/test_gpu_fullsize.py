"""Full-size parity at the bench workloads (64^3 slip-front, 160^3 inclined,
the 128x256x256 faulted aquifer):
the GPU applies, in the launch configuration the bench uses, are compared with
the oracle on sampled rows that the oracle evaluates from the elements around
each sampled node (too large to assemble whole).  The implicit step at 64^3 is
checked through properties that hold at any size."""
import numpy as np
import pytest

import workloads as W
from oracle import fem, solve as osolve

from gpu_common import cuda, need_gpu, rel, solver_for, torch

pytestmark = pytest.mark.gpu


def sample_nodes(prob, seed, k=400):
    rng = np.random.default_rng(seed)
    N = prob.n_nodes
    nb = (prob.nx + 1) * (prob.ny + 1)
    picks = [rng.integers(0, N, k)]
    if prob.kf is not None:                      # both lips, edges and corners included
        lip = rng.integers(0, nb, k // 4)
        picks += [lip + nb * prob.kf, lip + nb * (prob.kf + 1), np.array([nb * prob.kf, nb * (prob.kf + 2) - 1])]
    picks.append(np.array([0, N - 1, nb - 1, N - nb]))
    return np.unique(np.concatenate(picks))


@pytest.mark.parametrize("cfg", ["slipfront64", "inclined160", "aquifer"])
def test_fullsize_sampled_apply(cfg):
    need_gpu()
    prob = {"slipfront64": lambda: W.slip_front(n=64), "inclined160": lambda: W.inclined_lognormal(n=160),
            "aquifer": lambda: W.faulted_aquifer()}[cfg]()
    dt = prob.dts[0]
    s = solver_for(prob)
    s.timestep(dt)
    nodes = sample_nodes(prob, 5)
    mesh = fem.Mesh(prob.nx, prob.ny, prob.nz, prob.origin, prob.h, prob.shear, prob.kf)
    model = fem.Model(prob, elements=fem.elements_touching(mesh, nodes))
    N = model.N
    u = W.random_vectors(N, 71, scale_u=1e-5)[0] + W.random_displacement_jump(prob, 72, scale=3e-6)
    st = osolve.initial_state(model)
    r, _, Kcoh = osolve.fault_terms(model, u.reshape(-1), st.dlie)
    g = s.fault_update(cuda(u))
    assert np.array_equal(g["flags"].cpu().numpy().astype(np.int64), r["state"])
    x_u, x_p = W.random_vectors(N, 73)
    yu_o, yp_o = osolve.apply(model, "J", x_u.reshape(-1), x_p, dt=dt, Kcoh=Kcoh)
    yu_o = yu_o.reshape(3, N)[:, nodes]
    yp_o = yp_o[nodes]
    x = np.concatenate([x_u, x_p[None]], axis=0)
    y64 = s.apply("J", cuda(x)).cpu().numpy()
    assert rel(y64[:3, nodes], yu_o) < 1e-12
    assert rel(y64[3, nodes], yp_o) < 1e-12
    y32 = s.apply("J", cuda(x, torch.float32)).cpu().numpy()
    assert rel(y32[:3, nodes], yu_o) < 2e-5
    assert rel(y32[3, nodes], yp_o) < 2e-5
    # operator symmetry of K_T and A22 at full size: <a, A b> = <b, A a>
    a_u, a_p = W.random_vectors(N, 74)
    Ka = s.apply("KT", cuda(a_u)).cpu().numpy()
    Kx = s.apply("KT", cuda(x_u)).cpu().numpy()
    fu = np.asarray(prob.fixed[0:3], bool)
    au0, xu0 = np.where(fu, 0, a_u), np.where(fu, 0, x_u)
    assert abs(np.sum(xu0 * Ka) - np.sum(au0 * Kx)) <= 1e-12 * np.sqrt(np.sum(Ka * Ka) * np.sum(xu0 * xu0))


def test_fullsize_slipfront_step_properties():
    """64^3 slip-front, FP32-refined and FP64 steps: both reach the Newton
    tolerance, agree to well inside it, report identical fault states, and the
    accepted state satisfies the residual and the fault law (recomputed by the
    library from the accepted fields)."""
    need_gpu()
    prob = W.slip_front(n=64)
    s32 = solver_for(prob)
    s64 = solver_for(prob)
    for k in range(3):
        r32 = s32.step(prob.dts[k], newton_rtol=1e-10, precision=1)
        r64 = s64.step(prob.dts[k], newton_rtol=1e-10)
        assert (r32["n_slip"], r32["n_stick"], r32["n_open"]) == (r64["n_slip"], r64["n_stick"], r64["n_open"])
    a, b = s32.get_state(), s64.get_state()
    assert rel(a["u"], b["u"]) < 1e-7 and rel(a["p"], b["p"]) < 1e-7
    assert np.array_equal(a["flags"], b["flags"])
    # the residual entry point at zero increments is the next step's initial residual
    z3 = torch.zeros((3, s64.N), dtype=torch.float64, device="cuda")
    z1 = torch.zeros(s64.N, dtype=torch.float64, device="cuda")
    s64.timestep(prob.dts[3])
    _, rh = s64.residual(z3, z1)
    nxt = s64.step(prob.dts[3], newton_rtol=1e-10)
    assert abs(rh - nxt["rhat0"]) <= 1e-12 * nxt["rhat0"]
    # pressure maximum at the injection pair, decreasing outwards along x
    st = s64.get_state()
    nb = 65 * 65
    p = st["p"][32 * nb: 33 * nb].reshape(65, 65)
    assert p.argmax() == 32 * 65 + 32
    row = p[32, 32:]
    # monotone decay where the pressure is significant (ahead of the front the
    # consistent-mass Galerkin scheme leaves undershoots of ~1e-9 of the peak)
    sig = row > 1e-6 * row[0]
    assert sig[:3].all() and np.all(np.diff(row[sig]) < 0)
    assert row.min() > -1e-6 * row[0]


def test_fullsize_slip_front_matches_closed_form():
    """The 64^3 slip-front workload run through its 50-step schedule on the GPU
    (FP32-refined, Newton 1e-8): the pressure front L(t) (where p = dp* E1(1))
    and the rupture radius R(t) (farthest slipping pair) agree with
    L = sqrt(4 D t), R = lambda(T) L (Sec. 4.2) within the paper's bounds
    (8 % for L, 5 % for R) once the fronts span several cells (t > 1000 s)."""
    import math
    from oracle import analytic as A
    need_gpu()
    n = 64
    prob = W.slip_front(n=n)
    s = solver_for(prob)
    fp = prob.fault
    D = A.fault_diffusivity(fp.wk_par, fp.MF, prob.mu_f, fp.w0)
    dps = A.theis_dpstar(prob.fp.sum(), prob.mu_f, fp.wk_par)
    lam = A.lambda_of_T(0.1)
    h = prob.h[0]
    x = (np.arange(n + 1) - n // 2) * h
    X, Y = np.meshgrid(x, x, indexing="xy")
    r = np.sqrt(X ** 2 + Y ** 2).ravel()
    nb = (n + 1) ** 2
    t = 0.0
    checked = 0
    for k, dt in enumerate(prob.dts):
        s.step(dt, newton_rtol=1e-8, precision=1)
        t += dt
        if t < 1000.0:
            continue
        st = s.get_state()
        p = st["p"][prob.kf * nb:(prob.kf + 1) * nb]
        row = p.reshape(n + 1, n + 1)[n // 2, n // 2:]
        target = dps * 0.21938393439552          # E1(1)
        i = int(np.where(row < target)[0][0])
        L = h * (i - 1 + (row[i - 1] - target) / (row[i - 1] - row[i]))
        R = r[st["flags"] == 2].max()
        La = math.sqrt(4 * D * t)
        assert abs(L - La) / La < 0.08, (t, L, La)
        assert abs(R - lam * La) / (lam * La) < 0.05, (t, R, lam * La)
        checked += 1
    assert checked >= 5


def test_marginally_pressurised_rupture_matches_lambda_4():
    """The marginally pressurised case of Sec. 4.2 (tau0 = 47.830 MPa, Q = 1e-6
    m^3/s: T = 4) on 256^3 hexes of the 40 m cube through its 64 geometric steps
    (FP32-refined, Newton 1e-8).  The rupture stays far behind the pressure
    front, R = lambda(4) L with lambda(4) = 0.1387.  Checked from the paper's
    final time of this case (t_f = 5400 s) to the end of the schedule: the
    pressure front L (p = dp* E1(1) on the fault, interpolated along a grid
    line through the injection point) within 8 % of sqrt(4 D t) at every step;
    the rupture inside the pressurised region (R < L, the MP ordering); and the
    rupture radius R = h sqrt(n_slip / pi) (the slipping area: the farthest
    slipping node quantises R to whole cells, 11 % of R here) within 8 % of
    lambda(4) sqrt(4 D t) on average over those steps and 10 % at each.  The
    paper bounds the front errors (8 % for L, 5 % for R) for the critically
    stressed case only (Sec. 4.2, the front-history figure); for this case the
    numerical R stays 5-6 % below lambda(4) L at 256^3, 384^3 and 512^3 alike,
    a deficit that does not shrink with the mesh.  The history is printed."""
    import math
    from oracle import analytic as A
    need_gpu()
    n = 256
    prob = W.marginally_pressurised(n=n)
    s = solver_for(prob)
    fp = prob.fault
    D = A.fault_diffusivity(fp.wk_par, fp.MF, prob.mu_f, fp.w0)
    dps = A.theis_dpstar(prob.fp.sum(), prob.mu_f, fp.wk_par)
    lam = A.lambda_of_T(A.stress_injection_parameter(fp.tau0[0], fp.f, fp.tn0, prob.fp.sum(), prob.mu_f, fp.wk_par))
    assert abs(lam - 0.1387) < 1e-3
    h = prob.h[0]
    nb = (n + 1) ** 2
    t = 0.0
    late = []
    for k, dt in enumerate(prob.dts):
        s.step(dt, newton_rtol=1e-8, precision=1)
        t += dt
        st = s.get_state()
        nslip = int((st["flags"] == 2).sum())
        if nslip == 0:
            continue
        R = h * math.sqrt(nslip / math.pi)
        p = st["p"][prob.kf * nb:(prob.kf + 1) * nb]
        row = p.reshape(n + 1, n + 1)[n // 2, n // 2:]
        target = dps * 0.21938393439552          # E1(1)
        i = int(np.where(row < target)[0][0])
        L = h * (i - 1 + (row[i - 1] - target) / (row[i - 1] - row[i]))
        La = math.sqrt(4 * D * t)
        eL, eR = (L - La) / La, (R - lam * La) / (lam * La)
        print(f"step {k} t {t:9.1f} s  L {L:6.3f} m ({100 * eL:+5.1f} %)  R {R:6.3f} m = {R / h:5.2f} cells "
              f"({100 * eR:+5.1f} % of lambda(4) sqrt(4Dt))")
        if t >= 5400.0:
            late.append((t, eL, eR, R, L))
    assert len(late) >= 5
    for t, eL, eR, R, L in late:
        assert abs(eL) < 0.08 and abs(eR) < 0.10 and R < L, (t, eL, eR, R, L)
    mean_eR = sum(e[2] for e in late) / len(late)
    print(f"mean R error from t_f = 5400 s: {100 * mean_eR:+.1f} %")
    assert abs(mean_eR) < 0.08, mean_eR
