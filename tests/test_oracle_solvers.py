"""Pins for the oracle's solvers: dense LU, sparse direct and Prevost's
partitioned CG agree (Sec. 3.3.2: the Schur-complement reduction is exact),
Newton converges on the nonlinear fault problem, and the discretisation
reproduces 1-D consolidation and the line-source fault pressure."""
import math

import numpy as np
from scipy import special
import pytest

import workloads as W
from oracle import analytic, fem, solve


@pytest.mark.parametrize("dims,shear,kperp", [((1, 1, 2), (0, 0), 0.0),
                                              ((2, 2, 2), (0.5, 0), 0.0),
                                              ((2, 2, 2), (0, 0), 1e-12),
                                              ((4, 4, 4), (0, 0), 0.0)])
def test_direct_vs_partitioned(dims, shear, kperp):
    prob = W.tiny_faulted(*dims, shear=shear, k_perp=kperp, seed=7, Q=2e-4)
    model = fem.Model(prob)
    st = solve.initial_state(model)
    rng = np.random.default_rng(3)
    u = rng.normal(size=3 * model.N) * 1e-6
    r, force, Kcoh = solve.fault_terms(model, u, st.dlie)
    KT, Apu, A22 = solve.jacobian_blocks(model, Kcoh, 1.5)
    b1 = rng.normal(size=KT.shape[0]) * 1e3
    b2 = rng.normal(size=A22.shape[0]) * 1e-9
    x1a, x2a = solve.solve_monolithic(KT, Apu, A22, b1, b2, dense=True)
    x1b, x2b = solve.solve_monolithic(KT, Apu, A22, b1, b2, dense=False)
    x1c, x2c, it = solve.solve_prevost(KT, Apu, A22, b1, b2, rtol=1e-14)
    for x1, x2 in ((x1b, x2b), (x1c, x2c)):
        assert np.linalg.norm(x1 - x1a) <= 1e-10 * np.linalg.norm(x1a)
        assert np.linalg.norm(x2 - x2a) <= 1e-10 * np.linalg.norm(x2a)
    assert it <= A22.shape[0] + 1


def test_newton_paths_agree_across_linear_solvers():
    prob = W.tiny_faulted(4, 4, 4, seed=11, Q=4e-4, steps=3)
    _, ra = solve.run(prob, solver="lu")
    _, rb = solve.run(prob, solver="prevost")
    for a, b in zip(ra, rb):
        assert np.array_equal(a.flags, b.flags)
        assert np.linalg.norm(a.u - b.u) <= 1e-10 * np.linalg.norm(a.u)
        assert np.linalg.norm(a.p - b.p) <= 1e-10 * np.linalg.norm(a.p)


def test_fault_small_reaches_all_states_without_ties():
    """The 8^3 faulted cube: final step has OPEN, STICK and >= 4 SLIP pairs, and no
    pair within 1e-8 of a state boundary at any step."""
    prob = W.fault_small()
    _, res = solve.run(prob)
    fp = prob.fault
    for r in res:
        c = r.tn > 0
        assert np.all(np.abs(r.F[c]) / (fp.f * r.tn[c]) > 1e-8)
        assert np.all(np.abs(fp.tn0 - fp.kn * r.dn) / fp.tn0 > 1e-8)
        assert r.rhat <= 1e-12 * r.rhat0
    fl = res[-1].flags
    assert (fl == 0).sum() >= 1 and (fl == 1).sum() >= 4 and (fl == 2).sum() >= 4


def terzaghi_error(nz, steps=400, tstar=0.2):
    H = 1.0
    E, nu, alpha, M, k, mu, F = 20e9, 0.25, 0.8, 50e9, 1e-15, 1e-3, 1e6
    p0, cv = analytic.terzaghi_params(E, nu, alpha, M, k, mu, F)
    t_end = tstar * H * H / cv
    prob = W.column_terzaghi(nz=nz, H=H, load=F, steps=steps, dt=t_end / steps)
    model, res = solve.run(prob)
    X = model.mesh.coords()
    nb = model.mesh.nb
    z = X[::nb, 2]
    p_num = res[-1].p[::nb]
    p_an = analytic.terzaghi_pressure(z, t_end, H, p0, cv)
    return np.abs(p_num - p_an).max() / p0


def test_terzaghi_consolidation_converges_at_second_order():
    e8 = terzaghi_error(8)
    e16 = terzaghi_error(16)
    assert e16 < 0.01
    assert e8 / e16 > 2.5


def pressure_front(xy, p_rel):
    """Radius where the fault pressure falls to dp* E1(1) along the +x and +y
    rays through the source (linear interpolation between nodes)."""
    level = special.exp1(1.0)
    out = []
    for ax in (0, 1):
        ray = (np.abs(xy[:, 1 - ax]) < 1e-9) & (xy[:, ax] > 0)
        o = np.argsort(xy[ray, ax])
        rr, pp = xy[ray, ax][o], p_rel[ray][o]
        k = np.nonzero(pp < level)[0][0]
        out.append(rr[k - 1] + (pp[k - 1] - level) / (pp[k - 1] - pp[k]) * (rr[k] - rr[k - 1]))
    return np.array(out)


def test_theis_fault_pressure():
    """Impermeable, uncoupled matrix (Sec. 4.2): after 50 steps (t = 3600 s)
    the pressure front, where p = dp* E1(1), lies within the paper's 8 % of
    L = sqrt(4Dt) (4.6 cells here) on both grid axes, and the pressure at
    radii of 3 to 8 cells, where it spans 0.01 to 0.65 dp*, is within 6 % of
    dp* of dp* E1(r^2/4Dt) (the log-singular point source on 1.25 m cells
    costs 5 % at 3 cells)."""
    prob = W.theis_plate(n=32, steps=50)
    model, res = solve.run(prob)
    fp = prob.fault
    t = sum(prob.dts)
    X = model.mesh.coords()
    pairs = model.fg["pairs"]
    Q = prob.fp.sum()
    dps = analytic.theis_dpstar(Q, prob.mu_f, fp.wk_par)
    r = np.linalg.norm(X[pairs[:, 0], :2], axis=1)
    p = res[-1].p[pairs[:, 0]]
    D = analytic.fault_diffusivity(fp.wk_par, fp.MF, prob.mu_f, fp.w0)
    L = math.sqrt(4 * D * t)
    assert 4 * prob.h[0] < L < 10.0                     # resolved, and well inside 20 m
    assert np.abs(pressure_front(X[pairs[:, 0], :2], p / dps) / L - 1).max() < 0.08
    h = prob.h[0]
    sel = (r >= 3 * h - 1e-9) & (r <= 8 * h + 1e-9)
    pan = analytic.theis_pressure(r[sel], t, Q, prob.mu_f, fp.wk_par, fp.MF, fp.w0)
    assert pan.max() > 0.5 * dps
    assert (np.abs(p[sel] - pan) / dps).max() < 0.06
