"""Pins for the oracle's fault law: hand-worked single-pair cases of Sec. 2.2.1
(Eqs. normal_traction, yield_function, slip_split, plastic_slip_increment,
corrector) with exactly representable numbers, and the tangent reading checked
against finite differences."""
import numpy as np
import pytest

from oracle.law import OPEN, SLIP, STICK, return_map

n = np.array([[0.0, 0.0, 1.0]])
t1 = np.array([[1.0, 0.0, 0.0]])
t2 = np.array([[0.0, 1.0, 0.0]])
kn, ks, f, tn0 = 1000.0, 100.0, 0.5, 10.0
tau0 = np.array([3.0, 0.0])


def rm(jump, dlie=(0.0, 0.0), tau=tau0):
    return return_map(np.array([jump], float), n, t1, t2, kn, ks, f, tn0, tau,
                      np.array([dlie], float))


def test_stick_at_rest():
    r = rm([0, 0, 0])
    assert r["state"][0] == STICK
    assert r["tn"][0] == 10.0 and np.all(r["ts"][0] == [3.0, 0.0])
    assert np.all(r["T"][0] == 0.0)                 # in-situ state is the offset


def test_slip_hand_worked():
    # jump 0.04 along x: t_tr = 3 + 100*0.04 = 7 > f tn = 5  ->  slip
    r = rm([0.04, 0, 0])
    assert r["state"][0] == SLIP
    assert r["dlam"][0] == pytest.approx((7.0 - 5.0) / ks)       # Eq. corrector
    assert np.allclose(r["ts"][0], [5.0, 0.0])
    assert np.allclose(r["dlie"][0], [0.02, 0.0])
    assert np.allclose(r["T"][0], [2.0, 0.0, 0.0])               # t_s - tau0


def test_slip_direction_2d_and_normal_change():
    # jump (0.0, 0.04, -0.002): tn = 10 + 2 = 12, strength 6; t_tr = (3, 4): |t_tr| = 5 < 6 stick
    r = rm([0.0, 0.04, -0.002])
    assert r["state"][0] == STICK and r["tn"][0] == pytest.approx(12.0)
    # jump (0.0, 0.09, 0.0): t_tr = (3, 9), |.| = sqrt(90) > 5: slip along t_tr
    r = rm([0.0, 0.09, 0.0])
    assert r["state"][0] == SLIP
    tau = np.array([3.0, 9.0]) / np.sqrt(90.0)
    assert np.allclose(r["ts"][0], 5.0 * tau)
    assert np.allclose(r["dlie"][0], (np.sqrt(90.0) - 5.0) / ks * tau)


def test_yield_boundary_is_stick():
    # t_tr = 3 + 100*0.02 = 5 = f tn exactly -> F = 0 -> STICK (tie rule)
    r = rm([0.02, 0, 0])
    assert r["F"][0] == 0.0 and r["state"][0] == STICK


def test_open_releases_insitu_tractions():
    r = rm([0.0, 0.0, 0.02])                         # tn_c = 10 - 20 < 0
    assert r["state"][0] == OPEN
    assert r["tn"][0] == 0.0 and np.all(r["ts"][0] == 0.0)
    assert np.allclose(r["T"][0], [-3.0, 0.0, 10.0])
    # contact exactly at zero gap is contact (tn = 0), per the tie rule
    r = rm([0.0, 0.0, 0.01])
    assert r["state"][0] != OPEN and r["tn"][0] == 0.0


def test_unloading_keeps_inelastic_slip():
    r1 = rm([0.04, 0, 0])
    r2 = rm([0.0, 0, 0], dlie=r1["dlie"][0])
    # t_tr = 3 + 100*(0 - 0.02) = 1 -> stick, elastic recovery only
    assert r2["state"][0] == STICK
    assert np.allclose(r2["ts"][0], [1.0, 0.0])
    assert np.allclose(r2["dlie"][0], [0.02, 0.0])


def fd_jac(jump, h=1e-7):
    J = np.zeros((3, 3))
    for b in range(3):
        e = np.zeros(3); e[b] = h
        J[:, b] = (rm(jump + e)["T"][0] - rm(jump - e)["T"][0]) / (2 * h)
    return J


def test_tangent_stick_exact_and_slip_symmetric_reading():
    j = np.array([0.001, -0.002, 0.0005])
    assert rm(j)["state"][0] == STICK
    assert np.allclose(rm(j)["D"][0], fd_jac(j), rtol=1e-6, atol=1e-6)
    j = np.array([0.05, 0.03, -0.001])
    r = rm(j)
    assert r["state"][0] == SLIP
    tau = r["ts"][0] / np.linalg.norm(r["ts"][0])
    taug = tau[0] * t1[0] + tau[1] * t2[0]
    # the consistent tangent is D - f kn tau n^T; the symmetric reading drops that term
    assert np.allclose(r["D"][0] - f * kn * np.outer(taug, n[0]), fd_jac(j), rtol=1e-5, atol=1e-5)
    assert np.allclose(r["D"][0], r["D"][0].T)
    assert np.all(rm([0, 0, 0.05])["D"][0] == 0.0)


def test_per_pair_insitu_equals_pairwise_scalar_calls():
    """Per-pair in-situ tractions (depth-dependent stress) give, pair by pair,
    the result of the pinned single-pair law with that pair's scalars."""
    rng = np.random.default_rng(11)
    P = 9
    nn = np.repeat(n, P, 0)
    tt1 = np.repeat(t1, P, 0)
    tt2 = np.repeat(t2, P, 0)
    tn0p = rng.uniform(5.0, 15.0, P)
    tau0p = np.stack([rng.uniform(1.0, 6.0, P), rng.uniform(-1.0, 1.0, P)], 1)
    jump = np.stack([rng.uniform(-0.05, 0.05, P), rng.uniform(-0.05, 0.05, P),
                     rng.uniform(-0.004, 0.02, P)], 1)
    dlie = rng.uniform(-0.01, 0.01, (P, 2))
    r = return_map(jump, nn, tt1, tt2, kn, ks, f, tn0p, tau0p, dlie)
    assert len(set(r["state"].tolist())) == 3          # open, stick and slip all present
    for i in range(P):
        ri = return_map(jump[i:i + 1], n, t1, t2, kn, ks, f, tn0p[i], tau0p[i], dlie[i:i + 1])
        for key in ("state", "tn", "ts", "dlie", "T", "D", "F"):
            assert np.array_equal(r[key][i], ri[key][0]), (i, key)
