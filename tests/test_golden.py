"""Values printed in the paper (tests/golden/), checked against the workloads
and the oracle's closed forms."""
import json
import os

import pytest

import workloads as W
from oracle import analytic

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def load(name):
    with open(os.path.join(GOLD, name)) as f:
        return json.load(f)


def test_slip_front_workload_uses_table1():
    g = load("table1_slip_benchmark.json")
    prob = W.slip_front(n=8, steps=1)
    fp = prob.fault
    assert (prob.E[0], prob.nu, prob.alpha, prob.M, prob.mu_f) == (g["E"], g["nu"], g["alpha"], g["M"], g["mu_f"])
    assert prob.k.max() == g["k_matrix"]
    assert (fp.f, fp.kn, fp.ks, fp.wk_par, fp.MF, fp.tn0) == (g["f"], g["kn"], g["ks"], g["wk_par"], g["MF"], g["sigma0"])
    assert fp.k_perp <= 0                       # infinite transverse permeability: tied
    assert prob.nx * prob.h[0] == g["box"]


def test_printed_marginally_pressurised_case_has_T_4():
    g = load("table1_slip_benchmark.json")
    T = analytic.stress_injection_parameter(g["tau0_MP"], g["f"], g["sigma0"], g["Q"], g["mu_f"], g["wk_par"])
    assert T == pytest.approx(g["T_MP"], rel=2e-3)


def test_printed_critically_stressed_tau0_is_rounded():
    """With the printed tau0 = 47.999 MPa the parameter evaluates to ~0.024, not
    the stated 0.01: the printed shear load is rounded, so the slip-front
    workload sets tau0 from the stated ratio and T instead."""
    g = load("table1_slip_benchmark.json")
    T = analytic.stress_injection_parameter(g["tau0_CS"], g["f"], g["sigma0"], g["Q"], g["mu_f"], g["wk_par"])
    assert 0.02 < T < 0.03
