"""The seeded workload generators agree with the oracle's geometry: the
faulted-aquifer workload projects its in-situ stress on the same fault frame
(n, t1, t2) that the oracle (and the library) build from the grid, its line
source injects exactly Q, and its layers are where they are stated."""
import numpy as np
import pytest

import workloads as W
from oracle import fem


def test_faulted_aquifer_frame_source_and_layers():
    p = W.faulted_aquifer(nv=20, ny=6, nz=8, steps=1, Q=0.5)
    mesh = fem.Mesh(p.nx, p.ny, p.nz, p.origin, p.h, p.shear, p.kf)
    fg = fem.fault_geometry(mesh)
    # rebuild the tractions from the oracle's frame and a stress tensor with the
    # stated gradients: they must equal the workload's
    depth = 500.0 + 2000.0 - (np.arange(p.n_pairs) % (p.nx + 1)) * p.h[0]
    p0 = 9.81e3 * depth
    S = np.zeros((p.n_pairs, 3, 3))
    S[:, 0, 0] = -(18.75e3 * depth - p0)
    S[:, 1, 1] = -(20.4e3 * depth - p0)
    S[:, 2, 2] = -(11.9e3 * depth - p0)
    tr = np.einsum("pij,pj->pi", S, fg["n"])
    assert np.allclose(-np.sum(tr * fg["n"], 1), p.fault.tn0, rtol=1e-12)
    assert np.allclose(np.sum(tr * fg["t1"], 1), p.fault.tau0[:, 0], rtol=1e-12, atol=1e-6)
    assert np.allclose(np.sum(tr * fg["t2"], 1), p.fault.tau0[:, 1], atol=1e-6)
    # normal faulting: the footwall (+ side) carries shear up-dip, i.e. the
    # hanging wall is driven down; everywhere 0.85 of the frictional strength
    assert np.all(p.fault.tau0[:, 0] > 0)
    assert np.allclose(np.hypot(*p.fault.tau0.T) / (0.6 * p.fault.tn0), 0.85, rtol=1e-3)
    assert np.isclose(p.fp.sum(), 0.5)
    assert np.unique(p.E).tolist() == [15e9, 25e9, 40e9]
    k_aq = p.k[p.E == 15e9]
    assert k_aq.min() > 1e-16 and p.k[p.E == 25e9].max() == 1e-19


def test_marginally_pressurised_case_matches_the_printed_parameters():
    """The T = 4 workload restates the paper's marginally pressurised case
    (Sec. 4.2, Table 1; golden file): tau0, sigma'_0, Q and the Table-1 fault
    values as printed, T = 4 from them within the printing's 2e-3, and a time
    schedule whose pressure front ends near 10 m (inside the 20 m half-width)
    with the closed-form rupture radius lambda(4) L spanning at least 8 cells."""
    import json
    import math
    import os
    from oracle import analytic as A
    g = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "table1_slip_benchmark.json")))
    p = W.marginally_pressurised()
    fp = p.fault
    assert abs(fp.tau0[0] / g["tau0_MP"] - 1) < 1e-12        # tau0 = ratio * f * sigma'_0
    assert fp.tn0 == g["sigma0"] and fp.f == g["f"]
    assert (fp.kn, fp.ks, fp.wk_par, fp.MF) == (g["kn"], g["ks"], g["wk_par"], g["MF"])
    assert abs(p.fp.sum() / g["Q"] - 1) < 1e-12
    assert p.mu_f == g["mu_f"] and p.E[0] == g["E"] and p.nu == g["nu"] and p.alpha == g["alpha"]
    T = A.stress_injection_parameter(fp.tau0[0], fp.f, fp.tn0, p.fp.sum(), p.mu_f, fp.wk_par)
    assert abs(T / g["T_MP"] - 1) < 2e-3
    D = A.fault_diffusivity(fp.wk_par, fp.MF, p.mu_f, fp.w0)
    L = math.sqrt(4 * D * sum(p.dts))
    assert 9.5 < L < 10.5 < g["box"] / 2
    assert A.lambda_of_T(T) * L / p.h[0] > 8.0


def test_stress_rotation_matches_the_papers_orientation_statements():
    """Sec. 5's stress-rotation study: rotating the horizontal stresses by beta
    from the strike, the Coulomb ratio |tau0| / (f t'_n0) of the fault is
    smallest at beta = 90 (the larger horizontal stress across the fault, the
    paper's most stable orientation) and largest between 20 and 40 degrees
    and, mirrored, between 140 and 160 (the paper: slip is promoted around 30
    and 150); beta and 180 - beta give the same ratio; beta = 0 is the default
    set-up; and the rotated tractions equal the rotated tensor projected on
    the oracle's fault frame."""
    def ratio(beta):
        p = W.faulted_aquifer(nv=20, ny=2, nz=2, steps=1, Q=0.5, beta_deg=beta)
        return float(np.max(np.linalg.norm(p.fault.tau0, axis=1) / (p.fault.f * p.fault.tn0)))
    bs = np.arange(0.0, 180.5, 1.0)
    rs = np.array([ratio(b) for b in bs])
    assert bs[np.argmin(rs)] == 90.0
    first = bs[np.argmax(np.where(bs < 90, rs, -1))]
    second = bs[np.argmax(np.where(bs > 90, rs, -1))]
    assert 20.0 <= first <= 40.0 and 140.0 <= second <= 160.0
    assert np.allclose(rs, rs[::-1], rtol=1e-12)
    d0 = W.faulted_aquifer(nv=20, ny=6, nz=8, steps=1, Q=0.5)
    d1 = W.faulted_aquifer(nv=20, ny=6, nz=8, steps=1, Q=0.5, beta_deg=0.0)
    assert np.array_equal(d0.fault.tn0, d1.fault.tn0) and np.array_equal(d0.fault.tau0, d1.fault.tau0)
    p = W.faulted_aquifer(nv=20, ny=6, nz=8, steps=1, Q=0.5, beta_deg=30.0)
    mesh = fem.Mesh(p.nx, p.ny, p.nz, p.origin, p.h, p.shear, p.kf)
    fg = fem.fault_geometry(mesh)
    depth = 500.0 + 2000.0 - (np.arange(p.n_pairs) % (p.nx + 1)) * p.h[0]
    p0 = 9.81e3 * depth
    b = np.radians(30.0)
    Rz = np.array([[1.0, 0.0, 0.0], [0.0, np.cos(b), -np.sin(b)], [0.0, np.sin(b), np.cos(b)]])
    S = np.zeros((p.n_pairs, 3, 3))
    S[:, 0, 0] = -(18.75e3 * depth - p0)
    S[:, 1, 1] = -(20.4e3 * depth - p0)
    S[:, 2, 2] = -(11.9e3 * depth - p0)
    S = np.einsum("ij,pjk,lk->pil", Rz, S, Rz)
    tr = np.einsum("pij,pj->pi", S, fg["n"])
    assert np.allclose(-np.sum(tr * fg["n"], 1), p.fault.tn0, rtol=1e-12)
    assert np.allclose(np.sum(tr * fg["t1"], 1), p.fault.tau0[:, 0], rtol=1e-10, atol=1e-6)
    assert np.allclose(np.sum(tr * fg["t2"], 1), p.fault.tau0[:, 1], rtol=1e-10, atol=1e-6)


def test_tetrahedralized_box_is_conforming():
    """Kuhn tetrahedralisation of a sheared faulted box: positive volumes that
    sum to the box volume; every fault triangle is a face of exactly one
    tetrahedron on each lip (interior faces are shared by two, so the fault
    surface is the only internal boundary); no tetrahedron holds both lips of
    a pair (the tetrahedral fault kernels rely on it)."""
    base = W.tiny_faulted(3, 2, 4, shear=(0.3, 0.2), h=(0.5, 0.4, 0.25))
    p = W.tetrahedralize(base)
    a, b, c, d = (p.nodes[p.tets[:, q]] for q in range(4))
    vol = np.einsum("ij,ij->i", np.cross(b - a, c - a), d - a) / 6.0
    assert vol.min() > 0
    assert vol.sum() == pytest.approx(1.5 * 0.8 * 1.0, rel=1e-12)
    faces = {}
    for t in p.tets:
        for f in ((0, 1, 2), (0, 1, 3), (0, 2, 3), (1, 2, 3)):
            key = tuple(sorted(t[list(f)]))
            faces[key] = faces.get(key, 0) + 1
    for lip in (0, 1):
        assert all(faces.get(tuple(sorted(p.pairs[tri, lip])), 0) == 1 for tri in p.fault_tris)
    boundary = [k for k, v in faces.items() if v == 1]
    n_outer = 2 * (2 * (3 * 2 + 3 * 4 + 2 * 4))          # two triangles per outer quad face
    assert len(boundary) == n_outer + 2 * len(p.fault_tris)
    lipm, lipp = set(p.pairs[:, 0]), set(p.pairs[:, 1])
    assert not any(lipm & set(t) and lipp & set(t) for t in p.tets)
