"""Seeded synthetic inputs shared by the oracle and the GPU library.

This module only *describes* problems: grid sizes, material values, fault
parameters, boundary masks, nodal loads, time-step schedules and seeded random
fields.  It contains none of the method's arithmetic (no element matrices, no
fault law, no solver), so that the CPU oracle and the CUDA path can both start
from the same numbers while sharing no computation.

Node numbering (used by both sides, and by the C-ABI):
  a structured grid of nx x ny x nz hexahedra.  Node planes are counted along z.
  When a fault plane at original node plane ``kf`` is present, that plane is
  duplicated: extended plane ``kf`` is the lower lip ("-" side) and extended
  plane ``kf + 1`` is the upper lip ("+" side), so there are nz + 2 planes.
  node id n = i + (nx + 1) * (j + (ny + 1) * kk),  kk in [0, n_planes).
  Element (ei, ej, ek) uses extended planes kb, kb + 1 with
  kb = ek + (1 if fault and ek >= kf else 0).
  Element id e = ei + nx * (ej + ny * ek).
Vectors are stored field-major ("SoA"): u as (3, N), p as (N,).

The workloads restate the paper's verification and application set-ups
(Sec. 4.2 injection-induced slip, Table 1; Sec. 5 faulted aquifer) on
structured grids, and Cryer's sphere (Sec. 4.1) on a generated tetrahedral
mesh of one octant; the paper's own meshes and datasets are not used.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Optional

import numpy as np

__all__ = [
    "FaultParams",
    "Problem",
    "node_id",
    "n_planes",
    "fault_small",
    "slip_front",
    "marginally_pressurised",
    "inclined_lognormal",
    "adjoint_lognormal",
    "adjoint_objective",
    "faulted_aquifer",
    "TetProblem",
    "cryer_octant",
    "FaultedTetProblem",
    "tetrahedralize",
    "column_terzaghi",
    "column_terzaghi_tet",
    "theis_plate",
    "tiny_faulted",
    "random_vectors",
    "random_displacement_jump",
    "CONFIGS",
]


@dataclasses.dataclass
class FaultParams:
    """Cohesive-fault and fracture-flow parameters (Sec. 2.2, Table 1).

    kn, ks   normal / shear penalty stiffness [Pa/m]
    f        Coulomb friction coefficient [-]
    w0       hydraulic aperture used by the fault flow operators [m]
    wk_par   longitudinal transmissibility w * k_par [m^3]
    k_perp   transverse permeability [m^2]; <= 0 means infinite (tied p+ = p-)
    MF       fracture Biot modulus [Pa]
    tn0      in-situ effective normal traction, compression positive [Pa]
    tau0     in-situ shear traction in the fault frame (t1, t2) [Pa]
    """

    kn: float
    ks: float
    f: float
    w0: float
    wk_par: float
    k_perp: float
    MF: float
    tn0: float
    tau0: tuple

    def as_tuple(self):
        return (self.kn, self.ks, self.f, self.w0, self.wk_par, self.k_perp,
                self.MF, self.tn0, float(self.tau0[0]), float(self.tau0[1]))


@dataclasses.dataclass
class Problem:
    """One synthetic problem: grid, materials, fault, constraints, loads, steps."""

    name: str
    nx: int
    ny: int
    nz: int
    origin: tuple
    h: tuple
    shear: tuple            # (dz/dx, dz/dy) of the affine map
    kf: Optional[int]       # original node-plane index of the fault, or None
    fault: Optional[FaultParams]
    E: np.ndarray           # Young's modulus per element [Pa]
    k: np.ndarray           # permeability per element [m^2]
    nu: float
    alpha: float
    M: float                # Biot modulus [Pa]
    mu_f: float             # fluid viscosity [Pa s]
    fixed: np.ndarray       # uint8 (4, N): 1 = homogeneous Dirichlet on (ux,uy,uz,p)
    fu: np.ndarray          # (3, N) nodal forces [N]
    fp: np.ndarray          # (N,) nodal fluid sources [m^3/s]
    dts: list               # time-step sizes [s]
    notes: str = ""

    @property
    def n_planes(self) -> int:
        return n_planes(self.nz, self.kf)

    @property
    def n_nodes(self) -> int:
        return (self.nx + 1) * (self.ny + 1) * self.n_planes

    @property
    def n_el(self) -> int:
        return self.nx * self.ny * self.nz

    @property
    def n_pairs(self) -> int:
        return 0 if self.kf is None else (self.nx + 1) * (self.ny + 1)

    @property
    def n_dof(self) -> int:
        return 4 * self.n_nodes


def n_planes(nz: int, kf: Optional[int]) -> int:
    return nz + 1 + (0 if kf is None else 1)


def node_id(nx: int, ny: int, i, j, kk):
    return np.asarray(i) + (nx + 1) * (np.asarray(j) + (ny + 1) * np.asarray(kk))


def _empty(nx, ny, nz, kf):
    N = (nx + 1) * (ny + 1) * n_planes(nz, kf)
    return (np.zeros((4, N), np.uint8), np.zeros((3, N)), np.zeros(N))


def _fix_bottom(fixed, nx, ny):
    """u = 0 on the bottom face (extended plane 0)."""
    nb = (nx + 1) * (ny + 1)
    fixed[0:3, :nb] = 1


def _inject_centre(fp, nx, ny, kf, Q):
    """Constant-rate injection at the centre fault pair, split half/half
    between the two lips (Sec. 4.2)."""
    ic, jc = nx // 2, ny // 2
    fp[node_id(nx, ny, ic, jc, kf)] += 0.5 * Q
    fp[node_id(nx, ny, ic, jc, kf + 1)] += 0.5 * Q


# ---------------------------------------------------------------------------
# Workload definitions
# ---------------------------------------------------------------------------

def fault_small(n: int = 8, Q: float = 5e-5, steps: int = 5, dt: float = 2.0) -> Problem:
    """Unit cube, n^3 Q1 hexes, horizontal fault at mid-height, centre injection.

    E=20 GPa, nu=0.25, alpha=0.8, M=50 GPa, k=1e-15 m^2, mu=1e-3 Pa s;
    fault f=0.6, in-situ sigma'_n0=10 MPa, tau0=5.4 MPa along x, Table-1
    fracture-flow values, tied lip pressures; 5 steps of 2 s.  Penalties
    follow Table 1's kn/E and ks/E ratios per metre: kn=2e12, ks=2e11 Pa/m.
    """
    nx = ny = nz = n
    kf = n // 2
    fixed, fu, fp = _empty(nx, ny, nz, kf)
    _fix_bottom(fixed, nx, ny)
    _inject_centre(fp, nx, ny, kf, Q)
    nel = nx * ny * nz
    fault = FaultParams(kn=2e12, ks=2e11, f=0.6, w0=1e-4, wk_par=1e-15, k_perp=0.0,
                        MF=0.2e6, tn0=10e6, tau0=(5.4e6, 0.0))
    return Problem(name=f"fault{n}", nx=nx, ny=ny, nz=nz, origin=(0.0, 0.0, 0.0),
                   h=(1.0 / n,) * 3, shear=(0.0, 0.0), kf=kf, fault=fault,
                   E=np.full(nel, 20e9), k=np.full(nel, 1e-15), nu=0.25, alpha=0.8,
                   M=50e9, mu_f=1e-3, fixed=fixed, fu=fu, fp=fp, dts=[dt] * steps,
                   notes="unit cube, mid-height fault, centre injection")


def slip_front(n: int = 64, steps: int = 50, ratio: float = 0.99, T: float = 0.1,
               dt0: float = 1.0, growth: float = 1.115) -> Problem:
    """Sec. 4.2 restated on a structured grid: 40 m cube, n^3 hexes, fault at z=0.

    Table 1 values (E=60 GPa, nu=0, k_M=0, alpha=0, M=1e5 GPa, mu=0.89 mPa s,
    f=0.6, kn=6e3 GPa/m, ks=6e2 GPa/m, wk_par=1e-15 m^3, k_perp infinite,
    M_F=0.2 MPa), sigma'_0 = 80 MPa.  tau0 = ratio * f * sigma'_0 and the
    injection rate Q is chosen so that the stress-injection parameter equals T,
    i.e. Q = 4 pi wk_par dp* / mu with dp* = (1 - ratio) sigma'_0 / T.
    Geometric time steps dt_k = dt0 * growth^k.
    """
    nx = ny = nz = n
    kf = n // 2
    L = 40.0
    fixed, fu, fp = _empty(nx, ny, nz, kf)
    _fix_bottom(fixed, nx, ny)
    mu = 0.89e-3
    wk = 1e-15
    sig0 = 80e6
    dpstar = (1.0 - ratio) * sig0 / T
    Q = 4.0 * math.pi * wk * dpstar / mu
    _inject_centre(fp, nx, ny, kf, Q)
    nel = nx * ny * nz
    fault = FaultParams(kn=6e12, ks=6e11, f=0.6, w0=1e-4, wk_par=wk, k_perp=0.0,
                        MF=0.2e6, tn0=sig0, tau0=(ratio * 0.6 * sig0, 0.0))
    dts = [dt0 * growth ** s for s in range(steps)]
    return Problem(name=f"slipfront{n}", nx=nx, ny=ny, nz=nz,
                   origin=(-L / 2, -L / 2, -L / 2), h=(L / n,) * 3, shear=(0.0, 0.0),
                   kf=kf, fault=fault, E=np.full(nel, 60e9), k=np.zeros(nel),
                   nu=0.0, alpha=0.0, M=1e14, mu_f=mu, fixed=fixed, fu=fu, fp=fp,
                   dts=dts, notes=f"ratio={ratio} T={T} Q={Q:.6e}")


def marginally_pressurised(n: int = 256, steps: int = 64, dt0: float = 1.0,
                           growth: float = 1.119) -> Problem:
    """The marginally pressurised case of Sec. 4.2 (Table 1 values): tau0 =
    47.830 MPa against f sigma'_0 = 48 MPa and Q = 1e-6 m^3/s, i.e. the
    stress-injection parameter T = 4, on the 40 m cube of ``slip_front`` with
    n^3 hexes.  The rupture front stays far behind the pressure front here
    (R = lambda(4) L with lambda(4) = 0.139), so the grid must be fine: with
    n = 256 and the geometric steps dt_k = dt0 growth^k the pressure front
    reaches L = 10 m (half the half-width) near the last step, where R spans
    about nine cells."""
    sig0, tau0 = 80e6, 47.830e6
    mu, wk = 0.89e-3, 1e-15
    Q = 1e-6
    dpstar = Q * mu / (4.0 * math.pi * wk)
    T = (1.0 - tau0 / (0.6 * sig0)) * sig0 / dpstar
    prob = slip_front(n=n, steps=steps, ratio=tau0 / (0.6 * sig0), T=T, dt0=dt0, growth=growth)
    prob.name = f"marginal{n}"
    prob.notes = f"tau0={tau0} Q={Q} T={T:.4f}"
    return prob


def inclined_lognormal(n: int = 160, steps: int = 20, seed: int = 3,
                       dip_deg: float = 60.0, dt: float = 5.0, Q: float = 2e-4) -> Problem:
    """n^3 hexes on a sheared grid whose fault node plane dips ``dip_deg``.

    Per-element log10 k ~ N(-15, 0.5) and E ~ U[10, 30] GPa from
    numpy default_rng(seed); nu=0.25, alpha=0.8, M=50 GPa; fault f=0.6,
    sigma'_n0=10 MPa, tau0=5.4 MPa along the dip direction, tied lip pressures.
    The grid spacing is 1 m; the affine map adds dz = tan(dip) * x.
    """
    nx = ny = nz = n
    kf = n // 2
    fixed, fu, fp = _empty(nx, ny, nz, kf)
    _fix_bottom(fixed, nx, ny)
    _inject_centre(fp, nx, ny, kf, Q)
    rng = np.random.default_rng(seed)
    nel = nx * ny * nz
    logk = rng.normal(-15.0, 0.5, nel)
    E = rng.uniform(10e9, 30e9, nel)
    fault = FaultParams(kn=2e12, ks=2e11, f=0.6, w0=1e-4, wk_par=1e-15, k_perp=0.0,
                        MF=0.2e6, tn0=10e6, tau0=(5.4e6, 0.0))
    return Problem(name=f"inclined{n}", nx=nx, ny=ny, nz=nz, origin=(0.0, 0.0, 0.0),
                   h=(1.0, 1.0, 1.0), shear=(math.tan(math.radians(dip_deg)), 0.0),
                   kf=kf, fault=fault, E=E, k=10.0 ** logk, nu=0.25, alpha=0.8,
                   M=50e9, mu_f=1e-3, fixed=fixed, fu=fu, fp=fp, dts=[dt] * steps,
                   notes=f"seed={seed} dip={dip_deg}")


def adjoint_lognormal(n: int = 64, steps: int = 20, seed: int = 4, Q: float = 2e-5,
                      dt: float = 0.1) -> Problem:
    """The unit-cube faulted case of ``fault_small`` on n^3 hexes with a
    per-element log-normal permeability, log10 k ~ N(-15, 0.5) from numpy
    default_rng(seed); E=20 GPa, nu=0.25, alpha=0.8, M=50 GPa, mu=1e-3 Pa s,
    fault f=0.6, sigma'_n0=10 MPa, tau0=5.4 MPa, Table-1 fracture flow,
    constant injection Q at the centre pair, ``steps`` steps of ``dt``.
    The workload of gradient (adjoint) runs."""
    prob = fault_small(n=n, Q=Q, steps=steps, dt=dt)
    rng = np.random.default_rng(seed)
    prob.k = 10.0 ** rng.normal(-15.0, 0.5, prob.n_el)
    prob.name = f"adjoint{n}"
    prob.notes = f"seed={seed} Q={Q} dt={dt}"
    return prob


def adjoint_objective(prob: Problem, n_slip: int = 256, n_p: int = 64, seed: int = 44):
    """Observation sets of the gradient workload: ``n_slip`` random fault
    pairs (slip observed) and ``n_p`` random bulk nodes (pressure observed),
    from numpy default_rng(seed), without repetition."""
    rng = np.random.default_rng(seed)
    pairs = rng.choice(prob.n_pairs, min(n_slip, prob.n_pairs), replace=False)
    nb = (prob.nx + 1) * (prob.ny + 1)
    lo = nb * (prob.kf + 1)          # exclude both fault node planes
    bulk = np.concatenate([np.arange(0, nb * prob.kf), np.arange(lo + nb, prob.n_nodes)])
    nodes = rng.choice(bulk, min(n_p, bulk.size), replace=False)
    return pairs, nodes


def faulted_aquifer(nv: int = 128, ny: int = 256, nz: int = 256, steps: int = 100, seed: int = 5,
                    dt: float = 43200.0, Q: float = 0.01, throw: float = 150.0,
                    dip_deg: float = 80.0, sv_grad: float = 18.75e3, beta_deg: float = 0.0) -> Problem:
    """Faulted aquifer (Sec. 5 restated): 2000 m (vertical) x 4000 m x 4000 m.

    Grid axes: x is vertical (x = 0 at the bottom, H = 2000 m at the top, nv
    cells), y is the fault strike (ny cells), z crosses the fault (nz cells).
    The affine map z_phys = z + tan(90 deg - dip) x tilts the fault node plane
    kf = nz / 2 to the stated dip (80 deg: a mild 10 deg shear of the cells).
    Three layers by height: basement (E = 40 GPa, k = 1e-18 m^2), aquifer
    (E = 15 GPa, log10 k ~ N(-13, 0.7) from numpy default_rng(seed)) and
    caprock (E = 25 GPa, k = 1e-19 m^2); the aquifer spans 950-1050 m on the
    footwall and sits `throw` lower on the hanging wall (the grid-z < kf side,
    above the dipping plane), so the two segments meet only through the fault.
    nu = 0.15, alpha = 0.64, M = 22.7 GPa, mu = 0.89 mPa s; fault f = 0.6,
    kn = 27300 GPa/m, ks = 273 GPa/m, Table-1 fracture flow, tied lip pressures.
    In-situ stress grows with depth d below the ground surface (500 m of rock
    above the model top): vertical sv_grad * d, horizontal 11.9 kPa/m * d across
    the fault and 20.4 kPa/m * d along strike, hydrostatic pore pressure
    9.81 kPa/m * d; the fault carries the effective traction of that stress per
    pair, t'_n0 = -n.S'n and tau0 = (t1.S'n, t2.S'n) with S' the tension-positive
    effective stress and (n, t1, t2) the library's fault frame (n from the
    grid-z < kf side to the other, t1 the unit grid-x direction in the plane,
    t2 = n x t1).  beta_deg rotates the two horizontal principal stresses about
    the vertical by beta, the 20.4 kPa/m one from the strike towards the fault
    normal (Sec. 5's stress-rotation study; beta = 0 is the default set-up, 90
    puts the larger horizontal stress across the fault).  Injection Q as a line
    source over the hanging-wall aquifer at
    mid-strike, 250 m from the fault, split by nodal length.  Bottom face
    u = 0, all faces no-flow."""
    H, Ly, Lz = 2000.0, 4000.0, 4000.0
    nx = nv
    kf = nz // 2
    hx, hy, hz = H / nx, Ly / ny, Lz / nz
    sx = math.tan(math.radians(90.0 - dip_deg))
    fixed, fu, fp = _empty(nx, ny, nz, kf)
    # bottom face: grid x = 0, every extended plane
    nb = (nx + 1) * (ny + 1)
    planes = n_planes(nz, kf)
    bottom = (np.arange(ny + 1)[:, None] * (nx + 1) + nb * np.arange(planes)[None, :]).ravel()
    fixed[0:3, bottom] = 1
    # layers by element-centre height; hanging wall (k < kf) thrown down
    ex = (np.arange(nx) + 0.5) * hx
    nel = nx * ny * nz
    zc = np.broadcast_to(ex[None, None, :], (nz, ny, nx)).reshape(-1)
    kk = np.broadcast_to(np.arange(nz)[:, None, None], (nz, ny, nx)).reshape(-1)
    lo = np.where(kk < kf, 950.0 - throw, 950.0)
    layer = np.where(zc < lo, 0, np.where(zc < lo + 100.0, 1, 2))
    rng = np.random.default_rng(seed)
    k_aq = 10.0 ** rng.normal(-13.0, 0.7, nel)
    E = np.choose(layer, [40e9, 15e9, 25e9])
    k = np.choose(layer, [np.full(nel, 1e-18), k_aq, np.full(nel, 1e-19)])
    # per-pair in-situ effective traction on the fault
    n_ = np.array([-sx, 0.0, 1.0]) / math.hypot(sx, 1.0)
    t1 = np.array([1.0, 0.0, sx]) / math.hypot(sx, 1.0)
    t2 = np.cross(n_, t1)
    P = nb
    xi = (np.arange(P) % (nx + 1)) * hx
    depth = 500.0 + H - xi
    p0 = 9.81e3 * depth
    S = np.zeros((P, 3, 3))            # tension-positive effective stress, physical axes
    S[:, 0, 0] = -(sv_grad * depth - p0)
    sH = -(20.4e3 * depth - p0)
    sh = -(11.9e3 * depth - p0)
    cb, sb = math.cos(math.radians(beta_deg)), math.sin(math.radians(beta_deg))
    S[:, 1, 1] = cb * cb * sH + sb * sb * sh
    S[:, 2, 2] = sb * sb * sH + cb * cb * sh
    S[:, 1, 2] = S[:, 2, 1] = cb * sb * (sH - sh)
    tr = S @ n_
    tn0 = -(tr @ n_)
    tau0 = np.stack([tr @ t1, tr @ t2], 1)
    # line source over the hanging-wall aquifer
    kw = kf - max(1, int(round(250.0 / hz)))
    jw = ny // 2
    top = 950.0 - throw + 100.0
    iw = np.array([i for i in range(nx + 1) if 950.0 - throw - 1e-9 <= i * hx <= top + 1e-9])
    w = np.full(iw.size, hx)
    w[0] = w[-1] = 0.5 * hx
    fp[iw + (nx + 1) * (jw + (ny + 1) * kw)] = Q * w / w.sum()
    fault = FaultParams(kn=2.73e13, ks=2.73e11, f=0.6, w0=1e-4, wk_par=1e-15, k_perp=0.0,
                        MF=0.2e6, tn0=tn0, tau0=tau0)
    return Problem(name=f"aquifer{nv}x{ny}x{nz}", nx=nx, ny=ny, nz=nz, origin=(0.0, 0.0, -Lz / 2),
                   h=(hx, hy, hz), shear=(sx, 0.0), kf=kf, fault=fault, E=E, k=k, nu=0.15,
                   alpha=0.64, M=22.7e9, mu_f=0.89e-3, fixed=fixed, fu=fu, fp=fp,
                   dts=[dt] * steps, notes=f"seed={seed} dip={dip_deg} throw={throw} beta={beta_deg}")


@dataclasses.dataclass
class TetProblem:
    """An unstructured P1-tetrahedron problem without fault."""

    name: str
    nodes: np.ndarray       # (N, 3) coordinates [m]
    tets: np.ndarray        # (M, 4) vertex ids, positive orientation
    E: float
    nu: float
    alpha: float
    M: float
    k: float
    mu_f: float
    fixed: np.ndarray       # uint8 (4, N): 1 = homogeneous Dirichlet on (ux, uy, uz, p)
    load_tris: np.ndarray   # (T, 3) surface triangles carrying the normal traction, outward order
    sigma0: float           # compressive normal traction on load_tris [Pa]
    dts: list
    notes: str = ""


def cryer_octant(n: int = 8, R: float = 1.0, sigma0: float = 1e6, steps: int = 40,
                 E: float = 20e9, nu: float = 0.25, alpha: float = 0.8, M: float = 50e9,
                 k: float = 1e-15, mu_f: float = 1e-3) -> TetProblem:
    """Cryer's sphere (Sec. 4.1) as one octant of a ball of radius R.

    The unit cube [0, 1]^3 with n cells per edge is mapped onto the octant by
    x -> R x |x|_inf / |x|_2, so its faces x_i = 1 land on the sphere and its
    faces x_i = 0 on the symmetry planes; each cell is cut into the 6 Kuhn
    tetrahedra along its main diagonal (conforming between cells).  Symmetry
    planes: normal displacement 0; sphere: p = 0 and a compressive normal
    traction sigma0.  Time steps: a short first step (the undrained response)
    then a geometric series up to t* = c t / R^2 = 1 with c the consolidation
    coefficient (k/mu) / (1/M + alpha^2 / K_v)."""
    g = np.linspace(0.0, 1.0, n + 1)
    X, Y, Z = np.meshgrid(g, g, g, indexing="ij")
    P = np.stack([X.ravel(), Y.ravel(), Z.ravel()], 1)
    ninf = np.max(np.abs(P), axis=1)
    n2 = np.linalg.norm(P, axis=1)
    scale = np.where(n2 > 0, ninf / np.where(n2 > 0, n2, 1.0), 0.0)
    nodes = R * P * scale[:, None]
    idx = lambda i, j, kk: (i * (n + 1) + j) * (n + 1) + kk
    perms = [(0, 1, 2), (0, 2, 1), (1, 0, 2), (1, 2, 0), (2, 0, 1), (2, 1, 0)]
    tets = []
    for i in range(n):
        for j in range(n):
            for kk in range(n):
                for pm in perms:
                    v = [0, 0, 0]
                    path = [idx(i, j, kk)]
                    for ax in pm:
                        v[ax] += 1
                        path.append(idx(i + v[0], j + v[1], kk + v[2]))
                    tets.append(path)
    tets = np.array(tets)
    a, b, c, d = (nodes[tets[:, q]] for q in range(4))
    vol = np.einsum("ij,ij->i", np.cross(b - a, c - a), d - a)
    swap = vol < 0
    tets[swap, 1], tets[swap, 2] = tets[swap, 2].copy(), tets[swap, 1].copy()
    N = nodes.shape[0]
    fixed = np.zeros((4, N), np.uint8)
    for ax in range(3):
        fixed[ax, P[:, ax] == 0.0] = 1
    on_sphere = ninf == 1.0
    fixed[3, on_sphere] = 1
    # surface triangles: tetrahedron faces with all three vertices on one cube face x_i = 1
    tris = []
    faces = [(0, 1, 2, 3), (0, 1, 3, 2), (0, 2, 3, 1), (1, 2, 3, 0)]
    for t in tets:
        for f0, f1, f2, opp in faces:
            tri = [t[f0], t[f1], t[f2]]
            if any(np.all(P[tri, ax] == 1.0) for ax in range(3)):
                x0, x1, x2 = nodes[tri]
                nrm = np.cross(x1 - x0, x2 - x0)
                if np.dot(nrm, x0 - nodes[t[opp]]) < 0:
                    tri = [tri[0], tri[2], tri[1]]
                tris.append(tri)
    lam = E * nu / ((1 + nu) * (1 - 2 * nu))
    Kv = lam + E / (1 + nu)
    c = (k / mu_f) / (1.0 / M + alpha * alpha / Kv)
    t_end = R * R / c
    t0 = 1e-4 * t_end
    growth = (t_end / t0) ** (1.0 / (steps - 1))
    times = [t0 * growth ** s for s in range(steps)]
    dts = [times[0]] + [times[s] - times[s - 1] for s in range(1, steps)]
    return TetProblem(name=f"cryer{n}", nodes=nodes, tets=tets, E=E, nu=nu, alpha=alpha, M=M, k=k,
                      mu_f=mu_f, fixed=fixed, load_tris=np.array(tris), sigma0=sigma0, dts=dts,
                      notes="octant of a ball; Kuhn tetrahedra")


def column_terzaghi(nz: int = 16, H: float = 1.0, load: float = 1e6, steps: int = 200,
                    dt: float = None, E: float = 20e9, nu: float = 0.25,
                    alpha: float = 0.8, M: float = 50e9, k: float = 1e-15,
                    mu: float = 1e-3) -> Problem:
    """One-dimensional consolidation column: 1 x 1 x nz hexes of height H.

    Lateral displacements fixed everywhere (uniaxial strain), u_z = 0 at the
    bottom, a compressive traction ``load`` on the top face applied from the
    first step, the top face drained (p = 0), all other faces no-flow.
    """
    nx = ny = 1
    fixed, fu, fp = _empty(nx, ny, nz, None)
    fixed[0:2, :] = 1
    nb = (nx + 1) * (ny + 1)
    fixed[2, :nb] = 1
    top = slice(nz * nb, (nz + 1) * nb)
    fixed[3, top] = 1
    hx = H / nz
    # consistent nodal forces of a uniform traction on one bilinear face: area/4 each
    fu[2, top] = -load * (hx * hx) / 4.0
    nel = nz
    if dt is None:
        dt = 1.0
    return Problem(name=f"terzaghi{nz}", nx=1, ny=1, nz=nz, origin=(0.0, 0.0, 0.0),
                   h=(hx, hx, hx), shear=(0.0, 0.0), kf=None, fault=None,
                   E=np.full(nel, E), k=np.full(nel, k), nu=nu, alpha=alpha, M=M,
                   mu_f=mu, fixed=fixed, fu=fu, fp=fp, dts=[dt] * steps,
                   notes="1-D consolidation column")


def column_terzaghi_tet(nz: int = 16, H: float = 1.0, load: float = 1e6, steps: int = 200,
                        dt: float = None, E: float = 20e9, nu: float = 0.25, alpha: float = 0.8,
                        M: float = 50e9, k: float = 1e-15, mu: float = 1e-3) -> TetProblem:
    """``column_terzaghi`` on linear tetrahedra: the 1 x 1 x nz column of cubes
    of side H / nz, each cut into the 6 Kuhn tetrahedra along its (0,0,0)-(1,1,1)
    diagonal; lateral displacements fixed everywhere, u_z = 0 at the bottom,
    the top face drained (p = 0) and loaded by the compressive traction
    ``load`` on its two triangles (outward order), all other faces no-flow."""
    h = H / nz
    kk, j, i = np.meshgrid(np.arange(nz + 1), np.arange(2), np.arange(2), indexing="ij")
    i, j, kk = i.ravel(), j.ravel(), kk.ravel()
    nodes = np.stack([i * h, j * h, kk * h], axis=1).astype(float)
    nid = lambda a, b, c: a + 2 * (b + 2 * c)
    tets = []
    for c in range(nz):
        for path in _KUHN_PATHS:
            v = [0, 0, 0]
            corners = [nid(0, 0, c)]
            for ax in path:
                v[ax] += 1
                corners.append(nid(v[0], v[1], c + v[2]))
            tets.append(corners)
    tets = np.array(tets)
    a, b, cc, d = (nodes[tets[:, q]] for q in range(4))
    neg = np.einsum("ij,ij->i", np.cross(b - a, cc - a), d - a) < 0
    tets[neg, 1], tets[neg, 2] = tets[neg, 2].copy(), tets[neg, 1].copy()
    N = nodes.shape[0]
    fixed = np.zeros((4, N), np.uint8)
    fixed[0:2, :] = 1
    fixed[2, kk == 0] = 1
    fixed[3, kk == nz] = 1
    t0, t1, t2, t3 = nid(0, 0, nz), nid(1, 0, nz), nid(0, 1, nz), nid(1, 1, nz)
    tris = np.array([[t0, t1, t3], [t0, t3, t2]])
    return TetProblem(name=f"terzaghi_tet{nz}", nodes=nodes, tets=tets, E=E, nu=nu, alpha=alpha, M=M, k=k,
                      mu_f=mu, fixed=fixed, load_tris=tris, sigma0=load, dts=[1.0 if dt is None else dt] * steps,
                      notes="1-D consolidation column on Kuhn tetrahedra")


def theis_plate(n: int = 32, nz: int = 2, L: float = 40.0, Q: float = 1e-6,
                steps: int = 30, dt0: float = 0.5, growth: float = 1.15,
                tn0: float = 80e6) -> Problem:
    """Fault-plane flow with an impermeable, uncoupled matrix (k_M=0, alpha=0):
    the fault pressure follows the line-source (Theis) solution (Sec. 4.2).
    Table-1 fault values, shear far below the friction limit (no slip)."""
    nx = ny = n
    kf = nz // 2
    fixed, fu, fp = _empty(nx, ny, nz, kf)
    _fix_bottom(fixed, nx, ny)
    _inject_centre(fp, nx, ny, kf, Q)
    nel = nx * ny * nz
    fault = FaultParams(kn=6e12, ks=6e11, f=0.6, w0=1e-4, wk_par=1e-15, k_perp=0.0,
                        MF=0.2e6, tn0=tn0, tau0=(0.0, 0.0))
    dts = [dt0 * growth ** s for s in range(steps)]
    hz = L / n
    return Problem(name=f"theis{n}", nx=nx, ny=ny, nz=nz, origin=(-L / 2, -L / 2, -hz * kf),
                   h=(L / n, L / n, hz), shear=(0.0, 0.0), kf=kf, fault=fault,
                   E=np.full(nel, 60e9), k=np.zeros(nel), nu=0.0, alpha=0.0, M=1e14,
                   mu_f=0.89e-3, fixed=fixed, fu=fu, fp=fp, dts=dts,
                   notes="fault-only diffusion")


def tiny_faulted(nx: int = 2, ny: int = 2, nz: int = 2, shear=(0.0, 0.0), k_perp: float = 0.0,
                 seed: Optional[int] = None, Q: float = 2e-5, steps: int = 2,
                 dt: float = 1.0, h=(0.5, 0.5, 0.5)) -> Problem:
    """Small faulted box for direct-vs-partitioned and GPU parity checks.

    With ``seed`` the element E and k are drawn from default_rng(seed)
    (E ~ U[10, 30] GPa, log10 k ~ N(-15, 0.5)); otherwise uniform.
    """
    kf = nz // 2
    fixed, fu, fp = _empty(nx, ny, nz, kf)
    _fix_bottom(fixed, nx, ny)
    _inject_centre(fp, nx, ny, kf, Q)
    nel = nx * ny * nz
    if seed is None:
        E = np.full(nel, 20e9)
        k = np.full(nel, 1e-15)
    else:
        rng = np.random.default_rng(seed)
        E = rng.uniform(10e9, 30e9, nel)
        k = 10.0 ** rng.normal(-15.0, 0.5, nel)
    fault = FaultParams(kn=2e12, ks=2e11, f=0.6, w0=1e-4, wk_par=1e-15, k_perp=k_perp,
                        MF=0.2e6, tn0=10e6, tau0=(5.4e6, 0.0))
    return Problem(name=f"tiny{nx}x{ny}x{nz}", nx=nx, ny=ny, nz=nz, origin=(0.0, 0.0, 0.0),
                   h=tuple(h), shear=tuple(shear), kf=kf, fault=fault, E=E, k=k, nu=0.25,
                   alpha=0.8, M=50e9, mu_f=1e-3, fixed=fixed, fu=fu, fp=fp,
                   dts=[dt] * steps, notes="small faulted box")


@dataclasses.dataclass
class FaultedTetProblem:
    """A P1-tetrahedron problem with one planar fault of duplicated nodes.

    pairs[i] = (minus node, plus node) of fault node pair i; fault_tris holds
    the triangles of the fault surface as triples of pair ids, ordered so
    that the right-hand-rule normal points from the minus to the plus lip.
    t1_ref is the direction whose projection onto the fault is the first
    tangent t1 (tau0 is given in the frame t1, t2 = n x t1).  E and k are
    per tetrahedron; fixed, fu, fp and dts as in Problem."""

    name: str
    nodes: np.ndarray       # (N, 3) coordinates [m]; both lips at the same place
    tets: np.ndarray        # (M, 4) vertex ids, positive orientation
    pairs: np.ndarray       # (P, 2) node ids (minus, plus)
    fault_tris: np.ndarray  # (T, 3) pair ids, minus-to-plus right-hand order
    t1_ref: tuple
    fault: FaultParams
    E: np.ndarray           # (M,) [Pa]
    k: np.ndarray           # (M,) [m^2]
    nu: float
    alpha: float
    M: float
    mu_f: float
    fixed: np.ndarray       # uint8 (4, N)
    fu: np.ndarray          # (3, N)
    fp: np.ndarray          # (N,)
    dts: list
    notes: str = ""

    @property
    def n_nodes(self) -> int:
        return self.nodes.shape[0]


_KUHN_PATHS = [(0, 1, 2), (0, 2, 1), (1, 0, 2), (1, 2, 0), (2, 0, 1), (2, 1, 0)]


def tetrahedralize(prob: Problem, t1_ref=(1.0, 0.0, 0.0)) -> FaultedTetProblem:
    """The same faulted box on linear tetrahedra (the paper's element, Sec. 3.1):
    every hexahedron of the structured grid is cut into the six Kuhn
    tetrahedra along its diagonal from local corner (0,0,0) to (1,1,1), which
    is conforming between cells and cuts every fault quad along the same
    diagonal, into the triangles (b0, b1, b3) and (b0, b3, b2) of its corner
    pairs b = bx + 2 by.  Node numbering, lips, constraints, loads, sources,
    steps and fault parameters are those of ``prob``; each tetrahedron takes
    the E and k of its hexahedron."""
    nx, ny, nz, kf = prob.nx, prob.ny, prob.nz, prob.kf
    if kf is None:
        raise ValueError("tetrahedralize expects a faulted problem")
    nb = (nx + 1) * (ny + 1)
    npl = n_planes(nz, kf)
    kk, j, i = np.meshgrid(np.arange(npl), np.arange(ny + 1), np.arange(nx + 1), indexing="ij")
    i, j, kk = i.ravel(), j.ravel(), kk.ravel()
    korig = np.where(kk > kf, kk - 1, kk)
    hx, hy, hz = prob.h
    sx, sy = prob.shear
    ox, oy, oz = prob.origin
    nodes = np.stack([ox + i * hx, oy + j * hy,
                      oz + korig * hz + sx * i * hx + sy * j * hy], axis=1)
    ei, ej, ek = np.meshgrid(np.arange(nx), np.arange(ny), np.arange(nz), indexing="ij")
    ei, ej, ek = (a.transpose(2, 1, 0).ravel() for a in (ei, ej, ek))   # element id order
    kb = ek + (ek >= kf)
    tets = []
    for path in _KUHN_PATHS:
        v = [0, 0, 0]
        corners = [node_id(nx, ny, ei, ej, kb)]
        for ax in path:
            v[ax] += 1
            corners.append(node_id(nx, ny, ei + v[0], ej + v[1], kb + v[2]))
        tets.append(np.stack(corners, axis=1))
    tets = np.stack(tets, axis=1).reshape(-1, 4)                          # 6 per hex, hex-major
    a, b, c, d = (nodes[tets[:, q]] for q in range(4))
    neg = np.einsum("ij,ij->i", np.cross(b - a, c - a), d - a) < 0
    tets[neg, 1], tets[neg, 2] = tets[neg, 2].copy(), tets[neg, 1].copy()
    pid = np.arange(nb)
    pairs = np.stack([pid + nb * kf, pid + nb * (kf + 1)], axis=1)
    qi, qj = np.meshgrid(np.arange(nx), np.arange(ny), indexing="xy")
    qi, qj = qi.ravel(), qj.ravel()
    b0 = qi + (nx + 1) * qj
    b1, b2, b3 = b0 + 1, b0 + (nx + 1), b0 + (nx + 2)
    tris = np.concatenate([np.stack([b0, b1, b3], 1), np.stack([b0, b3, b2], 1)])
    E = np.repeat(np.broadcast_to(np.asarray(prob.E, float), (prob.n_el,)), 6)
    k = np.repeat(np.broadcast_to(np.asarray(prob.k, float), (prob.n_el,)), 6)
    return FaultedTetProblem(name=prob.name + "_tet", nodes=nodes, tets=tets, pairs=pairs,
                             fault_tris=tris, t1_ref=tuple(float(x) for x in t1_ref),
                             fault=prob.fault, E=E, k=k, nu=prob.nu, alpha=prob.alpha, M=prob.M,
                             mu_f=prob.mu_f, fixed=prob.fixed.copy(), fu=prob.fu.copy(),
                             fp=prob.fp.copy(), dts=list(prob.dts),
                             notes=prob.notes + "; Kuhn tetrahedra")


def random_vectors(n_nodes: int, seed: int, scale_u: float = 1e-4, scale_p: float = 1e6):
    """Seeded random (u, p) fields: u ~ U[-1,1] * scale_u (3, N), p ~ U[-1,1] * scale_p."""
    rng = np.random.default_rng(seed)
    u = rng.uniform(-1.0, 1.0, (3, n_nodes)) * scale_u
    p = rng.uniform(-1.0, 1.0, n_nodes) * scale_p
    return u, p


def random_displacement_jump(prob: Problem, seed: int, scale: float = 1e-6):
    """A displacement field that is zero except on the upper fault lip, where it
    is U[-1,1] * scale per component: prescribes arbitrary lip jumps."""
    rng = np.random.default_rng(seed)
    u = np.zeros((3, prob.n_nodes))
    if prob.kf is not None:
        nb = (prob.nx + 1) * (prob.ny + 1)
        plus = slice((prob.kf + 1) * nb, (prob.kf + 2) * nb)
        u[:, plus] = rng.uniform(-1.0, 1.0, (3, nb)) * scale
    return u


CONFIGS = {
    "fault8": fault_small,
    "slipfront64": slip_front,
    "inclined160": inclined_lognormal,
    "aquifer": faulted_aquifer,
    "adjoint64": adjoint_lognormal,
}
