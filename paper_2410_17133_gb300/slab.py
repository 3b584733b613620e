"""Slab decomposition of the structured grid over several ranks (one GPU each).

The grid is cut along y, parallel to the fault plane (every horizontal or
x-z-sheared fault spans the whole y range), so each slab holds a share of the
fault pairs and the cut never crosses a fault element.  Rank r owns the element
rows [j0_r, j1_r) and the node rows [j0_r, j1_r) (the last rank also the top
row ny); node row j0_r (r > 0) is shared with rank r - 1, which holds it as its
top row without owning it.

Each rank binds an ordinary context on its slab (the sub-problem below).  An
operator product on the slab gives complete rows everywhere except on the
shared node rows, which lack the elements (and the fault quads) of the other
side: one exchange of those rows' partial sums with each neighbour (all fields,
all node planes) completes them on both copies.  Fault pairs on a shared row
are computed by both ranks: each side integrates its own quads (half of the
pair's tributary area), and the exchange adds the halves.  Dot products sum
over owned nodes and are all-reduced.  This is the parallel layout of the
paper's solver (Sec. 3.3.2 partitioned CG; the strong-scaling set-up of
Sec. 4), restated for slabs of a structured grid.

Communication goes through torch.distributed point-to-point and all-reduce on
the tensors' device: gloo on CPU tensors (how the decomposition is tested),
NCCL on GPU tensors.  The local operator product is a callable, so the same
driver runs on a rank's libgm context or on any other local operator.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Callable, Optional, Sequence, Tuple

import numpy as np


def partition(ny: int, world: int) -> list:
    """Element-row ranges [j0, j1) of the ranks, balanced, each non-empty."""
    if world < 1 or ny < world:
        raise ValueError(f"cannot cut {ny} element rows into {world} slabs")
    edges = [round(r * ny / world) for r in range(world + 1)]
    return [(edges[r], edges[r + 1]) for r in range(world)]


@dataclasses.dataclass
class Slab:
    rank: int
    world: int
    j0: int              # first element row (= first node row) of the slab
    j1: int              # one past the last element row (= the top node row)
    nx: int
    ny: int              # global element rows
    nplanes: int

    @property
    def ny_local(self) -> int:
        return self.j1 - self.j0

    @property
    def nb_local(self) -> int:
        return (self.nx + 1) * (self.ny_local + 1)

    @property
    def n_local(self) -> int:
        return self.nb_local * self.nplanes

    def global_nodes(self) -> np.ndarray:
        """Global node ids of the slab's nodes in local order."""
        kk, jl, i = np.meshgrid(np.arange(self.nplanes), np.arange(self.ny_local + 1), np.arange(self.nx + 1),
                                indexing="ij")
        return (i + (self.nx + 1) * ((jl + self.j0) + (self.ny + 1) * kk)).ravel()

    def owned(self) -> np.ndarray:
        """Local nodes this rank owns (its bottom row only on rank 0 is shared-free;
        the top row only on the last rank)."""
        jl = (np.arange(self.n_local) // (self.nx + 1)) % (self.ny_local + 1)
        top = self.ny_local if self.rank == self.world - 1 else self.ny_local - 1
        return jl <= top

    def global_elements(self, nz: int) -> np.ndarray:
        ek, ej, ei = np.meshgrid(np.arange(nz), np.arange(self.j0, self.j1), np.arange(self.nx), indexing="ij")
        return (ei + self.nx * (ej + self.ny * ek)).ravel()

    def global_pairs(self) -> np.ndarray:
        jl, i = np.meshgrid(np.arange(self.ny_local + 1), np.arange(self.nx + 1), indexing="ij")
        return (i + (self.nx + 1) * (jl + self.j0)).ravel()


def make_slab(prob, rank: int, world: int) -> Slab:
    j0, j1 = partition(prob.ny, world)[rank]
    nplanes = prob.nz + 1 + (0 if prob.kf is None else 1)
    return Slab(rank, world, j0, j1, prob.nx, prob.ny, nplanes)


def sub_problem(prob, slab: Slab):
    """The slab's own problem: the sub-grid, its materials, constraints and
    per-pair in-situ tractions, and the loads of the nodes it owns (loads of a
    shared row are applied once, by its owner)."""
    nodes = slab.global_nodes()
    elems = slab.global_elements(prob.nz)
    own = slab.owned()
    N = (prob.nx + 1) * (prob.ny + 1) * slab.nplanes
    fixed = np.asarray(prob.fixed).reshape(4, N)[:, nodes].copy()
    fu = np.asarray(prob.fu, float).reshape(3, N)[:, nodes] * own[None, :]
    fp = np.asarray(prob.fp, float).reshape(N)[nodes] * own
    E = np.broadcast_to(np.asarray(prob.E, float), (prob.nx * prob.ny * prob.nz,))[elems].copy()
    k = np.broadcast_to(np.asarray(prob.k, float), (prob.nx * prob.ny * prob.nz,))[elems].copy()
    fault = prob.fault
    if fault is not None and (np.ndim(fault.tn0) > 0 or np.ndim(fault.tau0) > 1):
        pairs = slab.global_pairs()
        P = (prob.nx + 1) * (prob.ny + 1)
        tn0 = np.broadcast_to(np.asarray(fault.tn0, float), (P,))[pairs].copy()
        tau0 = np.broadcast_to(np.asarray(fault.tau0, float).reshape(-1, 2), (P, 2))[pairs].copy()
        fault = dataclasses.replace(fault, tn0=tn0, tau0=tau0)
    o = np.asarray(prob.origin, float)
    origin = (o[0], o[1] + slab.j0 * prob.h[1], o[2] + prob.shear[1] * slab.j0 * prob.h[1])
    return dataclasses.replace(prob, name=f"{prob.name}.slab{slab.rank}of{slab.world}", ny=slab.ny_local,
                               origin=origin, fault=fault, E=E, k=k, fixed=fixed, fu=fu, fp=fp)


class HaloExchanger:
    """Completes the shared node rows of a slab's operator products by adding
    the neighbour's partial sums (one row of every field and node plane per
    neighbour and exchange), and sums owned-node dot products over ranks."""

    def __init__(self, slab: Slab, dist, group=None):
        self.slab = slab
        self.dist = dist
        self.group = group
        self.down = slab.rank - 1 if slab.rank > 0 else None
        self.up = slab.rank + 1 if slab.rank < slab.world - 1 else None
        import torch
        self._own = torch.from_numpy(slab.owned())
        self.exchanges = 0

    def _rows(self, y, jl):
        s = self.slab
        return y.reshape(y.shape[0], s.nplanes, s.ny_local + 1, s.nx + 1)[:, :, jl, :]

    def complete(self, y):
        """y: (F, n_local) partial sums -> complete sums on every local node (in place)."""
        import torch
        s = self.slab
        F = y.shape[0]
        v = y.reshape(F, s.nplanes, s.ny_local + 1, s.nx + 1)
        ops, bufs = [], []
        if self.down is not None:
            send_d = v[:, :, 0, :].contiguous()
            recv_d = torch.empty_like(send_d)
            ops += [self.dist.P2POp(self.dist.isend, send_d, self.down, self.group),
                    self.dist.P2POp(self.dist.irecv, recv_d, self.down, self.group)]
            bufs.append((0, recv_d))
        if self.up is not None:
            send_u = v[:, :, s.ny_local, :].contiguous()
            recv_u = torch.empty_like(send_u)
            ops += [self.dist.P2POp(self.dist.isend, send_u, self.up, self.group),
                    self.dist.P2POp(self.dist.irecv, recv_u, self.up, self.group)]
            bufs.append((s.ny_local, recv_u))
        if ops:
            for req in self.dist.batch_isend_irecv(ops):
                req.wait()
            for jl, r in bufs:
                v[:, :, jl, :] += r
        self.exchanges += 1
        return y

    def dot(self, a, b) -> float:
        """sum over owned nodes of a * b (fields summed), in FP64, over all ranks."""
        import torch
        own = self._own.to(a.device)
        loc = (a.double() * b.double()).reshape(-1, self.slab.n_local)[:, own].sum().reshape(1)
        self.dist.all_reduce(loc, group=self.group)
        return float(loc.item())


@dataclasses.dataclass
class PartitionedOps:
    """The blocks of one Jacobian system (Eq. linear_system) on a slab:
    local products (partial sums) and local diagonals, and the free-dof masks."""
    apply_KT: Callable        # (3, n) -> (3, n) partial K_T x
    apply_Apu: Callable       # (n,) -> (3, n) partial A_pu x
    apply_Aup: Callable       # (3, n) -> (n,) partial A_up x
    apply_A22: Callable       # (n,) -> (n,) partial (S + dt C) x
    diag_KT: object           # (3, n) partial diagonal of K_T
    diag_A22: object          # (n,) partial diagonal of A22
    free_u: object            # (3, n) bool
    free_p: object            # (n,) bool


class PartitionedSystem:
    """Products and reductions of the partitioned Jacobian system; every
    product is completed by one halo exchange."""

    def __init__(self, ops: PartitionedOps, exch: HaloExchanger):
        self.ops = ops
        self.x = exch
        fu, fp = ops.free_u, ops.free_p
        dK = exch.complete(ops.diag_KT.clone())
        dA = exch.complete(ops.diag_A22.clone()[None])[0]
        self.inv_dK = (1.0 / dK.where(fu, dK.new_ones(()))) * fu
        self.inv_dA = (1.0 / dA.where(fp, dA.new_ones(()))) * fp

    def KT(self, x):
        return self.x.complete(self.ops.apply_KT(x * self.ops.free_u)) * self.ops.free_u

    def Apu(self, x):
        return self.x.complete(self.ops.apply_Apu(x * self.ops.free_p)) * self.ops.free_u

    def Aup(self, x):
        return self.x.complete(self.ops.apply_Aup(x * self.ops.free_u)[None])[0] * self.ops.free_p

    def A22(self, x):
        return self.x.complete(self.ops.apply_A22(x * self.ops.free_p)[None])[0] * self.ops.free_p

    def J(self, xu, xp):
        """[K_T  -A_pu; A_up  A22] [xu; xp] (Eq. linear_system)."""
        return self.KT(xu) - self.Apu(xp), self.Aup(xu) + self.A22(xp)

    def pcg(self, op, inv_diag, b, rtol, maxit):
        """Jacobi PCG from zero; returns (x, iterations)."""
        x = b.new_zeros(b.shape)
        r = b.clone()
        bb = self.x.dot(b, b)
        if bb == 0.0:
            return x, 0
        z = inv_diag * r
        p = z.clone()
        rz = self.x.dot(r, z)
        for it in range(1, maxit + 1):
            q = op(p)
            pq = self.x.dot(p, q)
            if not pq > 0.0:
                raise RuntimeError("partitioned PCG: loss of positive definiteness")
            a = rz / pq
            x += a * p
            r -= a * q
            if self.x.dot(r, r) <= rtol * rtol * bb:
                return x, it
            z = inv_diag * r
            rz_new = self.x.dot(r, z)
            p = z + (rz_new / rz) * p
            rz = rz_new
        raise RuntimeError("partitioned PCG: no convergence")

    def prevost(self, b1, b2, outer_rtol=1e-10, inner_rtol=1e-13, maxit=500, inner_maxit=20000):
        """Prevost's partitioned CG (Eqs. prevost_system, schur_system): CG on
        (A22 + A_up K_T^-1 A_pu) x2 = b2 - A_up K_T^-1 b1, preconditioned with
        A22^-1, then x1 = K_T^-1 (b1 + A_pu x2).  Inner solves by Jacobi PCG.
        Returns (x1, x2, outer iterations)."""
        solve_K = lambda v: self.pcg(self.KT, self.inv_dK, v, inner_rtol, inner_maxit)[0]
        solve_A = lambda v: self.pcg(self.A22, self.inv_dA, v, inner_rtol, inner_maxit)[0]
        schur = lambda v: self.A22(v) + self.Aup(solve_K(self.Apu(v)))
        r = b2 - self.Aup(solve_K(b1))
        x2 = r.new_zeros(r.shape)
        rr0 = self.x.dot(r, r)
        it = 0
        if rr0 > 0.0:
            z = solve_A(r)
            p = z.clone()
            rz = self.x.dot(r, z)
            for it in range(1, maxit + 1):
                q = schur(p)
                a = rz / self.x.dot(p, q)
                x2 += a * p
                r -= a * q
                if self.x.dot(r, r) <= outer_rtol * outer_rtol * rr0:
                    break
                z = solve_A(r)
                rz_new = self.x.dot(r, z)
                p = z + (rz_new / rz) * p
                rz = rz_new
            else:
                raise RuntimeError("partitioned Prevost CG: no convergence")
        x1 = solve_K(b1 + self.Apu(x2))
        return x1, x2, it
