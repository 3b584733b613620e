"""Slab decomposition on CPU ranks (gloo): the partitioned Jacobian product
equals the single-domain one, and Prevost's partitioned CG over 2 and 3 slabs
solves the single-domain system.  Each rank's local operator is the oracle's
assembly on its slab (its own elements and fault quads only), so the partial
sums on the shared node rows and the halved tributary areas of the fault pairs
there are exactly what a rank's GPU context computes; the halo exchange and
the all-reduced dot products are the decomposition under test."""
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp

CASES = {
    # tied lip pressures, box cells, seeded materials
    "box_tied": dict(nx=4, ny=7, nz=4, seed=11),
    # double-node pressures on an x-z sheared grid (the inclined-fault class)
    "sheared_untied": dict(nx=3, ny=8, nz=4, seed=12, shear=(1.7320508075688772, 0.0), k_perp=1e-13),
}


def _problem(name):
    import workloads as W
    kw = dict(CASES[name])
    p = W.tiny_faulted(kw.pop("nx"), kw.pop("ny"), kw.pop("nz"), Q=2e-4, **kw)
    # a load on a node of the row shared by the first two slabs of a 2-way cut
    N = p.n_nodes
    j = p.ny // 2
    node = 1 + (p.nx + 1) * (j + (p.ny + 1) * (p.n_planes - 1))
    p.fu = np.asarray(p.fu, float).reshape(3, N)
    p.fu[2, node] = -3e5
    return p


def _run(rank, world, name):
    import workloads as W
    from oracle import fem, solve as osolve
    from paper_2410_17133_gb300 import slab as S

    dt = 1.7
    prob = _problem(name)
    model = fem.Model(prob)
    N = model.N
    u = W.random_vectors(N, 5, scale_u=1e-5)[0] + W.random_displacement_jump(prob, 6, scale=5e-6)
    st = osolve.initial_state(model)
    r, _, Kcoh = osolve.fault_terms(model, u.reshape(-1), st.dlie)
    states = set(r["state"].tolist())
    xu, xp = W.random_vectors(N, 7)
    yu, yp = osolve.apply(model, "J", xu.reshape(-1), xp, dt=dt, Kcoh=Kcoh)
    bu, bp = W.random_vectors(N, 8, scale_u=1e3, scale_p=1e-9)
    b1 = np.where(model.free_u, bu.reshape(-1), 0.0)
    b2 = np.where(model.free_p, bp, 0.0)
    KT, Apu, A22 = osolve.jacobian_blocks(model, Kcoh, dt)
    x1f, x2f = osolve.solve_monolithic(KT, Apu, A22, b1[model.free_u], b2[model.free_p], dense=False)
    x1 = np.zeros(3 * N); x1[model.free_u] = x1f
    x2 = np.zeros(N); x2[model.free_p] = x2f

    sl = S.make_slab(prob, rank, world)
    sub = S.sub_problem(prob, sl)
    ml = fem.Model(sub)
    gn = sl.global_nodes()
    n = sl.n_local
    assert ml.N == n
    _, _, Kl = osolve.fault_terms(ml, u.reshape(3, N)[:, gn].reshape(-1), osolve.initial_state(ml).dlie)
    KTl = (ml.Kb + Kl).tocsr()
    Apul = ml.Apu.tocsr()
    A22l = ml.A22(dt)
    T = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64))
    ops = S.PartitionedOps(
        apply_KT=lambda x: T(KTl @ x.numpy().reshape(-1)).reshape(3, n),
        apply_Apu=lambda x: T(Apul @ x.numpy()).reshape(3, n),
        apply_Aup=lambda x: T(Apul.T @ x.numpy().reshape(-1)),
        apply_A22=lambda x: T(A22l @ x.numpy()),
        diag_KT=T(KTl.diagonal()).reshape(3, n), diag_A22=T(A22l.diagonal()),
        free_u=torch.from_numpy(ml.free_u.reshape(3, n)), free_p=torch.from_numpy(ml.free_p))
    ex = S.HaloExchanger(sl, dist)
    sysm = S.PartitionedSystem(ops, ex)

    ju, jp = sysm.J(T(xu[:, gn]), T(xp[gn]))
    ref_u, ref_p = yu.reshape(3, N)[:, gn], yp[gn]
    e_apply = max(np.linalg.norm(ju.numpy() - ref_u) / np.linalg.norm(ref_u),
                  np.linalg.norm(jp.numpy() - ref_p) / np.linalg.norm(ref_p))
    # the loads of the sub-problems add up to the global loads (shared rows once)
    fsum = torch.tensor([float(np.asarray(sub.fu).sum()), float(np.asarray(sub.fp).sum())], dtype=torch.float64)
    dist.all_reduce(fsum)
    loads_ok = np.allclose(fsum.numpy(), [np.asarray(prob.fu).sum(), np.asarray(prob.fp).sum()], rtol=1e-14, atol=0)
    # the owned nodes of all ranks partition the global nodes
    cnt = torch.zeros(N, dtype=torch.float64)
    cnt[torch.from_numpy(gn[sl.owned()])] = 1.0
    dist.all_reduce(cnt)
    partition_ok = bool(torch.all(cnt == 1.0))

    s1, s2, its = sysm.prevost(T(b1.reshape(3, N)[:, gn]), T(b2[gn]), outer_rtol=1e-12, inner_rtol=1e-14)
    r1, r2 = x1.reshape(3, N)[:, gn], x2[gn]
    e_solve = max(np.linalg.norm(s1.numpy() - r1) / np.linalg.norm(x1), np.linalg.norm(s2.numpy() - r2) / np.linalg.norm(x2))
    return dict(e_apply=e_apply, e_solve=e_solve, its=its, loads_ok=loads_ok, partition_ok=partition_ok,
                states=sorted(states), exchanges=ex.exchanges, pairs=int(ml.fg["pairs"].shape[0]))


def _worker(rank, world, port, name, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        q.put((rank, _run(rank, world, name)))
    except Exception as e:          # report instead of hanging the other ranks' queue reads
        import traceback
        q.put((rank, "error: " + repr(e) + "\n" + traceback.format_exc()))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
@pytest.mark.parametrize("name", list(CASES))
def test_partitioned_apply_and_prevost_match_single_domain(name, world):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29600 + (os.getpid() * 7 + 13 * world + len(name)) % 2000
    procs = [ctx.Process(target=_worker, args=(r, world, port, name, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = dict(q.get(timeout=600) for _ in range(world))
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    for rank in range(world):
        res = out[rank]
        assert isinstance(res, dict), res
        assert res["e_apply"] < 1e-14, (rank, res)
        assert res["e_solve"] < 1e-8, (rank, res)
        assert res["loads_ok"] and res["partition_ok"], (rank, res)
        assert res["pairs"] > 0
        assert len(res["states"]) >= 2         # the lip jumps put pairs in more than one state
    its = {out[r]["its"] for r in range(world)}
    assert len(its) == 1                        # every rank ran the same iterations


def test_partition_is_balanced_and_covers_the_rows():
    from paper_2410_17133_gb300 import slab as S
    for ny, world in ((7, 2), (8, 3), (160, 8), (5, 5)):
        parts = S.partition(ny, world)
        assert parts[0][0] == 0 and parts[-1][1] == ny
        assert all(a[1] == b[0] for a, b in zip(parts, parts[1:]))
        sizes = [b - a for a, b in parts]
        assert min(sizes) >= 1 and max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        S.partition(2, 3)
