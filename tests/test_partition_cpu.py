"""Domain decomposition on the CPU: the partition plan of gks_partition_create (host code of the
library) with its halo moved by torch.distributed point-to-point messages between gloo ranks
(world size 2), the residual and one two-stage step of each rank's cells computed by the FP64
oracle from the rank's own columns only. Columns outside a rank's owned and halo cells are NaN,
so a halo that misses a cell the residual reads poisons that rank's result; the test requires
the decomposed residual and step to equal the one-rank ones bit for bit.
"""
import os
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CASES = [  # (cubes, layers, bc, min_stencil, params)
    (8, "hybrid8", (0, 0, 0), 0, dict(flux_mode=1, tau_model=2, mu=1e-3)),
    (8, "hybrid8", (1, 1, 1), 18, dict(flux_mode=1, tau_model=1)),
]


def _rank(rank, world, port, case, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    sys.path.insert(0, ROOT)
    import oracle
    import paper_2203_09047_gb300 as gks
    from paper_2203_09047_gb300 import inputs as I
    from paper_2203_09047_gb300.partition import Partition, global_min_dt, halo_exchange
    n, layers, bc, ms, kw = CASES[case]
    lo, hi = ((0, 0, 0), (2, 2, 2)) if bc[0] == 0 else ((-1, -1, -1), (1, 1, 1))
    m = I.layered_box_mesh(n, layers, lo=lo, hi=hi, bc=bc)
    part = Partition(gks.Mesh(m, min_stencil=ms), world, rank)
    om = oracle.Mesh(m, lazy=True, min_stencil=ms)
    P = oracle.params_vec(**kw)
    base = oracle.Mesh(m).advection_average() if bc[0] == 0 else \
        np.tile(np.array([[0.8], [0.05], [-0.02], [0.03], [1.1 / 0.4]]), (1, om.n_cells))
    Qf = I.perturbed_state(base, seed=81, amp=0.02)  # the same on every rank
    own, halo = part.owned, part.halo
    # this rank's columns only
    Q = torch.full(Qf.shape, float("nan"), dtype=torch.float64)
    Q[:, own] = torch.from_numpy(Qf[:, own])
    halo_exchange(Q, part, dist)
    res = {"halo_ok": bool(torch.equal(Q[:, halo], torch.from_numpy(Qf[:, halo])))}
    dt = 0.004
    L, Lt = om.residual_cells(P, Q.numpy(), dt, own)
    Lr, Ltr = om.residual_cells(P, Qf, dt, own)
    res["residual_bitwise"] = bool(np.array_equal(L, Lr) and np.array_equal(Lt, Ltr))
    # one two-stage step (Section 3.3): stage 1 on the owned cells, halo exchange of Q*, stage 2
    def stages(Qa, Lx, Ltx, Ltsx):
        return oracle.s2o4(Qa, Lx, Ltx, Ltsx, dt)
    Qs_own, _ = stages(Qf[:, own], L.T, Lt.T, np.zeros_like(Lt.T))
    Qs = torch.full(Qf.shape, float("nan"), dtype=torch.float64)
    Qs[:, own] = torch.from_numpy(Qs_own)
    halo_exchange(Qs, part, dist)
    _, Lts = om.residual_cells(P, Qs.numpy(), dt, own)
    _, Qn_own = stages(Qf[:, own], L.T, Lt.T, Lts.T)
    # the same step on the whole state, restricted to this rank's cells
    allc = np.arange(om.n_cells)
    La, Lta = om.residual_cells(P, Qf, dt, allc)
    Qs_all, _ = stages(Qf, La.T, Lta.T, np.zeros_like(Lta.T))
    _, Ltsa = om.residual_cells(P, Qs_all, dt, allc)
    _, Qn_all = stages(Qf, La.T, Lta.T, Ltsa.T)
    res["step_bitwise"] = bool(np.array_equal(Qn_own, Qn_all[:, own]))
    # the time step is the minimum of the ranks' bounds
    res["dt"] = global_min_dt(0.01 + 0.001 * rank, dist)
    res["n_owned"], res["n_halo"] = len(own), len(halo)
    out[rank] = res
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("case", range(len(CASES)))
def test_two_rank_residual_and_step_equal_one_rank_bitwise(case):
    world, port = 2, 29541 + case
    with mp.Manager() as man:
        out = man.dict()
        mp.spawn(_rank, args=(world, port, case, out), nprocs=world, join=True)
        res = dict(out)
    n_cells = sum(res[r]["n_owned"] for r in range(world))
    assert n_cells == 4 * CASES[case][0] ** 3
    for r in range(world):
        assert res[r]["halo_ok"] and res[r]["residual_bitwise"] and res[r]["step_bitwise"], res[r]
        assert res[r]["dt"] == 0.01
        assert 0 < res[r]["n_halo"] < n_cells - res[r]["n_owned"]


def test_partition_plan_is_consistent():
    """Owned sets are disjoint and cover the mesh, sizes differ by at most one cell, and what a
    rank sends a peer is exactly that peer's halo entries owned by the rank, in order."""
    sys.path.insert(0, ROOT)
    import paper_2203_09047_gb300 as gks
    from paper_2203_09047_gb300 import inputs as I
    from paper_2203_09047_gb300.partition import Partition
    m = I.layered_box_mesh(8, "hybrid8")
    M = gks.Mesh(m)
    for world in (1, 3, 4):
        parts = [Partition(M, world, r) for r in range(world)]
        owned = np.concatenate([p.owned for p in parts])
        assert np.array_equal(np.sort(owned), np.arange(2048))
        sizes = [len(p.owned) for p in parts]
        assert max(sizes) - min(sizes) <= 1
        for p in parts:
            assert not np.isin(p.halo, p.owned).any()
            for q in range(world):
                if q != p.rank:
                    assert np.array_equal(parts[q].send[p.rank], p.recv[q])
        if world == 1:
            assert len(parts[0].halo) == 0
    with pytest.raises(gks.GksError):
        Partition(M, 2, 2)
