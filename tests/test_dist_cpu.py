"""Multi-rank host logic on CPU (gloo, world size 2; no GPU).

One horizon split across two ranks: each rank computes the VJP of its own
interval range (here with the oracle, standing in for a GPU), the ranks combine
the gradient row of the node they share with dist.merge_cut_rows, and the
result must equal the VJP of the unsplit horizon.  Also: balanced instance
ranges and the max-over-ranks timing reduction.
"""
import os
import socket

import numpy as np
import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import torch
    import torch.distributed as dist

    import oracle
    from paper_2604_09993_gb300 import dist as pdist
    from paper_2604_09993_gb300 import synth
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        p = synth.hopper_fp64(seed=3, N=11, n_sub=3)
        R = p.robot.as_dict()
        k0, k1 = pdist.interval_ranges(p.N, world)[rank]
        gX, gU, gs, L = oracle.vjp(R, p.X[k0:k1 + 1], p.U[k0:k1 + 1], p.s[k0:k1], p.w[k0:k1],
                                   p.rho[k0:k1], p.n_sub, threads=1)
        gXo, gUo, Lt = pdist.merge_cut_rows(torch.tensor(gX), torch.tensor(gU),
                                            torch.tensor(L, dtype=torch.float64))
        t = pdist.max_over_ranks([0.5 + rank, 3.0 - rank])
        rows = [None] * world
        dist.all_gather_object(rows, (k0, k1, gXo.numpy(), gUo.numpy(), gs, float(Lt), t))
        if rank == 0:
            q.put(rows)
    finally:
        dist.destroy_process_group()


@pytest.mark.timeout(300)
def test_split_horizon_vjp_matches_unsplit():
    import torch.multiprocessing as mp

    import oracle
    from paper_2604_09993_gb300 import synth
    oracle.build()
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for pr in procs:
        pr.start()
    rows = q.get(timeout=240)
    for pr in procs:
        pr.join(timeout=60)
        assert pr.exitcode == 0
    p = synth.hopper_fp64(seed=3, N=11, n_sub=3)
    gX, gU, gs, L = oracle.vjp(p.robot.as_dict(), p.X, p.U, p.s, p.w, p.rho, p.n_sub, threads=1)
    gXm = np.concatenate([r[2] for r in rows])
    gUm = np.concatenate([r[3] for r in rows])
    gsm = np.concatenate([r[4] for r in rows])
    assert gXm.shape == gX.shape and gUm.shape == gU.shape
    assert np.allclose(gXm, gX, rtol=0, atol=1e-12 * max(1, np.abs(gX).max()))
    assert np.allclose(gUm, gU, rtol=0, atol=1e-12 * max(1, np.abs(gU).max()))
    assert np.allclose(gsm, gs, rtol=0, atol=1e-12 * max(1, np.abs(gs).max()))
    assert abs(rows[0][5] - L) <= 1e-12 * max(1.0, abs(L))
    assert rows[0][6] == [1.5, 3.0] and rows[1][6] == [1.5, 3.0]


def test_interval_and_instance_ranges():
    from paper_2604_09993_gb300 import dist as pdist
    assert pdist.interval_ranges(10, 3) == [(0, 4), (4, 7), (7, 10)]
    with pytest.raises(ValueError):
        pdist.interval_ranges(2, 3)
    costs = [1, 1, 1, 1, 10, 1, 1, 1]
    parts = [pdist.instance_range(costs, r, 2) for r in range(2)]
    assert parts[0][0] == 0 and parts[-1][1] == len(costs)
    assert parts[0][1] == parts[1][0]
    # every instance is covered exactly once
    cover = sum((list(range(a, b)) for a, b in parts), [])
    assert cover == list(range(len(costs)))
