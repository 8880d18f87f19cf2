"""The multi-rank path of bench.py on CPU: world size 2 over gloo (no GPU, no kernels).

Each rank of a weak-scaling run takes a batch of the same channel widths with its own draw
of (M, Ca, theta); rank 0 reports the maximum of the ranks' timed regions and the fluid
nodes of all ranks.
"""
import os
import socket

import numpy as np
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, ws, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        import bench
        (geoms, prms), _ = bench.workload("batched_sweep", rank=rank, lattices=6)
        nf = bench.fluid_nodes(geoms)
        ms_max, nf_total = bench.reduce_over_ranks(10.0 + rank, nf, ws, "cpu")
        out[rank] = (nf, ms_max, nf_total, tuple((p.nu_B, p.sigma, p.theta) for p in prms),
                     tuple(g.nx for g in geoms))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_weak_scaling_reduction():
    ws = 2
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank_main, args=(ws, port, out), nprocs=ws, join=True)
        res = dict(out)
    nf0, ms0, tot0, par0, nx0 = res[0]
    nf1, ms1, tot1, par1, nx1 = res[1]
    assert nx0 == nx1 and nf0 == nf1            # equal work per rank
    assert par0 != par1                          # independent parameter draws
    assert ms0 == ms1 == 11.0                    # max over ranks
    assert tot0 == tot1 == nf0 + nf1             # all ranks' nodes


def test_single_rank_reduction_is_the_identity():
    import bench
    assert bench.reduce_over_ranks(7.5, 1234, 1, "cpu") == (7.5, 1234)
