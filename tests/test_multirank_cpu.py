"""Sharded SCMF cycle on CPU ranks (gloo, world size 2).

The method shards by whole chains with one exchange per cycle: every rank
moves its own chains against the shared fields, counts its particles, and
one all-reduce (sum) of the packed occupation grid (A | B<<16) gives every
rank the full counts, from which each computes the fields (Sec. 3.1.1).  Each
rank runs the oracle on its chain range; after three cycles the positions of
each shard and the all-reduced counts must equal the monolithic run bit for
bit (chains are independent under frozen fields, integer addition is
associative, and the random-number counters are global particle indices).
"""
import os
import socket

import numpy as np
import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _desc():
    from paper_1711_03828_gb300 import workloads
    return workloads.melt_small(n_chains=512, chiN=25.0)


def _rank_main(rank, world, port, out_dir):
    import torch
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from oracle import Positions
    from tests.conftest import oracle_system
    d = _desc()
    full = oracle_system(d)
    p = full.initial_state()
    per = d.n_chains // world
    c0, c1 = rank * per, (rank + 1) * per
    shard_desc = type(d)(**{**d.__dict__, "n_chains": per})
    shard = oracle_system(shard_desc)

    def shard_counts():
        sl = slice(c0 * d.N, c1 * d.N)
        sp = Positions(p.x[sl].copy(), p.y[sl].copy(), p.z[sl].copy())
        nA, nB = shard.histogram(sp)
        packed = nA.astype(np.int64) | (nB.astype(np.int64) << 16)
        t = torch.from_numpy(packed)
        dist.all_reduce(t, op=dist.ReduceOp.SUM)
        n = t.numpy()
        return (n & 0xFFFF).astype(np.uint32), (n >> 16).astype(np.uint32)

    nA, nB = shard_counts()
    for sweep in range(3):
        wA, wB = full.fields(nA, nB)
        full.sweep(p, wA, wB, sweep, c0=c0, c1=c1)   # only this rank's chains
        nA, nB = shard_counts()
    sl = slice(c0 * d.N, c1 * d.N)
    np.save(os.path.join(out_dir, f"pos{rank}.npy"), np.stack([p.x[sl], p.y[sl], p.z[sl]]))
    np.save(os.path.join(out_dir, f"n{rank}.npy"), np.stack([nA, nB]))
    dist.barrier()
    dist.destroy_process_group()


def test_sharded_cycle_equals_monolithic(oracle_lib, tmp_path):
    import torch.multiprocessing as mp
    world = 2
    mp.start_processes(_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world,
                       join=True, start_method="spawn")
    from tests.conftest import oracle_system
    d = _desc()
    full = oracle_system(d)
    p = full.initial_state()
    nA, nB = full.histogram(p)
    for sweep in range(3):
        wA, wB = full.fields(nA, nB)
        full.sweep(p, wA, wB, sweep)
        nA, nB = full.histogram(p)
    per = d.n_chains // world
    for r in range(world):
        pos = np.load(tmp_path / f"pos{r}.npy")
        sl = slice(r * per * d.N, (r + 1) * per * d.N)
        np.testing.assert_array_equal(pos, np.stack([p.x[sl], p.y[sl], p.z[sl]]))
        n = np.load(tmp_path / f"n{r}.npy")
        np.testing.assert_array_equal(n[0], nA)
        np.testing.assert_array_equal(n[1], nB)
