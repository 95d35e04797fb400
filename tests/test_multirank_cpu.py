"""Sharded SCMF cycle on CPU ranks (gloo, world size 2).

The method shards by whole chains with one exchange per cycle: every rank
moves its own chains against the shared fields, counts its particles, and
one all-reduce (sum) of the packed occupation grid (A | B<<16) gives every
rank the full counts, from which each computes the fields (Sec. 3.1.1).

Each rank drives its shard through ``paper_1711_03828_gb300.shard.ShardedRun``
-- the driver ``bench.py --gpus N`` runs over NCCL -- with a stand-in shard
that has the library's three ``shard_*`` calls but computes with the oracle on
the rank's chain range.  After three cycles the positions of each shard and
the all-reduced counts must equal the monolithic run bit for bit (chains are
independent under frozen fields, integer addition is associative, and the
random-number counters are global particle indices).  A third rank count
(three ranks on 512 chains) leaves shards of unequal size.  The same holds
for molecules of several architectures under smart Monte Carlo moves (each
rank holding its molecules' architecture bytes).
"""
import os
import socket

import numpy as np
import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _desc(case="diblock"):
    from paper_1711_03828_gb300 import SystemDesc, workloads
    if case == "diblock":
        return workloads.melt_small(n_chains=512, chiN=25.0)
    return SystemDesc(n_chains=600, N=16, f=0.5, box_Re=(2.0, 2.0, 1.0), grid=(12, 12, 6),
                      chiN=25.0, kappaN=50.0, move=1, seed=5)


def _setup(case, orc, c0, c1):
    """The molecules' architectures of chains [c0, c1) for the architecture case."""
    if case == "diblock":
        return
    from paper_1711_03828_gb300 import workloads
    mols = [workloads.star_architecture(3, 5), workloads.ring_architecture(16),
            workloads.comb_architecture(8, 4, 2), workloads.linear_architecture(16)]
    words, starts = workloads.encode_architectures(mols)
    arch = np.random.default_rng(3).integers(0, len(mols), 600).astype(np.uint8)
    orc.set_topology(words, starts, arch[c0:c1])


class OracleShard:
    """The oracle behind the shard calls of ``System``: chains [c0, c1) of the
    whole system's positions move, their counts are packed A | B<<16."""

    def __init__(self, d, c0, c1, case="diblock"):
        from tests.conftest import oracle_system
        self.d, self.c0, self.c1 = d, c0, c1
        self.full = oracle_system(d)
        _setup(case, self.full, 0, d.n_chains)
        self.p = self.full.initial_state()
        self.own = oracle_system(type(d)(**{**d.__dict__, "n_chains": c1 - c0}))
        _setup(case, self.own, c0, c1)
        self.sweep_no = 0
        self.wA = self.wB = None

    def _counts(self, buf):
        from oracle import Positions
        sl = slice(self.c0 * self.d.N, self.c1 * self.d.N)
        nA, nB = self.own.histogram(Positions(self.p.x[sl].copy(), self.p.y[sl].copy(),
                                              self.p.z[sl].copy()))
        packed = (nA.astype(np.uint32) | (nB.astype(np.uint32) << 16)).view(np.int32)
        buf.copy_(__import__("torch").from_numpy(packed))

    def shard_counts(self, buf):
        self._counts(buf)

    def shard_sweep(self, buf):
        self.full.sweep(self.p, self.wA, self.wB, self.sweep_no, c0=self.c0, c1=self.c1)
        self.sweep_no += 1
        self._counts(buf)

    def shard_fields(self, summed):
        n = summed.numpy().view(np.uint32)
        self.nA, self.nB = n & 0xFFFF, n >> 16
        self.wA, self.wB = self.full.fields(self.nA, self.nB)


def _rank_main(rank, world, port, out_dir, case="diblock"):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from paper_1711_03828_gb300.shard import ShardedRun, shard_desc
    d = _desc(case)
    sd = shard_desc(d, world, rank)
    shard = OracleShard(d, sd.chain_offset, sd.chain_offset + sd.n_chains, case)
    run = ShardedRun(shard, d.cells, "cpu")
    run.start()
    run.cycle(3)
    sl = slice(shard.c0 * d.N, shard.c1 * d.N)
    np.save(os.path.join(out_dir, f"pos{rank}.npy"),
            np.stack([shard.p.x[sl], shard.p.y[sl], shard.p.z[sl]]))
    np.save(os.path.join(out_dir, f"n{rank}.npy"), np.stack([shard.nA, shard.nB]))
    np.save(os.path.join(out_dir, f"range{rank}.npy"), np.array([shard.c0, shard.c1]))
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("world,case", [(2, "diblock"), (3, "diblock"), (2, "architectures_smc")])
def test_sharded_cycle_equals_monolithic(oracle_lib, tmp_path, world, case):
    import torch.multiprocessing as mp
    mp.start_processes(_rank_main, args=(world, _free_port(), str(tmp_path), case), nprocs=world,
                       join=True, start_method="spawn")
    from tests.conftest import oracle_system
    d = _desc(case)
    full = oracle_system(d)
    _setup(case, full, 0, d.n_chains)
    p = full.initial_state()
    nA, nB = full.histogram(p)
    for sweep in range(3):
        wA, wB = full.fields(nA, nB)
        full.sweep(p, wA, wB, sweep)
        nA, nB = full.histogram(p)
    covered = 0
    for r in range(world):
        c0, c1 = np.load(tmp_path / f"range{r}.npy")
        assert c0 == covered
        covered = c1
        pos = np.load(tmp_path / f"pos{r}.npy")
        sl = slice(c0 * d.N, c1 * d.N)
        np.testing.assert_array_equal(pos, np.stack([p.x[sl], p.y[sl], p.z[sl]]))
        n = np.load(tmp_path / f"n{r}.npy")
        np.testing.assert_array_equal(n[0], nA)
        np.testing.assert_array_equal(n[1], nB)
    assert covered == d.n_chains


def test_shard_ranges_cover_the_chains_once():
    from paper_1711_03828_gb300 import workloads
    from paper_1711_03828_gb300.shard import shard_desc, shard_range
    for total in (1, 7, 512, 4_194_304, 4_194_305):
        for world in (1, 2, 3, 8):
            if total < world:
                continue
            spans = [shard_range(total, world, r) for r in range(world)]
            assert spans[0][0] == 0
            for (o0, c0), (o1, _) in zip(spans, spans[1:]):
                assert o0 + c0 == o1
            assert spans[-1][0] + spans[-1][1] == total
            assert max(c for _, c in spans) - min(c for _, c in spans) <= 1
    d = workloads.melt_small(n_chains=10)
    s = shard_desc(d, 3, 2)
    assert (s.chain_offset, s.n_chains, s.n_chains_total) == (7, 3, 10)
    with pytest.raises(ValueError):
        shard_desc(s, 2, 0)
    with pytest.raises(ValueError):
        shard_range(10, 2, 2)
