"""Chain sharding on one GPU (Sec. 3.1.1: molecules distributed over ranks,
one sum of the occupation numbers per cycle).

Shards of a system -- handles whose description carries chain_offset and
n_chains_total -- are driven through the library's exchange calls
(soma_shard_counts, soma_shard_sweep, soma_shard_fields) with their count
buffers summed on the device between the calls, the exchange an all-reduce
over ranks performs.  They run one after another on one stream (no kernel
waits on another), from the positions of a handle holding the whole system,
which runs beside them.  Every cycle the shards' positions, taken together,
must equal the whole system's bit for bit, and so must the summed counts and
every shard's occupation numbers; the accepted moves add up.  The whole
system's cycles are compared with the oracle elsewhere; one shard cycle is
compared with the oracle here as well.
"""
import numpy as np
import pytest
import torch

from paper_1711_03828_gb300 import (ITERATION_MOLECULE, MOVE_LEARNED, MOVE_SMC, SET_ORDER_FIXED,
                                    SomaError, System, SystemDesc, _abi, workloads)
from paper_1711_03828_gb300.shard import ShardedRun, shard_desc
from tests.conftest import oracle_system
from tests.test_gpu_parity import _pos, check_decisions

pytestmark = pytest.mark.gpu


@pytest.fixture
def on_stream(cuda_device):
    """A stream of its own, current for torch during the test: the handles
    run on it (a NULL stream would give each handle a private stream that
    torch's operations are not ordered with)."""
    st = torch.cuda.Stream()
    with torch.cuda.stream(st):
        yield st
    st.synchronize()


def _arch_setup(d):
    mols = [workloads.star_architecture(3, 5), workloads.ring_architecture(16),
            workloads.comb_architecture(8, 4, 2), workloads.linear_architecture(16)]
    words, starts = workloads.encode_architectures(mols)
    arch = np.random.default_rng(3).integers(0, len(mols), d.n_chains).astype(np.uint8)

    def setup(s, c0, c1):
        s.set_topology(words, starts, arch[c0:c1])
    return setup


def _learned_setup(d):
    W = workloads.random_mlp(5, scale=0.2).astype(np.float32)

    def setup(s, c0, c1):
        s.set_proposal_weights(W)
    return setup


CASES = {
    "uniform_pair": (SystemDesc(n_chains=1001, N=32, box_Re=(2.0, 2.0, 2.0), grid=(12, 12, 12),
                                chiN=25.0, seed=3), None, 2),
    "uniform_three_shards": (SystemDesc(n_chains=1001, N=32, box_Re=(2.0, 2.0, 2.0),
                                        grid=(12, 12, 12), chiN=25.0, seed=3), None, 3),
    "uniform_any_N": (SystemDesc(n_chains=1500, N=7, box_Re=(1.5, 1.5, 1.0), grid=(9, 9, 6),
                                 chiN=20.0, seed=5, set_order=SET_ORDER_FIXED), None, 2),
    "smc": (SystemDesc(n_chains=1000, N=32, box_Re=(2.0, 2.0, 2.0), grid=(12, 12, 12),
                       chiN=25.0, move=MOVE_SMC, seed=7), None, 2),
    "learned": (SystemDesc(n_chains=1000, N=16, box_Re=(2.0, 2.0, 1.0), grid=(12, 12, 6),
                           chiN=25.0, move=MOVE_LEARNED, seed=9), _learned_setup, 2),
    "molecule_parallel": (SystemDesc(n_chains=999, N=32, box_Re=(2.0, 2.0, 2.0),
                                     grid=(12, 12, 12), chiN=25.0, seed=11,
                                     set_order=ITERATION_MOLECULE), None, 2),
    "architectures": (SystemDesc(n_chains=2000, N=16, box_Re=(2.0, 2.0, 1.0), grid=(12, 12, 6),
                                 chiN=25.0, seed=13), _arch_setup, 2),
    "architectures_smc": (SystemDesc(n_chains=2000, N=16, box_Re=(2.0, 2.0, 1.0),
                                     grid=(12, 12, 6), chiN=25.0, move=MOVE_SMC, seed=15),
                          _arch_setup, 2),
}


def _shards_from_whole(d, world, setup_factory):
    st = torch.cuda.current_stream()
    assert st.cuda_stream != 0
    setup = setup_factory(d) if setup_factory else None
    whole = System(d, stream=st)
    if setup:
        setup(whole, 0, d.n_chains)
        whole.update_fields()
    pos = whole.get_positions()
    shards = []
    for r in range(world):
        sd = shard_desc(d, world, r)
        s = System(sd, stream=st)
        c0, c1 = sd.chain_offset, sd.chain_offset + sd.n_chains
        if setup:
            setup(s, c0, c1)
        s.set_positions(np.ascontiguousarray(pos[:, c0 * d.N:c1 * d.N]))
        shards.append(s)
    return whole, shards


def _exchange(shards, call, cells):
    bufs = [torch.zeros(cells, dtype=torch.int32, device="cuda") for _ in shards]
    for s, b in zip(shards, bufs):
        call(s, b)
    tot = bufs[0].clone()
    for b in bufs[1:]:
        tot += b                     # the packed halves add as 32-bit integers
    for s in shards:
        s.shard_fields(tot)
    return tot


@pytest.mark.parametrize("case", list(CASES))
def test_shards_equal_the_whole_system_bit_for_bit(on_stream, case):
    d, setup_factory, world = CASES[case]
    whole, shards = _shards_from_whole(d, world, setup_factory)
    _exchange(shards, lambda s, b: s.shard_counts(b), d.cells)
    n_whole = whole.get_density()
    for s in shards:
        np.testing.assert_array_equal(s.get_density(), n_whole)
    for cycle in range(6):
        tot = _exchange(shards, lambda s, b: s.shard_sweep(b), d.cells)
        whole.sweep(1)
        g = whole.get_positions()
        parts = np.concatenate([s.get_positions() for s in shards], axis=1)
        assert np.array_equal(parts, g), f"cycle {cycle}: positions differ"
        n_whole = whole.get_density()
        np.testing.assert_array_equal(tot.cpu().numpy().view(np.uint32), n_whole)
        for s in shards:
            np.testing.assert_array_equal(s.get_density(), n_whole)
    ow = whole.observables()
    os_ = [s.observables() for s in shards]
    assert sum(o["accepted"] for o in os_) == ow["accepted"]
    assert all(o["sweeps"] == ow["sweeps"] for o in os_)
    assert sum(o["E_b"] for o in os_) == pytest.approx(ow["E_b"], rel=1e-9)
    assert all(o["E_nb"] == pytest.approx(ow["E_nb"], rel=1e-12) for o in os_)
    print(f"{case}: {world} shards, 6 cycles bit-identical, accepted {ow['accepted']}")
    for s in shards:
        s.close()
    whole.close()


def test_sharded_run_one_cycle_matches_oracle(on_stream):
    """Two shards driven by ShardedRun (the summing done by a device add in
    place of the all-reduce) against the oracle's whole-system cycle from the
    same positions: counts bit-exact, decisions equal except at near-ties,
    positions bit-equal where the decisions agree."""
    d = workloads.melt_small(n_chains=1024, chiN=25.0)
    world = 2
    pos0 = workloads.random_walk_positions(d, seed=41)
    st = torch.cuda.current_stream()
    shards = []
    for r in range(world):
        sd = shard_desc(d, world, r)
        s = System(sd, stream=st)
        s.set_positions(np.ascontiguousarray(
            pos0[:, sd.chain_offset * d.N:(sd.chain_offset + sd.n_chains) * d.N]))
        shards.append(s)

    class Pair:                       # both shards behind one set of shard calls
        def __init__(self):
            self.bufs = [torch.zeros(d.cells, dtype=torch.int32, device="cuda") for _ in shards]

        def _sum(self, call, buf):
            for s, b in zip(shards, self.bufs):
                call(s, b)
            buf.copy_(self.bufs[0] + self.bufs[1])

        def shard_counts(self, buf):
            self._sum(lambda s, b: s.shard_counts(b), buf)

        def shard_sweep(self, buf):
            self._sum(lambda s, b: s.shard_sweep(b), buf)

        def shard_fields(self, buf):
            for s in shards:
                s.shard_fields(buf)

    run = ShardedRun(Pair(), d.cells, "cuda", allreduce=lambda t: None)
    run.start()
    orc = oracle_system(d)
    p = _pos(pos0)
    nA, nB = orc.histogram(p)
    n = shards[0].get_density()
    np.testing.assert_array_equal(n & 0xFFFF, nA)
    np.testing.assert_array_equal(n >> 16, nB)
    wA, wB = orc.fields(nA, nB)
    _, margin, acc = orc.sweep(p, wA, wB, 0, want_margin=True, want_acc=True)
    run.cycle(1)
    g = np.concatenate([s.get_positions() for s in shards], axis=1)
    gacc = np.any(g != pos0, axis=0).astype(np.uint8)
    bad = np.nonzero(gacc != acc)[0]
    ties = check_decisions(bad, margin, d.N)
    keep = np.ones(d.M, bool)
    keep[np.repeat(np.isin(np.arange(d.n_chains), np.unique(bad // d.N)), d.N)] = False
    np.testing.assert_array_equal(g[:, keep], p.stacked()[:, keep])
    nA, nB = orc.histogram(p)
    n = shards[1].get_density()
    if len(bad) == 0:
        np.testing.assert_array_equal(n & 0xFFFF, nA)
        np.testing.assert_array_equal(n >> 16, nB)
    print(f"sharded cycle vs oracle: {d.M} moves, mismatches {len(bad)} ({ties} near-ties)")
    for s in shards:
        s.close()


def test_shard_calls_are_refused_out_of_order(on_stream):
    d = workloads.melt_small(n_chains=64)
    sd = shard_desc(d, 2, 1)
    s = System(sd, stream=torch.cuda.current_stream())
    buf = torch.zeros(d.cells, dtype=torch.int32, device="cuda")
    for call in (lambda: s.sweep(1), lambda: s.update_fields(), lambda: s.shard_fields(buf)):
        with pytest.raises(SomaError) as e:
            call()
        assert e.value.status == _abi.SOMA_ESTATE
    with pytest.raises(SomaError) as e:
        s.set_types(3, np.zeros((3, 3)))
    assert e.value.status == _abi.SOMA_ESTATE
    s.shard_sweep(buf)
    with pytest.raises(SomaError) as e:
        s.shard_counts(buf)           # a fields call must come first
    assert e.value.status == _abi.SOMA_ESTATE
    s.shard_fields(buf)
    with pytest.raises(SomaError) as e:
        _abi.soma_shard_sweep(s.h, buf.data_ptr(), d.cells - 1)
    assert e.value.status == _abi.SOMA_EINVAL
    whole = System(d, stream=torch.cuda.current_stream())
    with pytest.raises(SomaError) as e:
        whole.shard_sweep(buf)        # not a shard
    assert e.value.status == _abi.SOMA_ESTATE
    # molecules of fewer than N particles: a shard's density counts the whole system
    mols = [workloads.linear_architecture(d.N), workloads.linear_architecture(d.N // 2, 0)]
    words, starts = workloads.encode_architectures(mols)
    with pytest.raises(SomaError) as e:
        s.set_topology(words, starts, np.arange(sd.n_chains, dtype=np.uint8) % 2)
    assert e.value.status == _abi.SOMA_EINVAL
    s.set_topology(words, starts, np.zeros(sd.n_chains, np.uint8))   # all of N: taken
    s.close()
    whole.close()
