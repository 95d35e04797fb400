"""Batched launch of many independent systems (soma_batch_*).

Every member must evolve exactly as the same system run alone: the batch runs
the same tile body with the same random-number counters, so positions,
occupation numbers and acceptance counts are compared bit for bit, before and
after the autotuner changes the launch shape.  One member is also checked
against the FP64 oracle for one cycle.
"""
import numpy as np
import pytest

from paper_1711_03828_gb300 import Batch, System, SystemDesc, workloads
from tests.conftest import oracle_system
from tests.test_gpu_parity import TIE, check_decisions

pytestmark = pytest.mark.gpu


def _small_batch(n=6):
    descs = []
    rng = np.random.default_rng(5)
    for i in range(n):
        L = int(rng.choice([1, 2]))
        N = int(rng.choice([16, 32, 64]))
        descs.append(SystemDesc(n_chains=max(1, 4096 * L**3 // N // 4) + i, N=N,
                                f=float(rng.choice([0.3, 0.5])), box_Re=(float(L),) * 3,
                                grid=(6 * L,) * 3, chiN=float(rng.uniform(10, 40)), kappaN=50.0,
                                seed=3, replica_id=i))
    return descs


def _compare(batch, singles):
    for m, s in zip(batch.members, singles):
        np.testing.assert_array_equal(m.get_positions(), s.get_positions())
        np.testing.assert_array_equal(m.get_density(), s.get_density())
        om, os_ = m.observables(), s.observables()
        assert om["accepted"] == os_["accepted"] and om["sweeps"] == os_["sweeps"]


def test_batch_members_match_single_systems(cuda_device):
    descs = _small_batch()
    b = Batch(descs)
    singles = [System(d) for d in descs]
    _compare(b, singles)
    b.sweep(3)                 # eager launches
    for s in singles:
        s.sweep(3)
    _compare(b, singles)
    b.sweep(16)                # one graph replay
    for s in singles:
        s.sweep(16)
    _compare(b, singles)
    # sweeping a lent member alone is refused
    from paper_1711_03828_gb300 import SomaError
    with pytest.raises(SomaError):
        b.members[0].sweep(1)
    b.close()


def test_batch_autotune_keeps_results(cuda_device):
    descs = _small_batch(4)
    b = Batch(descs)
    table = b.autotune(cycles_per_candidate=2)
    assert len(table) >= 3
    best = min(table, key=lambda t: t["ms_per_cycle"])
    sh = b.shape()
    assert (sh["block"], sh["blocks_per_sm"], sh["item_tiles"]) == \
        (best["block"], best["blocks_per_sm"], best["item_tiles"])
    cycles = b.members[0].observables()["sweeps"]
    singles = [System(d) for d in descs]
    for s in singles:
        s.sweep(int(cycles))
    _compare(b, singles)
    b.sweep(17)
    for s in singles:
        s.sweep(17)
    _compare(b, singles)
    b.close()


@pytest.mark.parametrize("shape", [(256, 3, 0), (128, 5, 0), (64, 1, 0), (256, 2, 16), (128, 4, 7)])
def test_batch_shapes_keep_results(cuda_device, shape):
    """Every launch shape covers every tile exactly once: the balanced split
    (item_tiles 0: one equal contiguous range of the members' tiles per block,
    cut at member boundaries; with fewer tiles than blocks some ranges are
    empty, with 64 x 1 per SM a range holds a few tiles and some cross a
    member boundary) and work items taken in turn, eager and replayed."""
    from paper_1711_03828_gb300 import SomaError
    descs = _small_batch(7)
    b = Batch(descs)
    b.set_shape(*shape)
    sh = b.shape()
    assert (sh["block"], sh["blocks_per_sm"], sh["item_tiles"]) == shape
    singles = [System(d) for d in descs]
    b.sweep(2)
    b.sweep(16)
    for s in singles:
        s.sweep(18)
    _compare(b, singles)
    for bad in [(100, 1, 0), (256, 0, 0), (256, 64, 0), (512, 1, 0), (256, 1, -1)]:
        with pytest.raises(SomaError):
            b.set_shape(*bad)
    assert b.shape() == sh
    b.close()


def test_batch_members_match_oracle(cuda_device):
    """The members' initial states are the oracle's (to one FP32 ulp); one
    batched cycle from those states matches the oracle's cycle per member."""
    from oracle import Positions
    descs = _small_batch(3)
    b = Batch(descs)
    before = []
    for k, d in enumerate(descs):
        orc = oracle_system(d)
        p = orc.initial_state()
        g0 = b.members[k].get_positions()
        ulp = np.spacing(np.abs(p.stacked()).astype(np.float32))
        assert np.all(np.abs(g0 - p.stacked()) <= ulp)
        n = b.members[k].get_density()
        pg = Positions(g0[0].copy(), g0[1].copy(), g0[2].copy())
        nA, nB = orc.histogram(pg)
        np.testing.assert_array_equal(n & 0xFFFF, nA)
        np.testing.assert_array_equal(n >> 16, nB)
        before.append((orc, pg, nA, nB))
    b.sweep(1)
    for k, (orc, p, nA, nB) in enumerate(before):
        wA, wB = orc.fields(nA, nB)
        old = p.copy()
        _, margin, acc = orc.sweep(p, wA, wB, 0, want_margin=True, want_acc=True)
        g = b.members[k].get_positions()
        gacc = np.any(g != old.stacked(), axis=0).astype(np.uint8)
        bad = np.nonzero(gacc != acc)[0]
        check_decisions(bad, margin, descs[k].N)
        if len(bad) == 0:
            np.testing.assert_array_equal(g, p.stacked())
    b.close()
