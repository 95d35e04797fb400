"""Mixtures of linear architectures (any A/B sequence per chain) on the GPU
against the FP64 oracle, through the C ABI: the SET sweep (even N), the
molecule-parallel iteration (odd N) and smart Monte Carlo moves (the mixture
run as linear architectures on the architecture path)."""
import numpy as np
import pytest

from paper_1711_03828_gb300 import (ITERATION_MOLECULE, MOVE_LEARNED, MOVE_SMC, SomaError,
                                    System, SystemDesc, _abi, workloads)
from tests.conftest import oracle_system
from tests.test_gpu_parity import TIE, Runner, _pos

pytestmark = pytest.mark.gpu


def _sequences(N):
    """Diblock, homopolymer A, homopolymer B, ABA triblock, alternating."""
    full = (1 << N) - 1
    third = N // 3
    return np.array([full & ~((1 << (N // 2)) - 1), 0, full,
                     ((1 << (2 * third)) - 1) & ~((1 << third) - 1), 0xAAAAAAAAAAAAAAAA & full],
                    np.uint64)


def test_mixture_set_sweeps_match_oracle(cuda_device):
    d = workloads.melt_small(chiN=30.0)
    seq = _sequences(d.N)
    arch = np.random.default_rng(4).integers(0, len(seq), d.n_chains).astype(np.uint8)
    r = Runner(d)
    r.gpu.set_architectures(seq, arch)
    r.gpu.update_fields()
    r.orc.set_architectures(seq, arch)
    r.nA, r.nB = r.orc.histogram(r.p)
    r.wA, r.wB = r.orc.fields(r.nA, r.nB)
    r.check_grid()
    live = True
    for _ in range(20):
        live = r.step(1)
        if not live:
            break
    if live:
        r.step(16)
    print(f"mixture (SET): {r.moves} moves, tolerated mismatches {r.mismatch}")
    assert r.moves >= 5 * d.M


def test_mixture_molecule_iteration_matches_oracle(cuda_device):
    d = SystemDesc(n_chains=1500, N=7, f=0.5, box_Re=(1.5, 1.5, 1.0), grid=(9, 9, 6),
                   chiN=25.0, kappaN=40.0, set_order=ITERATION_MOLECULE, seed=21)
    seq = _sequences(d.N)
    arch = np.random.default_rng(8).integers(0, len(seq), d.n_chains).astype(np.uint8)
    pos0 = workloads.random_walk_positions(d, seed=61)
    s = System(d)
    s.set_architectures(seq, arch)
    s.set_positions(pos0)
    s.update_fields()
    s.sweep(1)
    g = s.get_positions()
    n = s.get_density()
    s.close()
    orc = oracle_system(d)
    orc.set_architectures(seq, arch)
    p = _pos(pos0)
    nA, nB = orc.histogram(p)
    wA, wB = orc.fields(nA, nB)
    st, margin, acc, chosen = orc.sweep(p, wA, wB, 0, want_margin=True, want_acc=True,
                                        want_chosen=True)
    keep = ~(np.abs(margin.reshape(d.n_chains, d.N)) < TIE).any(axis=1)
    np.testing.assert_array_equal(g.reshape(3, d.n_chains, d.N)[:, keep],
                                  p.stacked().reshape(3, d.n_chains, d.N)[:, keep])
    gA, gB = orc.histogram(_pos(g))
    np.testing.assert_array_equal(n & 0xFFFF, gA)
    np.testing.assert_array_equal(n >> 16, gB)
    assert (~keep).sum() <= 3


def test_mixture_arguments_are_checked(cuda_device):
    d = workloads.melt_small(n_chains=64)
    s = System(d)
    seq = _sequences(d.N)
    bad = np.zeros(d.n_chains, np.uint8)
    bad[7] = len(seq)
    with pytest.raises(SomaError) as e:
        s.set_architectures(seq, bad)
    assert e.value.status == _abi.SOMA_EINVAL
    s.close()
    learned = System(workloads.melt_small(n_chains=64, move=MOVE_LEARNED))
    with pytest.raises(SomaError) as e:
        learned.set_architectures(seq, np.zeros(64, np.uint8))
    assert e.value.status == _abi.SOMA_EINVAL
    learned.close()


@pytest.mark.parametrize("N,n_chains,grid,box", [(32, 1024, (12, 12, 12), (2.0, 2.0, 2.0)),
                                                 (7, 1500, (9, 9, 6), (1.5, 1.5, 1.0))])
def test_mixture_smc_matches_oracle(cuda_device, N, n_chains, grid, box):
    """Smart Monte Carlo on a mixture (even and odd N): one cycle from each of
    three starts against the oracle's mixture path, with the tolerances of
    the SMC parity tests; the counts follow the sequences."""
    from tests.test_gpu_smc import compare_smc_cycle
    moves = mism = accepted = 0
    for k, sweep in enumerate((0, 5, 300)):
        d = SystemDesc(n_chains=n_chains, N=N, f=0.5, box_Re=box, grid=grid, chiN=30.0,
                       kappaN=50.0, move=MOVE_SMC, seed=31 + k)
        seq = _sequences(N)
        arch = np.random.default_rng(9 + k).integers(0, len(seq), d.n_chains).astype(np.uint8)
        s = System(d)
        s.set_architectures(seq, arch)
        orc = oracle_system(d)
        orc.set_architectures(seq, arch)
        m, b, a = compare_smc_cycle(d, s, orc, workloads.random_walk_positions(d, seed=71 + k),
                                    sweep)
        moves += m
        mism += b
        accepted += a
    print(f"SMC mixture N={N}: {moves} moves, acceptance {accepted / moves:.3f}, mismatches {mism}")
    assert mism <= max(3, 2e-4 * moves)
    assert 0.3 < accepted / moves < 0.999
