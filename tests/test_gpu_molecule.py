"""Molecule-parallel iteration (Sec. 3.1.2, first scheme) on the GPU against
the FP64 oracle, through the C ABI.

One cycle from the same positions and fields: every chain in which no attempt
came within 1e-4 kT of its acceptance threshold (the oracle's margin
|dE + ln u|) ends bit-equal to the oracle's chain (the trial positions round
identically on both sides); the other chains are counted and must be rare.
The occupation numbers the kernel counts equal the histogram of its own final
positions.  Sizes cover staged chains (N <= 64, several blocks, a ragged last
block), odd N and long chains read in place (N > 64).
"""
import math

import numpy as np
import pytest

from paper_1711_03828_gb300 import ITERATION_MOLECULE, System, SystemDesc, workloads
from tests.conftest import oracle_system
from tests.test_gpu_parity import TIE, _pos

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("N,n_chains,grid,box", [
    (32, 1000, (12, 12, 12), (2.0, 2.0, 2.0)),     # staged, 8 blocks, ragged last block
    (7, 1500, (9, 9, 6), (1.5, 1.5, 1.0)),         # odd N, staged
    (2, 300, (4, 4, 4), (1.0, 1.0, 1.0)),          # dimers
    (100, 40, (8, 8, 8), (1.0, 1.0, 1.0)),         # read in place (N > 64)
    (256, 9, (6, 6, 6), (1.0, 1.0, 1.0)),          # longest chains
])
def test_molecule_cycle_matches_oracle(cuda_device, N, n_chains, grid, box):
    d = SystemDesc(n_chains=n_chains, N=N, f=0.5, box_Re=box, grid=grid, chiN=25.0,
                   kappaN=40.0, set_order=ITERATION_MOLECULE, seed=19)
    attempts = tied_chains = 0
    for k, sweep in enumerate((0, 5, 1000)):
        pos0 = workloads.random_walk_positions(d, seed=500 + k)
        s = System(d)
        s.set_positions(pos0)
        s.set_sweep(sweep)
        s.update_fields()
        s.sweep(1)
        g = s.get_positions()
        n = s.get_density()
        s.close()
        orc = oracle_system(d)
        p = _pos(pos0)
        nA, nB = orc.histogram(p)
        wA, wB = orc.fields(nA, nB)
        st, margin, acc, chosen = orc.sweep(p, wA, wB, sweep, want_margin=True, want_acc=True,
                                            want_chosen=True)
        assert st.attempted == d.M
        near = np.abs(margin.reshape(n_chains, N)) < TIE
        keep = ~near.any(axis=1)
        ref = p.stacked().reshape(3, n_chains, N)
        G = g.reshape(3, n_chains, N)
        np.testing.assert_array_equal(G[:, keep, :], ref[:, keep, :])
        # the fused count is the histogram of the kernel's own final positions
        gA, gB = orc.histogram(_pos(g))
        np.testing.assert_array_equal(n & 0xFFFF, gA)
        np.testing.assert_array_equal(n >> 16, gB)
        attempts += d.M
        tied_chains += int((~keep).sum())
    print(f"molecule N={N}: {attempts} attempts, chains with a near-tie {tied_chains}")
    assert tied_chains <= max(2, 2e-3 * (attempts // N))


def test_molecule_two_particle_balance_brute_force(cuda_device):
    """Dimers with chiN = kappaN = 0 on a periodic 2^3 grid: the visited cell
    pairs follow the exact distribution (erf quadrature)."""
    from tests.test_gpu_learned import _pair_probabilities
    L, Re = 2, 1.5
    d = SystemDesc(n_chains=16384, N=2, f=0.5, box_Re=(L / Re,) * 3, grid=(L,) * 3, chiN=0.0,
                   kappaN=0.0, set_order=ITERATION_MOLECULE, seed=29)
    s = System(d)
    s.sweep(100)
    T = 400
    counts = np.zeros((d.n_chains, L**6))
    for _ in range(T):
        s.sweep(1)
        P = s.get_positions().reshape(3, d.n_chains, 2).astype(np.float64)
        c = np.floor(P).astype(np.int64) % L
        ci = (c[2] * L + c[1]) * L + c[0]
        counts[np.arange(d.n_chains), ci[:, 0] * L**3 + ci[:, 1]] += 1
    s.close()
    K = 3.0 / (2 * Re * Re)
    Pex = _pair_probabilities(K, L).reshape(-1)
    freq = counts / T
    est = freq.mean(0)
    se = freq.std(0) / math.sqrt(d.n_chains)
    z = (est - Pex) / np.maximum(se, 1e-12)
    print(f"molecule iteration: max |z| {np.max(np.abs(z)):.2f}")
    assert np.max(np.abs(z)) < 5.0
