"""Smart Monte Carlo moves (Sec. 2.2, the force-biased proposal) on molecules
of any architecture (Sec. 3.2.1) and of n_t types, CUDA path against the FP64
oracle through the C ABI.

The trial position r + A F + sqrt(2A) xi is evaluated in FP32 on the GPU and
in FP64 in the oracle, so, as for linear chains, each check starts both sides
from the same seeded positions and compares ONE cycle:
  * occupation numbers: bit-exact (same positions);
  * decisions: equal, except near-ties (|ln u - ln alpha| < 1e-4 kT), moves
    whose oracle trial position lies within 4 ulps of a cell face, and the
    molecules of those (their partners move later in the sweep against a
    position that differs);
  * positions: in every other molecule rejected moves leave the position
    bit-identical and accepted ones agree with the oracle's trial position to
    1e-6 R_e0; absent slots never move.
"""
import numpy as np
import pytest

from paper_1711_03828_gb300 import MOVE_SMC, SET_ORDER_FIXED, System, workloads
from tests.conftest import oracle_system
from tests.test_gpu_parity import _pos
from tests.test_gpu_smc import TIE_SMC, _near_face, _tol
from tests.test_gpu_topology import CASES, _setup
from tests.test_gpu_types import CHI3, _molecules

pytestmark = pytest.mark.gpu


def _one_cycle(d, words, starts, arch, pos0, sweep, n_types=0, chi=None):
    orc = oracle_system(d)
    orc.set_topology(words, starts, arch)
    s = System(d)
    if n_types:
        orc.set_types(n_types, chi)
        s.set_types(n_types, chi)
    s.set_topology(words, starts, arch)
    s.set_positions(pos0)
    s.set_sweep(sweep)              # counts, fields and the SMC table of pos0
    p = _pos(pos0)
    if n_types:
        n = orc.histogram_types(p)
        np.testing.assert_array_equal(s.get_type_counts(), n)
        w = orc.fields_types(n)
        st, margin, acc, trial = orc.sweep(p, None, None, sweep, want_margin=True, want_acc=True,
                                           want_trial=True, w_types=w)
    else:
        nA, nB = orc.histogram(p)
        n = s.get_density()
        np.testing.assert_array_equal(n & 0xFFFF, nA)
        np.testing.assert_array_equal(n >> 16, nB)
        wA, wB = orc.fields(nA, nB)
        st, margin, acc, trial = orc.sweep(p, wA, wB, sweep, want_margin=True, want_acc=True,
                                           want_trial=True)
    s.sweep(1)
    g = s.get_positions()
    s.close()
    gacc = np.any(g != pos0, axis=0).astype(np.uint8)
    bad = np.nonzero(gacc != acc)[0]
    ok = set(bad[np.abs(margin[bad]) < TIE_SMC].tolist())
    face = _near_face(np.nan_to_num(trial))
    ok |= {int(m) for m in bad if face[m]}
    ok_mol = {m // d.N for m in ok}
    for m in bad.tolist():
        if m not in ok:
            assert m // d.N in ok_mol, (m, margin[m])
    keep = np.ones(d.n_chains, bool)
    keep[np.unique(bad // d.N)] = False
    keep = np.repeat(keep, d.N)
    rej = keep & (acc == 0)
    np.testing.assert_array_equal(g[:, rej], pos0[:, rej])
    accd = keep & (acc == 1)
    err = np.abs(g[:, accd].astype(np.float64) - trial[:, accd]) / _tol(trial[:, accd])
    assert err.max(initial=0) <= 1.0, err.max()
    attempted = int(np.isfinite(margin).sum())
    return attempted, len(bad), int(acc.sum())


@pytest.mark.parametrize("name,set_order", [(n, 0) for n in CASES] +
                         [("N9_odd_ring_star", SET_ORDER_FIXED)])
def test_topology_smc_one_cycle_matches_oracle(cuda_device, name, set_order):
    moves = mism = accepted = 0
    for k, sweep in enumerate((0, 1, 17, 1000)):
        d, mols, arch, words, starts, pos0 = _setup(name, set_order, seed=5 + k, move=MOVE_SMC)
        m, b, a = _one_cycle(d, words, starts, arch, pos0, sweep)
        moves += m
        mism += b
        accepted += a
    print(f"SMC {name} set_order={set_order}: {moves} moves, acceptance {accepted / moves:.3f}, "
          f"mismatches {mism}")
    assert mism <= max(3, 2e-4 * moves)
    assert 0.3 < accepted / moves < 0.999


@pytest.mark.parametrize("hamiltonian", [0, 1])
def test_types_smc_one_cycle_matches_oracle(cuda_device, hamiltonian):
    """Three types: field and field force from the plane of each particle's
    type (the table has one plane per type)."""
    from paper_1711_03828_gb300 import SystemDesc
    mols = _molecules(3)
    words, starts = workloads.encode_architectures(mols)
    moves = mism = accepted = 0
    for k, sweep in enumerate((0, 3, 250)):
        d = SystemDesc(n_chains=2048, N=16, f=0.5, box_Re=(2.0, 2.0, 2.0), grid=(12, 12, 12),
                       chiN=20.0, kappaN=50.0, seed=5 + k, hamiltonian=hamiltonian, move=MOVE_SMC)
        arch = np.random.default_rng(5 + k).integers(0, len(mols), d.n_chains).astype(np.uint8)
        pos0 = workloads.architecture_positions(d, mols, arch, seed=105 + k)
        m, b, a = _one_cycle(d, words, starts, arch, pos0, sweep, 3, CHI3)
        moves += m
        mism += b
        accepted += a
    print(f"SMC three types K{hamiltonian}: {moves} moves, acceptance {accepted / moves:.3f}, "
          f"mismatches {mism}")
    assert mism <= max(3, 2e-4 * moves)
    assert 0.3 < accepted / moves < 0.999


def test_topology_smc_graph_replay_is_identical(cuda_device):
    """soma_sweep(32) replays the captured cycle graph (sweep, fields, table);
    32 single cycles give the same positions bit for bit."""
    d, mols, arch, words, starts, pos0 = _setup("N9_odd_ring_star", move=MOVE_SMC)
    out = []
    for chunked in (True, False):
        s = System(d)
        s.set_topology(words, starts, arch)
        s.set_positions(pos0)
        s.update_fields()
        if chunked:
            s.sweep(32)
        else:
            for _ in range(32):
                s.sweep(1)
        out.append(s.get_positions())
        s.close()
    np.testing.assert_array_equal(out[0], out[1])


def test_ideal_star_and_ring_statistics_smc(cuda_device):
    """chiN = kappaN = 0 under SMC: <|r_i - r_j|^2> = d_ij b0^2 on a star and
    b0^2 d (N - d)/N on a ring (the closed forms of Gaussian trees and rings;
    the bonded force and energy follow the listed bonds)."""
    from tests.test_gpu_topology import check_ideal_closed_forms
    check_ideal_closed_forms(move=MOVE_SMC)
