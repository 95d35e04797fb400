"""Interaction option K^1 and the external fields of Sec. 4 (a potential per
type and cell, cells no particle may enter) on the GPU against the FP64
oracle, through the C ABI."""
import numpy as np
import pytest

from paper_1711_03828_gb300 import Batch, System, SystemDesc, workloads
from tests.conftest import oracle_system
from tests.test_gpu_parity import Runner, _fields_tol, _pos

pytestmark = pytest.mark.gpu


def _external(d, seed):
    """A linear attraction of A to the x = 0 face (the potential falls off
    linearly over three cells), a weak random potential for B, and a wall:
    the plane of cells at z = 0."""
    nx, ny, nz = d.grid
    cx = np.arange(d.cells) % nx
    cz = np.arange(d.cells) // (nx * ny)
    ext = np.zeros((2, d.cells), np.float32)
    ext[0] = np.where(cx < 3, -0.4 * (3 - cx) / 3.0, 0.0)
    ext[1] = np.random.default_rng(seed).uniform(-0.1, 0.1, d.cells)
    forbidden = (cz == 0).astype(np.uint8)
    return ext, forbidden


def _check_fields(r, forbidden):
    gA, gB = r.gpu.get_fields()
    closed = forbidden != 0
    tol = np.broadcast_to(_fields_tol(r.d, r.nA, r.nB, r.orc.params.rho_cell), closed.shape)
    tol = tol[~closed] + 4 * 2.0**-24 * 0.4
    assert np.all(np.isinf(gA[closed])) and np.all(np.isinf(gB[closed]))
    assert np.all(np.abs(gA[~closed] - r.wA[~closed]) <= tol)
    assert np.all(np.abs(gB[~closed] - r.wB[~closed]) <= tol)


@pytest.mark.parametrize("hamiltonian", [0, 1])
def test_external_fields_and_k1_cycles_match_oracle(cuda_device, hamiltonian):
    d = workloads.melt_small(hamiltonian=hamiltonian, chiN=25.0)
    ext, forbidden = _external(d, 3)
    r = Runner(d)
    r.gpu.set_external(ext, forbidden)
    r.gpu.update_fields()
    r.orc.set_external(ext.astype(np.float64), forbidden)
    r.wA, r.wB = r.orc.fields(r.nA, r.nB)
    _check_fields(r, forbidden)
    o = r.gpu.observables()
    ref = r.orc.observables(r.p, r.nA, r.nB)
    for k in ("E_nb", "E_ext", "E_tot"):
        assert o[k] == pytest.approx(ref[k], rel=1e-9, abs=1e-9), k
    for _ in range(12):
        if not _step(r, forbidden):
            break
    print(f"K{hamiltonian} with external fields: {r.moves} moves, tolerated mismatches {r.mismatch}")
    assert r.moves >= 6 * d.M


@pytest.mark.parametrize("hamiltonian", [0, 1])
def test_external_potential_smc_matches_oracle(cuda_device, hamiltonian):
    """Smart Monte Carlo in an external potential (no closed cells: their
    infinite fields have no gradient): the field force includes the
    potential's central difference; one cycle from each of three starts
    against the oracle with the SMC tolerances."""
    from paper_1711_03828_gb300 import MOVE_SMC
    from tests.test_gpu_smc import compare_smc_cycle
    moves = mism = 0
    for k, sweep in enumerate((0, 7, 500)):
        d = workloads.melt_small(hamiltonian=hamiltonian, chiN=25.0, move=MOVE_SMC, seed=41 + k)
        ext, _ = _external(d, 5 + k)
        s = System(d)
        s.set_external(ext, None)
        orc = oracle_system(d)
        orc.set_external(ext.astype(np.float64), None)
        m, b, _ = compare_smc_cycle(d, s, orc, workloads.random_walk_positions(d, seed=81 + k),
                                    sweep)
        moves += m
        mism += b
    print(f"SMC K{hamiltonian} with an external potential: {moves} moves, mismatches {mism}")
    assert mism <= max(3, 2e-4 * moves)


def _step(r, forbidden):
    """One cycle in both; positions compared as in Runner.step, the grid with
    the infinite walls taken into account."""
    old = r.p.copy()
    st, margin, acc = r.orc.sweep(r.p, r.wA, r.wB, r.sweep, want_margin=True, want_acc=True)
    r.sweep += 1
    r.gpu.sweep(1)
    g = r.gpu.get_positions()
    gacc = ((g[0] != old.x) | (g[1] != old.y) | (g[2] != old.z)).astype(np.uint8)
    bad = np.nonzero(gacc != acc)[0]
    r.moves += r.d.M
    if len(bad):
        from tests.test_gpu_parity import check_decisions
        check_decisions(bad, margin, r.d.N)
        r.mismatch += len(bad)
        return False
    np.testing.assert_array_equal(g, r.p.stacked())
    r.nA, r.nB = r.orc.histogram(r.p)
    r.wA, r.wB = r.orc.fields(r.nA, r.nB)
    n = r.gpu.get_density()
    np.testing.assert_array_equal(n & 0xFFFF, r.nA)
    np.testing.assert_array_equal(n >> 16, r.nB)
    _check_fields(r, forbidden)
    return True


def test_walls_are_never_entered(cuda_device):
    """A slab of closed cells through a melt: particles that start inside may
    only leave (they cannot move within the wall, where both energies are
    infinite), and no particle enters, over 200 cycles."""
    d = workloads.melt_small(n_chains=512, chiN=10.0)
    _, forbidden = _external(d, 1)
    forbidden |= ((np.arange(d.cells) // d.grid[0]) % d.grid[1] == 5).astype(np.uint8)
    s = System(d)
    s.set_external(None, forbidden)
    s.update_fields()
    nx, ny = d.grid[0], d.grid[1]

    def inside(P):
        c = np.floor(P.astype(np.float64)).astype(np.int64) % np.asarray(d.grid)[:, None]
        return forbidden[(c[2] * ny + c[1]) * nx + c[0]] != 0

    P = s.get_positions()
    was = inside(P)
    start = int(was.sum())
    for _ in range(200):
        s.sweep(1)
        Q = s.get_positions()
        now = inside(Q)
        assert not (now & ~was).any()
        np.testing.assert_array_equal(Q[:, now], P[:, now])
        P, was = Q, now
    print(f"walls: {start} particles inside at the start, {int(was.sum())} after 200 cycles")
    assert int(was.sum()) < max(1, start // 4)
    s.close()


def test_k1_batch_members_match_single_systems(cuda_device):
    descs = [workloads.melt_small(n_chains=256, hamiltonian=1, replica_id=k, chiN=15.0 + 5 * k)
             for k in range(3)]
    b = Batch(descs)
    b.sweep(20)
    got = [b.members[k].get_positions() for k in range(3)]
    b.close()
    for k, d in enumerate(descs):
        s = System(d)
        s.sweep(20)
        np.testing.assert_array_equal(s.get_positions(), got[k])
        s.close()
