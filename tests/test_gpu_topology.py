"""Molecules of any architecture (the architecture array of Sec. 3.2.1, the
independent sets of Sec. 3.1.2) on the GPU against the FP64 oracle, through
the C ABI: stars, combs, rings (odd rings need three sets), chains with
next-nearest bonds (triangles, three sets) and linear chains mixed in one
system."""
import math

import numpy as np
import pytest

from paper_1711_03828_gb300 import (ITERATION_MOLECULE, MOVE_LEARNED, SomaError, System,
                                    SystemDesc, _abi, workloads)
from tests.conftest import oracle_system
from tests.test_gpu_parity import TIE, _fields_tol, _pos

pytestmark = pytest.mark.gpu


def _triangles(N):
    """Linear chain with next-nearest bonds i - (i+2): triangles, three sets."""
    types = [0 if i < N // 2 else 1 for i in range(N)]
    bonds = [(i, i + 1) for i in range(N - 1)] + [(i, i + 2) for i in range(N - 2)]
    return types, bonds


CASES = {
    "N16_star_comb_ring_linear": (
        dict(n_chains=2048, N=16, box_Re=(2.0, 2.0, 2.0), grid=(12, 12, 12)),
        [workloads.star_architecture(3, 5), workloads.comb_architecture(8, 4, 2),
         workloads.ring_architecture(16), workloads.linear_architecture(16)]),
    "N9_odd_ring_star": (
        dict(n_chains=3000, N=9, box_Re=(1.5, 1.5, 1.0), grid=(9, 9, 6)),
        [workloads.ring_architecture(9), workloads.star_architecture(4, 2),
         workloads.linear_architecture(9)]),
    "N64_star_triangles_ring": (
        dict(n_chains=512, N=64, box_Re=(2.0, 2.0, 1.0), grid=(12, 12, 6)),
        [workloads.star_architecture(7, 9), _triangles(64), workloads.ring_architecture(64)]),
    "N5_ring_star": (
        dict(n_chains=6000, N=5, box_Re=(1.0, 1.0, 1.0), grid=(6, 6, 6)),
        [workloads.ring_architecture(5), workloads.star_architecture(4, 1)]),
    # molecules of several lengths in slots of N (the rest of a molecule's
    # slots absent): a diblock of 16, a B homopolymer of 8, a star of 10, a
    # ring of 12 and A monomers
    "N16_blend_lengths": (
        dict(n_chains=2400, N=16, box_Re=(2.0, 2.0, 2.0), grid=(12, 12, 12)),
        [workloads.linear_architecture(16), workloads.linear_architecture(8, 0),
         workloads.star_architecture(3, 3), workloads.ring_architecture(12), ([0], [])]),
    # a homopolymer blend of lengths 32 (A) and 11 (B)
    "N32_homopolymer_blend": (
        dict(n_chains=1500, N=32, box_Re=(2.0, 2.0, 2.0), grid=(12, 12, 12)),
        [workloads.linear_architecture(32, 32), workloads.linear_architecture(11, 0)]),
}


def _setup(name, set_order=0, seed=5, **over):
    kw, mols = CASES[name]
    kw = dict(kw, f=0.5, chiN=30.0, kappaN=50.0, seed=seed, set_order=set_order)
    kw.update(over)
    d = SystemDesc(**kw)
    arch = np.random.default_rng(seed).integers(0, len(mols), d.n_chains).astype(np.uint8)
    words, starts = workloads.encode_architectures(mols)
    pos0 = workloads.architecture_positions(d, mols, arch, seed=seed + 100)
    return d, mols, arch, words, starts, pos0


def _check_decisions(bad, margin, N):
    """Mismatched decisions only at near-ties and, downstream of a tie, in the
    same molecule (its partners move later in the sweep against a different
    position)."""
    bad = np.asarray(bad)
    tied = bad[np.abs(margin[bad]) < TIE]
    tied_mol = set((tied // N).tolist())
    for m in bad[np.abs(margin[bad]) >= TIE].tolist():
        assert m // N in tied_mol, (m, margin[m])


def _cycles(d, gpu, orc, p, n):
    """n cycles on both sides from the same state; returns (moves compared,
    tolerated mismatches, oracle acceptances)."""
    nA, nB = orc.histogram(p)
    wA, wB = orc.fields(nA, nB)
    moves = mism = acc_tot = 0
    for sweep in range(n):
        n_gpu = gpu.get_density()
        np.testing.assert_array_equal(n_gpu & 0xFFFF, nA)
        np.testing.assert_array_equal(n_gpu >> 16, nB)
        gA, gB = gpu.get_fields()
        tol = _fields_tol(d, nA, nB, orc.params.rho_cell)
        assert np.all(np.abs(gA - wA) <= tol) and np.all(np.abs(gB - wB) <= tol)
        old = p.copy()
        st, margin, acc = orc.sweep(p, wA, wB, sweep, want_margin=True, want_acc=True)
        gpu.sweep(1)
        g = gpu.get_positions()
        gacc = ((g[0] != old.x) | (g[1] != old.y) | (g[2] != old.z)).astype(np.uint8)
        bad = np.nonzero(gacc != acc)[0]
        moves += d.M
        acc_tot += int(acc.sum())
        if len(bad):
            _check_decisions(bad, margin, d.N)
            mism += len(bad)
            keep = np.ones(d.n_chains, bool)
            keep[np.unique(bad // d.N)] = False
            keep = np.repeat(keep, d.N)
            np.testing.assert_array_equal(g[:, keep], p.stacked()[:, keep])
            break
        np.testing.assert_array_equal(g, p.stacked())
        nA, nB = orc.histogram(p)
        wA, wB = orc.fields(nA, nB)
    return moves, mism, acc_tot


@pytest.mark.parametrize("name,set_order", [(n, 0) for n in CASES] +
                         [("N16_star_comb_ring_linear", 1), ("N9_odd_ring_star", 1)])
def test_topology_cycles_match_oracle(cuda_device, name, set_order):
    d, mols, arch, words, starts, pos0 = _setup(name, set_order)
    gpu = System(d)
    gpu.set_topology(words, starts, arch)
    gpu.set_positions(pos0)
    gpu.update_fields()
    orc = oracle_system(d)
    orc.set_topology(words, starts, arch)
    moves, mism, acc_tot = _cycles(d, gpu, orc, _pos(pos0), 12)
    o = gpu.observables()
    gpu.close()
    print(f"{name} set_order={set_order}: {moves} moves, acceptance {acc_tot / moves:.3f}, "
          f"tolerated mismatches {mism}")
    assert moves >= 6 * d.M
    assert 0.2 < acc_tot / moves < 0.95
    assert o["sweeps"] == moves // d.M


def test_sort_molecules_relabels_like_the_oracle(cuda_device):
    """soma_sort_molecules gives the oracle's spatial labelling of the same
    positions, the architectures follow their molecules (cycles after the sort
    match the oracle run with the permuted architectures), and the counts do
    not change."""
    d, mols, arch, words, starts, pos0 = _setup("N16_star_comb_ring_linear")
    gpu = System(d)
    gpu.set_topology(words, starts, arch)
    gpu.set_positions(pos0)
    gpu.update_fields()
    n0 = gpu.get_density()
    perm = gpu.sort_molecules()
    np.testing.assert_array_equal(gpu.get_density(), n0)
    orc = oracle_system(d)
    p = _pos(pos0)
    operm = orc.sort_chains(p)
    np.testing.assert_array_equal(perm, operm)
    np.testing.assert_array_equal(gpu.get_positions(), p.stacked())
    assert sorted(perm.tolist()) == list(range(d.n_chains))
    orc.set_topology(words, starts, arch[perm.astype(np.int64)])
    moves, mism, _ = _cycles(d, gpu, orc, p, 6)
    gpu.close()
    assert moves >= 3 * d.M


@pytest.mark.parametrize("name", ["N16_star_comb_ring_linear", "N9_odd_ring_star",
                                  "N64_star_triangles_ring", "N16_blend_lengths"])
def test_topology_molecule_iteration_matches_oracle(cuda_device, name):
    """The molecule-parallel iteration (N attempts per molecule on random
    particles) with molecules of any architecture: one cycle per start,
    decisions and positions against the oracle, counts bit-exact."""
    moves = mism = 0
    for k in range(3):
        d, mols, arch, words, starts, pos0 = _setup(name, ITERATION_MOLECULE, seed=5 + k)
        s = System(d)
        s.set_topology(words, starts, arch)
        s.set_positions(pos0)
        s.update_fields()
        s.sweep(1)
        g = s.get_positions()
        n = s.get_density()
        s.close()
        orc = oracle_system(d)
        orc.set_topology(words, starts, arch)
        p = _pos(pos0)
        nA, nB = orc.histogram(p)
        wA, wB = orc.fields(nA, nB)
        st, margin, acc, chosen = orc.sweep(p, wA, wB, 0, want_margin=True, want_acc=True,
                                            want_chosen=True)
        # attempts are indexed by molecule * N + j; a molecule with a near-tie
        # attempt may diverge after it
        tied = (np.abs(margin.reshape(d.n_chains, d.N)) < TIE).any(axis=1)
        G = g.reshape(3, d.n_chains, d.N)
        P = p.stacked().reshape(3, d.n_chains, d.N)
        np.testing.assert_array_equal(G[:, ~tied], P[:, ~tied])
        gA, gB = orc.histogram(_pos(g))
        np.testing.assert_array_equal(n & 0xFFFF, gA)
        np.testing.assert_array_equal(n >> 16, gB)
        moves += d.M
        mism += int((G != P).any(axis=0).any(axis=1).sum())
        assert 0.2 < st.accepted / st.attempted < 0.95
    print(f"{name}, molecule-parallel: {moves} attempts, molecules with a tolerated tie {mism}")
    assert mism <= 3


@pytest.mark.parametrize("name", ["N16_star_comb_ring_linear", "N16_blend_lengths"])
def test_topology_observables_match_oracle(cuda_device, name):
    """FP64 observables and S(q) against the oracle; with molecules of several
    lengths also the density (rho_0 dL^3 of the present particles), R_e^2 to
    each molecule's own last particle and the attempted moves."""
    d, mols, arch, words, starts, pos0 = _setup(name)
    gpu = System(d)
    gpu.set_topology(words, starts, arch)
    gpu.set_positions(pos0)
    gpu.update_fields()
    o = gpu.observables()
    m = [(1, 0, 0), (0, 1, 2), (3, 2, 1), (5, 5, 5)]
    sq = gpu.structure_factor(m)
    par = gpu.parameters()
    orc = oracle_system(d)
    orc.set_topology(words, starts, arch)
    p = _pos(pos0)
    nA, nB = orc.histogram(p)
    ref = orc.observables(p, nA, nB)
    for k in ("E_b", "E_nb", "Re2", "b2", "E_tot"):
        assert o[k] == pytest.approx(ref[k], rel=1e-9), k
    np.testing.assert_allclose(sq, orc.structure_factor(nA, nB, m), rtol=1e-9)
    assert par["rho_cell"] == pytest.approx(orc.params.rho_cell, rel=1e-15)
    present = int(np.array([len(t) for t, _ in mols])[arch].sum())
    gpu.sweep(2)
    assert gpu.observables()["attempted"] == 2 * present
    gpu.close()


def test_topology_graph_replay_is_identical(cuda_device):
    """soma_sweep(32) replays the captured cycle graph; 32 single cycles give
    the same positions bit for bit."""
    d, mols, arch, words, starts, pos0 = _setup("N9_odd_ring_star")
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


def check_ideal_closed_forms(move=0):
    """chiN = kappaN = 0: <|r_i - r_j|^2> = d_ij b0^2 on a star (graph distance
    d_ij) and b0^2 d (N - d)/N on an odd ring (three sets), b0^2 = R_e0^2/(N-1),
    over 16384 molecules and 1500 cycles of the given move."""
    Re = 6.0
    for mol in (workloads.star_architecture(3, 5), workloads.ring_architecture(15)):
        N = len(mol[0])
        d = SystemDesc(n_chains=16384, N=N, f=0.5, box_Re=(4.0, 4.0, 2.0), grid=(24, 24, 12),
                       chiN=0.0, kappaN=0.0, seed=9, move=move)
        words, starts = workloads.encode_architectures([mol])
        arch = np.zeros(d.n_chains, np.uint8)
        s = System(d)
        s.set_topology(words, starts, arch)
        s.set_positions(workloads.architecture_positions(d, [mol], arch, seed=4))
        s.update_fields()
        s.sweep(500)
        acc = np.zeros((d.n_chains, N, N))
        k = 0
        for _ in range(50):
            s.sweep(20)
            P = s.get_positions().astype(np.float64).reshape(3, d.n_chains, N)
            acc += ((P[:, :, :, None] - P[:, :, None, :]) ** 2).sum(0)
            k += 1
        s.close()
        r2 = acc / k
        D = np.full((N, N), 10**6)
        np.fill_diagonal(D, 0)
        for i, j in mol[1]:
            D[i, j] = D[j, i] = 1
        for m in range(N):
            D = np.minimum(D, D[:, m:m + 1] + D[m:m + 1, :])
        b02 = Re**2 / (N - 1)
        ring = len(mol[1]) == N
        for dist in range(1, int(D.max()) + 1):
            per_mol = r2[:, np.triu(D == dist, 1)].mean(axis=1)
            want = b02 * dist * (N - dist) / N if ring else dist * b02
            se = per_mol.std() / math.sqrt(len(per_mol))
            assert abs(per_mol.mean() - want) < 5 * se, (ring, dist, per_mol.mean(), want, se)


def test_ideal_star_and_ring_statistics(cuda_device):
    check_ideal_closed_forms()


def test_topology_arguments_are_checked(cuda_device):
    d, mols, arch, words, starts, pos0 = _setup("N9_odd_ring_star")
    s = System(d)

    def expect_einval(w, st, a):
        with pytest.raises(SomaError) as e:
            s.set_topology(w, st, a)
        assert e.value.status == _abi.SOMA_EINVAL, _abi.soma_last_error()

    ring = workloads.ring_architecture(9)
    good, gst = workloads.encode_architectures([ring])
    a0 = np.zeros(d.n_chains, np.uint8)
    s.set_topology(good, gst, a0)                       # valid
    bad = good.copy()
    bad[gst[0] + 1 + 3] = (int(bad[gst[0] + 1 + 3]) & 0xFFFFFF00) | 2      # type 2
    expect_einval(bad, gst, a0)
    first = int(good[gst[0] + 1] >> 8)                   # particle 0's first bond word
    bad = good.copy()
    bad[first] |= 1 << 1                                 # bond type 1
    expect_einval(bad, gst, a0)
    bad = good.copy()
    bad[first] = (int(bad[first]) & 0x1F) | (40 << 5)            # partner outside
    expect_einval(bad, gst, a0)
    bad = good.copy()
    bad[first] = (int(bad[first]) & 0x1F) | (4 << 5)             # 0-4 listed at 0 only
    expect_einval(bad, gst, a0)
    expect_einval(good, np.array([len(good) - 2], np.uint32), a0)   # block past the end
    lin10, st10 = workloads.encode_architectures([workloads.linear_architecture(10)])
    expect_einval(lin10, st10, a0)                       # 10 particles, more than N = 9
    lin8, st8 = workloads.encode_architectures([workloads.linear_architecture(8)])
    s.set_topology(lin8, st8, a0)                        # 8 of N = 9: the ninth slot absent
    K9 = ([0] * 9, [(i, j) for i in range(9) for j in range(i + 1, 9)])
    k9, k9s = workloads.encode_architectures([K9])
    expect_einval(k9, k9s, a0)                           # nine sets
    two, two_st = workloads.encode_architectures([ring, ring])
    a_bad = a0.copy()
    a_bad[17] = 2
    expect_einval(two, two_st, a_bad)                    # mol_arch >= n_arch
    s.set_topology(None)                                 # back to the diblock
    s.sweep(2)
    s.close()
    for kw in (dict(move=MOVE_LEARNED),):     # the learned proposal takes linear chains
        s = System(SystemDesc(**dict(CASES["N9_odd_ring_star"][0], f=0.5, chiN=10.0, kappaN=50.0,
                                     **kw)))
        with pytest.raises(SomaError) as e:
            s.set_topology(good, gst, a0)
        assert e.value.status == _abi.SOMA_EINVAL
        s.close()


@pytest.mark.parametrize("dtype", [1, 2])
def test_topology_reduced_precision_grids(cuda_device, dtype):
    """BF16 / FP16 omega with molecules of any architecture: decisions agree
    with the oracle's omega rounded to the same type except at near-ties, at
    particles whose old or new cell holds a value one storage ulp apart (FP32
    rounding boundary), and downstream of those in the same molecule."""
    from tests.test_gpu_precision import ROUND_MODE, _cells, _differing_cells, _trial_positions
    d, mols, arch, words, starts, pos0 = _setup("N16_star_comb_ring_linear", grid_dtype=dtype)
    s = System(d)
    s.set_topology(words, starts, arch)
    s.set_positions(pos0)
    s.update_fields()
    orc = oracle_system(d)
    orc.set_topology(words, starts, arch)
    p = _pos(pos0)
    compared = 0
    for sweep in range(4):
        nA, nB = orc.histogram(p)
        n = s.get_density()
        np.testing.assert_array_equal(n & 0xFFFF, nA)
        np.testing.assert_array_equal(n >> 16, nB)
        wA, wB = orc.fields(nA, nB, ROUND_MODE[dtype])
        gA, gB = s.get_fields()
        odd = _differing_cells(gA, wA, dtype) | _differing_cells(gB, wB, dtype)
        old = p.copy()
        _, margin, acc = orc.sweep(p, wA, wB, sweep, want_margin=True, want_acc=True)
        s.sweep(1)
        g = s.get_positions()
        gacc = (g != old.stacked()).any(axis=0).astype(np.uint8)
        bad = np.nonzero(gacc != acc)[0]
        compared += d.M
        if len(bad):
            trial = _trial_positions(orc, old, sweep, bad)
            c_old = _cells(d, old.stacked()[:, bad])
            c_new = _cells(d, trial)
            excused = (np.abs(margin[bad]) < TIE) | np.isin(c_old, list(odd)) | \
                np.isin(c_new, list(odd))
            mols_ok = set((bad[excused] // d.N).tolist())
            assert all(m // d.N in mols_ok for m in bad.tolist())
            break
        np.testing.assert_array_equal(g, p.stacked())
    s.close()
    print(f"architectures, grid dtype {dtype}: {compared} moves compared")
    assert compared >= 2 * d.M
