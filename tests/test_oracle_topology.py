"""Pins of the oracle's molecular architectures: the array layout of Sec. 3.2.1
(Fig. polyarch), the independent sets of Sec. 3.1.2 and their random visiting
order, the sweep over the bond lists and the bond observables.

Each check compares the oracle with something other than itself: words
encoded by hand, hand-derived sets, the linear-chain path of the oracle (pinned
by its own closed forms), the closed forms of ideal Gaussian trees and rings,
and the uniform distribution of permutations."""
import math

import numpy as np
import pytest

import oracle
from oracle import Positions
from paper_1711_03828_gb300 import SystemDesc, workloads
from tests.conftest import oracle_system

# A "T": 0(A) - 1(B), 1 - 2(B), 1 - 3(A), encoded by hand (block at word 0),
# followed by a block of two unbonded particles (B, A) at word 11.
T_WORDS = [4, 0x500, 0x601, 0x901, 0xA00,
           0x21,                                # particle 0: +1, last
           0xFFFFFFE0, 0x20, 0x41,              # particle 1: -1, +1, +2 (last)
           0xFFFFFFE1,                          # particle 2: -1, last
           0xFFFFFFC1,                          # particle 3: -2, last
           2, 0xFFFFFF01, 0xFFFFFF00]
T_MOLECULE = ([0, 1, 1, 0], [(0, 1), (1, 2), (1, 3)])


def _L(lib):
    return lib if lib is not None else oracle.lib()


def check_architecture_words_decode(lib=None):
    L = _L(lib)
    w = np.asarray(T_WORDS, np.uint32)
    assert [oracle.topo_type(w, 0, i, L) for i in range(4)] == [0, 1, 1, 0]
    assert [oracle.topo_partners(w, 0, i, L) for i in range(4)] == [[1], [0, 2, 3], [1], [1]]
    assert [oracle.topo_type(w, 11, i, L) for i in range(2)] == [1, 0]
    assert [oracle.topo_partners(w, 11, i, L) for i in range(2)] == [[], []]
    # the encoder of the seeded inputs writes the same words
    enc, starts = workloads.encode_architectures([T_MOLECULE])
    assert list(starts) == [0] and [int(v) for v in enc] == T_WORDS[:11]


def _sets(molecule, L):
    w, st = workloads.encode_architectures([molecule])
    s, n = oracle.topology_sets(w, int(st[0]), L)
    return [int(v) for v in s], n


def check_sets_hand_values(lib=None):
    L = _L(lib)
    K4 = ([0] * 4, [(0, 1), (0, 2), (0, 3), (1, 2), (1, 3), (2, 3)])
    centre_last = ([0] * 7, [(0, 1), (2, 3), (4, 5), (6, 0), (6, 2), (6, 4)])
    assert _sets(T_MOLECULE, L) == ([0, 1, 0, 0], 2)
    assert _sets(workloads.ring_architecture(5), L) == ([0, 1, 0, 1, 2], 3)
    assert _sets(workloads.ring_architecture(4), L) == ([0, 1, 0, 1], 2)
    assert _sets(K4, L) == ([0, 1, 2, 3], 4)
    assert _sets(workloads.star_architecture(3, 2), L) == ([0, 1, 0, 1, 0, 1, 0], 2)
    assert _sets(centre_last, L) == ([0, 1, 0, 1, 0, 1, 1], 2)
    assert _sets(workloads.linear_architecture(6), L) == ([0, 1, 0, 1, 0, 1], 2)
    assert _sets(([0], []), L) == ([0], 1)


def check_tree_sets_are_depth_parity(lib=None):
    """Random trees whose every particle hangs from an earlier one: two sets,
    set = depth mod 2; random graphs: no bond inside a set."""
    L = _L(lib)
    rng = np.random.default_rng(5)
    for _ in range(50):
        N = int(rng.integers(2, 65))
        parent = [int(rng.integers(0, i)) for i in range(1, N)]
        bonds = [(p, i + 1) for i, p in enumerate(parent)]
        depth = [0] * N
        for i in range(1, N):
            depth[i] = depth[parent[i - 1]] + 1
        s, n = _sets(([0] * N, bonds), L)
        assert n == 2 and s == [d % 2 for d in depth]
    for _ in range(50):
        N = int(rng.integers(2, 40))
        pairs = {(int(a), int(b)) for a, b in rng.integers(0, N, (2 * N, 2)) if a != b}
        bonds = sorted({(min(a, b), max(a, b)) for a, b in pairs})
        s, n = _sets(([0] * N, bonds), L)
        assert all(s[a] != s[b] for a, b in bonds)
        assert n == max(s) + 1


def check_set_order_is_a_uniform_permutation(lib=None):
    L = _L(lib)
    d = workloads.melt_small(n_chains=4096, N=4)
    s = oracle_system(d, L)
    for n_sets, draws in ((3, 24000), (4, 48000), (5, 60000)):
        counts = {}
        for k in range(draws):
            o = tuple(s.set_order(k % d.n_chains, k // d.n_chains, n_sets))
            assert sorted(o) == list(range(n_sets))
            counts[o] = counts.get(o, 0) + 1
        cells = math.factorial(n_sets)
        assert len(counts) == cells
        e = draws / cells
        chi2 = sum((c - e) ** 2 / e for c in counts.values())
        # 5 sigma of the chi-square distribution with cells - 1 degrees of freedom
        assert chi2 < (cells - 1) + 5 * math.sqrt(2 * (cells - 1)), (n_sets, chi2)
    # eight sets: the first visited set is uniform
    first = np.zeros(8)
    for k in range(16000):
        o = s.set_order(k % d.n_chains, k // d.n_chains, 8)
        assert sorted(o) == list(range(8))
        first[o[0]] += 1
    chi2 = ((first - 2000.0) ** 2 / 2000.0).sum()
    assert chi2 < 7 + 5 * math.sqrt(14), chi2
    # fixed order (set_order 1) visits the sets in index order
    f = oracle_system(workloads.melt_small(n_chains=4096, N=4, set_order=1), L)
    assert f.set_order(3, 9, 5) == [0, 1, 2, 3, 4]


def _cycle_both(a, b, p, q, sweeps):
    for sweep in range(sweeps):
        nA, nB = a.histogram(p)
        mA, mB = b.histogram(q)
        np.testing.assert_array_equal(nA, mA)
        np.testing.assert_array_equal(nB, mB)
        wA, wB = a.fields(nA, nB)
        st1, m1, acc1 = a.sweep(p, wA, wB, sweep, want_margin=True, want_acc=True)
        st2, m2, acc2 = b.sweep(q, wA, wB, sweep, want_margin=True, want_acc=True)
        np.testing.assert_array_equal(m1, m2)
        np.testing.assert_array_equal(acc1, acc2)
        np.testing.assert_array_equal(p.stacked(), q.stacked())
        assert st1.accepted == st2.accepted
    assert a.observables(p, nA, nB) == b.observables(q, nA, nB)


def check_linear_topology_is_the_linear_chain(lib=None, set_order=0, move=0):
    """The diblock written as an architecture array gives bit for bit the
    sweeps, occupation numbers and observables of the linear-chain path, and
    a mixture of two linear architectures those of the mixture path (SET
    scheme, or the molecule-parallel iteration with set_order 2; uniform or
    smart Monte Carlo moves, move 1)."""
    L = _L(lib)
    d = workloads.melt_small(n_chains=512, chiN=30.0, box_Re=(2.0, 2.0, 1.0), grid=(12, 12, 6),
                             set_order=set_order, move=move)
    pos0 = workloads.random_walk_positions(d, seed=3)
    lin = oracle_system(d, L)
    top = oracle_system(d, L)
    words, starts = workloads.encode_architectures([workloads.linear_architecture(d.N)])
    top.set_topology(words, starts, np.zeros(d.n_chains, np.uint8))
    p = Positions(*[pos0[k].copy() for k in range(3)])
    q = Positions(*[pos0[k].copy() for k in range(3)])
    _cycle_both(lin, top, p, q, 4)
    # two architectures: the diblock and a B homopolymer
    arch = np.random.default_rng(2).integers(0, 2, d.n_chains).astype(np.uint8)
    seq = np.array([((1 << d.N) - 1) & ~((1 << (d.N // 2)) - 1), (1 << d.N) - 1], np.uint64)
    mix = oracle_system(d, L)
    mix.set_architectures(seq, arch)
    words, starts = workloads.encode_architectures([workloads.linear_architecture(d.N),
                                                    workloads.linear_architecture(d.N, 0)])
    top2 = oracle_system(d, L)
    top2.set_topology(words, starts, arch)
    p = Positions(*[pos0[k].copy() for k in range(3)])
    q = Positions(*[pos0[k].copy() for k in range(3)])
    _cycle_both(mix, top2, p, q, 3)


def _ideal(molecule, n_mol, L, sweeps, first, move=0):
    N = len(molecule[0])
    d = SystemDesc(n_chains=n_mol, N=N, f=0.5, box_Re=(2.0, 2.0, 1.0), grid=(12, 12, 6),
                   chiN=0.0, kappaN=0.0, seed=7, move=move)
    s = oracle_system(d, L)
    words, starts = workloads.encode_architectures([molecule])
    s.set_topology(words, starts, np.zeros(n_mol, np.uint8))
    pos0 = workloads.architecture_positions(d, [molecule], np.zeros(n_mol, np.uint8), seed=13)
    p = Positions(*[pos0[k].copy() for k in range(3)])
    nA, nB = s.histogram(p)
    wA, wB = s.fields(nA, nB)
    assert np.all(wA == 0) and np.all(wB == 0)
    r2 = []
    for sweep in range(sweeps):
        s.sweep(p, wA, wB, sweep)
        if sweep >= first and sweep % 4 == 0:
            P = p.stacked().astype(np.float64).reshape(3, n_mol, N)
            r2.append(((P[:, :, :, None] - P[:, :, None, :]) ** 2).sum(0))
    return d, np.mean(r2, axis=0)     # per-molecule time averages, (n_mol, N, N)


def _graph_distance(N, bonds):
    D = np.full((N, N), 10**6)
    for i in range(N):
        D[i, i] = 0
    for i, j in bonds:
        D[i, j] = D[j, i] = 1
    for k in range(N):
        D = np.minimum(D, D[:, k:k + 1] + D[k:k + 1, :])
    return D


def check_ideal_star_and_ring_closed_forms(lib=None, move=0):
    """chiN = kappaN = 0: the bonds of a tree are independent Gaussians, so
    <|r_i - r_j|^2> = d_ij b0^2 with d_ij the graph distance; on a ring of N
    bonds the constraint that they sum to zero gives b0^2 d (N - d) / N.
    b0^2 = R_e0^2/(N-1) is the bond length the spring constant fixes.  Under
    either move (uniform, or smart Monte Carlo: the bonded energy over the
    architecture's partners decides the acceptance)."""
    L = _L(lib)
    Re = 6.0
    for molecule, closed in ((workloads.star_architecture(3, 5), "tree"),
                             (workloads.ring_architecture(9), "ring")):
        N = len(molecule[0])
        d, r2 = _ideal(molecule, 1024, L, 1400, 400, move)
        b02 = Re**2 / (N - 1)
        D = _graph_distance(N, molecule[1])
        for dist in range(1, int(D.max()) + 1):
            sel = np.triu(D == dist, 1)
            per_mol = r2[:, sel].mean(axis=1)
            want = dist * b02 if closed == "tree" else b02 * dist * (N - dist) / N
            se = per_mol.std() / math.sqrt(len(per_mol))
            assert abs(per_mol.mean() - want) < 5 * se, (closed, dist, per_mol.mean(), want, se)


def check_smc_force_follows_the_architecture(lib=None):
    """Smart Monte Carlo on branched and cyclic molecules at chiN = kappaN =
    0: any force keeps the move exact (the proposal densities enter the
    acceptance), so the force is pinned by efficiency.  With the force of the
    molecule's own bonds the drift follows the harmonic well and nearly every
    move is accepted (0.94-0.95 at the default step); a force taken from the
    linear neighbours i - 1, i + 1 instead pulls the star's centre, the comb's
    teeth and the ring's closing particles the wrong way (0.62-0.89)."""
    L = _L(lib)
    for molecule in (workloads.star_architecture(3, 5), workloads.star_architecture(7, 2),
                     workloads.ring_architecture(9), workloads.comb_architecture(8, 4, 2)):
        N = len(molecule[0])
        n_mol = 1024
        d = SystemDesc(n_chains=n_mol, N=N, f=0.5, box_Re=(2.0, 2.0, 1.0), grid=(12, 12, 6),
                       chiN=0.0, kappaN=0.0, move=1, seed=7)
        s = oracle_system(d, L)
        words, starts = workloads.encode_architectures([molecule])
        s.set_topology(words, starts, np.zeros(n_mol, np.uint8))
        pos0 = workloads.architecture_positions(d, [molecule], np.zeros(n_mol, np.uint8), seed=13)
        p = Positions(*[pos0[k].copy() for k in range(3)])
        w0 = np.zeros(s.cells)
        acc = att = 0
        for sweep in range(20):
            st, _, _ = s.sweep(p, w0, w0, sweep)
            acc += st.accepted
            att += st.attempted
        assert att == 20 * d.M
        assert acc / att > 0.93, (N, acc / att)


def check_topology_observables_hand_values(lib=None):
    L = _L(lib)
    d = SystemDesc(n_chains=2, N=4, f=0.5, box_Re=(1.0, 1.0, 1.0), grid=(6, 6, 6), chiN=0.0,
                   kappaN=0.0)
    s = oracle_system(d, L)
    words, starts = workloads.encode_architectures([T_MOLECULE])
    s.set_topology(words, starts, np.zeros(2, np.uint8))
    P = np.array([[0, 1, 1, 1], [0, 0, 2, 0], [0, 0, 0, 3]], np.float32)   # bonds 1, 4, 9
    pos = np.concatenate([P, P + 1.5], axis=1)
    p = Positions(*[pos[k].copy() for k in range(3)])
    nA, nB = s.histogram(p)
    o = s.observables(p, nA, nB)
    K_b = s.params.K_b
    assert o["E_b"] == pytest.approx(2 * 14 * K_b, rel=1e-15)
    assert o["b2"] == pytest.approx(28.0 / 6.0, rel=1e-15)
    assert o["Re2"] == pytest.approx(10.0, rel=1e-15)     # |r_3 - r_0|^2
    assert int(nA.sum()) == 4 and int(nB.sum()) == 4       # types from the words


def test_architecture_words_decode(oracle_lib):
    check_architecture_words_decode()


def test_sets_hand_values(oracle_lib):
    check_sets_hand_values()


def test_tree_sets_are_depth_parity(oracle_lib):
    check_tree_sets_are_depth_parity()


def test_set_order_is_a_uniform_permutation(oracle_lib):
    check_set_order_is_a_uniform_permutation()


@pytest.mark.parametrize("set_order,move", [(0, 0), (1, 0), (2, 0), (0, 1), (1, 1)])
def test_linear_topology_is_the_linear_chain(oracle_lib, set_order, move):
    check_linear_topology_is_the_linear_chain(set_order=set_order, move=move)


@pytest.mark.parametrize("move", [0, 1])
def test_ideal_star_and_ring_closed_forms(oracle_lib, move):
    check_ideal_star_and_ring_closed_forms(move=move)


def test_smc_force_follows_the_architecture(oracle_lib):
    check_smc_force_follows_the_architecture()


def test_topology_observables_hand_values(oracle_lib):
    check_topology_observables_hand_values()


# --------------------------------------------------------------------------
# Molecules of several lengths in one system (Sec. 2.1 mixtures, one
# architecture per molecule type, Sec. 3.2.1): an architecture of n < N
# particles fills the first n of a molecule's N slots, the rest are absent.
# --------------------------------------------------------------------------
def _blend(N, lengths, n_mol, L, chiN=0.0, kappaN=0.0, set_order=0, seed=7):
    mols = [workloads.linear_architecture(n, n) for n in lengths]   # homopolymers of A
    d = SystemDesc(n_chains=n_mol, N=N, f=0.5, box_Re=(2.0, 2.0, 1.0), grid=(12, 12, 6),
                   chiN=chiN, kappaN=kappaN, seed=seed, set_order=set_order)
    s = oracle_system(d, L)
    words, starts = workloads.encode_architectures(mols)
    arch = (np.arange(n_mol) % len(lengths)).astype(np.uint8)
    s.set_topology(words, starts, arch)
    pos0 = workloads.architecture_positions(d, mols, arch, seed=13)
    return d, s, arch, Positions(*[pos0[k].copy() for k in range(3)])


def check_blend_ideal_statistics(lib=None, set_order=0):
    """Ideal homopolymers of 8 and 4 particles in slots of N = 8 (chiN = kappaN
    = 0): each keeps Gaussian bonds of b0^2 = R_e0^2/(N-1) (the spring constant
    of the system), so <R_e^2> = (n-1) b0^2 per length, and the absent slots of
    the short molecules never move.  Also under the molecule-parallel
    iteration, whose attempts pick a particle of the molecule's own n."""
    L = _L(lib)
    N, lengths = 8, (8, 4)
    d, s, arch, p = _blend(N, lengths, 1024, L, set_order=set_order)
    absent = np.zeros((d.n_chains, N), bool)
    absent[arch == 1, 4:] = True
    absent = absent.reshape(-1)
    frozen = p.stacked()[:, absent].copy()
    nA, nB = s.histogram(p)
    assert int(nA.sum()) == 512 * 8 + 512 * 4 and int(nB.sum()) == 0
    wA, wB = s.fields(nA, nB)
    Re = 6.0
    b02 = Re**2 / (N - 1)
    re2 = {8: [], 4: []}
    att = 0
    for sweep in range(1600):
        st, _, _ = s.sweep(p, wA, wB, sweep)
        att += st.attempted
        if sweep >= 600 and sweep % 4 == 0:
            P = p.stacked().astype(np.float64).reshape(3, d.n_chains, N)
            for a, n in enumerate(lengths):
                sel = arch == a
                re2[n].append(((P[:, sel, n - 1] - P[:, sel, 0]) ** 2).sum(0))
    assert att == 1600 * (512 * 8 + 512 * 4)
    np.testing.assert_array_equal(p.stacked()[:, absent], frozen)
    for n in lengths:
        per = np.mean(re2[n], axis=0)
        se = per.std() / math.sqrt(per.size)
        assert abs(per.mean() - (n - 1) * b02) < 5 * se, (n, per.mean(), (n - 1) * b02, se)
    o = s.observables(p, *s.histogram(p))
    P = p.stacked().astype(np.float64).reshape(3, d.n_chains, N)
    last = np.where(arch == 1, 3, 7)
    want = ((P[:, np.arange(d.n_chains), last] - P[:, :, 0]) ** 2).sum(0).mean()
    assert o["Re2"] == pytest.approx(want, rel=1e-12)


def check_blend_monomer_dimer_balance(lib=None):
    """Monomers (n = 1) and dimers (n = 2) in slots of N = 2 in fixed random
    fields: a free A monomer visits cell c with probability exp(-wA(c)) / Z
    (uniform inside each cell), the dimers follow the exact cell-pair
    distribution of the two-particle test (erf quadrature)."""
    from tests.test_oracle_pins import _cells_of, _pair_cell_probabilities
    L = _L(lib)
    Lg, Re = 2, 1.5
    mols = [([0, 1], [(0, 1)]), ([0], [])]
    d = SystemDesc(n_chains=4096, N=2, f=0.5, box_Re=(Lg / Re,) * 3, grid=(Lg,) * 3, chiN=0.0,
                   kappaN=0.0, seed=19)
    s = oracle_system(d, L)
    words, starts = workloads.encode_architectures(mols)
    arch = (np.arange(d.n_chains) % 2).astype(np.uint8)
    s.set_topology(words, starts, arch)
    wA, wB = workloads.random_fields(Lg**3, seed=5, scale=1.0)
    p = Positions(*[a.copy() for a in workloads.architecture_positions(d, mols, arch, seed=3)])
    for sweep in range(100):
        s.sweep(p, wA, wB, sweep)
    T = 1500
    dim = np.nonzero(arch == 0)[0]
    mono = np.nonzero(arch == 1)[0]
    cpair = np.zeros((dim.size, Lg**6))
    cmono = np.zeros((mono.size, Lg**3))
    for sweep in range(100, 100 + T):
        s.sweep(p, wA, wB, sweep)
        P = p.stacked().reshape(3, d.n_chains, 2)
        c0, c1 = _cells_of(P[:, dim, 0], Lg), _cells_of(P[:, dim, 1], Lg)
        cpair[np.arange(dim.size), c0 * Lg**3 + c1] += 1
        cmono[np.arange(mono.size), _cells_of(P[:, mono, 0], Lg)] += 1
    K = s.params.K_b
    for counts, want in ((cpair, _pair_cell_probabilities(K, Lg, wA, wB).reshape(-1)),
                         (cmono, np.exp(-wA) / np.exp(-wA).sum())):
        freq = counts / T
        z = (freq.mean(0) - want) / np.maximum(freq.std(0) / math.sqrt(freq.shape[0]), 1e-12)
        assert np.max(np.abs(z)) < 5.0, np.max(np.abs(z))


def check_blend_histogram_and_density(lib=None):
    """Occupation numbers count the molecules' particles only (numpy binning
    of the present slots); S(q) divides by their number (numpy FFT); and
    rho_0 dL^3 is their number per cell: with 1152 molecules of 8 and 4
    particles in 864 cells it is 8, and counts of 4 A and 4 B in every cell
    give omega = 0 exactly (the field vanishes at the melt density)."""
    L = _L(lib)
    d, s, arch, p = _blend(8, (8, 3, 5), 999, L, chiN=20.0, kappaN=50.0)
    present = (np.arange(8)[None, :] < np.array([8, 3, 5])[arch][:, None]).reshape(-1)
    P = p.stacked().astype(np.float64)
    c = np.floor(P).astype(np.int64) % np.array(d.grid)[:, None]
    ci = (c[2] * d.grid[1] + c[1]) * d.grid[0] + c[0]
    nA, nB = s.histogram(p)
    np.testing.assert_array_equal(nA, np.bincount(ci[present], minlength=d.cells))
    assert int(nB.sum()) == 0
    M_real = int(np.array([8, 3, 5])[arch].sum())
    assert s.params.rho_cell == pytest.approx(M_real / d.cells, rel=1e-15)
    m = [(1, 0, 0), (0, 2, 1), (3, 1, 2)]
    grid = nA.reshape(d.grid[2], d.grid[1], d.grid[0]).astype(np.float64)
    F = np.fft.fftn(grid)
    want = [abs(F[k, j, i]) ** 2 / M_real for i, j, k in m]
    np.testing.assert_allclose(s.structure_factor(nA, nB, m), want, rtol=1e-12)
    d2, s2, arch2, _ = _blend(8, (8, 4), 1152, L, chiN=20.0, kappaN=50.0)
    assert s2.params.rho_cell == 8.0
    four = np.full(d2.cells, 4, np.uint32)
    wA, wB = s2.fields(four, four)
    assert np.all(wA == 0.0) and np.all(wB == 0.0)


@pytest.mark.parametrize("set_order", [0, 2])
def test_blend_ideal_statistics(oracle_lib, set_order):
    check_blend_ideal_statistics(set_order=set_order)


def test_blend_monomer_dimer_balance(oracle_lib):
    check_blend_monomer_dimer_balance()


def test_blend_histogram_and_density(oracle_lib):
    check_blend_histogram_and_density()
