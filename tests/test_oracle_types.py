"""Pins of the oracle's n_t particle types (Sec. 2.1: Eq. hamil-comp,
hamil-pair and omega-fields for n_t types, the types of the molecular
architectures): against the two-type path (pinned by its own closed forms),
the energy whose derivative the fields are, the collapse of two identical
types under K^1, and numpy binning."""
import numpy as np
import pytest

from oracle import Positions
from paper_1711_03828_gb300 import SystemDesc, workloads
from tests.conftest import oracle_system


def _system(L, hamiltonian, n_types, chiN, mols, n_chains=512, N=None, seed=3, move=0):
    N = N or len(mols[0][0])
    # the A/B path takes chi_01 N from the description
    d = SystemDesc(n_chains=n_chains, N=N, f=0.5, box_Re=(2.0, 2.0, 1.0), grid=(12, 12, 6),
                   chiN=float(np.asarray(chiN)[0][1]), kappaN=40.0, seed=seed, move=move)
    s = oracle_system(d, L)
    s.set_hamiltonian(hamiltonian)
    words, starts = workloads.encode_architectures(mols)
    arch = np.random.default_rng(seed).integers(0, len(mols), d.n_chains).astype(np.uint8)
    s.set_topology(words, starts, arch)
    if n_types:
        s.set_types(n_types, chiN)
    pos = workloads.architecture_positions(d, mols, arch, seed=seed + 1)
    return d, s, words, starts, arch, Positions(*[pos[k].copy() for k in range(3)])


def check_two_types_equal_the_AB_path(lib=None, hamiltonian=0, move=0):
    """n_t = 2 through the type planes: the occupation numbers, fields (bit
    for bit), energy and several cycles of sweeps of the A/B path (uniform
    or smart Monte Carlo moves: the field and its force come from the plane
    of the particle's type)."""
    mols = [workloads.linear_architecture(16), workloads.star_architecture(3, 5)]
    chi = [[0.0, 27.0], [27.0, 0.0]]
    d, t, words, starts, arch, p = _system(lib, hamiltonian, 2, chi, mols, move=move)
    _, ab, _, _, _, q = _system(lib, hamiltonian, 0, chi, mols, move=move)
    for sweep in range(3):
        n = t.histogram_types(p)
        nA, nB = ab.histogram(q)
        np.testing.assert_array_equal(n[0], nA)
        np.testing.assert_array_equal(n[1], nB)
        w = t.fields_types(n)
        wA, wB = ab.fields(nA, nB)
        np.testing.assert_array_equal(w[0], wA)
        np.testing.assert_array_equal(w[1], wB)
        assert t.energy_types(n) == pytest.approx(ab.observables(q, nA, nB)["E_nb"], rel=1e-13)
        _, m1, a1 = t.sweep(p, None, None, sweep, want_margin=True, want_acc=True, w_types=w)
        _, m2, a2 = ab.sweep(q, wA, wB, sweep, want_margin=True, want_acc=True)
        np.testing.assert_array_equal(m1, m2)
        np.testing.assert_array_equal(p.stacked(), q.stacked())


def check_type_fields_are_the_energy_derivative(lib=None, hamiltonian=0):
    """omega_t(c) = dE_nb/dn_t(c) for three and four types with unequal
    chi_ij: the energy is quadratic in the counts, so the central difference
    in the integer count is exact up to rounding."""
    for T in (3, 4):
        rng = np.random.default_rng(11 + T)
        chi = np.zeros((T, T))
        iu = np.triu_indices(T, 1)
        chi[iu] = rng.uniform(5.0, 40.0, len(iu[0]))
        chi = chi + chi.T
        d = SystemDesc(n_chains=300, N=10, f=0.5, box_Re=(1.5, 1.5, 1.0), grid=(3, 3, 2),
                       chiN=0.0, kappaN=35.0)
        s = oracle_system(d, lib)
        s.set_hamiltonian(hamiltonian)
        s.set_types(T, chi)
        n = rng.integers(5, 40, (T, s.cells)).astype(np.uint32)
        w = s.fields_types(n)
        for c in range(s.cells):
            for t in range(T):
                up, dn = n.copy(), n.copy()
                up[t, c] += 1
                dn[t, c] -= 1
                dE = (s.energy_types(up) - s.energy_types(dn)) / 2
                assert dE == pytest.approx(w[t, c], rel=1e-9, abs=1e-9), (T, t, c)


def check_identical_types_collapse_under_K1(lib=None):
    """K^1 with chi_01 = chi_02 = chi and chi_12 = 0: types 1 and 2 are the
    same species, so their fields equal the B field of the two-type system
    in which they are merged, type 0's equals its A field, and the sweeps are
    those of the merged system."""
    chi3 = [[0.0, 30.0, 30.0], [30.0, 0.0, 0.0], [30.0, 0.0, 0.0]]
    three = [([0] * 8 + [1] * 4 + [2] * 4, workloads.linear_architecture(16)[1]),
             ([0, 2, 2, 1, 1, 2, 2, 1, 1, 0, 0, 0, 0, 0, 0, 0], workloads.star_architecture(3, 5)[1])]
    two = [([0 if t == 0 else 1 for t in m[0]], m[1]) for m in three]
    d, t, _, _, _, p = _system(lib, 1, 3, chi3, three)
    _, ab, _, _, _, q = _system(lib, 1, 0, [[0.0, 30.0], [30.0, 0.0]], two)
    for sweep in range(3):
        n = t.histogram_types(p)
        nA, nB = ab.histogram(q)
        np.testing.assert_array_equal(n[0], nA)
        np.testing.assert_array_equal(n[1] + n[2], nB)
        w = t.fields_types(n)
        wA, wB = ab.fields(nA, nB)
        np.testing.assert_allclose(w[0], wA, rtol=1e-13, atol=1e-13)
        np.testing.assert_allclose(w[1], wB, rtol=1e-13, atol=1e-13)
        np.testing.assert_allclose(w[2], wB, rtol=1e-13, atol=1e-13)
        _, m1, _ = t.sweep(p, None, None, sweep, want_margin=True, w_types=w)
        _, m2, _ = ab.sweep(q, wA, wB, sweep, want_margin=True)
        assert np.all(np.abs(m1 - m2) < 1e-9)
        np.testing.assert_array_equal(p.stacked(), q.stacked())


def check_type_histogram_matches_numpy(lib=None):
    mols = [([0, 1, 2, 3, 2, 1, 0, 3], workloads.linear_architecture(8)[1]),
            ([3, 3, 0, 0, 1, 1, 2, 2], workloads.ring_architecture(8)[1])]
    chi = np.full((4, 4), 10.0) - 10.0 * np.eye(4)
    d, s, words, starts, arch, p = _system(lib, 0, 4, chi, mols)
    n = s.histogram_types(p)
    P = p.stacked().astype(np.float64)
    g = np.asarray(d.grid)[:, None]
    c = np.floor(P).astype(np.int64) % g
    cell = (c[2] * d.grid[1] + c[1]) * d.grid[0] + c[0]
    types = np.concatenate([mols[a][0] for a in arch])
    for t in range(4):
        want = np.bincount(cell[types == t], minlength=s.cells)
        np.testing.assert_array_equal(n[t], want)
    assert int(n.sum()) == d.M


@pytest.mark.parametrize("hamiltonian,move", [(0, 0), (1, 0), (0, 1)])
def test_two_types_equal_the_AB_path(oracle_lib, hamiltonian, move):
    check_two_types_equal_the_AB_path(hamiltonian=hamiltonian, move=move)


@pytest.mark.parametrize("hamiltonian", [0, 1])
def test_type_fields_are_the_energy_derivative(oracle_lib, hamiltonian):
    check_type_fields_are_the_energy_derivative(hamiltonian=hamiltonian)


def test_identical_types_collapse_under_K1(oracle_lib):
    check_identical_types_collapse_under_K1()


def test_type_histogram_matches_numpy(oracle_lib):
    check_type_histogram_matches_numpy()
