"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test checks one oracle function against something other than itself:
a closed form, an invariant, a library routine (numpy binning, numpy FFT,
erf quadrature) or brute force.  Statistical tests use 5-sigma bounds with the
standard error taken across independent chains.
"""
import math

import numpy as np
import pytest

from paper_1711_03828_gb300 import workloads
from paper_1711_03828_gb300 import SystemDesc
from tests.conftest import oracle_system


# --------------------------------------------------------------------------
# Initial configuration (Sec. 2.1: Gaussian chain, b0^2 = R_e0^2/(N-1))
# --------------------------------------------------------------------------
def check_init_bond_and_end_to_end_statistics(lib=None):
    d = workloads.melt_small(n_chains=16384)
    s = oracle_system(d, lib)
    pos = s.init_chains()
    P = pos.stacked().astype(np.float64).reshape(3, d.n_chains, d.N)
    Re = d.grid[0] / d.box_Re[0]
    sigma2 = Re**2 / (3 * (d.N - 1))
    b = np.diff(P, axis=2).reshape(3, -1)
    n = b.shape[1]
    for k in range(3):
        assert abs(b[k].mean()) < 5 * math.sqrt(sigma2 / n)
        var = b[k].var()
        assert abs(var / sigma2 - 1) < 5 * math.sqrt(2.0 / n)
        kurt = np.mean(b[k] ** 4) / var**2
        assert abs(kurt - 3.0) < 5 * math.sqrt(24.0 / n)
    # components independent: no correlation between the axes of one bond or
    # between consecutive bonds along the chain
    B = np.diff(P, axis=2)  # (3, chains, N-1)
    for k1 in range(3):
        for k2 in range(3):
            if k1 < k2:
                r = np.corrcoef(B[k1].ravel(), B[k2].ravel())[0, 1]
                assert abs(r) < 5 / math.sqrt(n)
        r = np.corrcoef(B[k1, :, 1:].ravel(), B[k1, :, :-1].ravel())[0, 1]
        assert abs(r) < 5 / math.sqrt(n)
    # <R_e^2> = R_e0^2 (sum of N-1 independent bonds)
    re2 = ((P[:, :, -1] - P[:, :, 0]) ** 2).sum(0)
    assert abs(re2.mean() / Re**2 - 1) < 5 * re2.std() / Re**2 / math.sqrt(d.n_chains)
    # first particles uniform in the box: mean L/2, variance L^2/12
    for k in range(3):
        L = d.grid[k]
        f = P[k, :, 0]
        assert f.min() > 0 and f.max() < L
        assert abs(f.mean() - L / 2) < 5 * L / math.sqrt(12 * d.n_chains)
        assert abs(f.var() / (L * L / 12) - 1) < 5 * math.sqrt(0.8 / d.n_chains)


# --------------------------------------------------------------------------
# Occupation numbers (Eq. density-characteristics)
# --------------------------------------------------------------------------
def _numpy_histogram(pos, d):
    g = np.asarray(d.grid)
    c = np.floor(pos.astype(np.float64)).astype(np.int64) % g[:, None]
    idx = (c[2] * g[1] + c[1]) * g[0] + c[0]
    typeA = (np.arange(d.M) % d.N) < int(math.floor(d.f * d.N + 0.5))
    cells = int(np.prod(g))
    return (np.bincount(idx[typeA], minlength=cells).astype(np.uint32),
            np.bincount(idx[~typeA], minlength=cells).astype(np.uint32))


def check_histogram_matches_numpy_binning_with_edge_cases(lib=None):
    d = SystemDesc(n_chains=600, N=7, f=0.3, box_Re=(3.0, 2.0, 1.0), grid=(9, 6, 3),
                   chiN=10.0, kappaN=50.0)
    pos = workloads.random_walk_positions(d, seed=3, spread=3.0)
    # positions on cell faces, just below zero, on far images, negative images
    edge = np.array([0.0, -0.0, 1.0, 3.0, -1e-7, -1.0, 9.0, 27.0 + 0.5, -45.25, 8.999999,
                     np.nextafter(np.float32(9.0), np.float32(0.0)), -9.0, 1e6 + 0.5], np.float32)
    pos[0, : len(edge)] = edge
    pos[1, 100: 100 + len(edge)] = edge
    pos[2, 200: 200 + len(edge)] = edge[::-1]
    s = oracle_system(d, lib)
    from oracle import Positions
    p = Positions(pos[0].copy(), pos[1].copy(), pos[2].copy())
    nA, nB = s.histogram(p)
    eA, eB = _numpy_histogram(pos, d)
    np.testing.assert_array_equal(nA, eA)
    np.testing.assert_array_equal(nB, eB)
    assert int(nA.sum()) + int(nB.sum()) == d.M
    assert int(nA.sum()) == d.n_chains * int(math.floor(d.f * d.N + 0.5))


# --------------------------------------------------------------------------
# Fields (Eq. omega-fields, K^0) against the energy (Eq. discrete-ham)
# --------------------------------------------------------------------------
def check_fields_closed_forms(lib=None):
    # rho_0 dL^3 = 20 particles per cell
    d = SystemDesc(n_chains=40, N=4, f=0.5, box_Re=(2.0, 2.0, 2.0), grid=(2, 2, 2),
                   chiN=20.0, kappaN=50.0)
    s = oracle_system(d, lib)
    assert s.params.rho_cell == 20.0
    cells = 8
    nA = np.full(cells, 10, np.uint32)
    nB = np.full(cells, 10, np.uint32)
    wA, wB = s.fields(nA, nB)
    assert np.all(wA == 0.0) and np.all(wB == 0.0)  # phi_A = phi_B = 1/2: no force
    nA[0], nB[0] = 20, 0   # pure A cell at the mean density
    nA[1], nB[1] = 0, 20   # pure B cell
    nA[2], nB[2] = 20, 20  # twice the density, symmetric
    wA, wB = s.fields(nA, nB)
    chi0, kappa0 = 20.0 / 4, 50.0 / 4
    assert wA[0] == pytest.approx(-chi0 / 2) and wB[0] == pytest.approx(chi0 / 2)
    assert wA[1] == pytest.approx(chi0 / 2) and wB[1] == pytest.approx(-chi0 / 2)
    assert wA[2] == pytest.approx(kappa0) and wB[2] == pytest.approx(kappa0)


def check_fields_are_the_energy_derivative(lib=None, hamiltonian=0, external=False):
    """omega_i(c) = d(H_nb/kT + E_ext)/d n_i(c): Eq. (omega-fields) with
    phi = n/(rho_0 dL^3), for either interaction option, plus the external
    potential.  The energy is quadratic in the counts, so the central
    difference in the integer count is exact."""
    d = SystemDesc(n_chains=300, N=10, f=0.4, box_Re=(1.5, 1.5, 1.0), grid=(3, 3, 2),
                   chiN=27.0, kappaN=35.0)
    s = oracle_system(d, lib)
    s.set_hamiltonian(hamiltonian)
    if external:
        s.set_external(np.random.default_rng(3).normal(size=(2, s.cells)))
    rng = np.random.default_rng(7)
    nA = rng.integers(5, 40, s.cells).astype(np.uint32)
    nB = rng.integers(5, 40, s.cells).astype(np.uint32)
    pos = s.empty_positions()
    wA, wB = s.fields(nA, nB)
    for c in range(s.cells):
        for which, w in ((0, wA), (1, wB)):
            up = [nA.copy(), nB.copy()]
            dn = [nA.copy(), nB.copy()]
            up[which][c] += 1
            dn[which][c] -= 1
            ou, od = s.observables(pos, *up), s.observables(pos, *dn)
            Eu, Ed = ou["E_nb"] + ou["E_ext"], od["E_nb"] + od["E_ext"]
            assert (Eu - Ed) / 2 == pytest.approx(w[c], rel=1e-9, abs=1e-9)


def check_field_rounding_modes(lib=None):
    d = workloads.melt_small()
    s = oracle_system(d, lib)
    rng = np.random.default_rng(2)
    nA = rng.integers(0, 40, s.cells).astype(np.uint32)
    nB = rng.integers(0, 40, s.cells).astype(np.uint32)
    w64, _ = s.fields(nA, nB, 0)
    w32, _ = s.fields(nA, nB, 1)
    wbf, _ = s.fields(nA, nB, 2)
    w16, _ = s.fields(nA, nB, 3)
    np.testing.assert_array_equal(w32, w64.astype(np.float32).astype(np.float64))
    # BF16 keeps 8 significant bits, FP16 11 (normal range)
    assert np.all(np.abs(wbf - w32) <= np.abs(w32) * 2.0**-8 + 1e-30)
    assert np.all(np.abs(w16 - w32) <= np.abs(w32) * 2.0**-11 + 2.0**-24)
    bits = wbf.astype(np.float32).view(np.uint32)
    assert np.all(bits & 0xFFFF == 0)


# --------------------------------------------------------------------------
# Moves: ideal chains (chiN = kappaN = 0) relax to the Gaussian closed forms
# --------------------------------------------------------------------------
def check_ideal_chain_relaxes_to_gaussian_statistics(lib=None, move=0, set_order=0):
    """With chiN = kappaN = 0 every field vanishes and the Metropolis chain
    samples exp(-K_b sum b^2): <b^2> = R_e0^2/(N-1) and, the bonds being
    independent, <R_e^2> = R_e0^2.  Start from bonds stretched by 1.6x so
    the test sees the sweep relax the bond length."""
    d = workloads.melt_small(n_chains=1024, N=8, chiN=0.0, kappaN=0.0, box_Re=(2.0, 2.0, 1.0),
                             grid=(12, 12, 6), move=move, set_order=set_order)
    s = oracle_system(d, lib)
    if move == 2:
        s.set_mlp(workloads.random_mlp(7, scale=0.1))
    Re = 6.0
    sigma = Re / math.sqrt(3 * (d.N - 1))
    pos0 = workloads.random_walk_positions(d, seed=11, bond_sigma=1.6 * sigma)
    from oracle import Positions
    p = Positions(pos0[0].copy(), pos0[1].copy(), pos0[2].copy())
    nA, nB = s.histogram(p)
    wA, wB = s.fields(nA, nB)
    assert np.all(wA == 0) and np.all(wB == 0)
    b2_t, re2_t = [], []
    acc = att = 0
    for sweep in range(1600):
        st, _, _ = s.sweep(p, wA, wB, sweep)
        acc += st.accepted
        att += st.attempted
        if sweep >= 600 and sweep % 4 == 0:
            P = p.stacked().astype(np.float64).reshape(3, d.n_chains, d.N)
            b2_t.append((np.diff(P, axis=2) ** 2).sum(0).mean(1))
            re2_t.append(((P[:, :, -1] - P[:, :, 0]) ** 2).sum(0))
    b2 = np.mean(b2_t, axis=0)      # per-chain time averages
    re2 = np.mean(re2_t, axis=0)
    se_b2 = b2.std() / math.sqrt(d.n_chains)
    se_re2 = re2.std() / math.sqrt(d.n_chains)
    assert abs(b2.mean() - Re**2 / (d.N - 1)) < 5 * se_b2, (b2.mean(), Re**2 / (d.N - 1), se_b2)
    assert abs(re2.mean() - Re**2) < 5 * se_re2, (re2.mean(), Re**2, se_re2)
    # force-biased proposals of a harmonic chain are accepted far more often
    lo_hi = {0: (0.2, 0.95), 1: (0.5, 0.999), 2: (0.02, 0.999)}[move]
    assert lo_hi[0] < acc / att < lo_hi[1]


# --------------------------------------------------------------------------
# Balance: brute force on two bonded particles in fixed random fields
# --------------------------------------------------------------------------
def _pair_cell_probabilities(K, L, wA, wB):
    """Stationary P(c0, c1) of a harmonic dimer, particle 0 of type A and 1 of
    type B, in fixed fields on a periodic L^3 grid of unit cells:
    P ∝ exp(-wA(c0) - wB(c1)) prod_axes g(c0_d, c1_d) with
    g(a, b) = int_a^{a+1} dx0 sum_k int_{b+kL}^{b+kL+1} exp(-K (x1-x0)^2) dx1."""
    from math import erf, sqrt, pi
    xs, ws = np.polynomial.legendre.leggauss(64)

    def g(a, b):
        tot = 0.0
        for x, w in zip(xs, ws):
            x0 = a + 0.5 * (x + 1.0)
            inner = 0.0
            for k in range(-6, 7):
                lo, hi = b + k * L - x0, b + k * L + 1 - x0
                inner += 0.5 * sqrt(pi / K) * (erf(sqrt(K) * hi) - erf(sqrt(K) * lo))
            tot += 0.5 * w * inner
        return tot

    G1 = np.array([[g(a, b) for b in range(L)] for a in range(L)])
    cells = L**3
    P = np.zeros((cells, cells))
    for c0 in range(cells):
        a = (c0 % L, (c0 // L) % L, c0 // (L * L))
        for c1 in range(cells):
            b = (c1 % L, (c1 // L) % L, c1 // (L * L))
            P[c0, c1] = (math.exp(-wA[c0] - wB[c1]) * G1[a[0], b[0]] * G1[a[1], b[1]]
                         * G1[a[2], b[2]])
    return P / P.sum()


def _cells_of(P3, L):
    c = np.floor(P3.astype(np.float64)).astype(np.int64) % L
    return (c[2] * L + c[1]) * L + c[0]


def check_two_particle_balance_brute_force(set_order, lib=None, move=0, bf16=False):
    L = 2
    Re = 1.5
    d = SystemDesc(n_chains=4096, N=2, f=0.5, box_Re=(L / Re,) * 3, grid=(L,) * 3,
                   chiN=0.0, kappaN=0.0, set_order=set_order, seed=17, move=move)
    s = oracle_system(d, lib)
    if move == 2:
        s.set_mlp(workloads.random_mlp(7, scale=0.1), bf16=bf16)
    K = s.params.K_b
    assert K == pytest.approx(3.0 / (2 * Re * Re))
    wA, wB = workloads.random_fields(L**3, seed=5, scale=1.0)
    Pex = _pair_cell_probabilities(K, L, wA, wB)
    p = s.init_chains()
    for sweep in range(100):
        s.sweep(p, wA, wB, sweep)
    counts = np.zeros((d.n_chains, L**3 * L**3))
    T = 1500
    for sweep in range(100, 100 + T):
        s.sweep(p, wA, wB, sweep)
        P = p.stacked().reshape(3, d.n_chains, 2)
        c0 = _cells_of(P[:, :, 0], L)
        c1 = _cells_of(P[:, :, 1], L)
        counts[np.arange(d.n_chains), c0 * L**3 + c1] += 1
    freq = counts / T
    est = freq.mean(0)
    se = freq.std(0) / math.sqrt(d.n_chains)
    z = (est - Pex.reshape(-1)) / np.maximum(se, 1e-12)
    assert np.max(np.abs(z)) < 5.0, (np.max(np.abs(z)), np.argmax(np.abs(z)))
    chi2 = float(np.sum(z**2))
    assert chi2 < 64 + 8 * math.sqrt(2 * 64)  # 64 bins, loose upper bound


def check_walls_and_external_field_balance(lib=None, move=0):
    """Dimers in an external potential with two forbidden cells (chiN = kappaN
    = 0, so omega is the external field, +inf in the forbidden cells): the
    stationary cell-pair distribution is the exact one with weight 0 in the
    forbidden cells (exp(-inf)), and no particle ever enters one."""
    L, Re = 2, 1.5
    d = SystemDesc(n_chains=4096, N=2, f=0.5, box_Re=(L / Re,) * 3, grid=(L,) * 3,
                   chiN=0.0, kappaN=0.0, seed=23, move=move)
    s = oracle_system(d, lib)
    rng = np.random.default_rng(9)
    ext = rng.normal(size=(2, L**3))
    forbidden = np.zeros(L**3, np.uint8)
    forbidden[[2, 5]] = 1
    s.set_external(ext, forbidden)
    nA, nB = s.histogram(s.empty_positions())
    wA, wB = s.fields(nA, nB)
    assert np.all(np.isinf(wA[[2, 5]])) and np.all(np.isinf(wB[[2, 5]]))
    np.testing.assert_array_equal(wA[forbidden == 0], ext[0][forbidden == 0])
    K = s.params.K_b
    Pex = _pair_cell_probabilities(K, L, wA, wB)
    p = s.init_chains()
    for sweep in range(100):
        s.sweep(p, wA, wB, sweep)
    T = 1500
    counts = np.zeros((d.n_chains, L**6))
    for sweep in range(100, 100 + T):
        s.sweep(p, wA, wB, sweep)
        P = p.stacked().reshape(3, d.n_chains, 2)
        c0 = _cells_of(P[:, :, 0], L)
        c1 = _cells_of(P[:, :, 1], L)
        assert not forbidden[c0].any() and not forbidden[c1].any()
        counts[np.arange(d.n_chains), c0 * L**3 + c1] += 1
    freq = counts / T
    est = freq.mean(0)
    se = freq.std(0) / math.sqrt(d.n_chains)
    z = (est - Pex.reshape(-1)) / np.maximum(se, 1e-12)
    z[(Pex.reshape(-1) == 0) & (est == 0)] = 0.0
    assert np.max(np.abs(z)) < 5.0, (np.max(np.abs(z)), np.argmax(np.abs(z)))


def test_walls_and_external_field_balance(oracle_lib):
    check_walls_and_external_field_balance()


def check_architecture_mixture(lib=None):
    """A mixture of linear architectures: the counts follow the per-chain type
    sequences (numpy binning), and a blend of dimers AA, BB, AB and BA in
    fixed random fields samples, for each architecture, the exact cell-pair
    distribution with the fields of its own two types."""
    L, Re = 2, 1.5
    d = SystemDesc(n_chains=4096, N=2, f=0.5, box_Re=(L / Re,) * 3, grid=(L,) * 3,
                   chiN=0.0, kappaN=0.0, seed=31)
    s = oracle_system(d, lib)
    seq = np.array([0b00, 0b11, 0b10, 0b01], np.uint64)    # AA, BB, AB, BA
    arch = (np.arange(d.n_chains) % 4).astype(np.uint8)
    s.set_architectures(seq, arch)
    p = s.init_chains()
    # counts: particle i of chain k is B iff bit i of seq[arch[k]]
    nA, nB = s.histogram(p)
    P3 = p.stacked().astype(np.float64)
    c = _cells_of(P3, L)
    isB = ((seq[arch][:, None] >> np.arange(d.N, dtype=np.uint64)[None, :]) & 1).reshape(-1)
    np.testing.assert_array_equal(nA, np.bincount(c[isB == 0], minlength=L**3))
    np.testing.assert_array_equal(nB, np.bincount(c[isB == 1], minlength=L**3))
    wA, wB = workloads.random_fields(L**3, seed=5, scale=1.0)
    K = s.params.K_b
    for sweep in range(100):
        s.sweep(p, wA, wB, sweep)
    T = 1500
    counts = np.zeros((d.n_chains, L**6))
    for sweep in range(100, 100 + T):
        s.sweep(p, wA, wB, sweep)
        P = p.stacked().reshape(3, d.n_chains, 2)
        counts[np.arange(d.n_chains), _cells_of(P[:, :, 0], L) * L**3 + _cells_of(P[:, :, 1], L)] += 1
    fields = {0: wA, 1: wB}
    for a in range(4):
        t0, t1 = int(seq[a]) & 1, (int(seq[a]) >> 1) & 1
        Pex = _pair_cell_probabilities(K, L, fields[t0], fields[t1]).reshape(-1)
        freq = counts[arch == a] / T
        z = (freq.mean(0) - Pex) / np.maximum(freq.std(0) / math.sqrt(len(freq)), 1e-12)
        assert np.max(np.abs(z)) < 5.0, (a, np.max(np.abs(z)))


def test_architecture_mixture(oracle_lib):
    check_architecture_mixture()


# --------------------------------------------------------------------------
# Sweep mechanics: displacements bounded by a, accepted moves land on the draw
# --------------------------------------------------------------------------
def _f32_nearest(q):
    """The FP32 value nearest to the rational q (ties to the even significand),
    found from exact rational distances rather than by floating-point rounding."""
    from fractions import Fraction
    t = np.float32(float(q))
    best = None
    for c in (np.nextafter(t, np.float32(-np.inf)), t, np.nextafter(t, np.float32(np.inf))):
        dist = abs(Fraction(float(c)) - q)
        even = (int(np.array(c, np.float32).view(np.uint32)) & 1) == 0
        if best is None or dist < best[0] or (dist == best[0] and even):
            best = (dist, c)
    return best[1]


def check_sweep_moves_follow_the_draws(lib=None):
    from fractions import Fraction
    d = workloads.melt_small(n_chains=64)
    s = oracle_system(d, lib)
    p = s.init_chains()
    nA, nB = s.histogram(p)
    wA, wB = s.fields(nA, nB)
    before = p.copy()
    st, margin, acc = s.sweep(p, wA, wB, 3, want_margin=True, want_acc=True)
    a32 = float(np.float32(s.params.a32))
    for k in range(d.M):
        w = s.draw(1, k, 3)
        # r + a v rounded once: the exact rational sum, rounded to FP32
        prop = [_f32_nearest(Fraction(float(getattr(before, ax)[k])) + Fraction(a32) *
                             (Fraction((int(w[j]) >> 8) * 2 + 1, 2**24) - 1))
                for j, ax in enumerate("xyz")]
        now = [getattr(p, ax)[k] for ax in "xyz"]
        old = [getattr(before, ax)[k] for ax in "xyz"]
        if acc[k]:
            assert now == prop
        else:
            assert now == old
        assert (margin[k] > 0) == (not acc[k]) or margin[k] <= 0
    assert st.accepted == int(acc.sum())
    assert st.attempted == d.M
    assert np.all(np.abs(p.stacked() - before.stacked()) <= a32 * (1 + 1e-6))


# --------------------------------------------------------------------------
# Molecule-parallel iteration (Sec. 3.1.2, first scheme): N attempts per chain
# and step, each on a particle chosen at random, every particle attempted once
# per step on average; an attempt moves only its chosen particle, onto the
# trial position of its own draw, or leaves the chain unchanged.
# --------------------------------------------------------------------------
def check_molecule_iteration_attempts(lib=None):
    from oracle import Positions
    for N, n_chains in ((32, 512), (7, 1500)):
        d = SystemDesc(n_chains=n_chains, N=N, f=0.5, box_Re=(2.0, 2.0, 2.0), grid=(12, 12, 12),
                       chiN=20.0, kappaN=50.0, set_order=2)
        s = oracle_system(d, lib)
        p = s.init_chains()
        nA, nB = s.histogram(p)
        wA, wB = s.fields(nA, nB)
        counts = np.zeros(N)
        for sweep in range(6):
            before = p.copy()
            st, margin, acc, trial, chosen = s.sweep(p, wA, wB, sweep, want_margin=True,
                                                     want_acc=True, want_trial=True,
                                                     want_chosen=True)
            assert st.attempted == d.M and st.accepted == int(acc.sum())
            assert chosen.max() < N
            counts += np.bincount(chosen, minlength=N)
            B = before.stacked().reshape(3, n_chains, N)
            A = p.stacked().reshape(3, n_chains, N)
            T = trial.reshape(3, n_chains, N)
            C = chosen.reshape(n_chains, N)
            ACC = acc.reshape(n_chains, N)
            for k in range(0, n_chains, 37):   # replay chains attempt by attempt
                cur = B[:, k, :].copy()
                for j in range(N):
                    if ACC[k, j]:
                        cur[:, C[k, j]] = T[:, k, j]
                np.testing.assert_array_equal(cur, A[:, k, :])
            moved = np.any(A != B, axis=0)
            assert moved.mean() > 0.2
        # the choice is uniform over the chain (exact for N = 2^k, within 1/256 otherwise)
        tot = counts.sum()
        expect = tot / N
        chi2 = float(((counts - expect) ** 2 / expect).sum())
        assert chi2 < (N - 1) + 6 * math.sqrt(2 * (N - 1)) + (tot / 256**2 * N if N & (N - 1) else 0), chi2
        assert counts.min() > 0


def test_molecule_iteration_attempts(oracle_lib):
    check_molecule_iteration_attempts()


# --------------------------------------------------------------------------
# Observables
# --------------------------------------------------------------------------
def check_observables_hand_values(lib=None):
    d = SystemDesc(n_chains=1, N=3, f=0.0, box_Re=(1.0, 1.0, 1.0), grid=(4, 4, 4),
                   chiN=0.0, kappaN=0.0)
    s = oracle_system(d, lib)
    from oracle import Positions
    p = Positions(np.array([0, 1, 1], np.float32), np.array([0, 0, 2], np.float32),
                  np.array([0, 0, 0], np.float32))
    nA, nB = s.histogram(p)
    o = s.observables(p, nA, nB)
    # R_e0 = 4 dL, k0/2 = 3(N-1)/(2 R_e0^2) = 6/32; bonds |b|^2 = 1 and 4
    assert o["E_b"] == pytest.approx(5 * 6 / 32)
    assert o["Re2"] == pytest.approx(5.0)
    assert o["b2"] == pytest.approx(2.5)


def check_structure_factor_matches_numpy_fft(lib=None):
    d = SystemDesc(n_chains=400, N=8, f=0.5, box_Re=(2.0, 1.0, 1.5), grid=(8, 4, 6),
                   chiN=10.0, kappaN=50.0)
    s = oracle_system(d, lib)
    p = s.init_chains()
    nA, nB = s.histogram(p)
    ms = [(0, 0, 0), (1, 0, 0), (0, 1, 0), (0, 0, 1), (2, 1, 3), (-1, 2, -3), (7, 3, 5)]
    got = s.structure_factor(nA, nB, ms)
    dn = (nA.astype(np.float64) - nB.astype(np.float64)).reshape(d.grid[2], d.grid[1], d.grid[0])
    F = np.fft.fftn(dn)
    for (mx, my, mz), v in zip(ms, got):
        ref = abs(F[mz % d.grid[2], my % d.grid[1], mx % d.grid[0]]) ** 2 / d.M
        assert v == pytest.approx(ref, rel=1e-10, abs=1e-9)


# --------------------------------------------------------------------------
# The pins as tests (the mutation tests run the same checks on planted mistakes)
# --------------------------------------------------------------------------

def test_init_bond_and_end_to_end_statistics(oracle_lib):
    check_init_bond_and_end_to_end_statistics()


def test_histogram_matches_numpy_binning_with_edge_cases(oracle_lib):
    check_histogram_matches_numpy_binning_with_edge_cases()


def test_fields_closed_forms(oracle_lib):
    check_fields_closed_forms()


@pytest.mark.parametrize("hamiltonian,external", [(0, False), (1, False), (0, True), (1, True)])
def test_fields_are_the_energy_derivative(oracle_lib, hamiltonian, external):
    check_fields_are_the_energy_derivative(hamiltonian=hamiltonian, external=external)


def check_k1_fields_closed_forms(lib=None):
    """Option K^1: a pure A cell at the mean density has omega_A = 0 and
    omega_B = chi_0 (the cost of one B among A); a symmetric cell at the mean
    density has omega_A = omega_B = chi_0 / 2."""
    d = SystemDesc(n_chains=40, N=4, f=0.5, box_Re=(2.0, 2.0, 2.0), grid=(2, 2, 2),
                   chiN=20.0, kappaN=50.0)
    s = oracle_system(d, lib)
    s.set_hamiltonian(1)
    nA = np.full(8, 10, np.uint32)
    nB = np.full(8, 10, np.uint32)
    nA[0], nB[0] = 20, 0
    wA, wB = s.fields(nA, nB)
    chi0 = 20.0 / 4
    assert wA[0] == pytest.approx(0.0, abs=1e-12) and wB[0] == pytest.approx(chi0)
    assert wA[1] == pytest.approx(chi0 / 2) and wB[1] == pytest.approx(chi0 / 2)


def test_k1_fields_closed_forms(oracle_lib):
    check_k1_fields_closed_forms()


def test_field_rounding_modes(oracle_lib):
    check_field_rounding_modes()


@pytest.mark.parametrize("move,set_order", [(0, 0), (1, 0), (2, 0), (0, 2)])
def test_ideal_chain_relaxes_to_gaussian_statistics(oracle_lib, move, set_order):
    check_ideal_chain_relaxes_to_gaussian_statistics(move=move, set_order=set_order)


@pytest.mark.parametrize("set_order,move", [(0, 0), (0, 1), (0, 2), (1, 0), (1, 1), (1, 2),
                                            (2, 0)])
def test_two_particle_balance_brute_force(oracle_lib, set_order, move):
    check_two_particle_balance_brute_force(set_order, move=move)


def test_sweep_moves_follow_the_draws(oracle_lib):
    check_sweep_moves_follow_the_draws()


def test_observables_hand_values(oracle_lib):
    check_observables_hand_values()


def test_structure_factor_matches_numpy_fft(oracle_lib):
    check_structure_factor_matches_numpy_fft()


# --------------------------------------------------------------------------
# Spatial labelling of chains
# --------------------------------------------------------------------------
def _morton_ref(b):
    key = 0
    for bit in range(10):
        for d in range(3):
            key |= ((int(b[d]) >> bit) & 1) << (3 * bit + d)
    return key


def check_sort_chains_is_a_spatial_permutation(lib=None):
    d = SystemDesc(n_chains=3000, N=6, f=0.5, box_Re=(3.0, 2.0, 4.0), grid=(30, 20, 40),
                   chiN=0.0, kappaN=0.0)
    s = oracle_system(d, lib)
    p = s.init_chains()
    before = p.copy()
    perm = s.sort_chains(p)
    # a permutation of whole chains
    assert sorted(perm.tolist()) == list(range(d.n_chains))
    P0 = before.stacked().reshape(3, d.n_chains, d.N)
    P1 = p.stacked().reshape(3, d.n_chains, d.N)
    np.testing.assert_array_equal(P1, P0[:, perm.astype(np.int64), :])
    # keys (numpy floor/mod of the first particle, 8^3 blocks, Morton order) ascend,
    # ties keep the old order
    first = P1[:, :, 0].astype(np.float64)
    c = np.floor(first).astype(np.int64) % np.asarray(d.grid)[:, None]
    keys = np.array([_morton_ref(c[:, k] // 8) for k in range(d.n_chains)])
    assert np.all(np.diff(keys) >= 0)
    same = np.diff(keys) == 0
    assert np.all(np.diff(perm.astype(np.int64))[same] > 0)


def test_sort_chains_is_a_spatial_permutation(oracle_lib):
    check_sort_chains_is_a_spatial_permutation()


# --------------------------------------------------------------------------
# Smart Monte Carlo: exactness is pinned by the balance tests above (the MH
# correction makes any force exact); the direction of the force is pinned by
# efficiency: force-biased trial moves down a field ramp and inside a harmonic
# chain are accepted far more often than moves biased the wrong way.
# --------------------------------------------------------------------------
def check_smc_force_direction(lib=None):
    d = SystemDesc(n_chains=4096, N=1, f=1.0, box_Re=(64 / 6, 8 / 6, 8 / 6), grid=(64, 8, 8),
                   chiN=0.0, kappaN=0.0, a_Re=0.15, move=1, seed=3)
    s = oracle_system(d, lib)
    p = s.empty_positions()
    rng = np.random.default_rng(1)
    p.x[:] = rng.uniform(20, 44, d.M)
    p.y[:] = rng.uniform(0, 8, d.M)
    p.z[:] = rng.uniform(0, 8, d.M)
    ramp = 0.8 * (np.arange(s.cells) % 64).astype(np.float64)  # omega = 0.8 kT per cell along x
    acc = att = 0
    for sweep in range(10):
        st, _, _ = s.sweep(p, ramp, ramp, sweep)
        acc += st.accepted
        att += st.attempted
    assert acc / att > 0.83, acc / att      # 0.87 with the force, 0.74 with it reversed
    d2 = SystemDesc(n_chains=1024, N=8, box_Re=(2.0, 2.0, 1.0), grid=(12, 12, 6), chiN=0.0,
                    kappaN=0.0, move=1)
    s2 = oracle_system(d2, lib)
    p2 = s2.init_chains()
    w0 = np.zeros(s2.cells)
    acc = att = 0
    for sweep in range(20):
        st, _, _ = s2.sweep(p2, w0, w0, sweep)
        acc += st.accepted
        att += st.attempted
    assert acc / att > 0.9, acc / att       # 0.95 with the bond force, 0.32 reversed


def test_smc_force_direction(oracle_lib):
    check_smc_force_direction()


def check_smc_moves_follow_the_draws(lib=None):
    """Free particles (N = 1) in a field ramp along x, away from its periodic
    seam, so that the field force is the same constant F = (-0.8, 0, 0) at
    the old and at the trial cell: every trial position is r + A F + sqrt(2A)
    xi with xi the Box-Muller normals of the top 24 bits of words (0, 1) and
    (2, 3) of the move draw, and the acceptance compares ln u, u the open
    uniform of the low bytes of words 0, 1, 2, with ln alpha = -dE -
    |r - r' - A F|^2/(4A) + |r' - r - A F|^2/(4A), all recomputed here in
    FP64 from the Philox words."""
    d = SystemDesc(n_chains=2000, N=1, f=1.0, box_Re=(64 / 6, 8 / 6, 8 / 6), grid=(64, 8, 8),
                   chiN=0.0, kappaN=0.0, a_Re=0.15, move=1, seed=5)
    s = oracle_system(d, lib)
    p = s.empty_positions()
    rng = np.random.default_rng(2)
    p.x[:] = rng.uniform(20, 44, d.M)
    p.y[:] = rng.uniform(0, 8, d.M)
    p.z[:] = rng.uniform(0, 8, d.M)
    before = p.copy()
    ramp = 0.8 * (np.arange(s.cells) % 64).astype(np.float64)
    sweep = 7
    st, margin, acc, trial = s.sweep(p, ramp, ramp, sweep, want_margin=True, want_acc=True,
                                     want_trial=True)
    a = float(s.params.a)
    A = a * a / 6.0
    F = np.array([-0.8, 0.0, 0.0])
    for k in range(d.M):
        w = [int(v) for v in s.draw(1, k, sweep)]
        u = [((v >> 8) + 0.5) / 2**24 for v in w]
        r1, r2 = math.sqrt(-2 * math.log(u[0])), math.sqrt(-2 * math.log(u[2]))
        xi = [r1 * math.cos(2 * math.pi * u[1]), r1 * math.sin(2 * math.pi * u[1]),
              r2 * math.cos(2 * math.pi * u[3])]
        r = np.array([before.x[k], before.y[k], before.z[k]], np.float64)
        want = np.float32(r + np.float32(A * F + math.sqrt(2 * A) * np.array(xi)))
        got = trial[:, k]
        assert np.all(np.abs(got - want) <= np.spacing(np.abs(want).astype(np.float32))), (k, got, want)
        rn = got.astype(np.float64)
        dE = 0.8 * (math.floor(rn[0]) - math.floor(r[0]))
        fwd = ((rn - r - A * F) ** 2).sum()
        rev = ((r - rn - A * F) ** 2).sum()
        log_alpha = -dE - rev / (4 * A) + fwd / (4 * A)
        low = (w[0] & 0xFF) | (w[1] & 0xFF) << 8 | (w[2] & 0xFF) << 16
        lnu = math.log((low + 0.5) / 2**24)
        assert abs(margin[k] - (lnu - log_alpha)) < 1e-9, (k, margin[k], lnu - log_alpha)
        assert bool(acc[k]) == (log_alpha >= 0 or lnu < log_alpha)
    assert 0.5 < acc.mean() < 0.999


def test_smc_moves_follow_the_draws(oracle_lib):
    check_smc_moves_follow_the_draws()


# --------------------------------------------------------------------------
# Learned proposal: the gradient of the expected-squared-jump objective
# (through both network evaluations) against central finite differences.
# --------------------------------------------------------------------------
def check_esjd_gradient_matches_finite_differences(lib=None):
    from oracle import Positions
    d = workloads.melt_small(n_chains=64, chiN=30.0, move=2)
    s = oracle_system(d, lib)
    W = workloads.random_mlp(3)
    p = workloads.random_walk_positions(d, seed=5)
    P = Positions(p[0].copy(), p[1].copy(), p[2].copy())
    nA, nB = s.histogram(P)
    wA, wB = s.fields(nA, nB)
    rng = np.random.default_rng(0)
    checked = 0
    for _ in range(40):
        chain, i = int(rng.integers(0, d.n_chains)), int(rng.integers(0, d.N))
        xi = rng.normal(size=3)
        J, g, la = s.esjd_sample(W, P, wA, wB, chain, i, xi)
        if abs(la) < 1e-2:      # stay away from the kink of min(1, e^l)
            continue
        for k in rng.choice(1604, 25, replace=False):
            eps = 1e-6
            Wp, Wm = W.copy(), W.copy()
            Wp[k] += eps
            Wm[k] -= eps
            Jp, _, lp = s.esjd_sample(Wp, P, wA, wB, chain, i, xi, False)
            Jm, _, lm = s.esjd_sample(Wm, P, wA, wB, chain, i, xi, False)
            fd = (Jp - Jm) / (2 * eps)
            assert abs(fd - g[k]) <= 1e-5 * max(1.0, abs(fd)) or \
                abs(fd - g[k]) <= 1e-4 * (abs(fd) + abs(g[k])), (chain, i, k, fd, g[k])
            checked += 1
    assert checked > 400


def test_esjd_gradient_matches_finite_differences(oracle_lib):
    check_esjd_gradient_matches_finite_differences()


# --------------------------------------------------------------------------
# Learned proposal: the network forward pass on hand-built weights whose
# output has a closed form, o_k = sum_j C_kj |x_j| + 0.75 (k+1) + 0.1 k:
# layer 1 routes relu(x_j) and relu(-x_j) to separate units and holds 0.5 in
# eight bias-only units, layer 2 is the identity on the first 24 units and
# turns one bias unit into relu(2*0.5 - 0.25) = 0.75, layer 3 sums.  A
# transposed weight matrix, a dropped bias or a missing ReLU changes it.
# --------------------------------------------------------------------------
def check_mlp_forward_closed_form(lib=None):
    import oracle
    rng = np.random.default_rng(11)
    C = rng.uniform(0.5, 2.0, (4, 12))
    W = np.zeros(oracle.MLP_PARAMS)
    W1 = W[0:384].reshape(32, 12)
    b1 = W[384:416]
    W2 = W[416:1440].reshape(32, 32)
    b2 = W[1440:1472]
    W3 = W[1472:1600].reshape(4, 32)
    b3 = W[1600:1604]
    for j in range(12):
        W1[j, j] = 1.0
        W1[12 + j, j] = -1.0
    b1[24:] = 0.5
    for j in range(24):
        W2[j, j] = 1.0
    W2[24, 24] = 2.0
    b2[24] = -0.25
    b2[25:] = -1.0
    for k in range(4):
        W3[k, :12] = C[k]
        W3[k, 12:24] = C[k]
        W3[k, 24] = k + 1.0
        b3[k] = 0.1 * k
    for _ in range(20):
        x = rng.normal(size=12) * 3.0
        want = C @ np.abs(x) + 0.75 * np.arange(1, 5) + 0.1 * np.arange(4)
        got = oracle.mlp_forward(W, x, L=lib)
        np.testing.assert_allclose(got, want, rtol=1e-13, atol=1e-13)


def test_mlp_forward_closed_form(oracle_lib):
    check_mlp_forward_closed_form()


# --------------------------------------------------------------------------
# Learned proposal: the features of a hand-placed 3-particle chain in the
# field omega(c) = 3 cx + cy^2 (8^3 grid), where the face differences are
# 3 along x (-21 across the periodic seam at cx = 0), 2cy-1 and 2cy+1 along y
# and 0 along z, so the interpolated gradient is known in closed form.
# --------------------------------------------------------------------------
def check_learned_features_hand_values(lib=None):
    d = SystemDesc(n_chains=1, N=3, f=0.5, box_Re=(8 / 6, 8 / 6, 8 / 6), grid=(8, 8, 8),
                   chiN=0.0, kappaN=0.0, move=2)
    s = oracle_system(d, lib)          # N_A = floor(1.5 + 0.5) = 2
    p = s.empty_positions()
    R = np.array([[1.25, 2.5, 3.5], [2.0, 2.25, 3.75], [2.5, 3.0, 3.0]], np.float32)
    p.x[:], p.y[:], p.z[:] = R[:, 0], R[:, 1], R[:, 2]
    c = np.arange(512)
    cx, cy = c % 8, (c // 8) % 8
    w = (3.0 * cx + cy.astype(np.float64) ** 2)

    def grad(r):
        fx, fy = math.floor(r[0]), math.floor(r[1])
        tx, ty = r[0] - fx, r[1] - fy
        lo_x = 3.0 if fx % 8 != 0 else -21.0
        hi_x = 3.0 if fx % 8 != 7 else -21.0
        cyy = fy % 8
        lo_y = cyy ** 2 - ((cyy - 1) % 8) ** 2
        hi_y = ((cyy + 1) % 8) ** 2 - cyy ** 2
        return [(1 - tx) * lo_x + tx * hi_x, (1 - ty) * lo_y + ty * hi_y, 0.0]

    cases = [
        (1, [2.3, 2.75, 3.1], [2.3, 2.75, 3.1] - R[0], R[2] - [2.3, 2.75, 3.1], 1, 1, 1),
        (0, [0.5, 5.5, 7.9], [0, 0, 0], R[1] - [0.5, 5.5, 7.9], 1, 0, 1),
        (2, [7.25, 0.75, 1.0], [7.25, 0.75, 1.0] - R[1], [0, 0, 0], 0, 1, 0),
    ]
    for i, r, bp, bn, isA, hp, hn in cases:
        r = np.asarray(r, np.float64)
        f = s.learned_features(p, w, 0, i, r)
        want = np.concatenate([np.asarray(bp, np.float64), np.asarray(bn, np.float64), grad(r),
                               [isA, hp, hn]])
        np.testing.assert_allclose(f, want, rtol=0, atol=1e-12, err_msg=f"particle {i}")


def test_learned_features_hand_values(oracle_lib):
    check_learned_features_hand_values()
