"""n_t particle types (Sec. 2.1: Eq. hamil-comp, hamil-pair, omega-fields for
n_t types) on the GPU against the FP64 oracle, through the C ABI: occupation
numbers per type bit-exact, fields per type within FP32 rounding, move
decisions and positions cycle by cycle, the non-bonded energy, and the
arguments the library refuses."""
import numpy as np
import pytest

from paper_1711_03828_gb300 import (GRID_BF16, ITERATION_MOLECULE, SomaError, System, SystemDesc,
                                    _abi, workloads)
from tests.conftest import oracle_system
from tests.test_gpu_parity import TIE, _pos

pytestmark = pytest.mark.gpu

CHI3 = [[0.0, 30.0, 15.0], [30.0, 0.0, 40.0], [15.0, 40.0, 0.0]]
CHI2 = [[0.0, 25.0], [25.0, 0.0]]


def _molecules(n_types):
    """Three architectures of N = 16 with types 0..n_types-1: a linear chain
    in blocks, a three-arm star whose arms carry different types, a ring."""
    lin = ([min(i * n_types // 16, n_types - 1) for i in range(16)],
           workloads.linear_architecture(16)[1])
    star_types = [0] + [1] * 5 + [(2 % n_types)] * 5 + [1] * 5
    star = (star_types, workloads.star_architecture(3, 5)[1])
    ring = ([i % n_types for i in range(16)], workloads.ring_architecture(16)[1])
    return [lin, star, ring]


def _setup(n_types, chi, hamiltonian=0, set_order=0, seed=5, n_chains=2048):
    d = SystemDesc(n_chains=n_chains, N=16, f=0.5, box_Re=(2.0, 2.0, 2.0), grid=(12, 12, 12),
                   chiN=20.0, kappaN=50.0, seed=seed, set_order=set_order, hamiltonian=hamiltonian)
    mols = _molecules(n_types)
    arch = np.random.default_rng(seed).integers(0, len(mols), d.n_chains).astype(np.uint8)
    words, starts = workloads.encode_architectures(mols)
    pos0 = workloads.architecture_positions(d, mols, arch, seed=seed + 100)
    gpu = System(d)
    gpu.set_types(n_types, chi)
    gpu.set_topology(words, starts, arch)
    gpu.set_positions(pos0)
    gpu.update_fields()
    orc = oracle_system(d)
    orc.set_topology(words, starts, arch)
    orc.set_types(n_types, chi)
    return d, gpu, orc, _pos(pos0)


def _fields_tol(d, n, rho, chi):
    phi = n.astype(np.float64) / rho
    k0 = d.kappaN / d.N
    c0 = np.max(np.abs(chi)) / d.N
    return 8 * 2.0**-24 * (abs(k0) * (phi.sum(0) + 1) + c0 * phi.sum(0) * len(n)) + 1e-30


def _cycles(d, gpu, orc, p, n_cycles, chi):
    n = orc.histogram_types(p)
    w = orc.fields_types(n)
    moves = mism = 0
    for sweep in range(n_cycles):
        np.testing.assert_array_equal(gpu.get_type_counts(), n)
        tol = _fields_tol(d, n, orc.params.rho_cell, chi)
        assert np.all(np.abs(gpu.get_type_fields() - w) <= tol)
        old = p.copy()
        st, margin, acc = orc.sweep(p, None, None, sweep, want_margin=True, want_acc=True,
                                    w_types=w)
        gpu.sweep(1)
        g = gpu.get_positions()
        moves += d.M
        if d.set_order == ITERATION_MOLECULE:
            tied = (np.abs(margin.reshape(d.n_chains, d.N)) < TIE).any(axis=1)
            G = g.reshape(3, d.n_chains, d.N)
            P = p.stacked().reshape(3, d.n_chains, d.N)
            np.testing.assert_array_equal(G[:, ~tied], P[:, ~tied])
            if (G != P).any():
                mism += 1
                break
        else:
            gacc = (g != old.stacked()).any(axis=0).astype(np.uint8)
            bad = np.nonzero(gacc != acc)[0]
            if len(bad):
                tied_mol = set((bad[np.abs(margin[bad]) < TIE] // d.N).tolist())
                assert all(m // d.N in tied_mol for m in bad.tolist())
                mism += len(bad)
                keep = np.repeat(~np.isin(np.arange(d.n_chains), bad // d.N), d.N)
                np.testing.assert_array_equal(g[:, keep], p.stacked()[:, keep])
                break
            np.testing.assert_array_equal(g, p.stacked())
        n = orc.histogram_types(p)
        w = orc.fields_types(n)
    return moves, mism


@pytest.mark.parametrize("n_types,hamiltonian,set_order", [
    (3, 0, 0), (3, 1, 0), (2, 0, 0), (3, 0, ITERATION_MOLECULE)])
def test_types_cycles_match_oracle(cuda_device, n_types, hamiltonian, set_order):
    chi = CHI3 if n_types == 3 else CHI2
    d, gpu, orc, p = _setup(n_types, chi, hamiltonian, set_order)
    moves, mism = _cycles(d, gpu, orc, p, 10, chi)
    gpu.close()
    print(f"{n_types} types, K{hamiltonian}, set_order {set_order}: {moves} moves, "
          f"tolerated mismatches {mism}")
    assert moves >= 5 * d.M


def test_types_observables_match_oracle(cuda_device):
    d, gpu, orc, p = _setup(3, CHI3, 0)
    o = gpu.observables()
    ref = orc.observables_types(p, orc.histogram_types(p))
    gpu.close()
    for k in ("E_b", "E_nb", "Re2", "b2", "E_tot"):
        assert o[k] == pytest.approx(ref[k], rel=1e-9), k
    assert o["E_ext"] == 0.0


def test_types_graph_replay_is_identical(cuda_device):
    out = []
    for chunked in (True, False):
        d, gpu, orc, p = _setup(3, CHI3, 1, n_chains=1024)
        if chunked:
            gpu.sweep(32)
        else:
            for _ in range(32):
                gpu.sweep(1)
        out.append((gpu.get_positions(), gpu.get_type_counts()))
        gpu.close()
    np.testing.assert_array_equal(out[0][0], out[1][0])
    np.testing.assert_array_equal(out[0][1], out[1][1])
    assert int(out[0][1].sum()) == 1024 * 16


def test_types_arguments_are_checked(cuda_device):
    d = SystemDesc(n_chains=256, N=16, box_Re=(1.0, 1.0, 1.0), grid=(6, 6, 6))
    s = System(d)

    def refused(status, fn, *a):
        with pytest.raises(SomaError) as e:
            fn(*a)
        assert e.value.status == status, _abi.soma_last_error()

    refused(_abi.SOMA_EINVAL, s.set_types, 9, np.zeros((9, 9)))
    refused(_abi.SOMA_EINVAL, s.set_types, 3, [[0, 1, 2], [1, 0, 3], [2, 4, 0]])   # not symmetric
    refused(_abi.SOMA_EINVAL, s.set_types, 3, [[1, 1, 2], [1, 0, 3], [2, 3, 0]])   # diagonal
    s.set_types(3, CHI3)
    refused(_abi.SOMA_ESTATE, s.sweep, 1)                       # no architectures yet
    mols = _molecules(3)
    words, starts = workloads.encode_architectures(mols)
    arch = np.zeros(d.n_chains, np.uint8)
    s.set_topology(words, starts, arch)
    s.update_fields()
    s.sweep(2)
    refused(_abi.SOMA_EINVAL, s.get_density)
    refused(_abi.SOMA_EINVAL, s.get_fields)
    refused(_abi.SOMA_EINVAL, s.structure_factor, [(1, 0, 0)])
    refused(_abi.SOMA_ESTATE, s.set_types, 0)                   # the architectures use type 2
    refused(_abi.SOMA_EINVAL, s.set_types, 2, CHI2)             # type 2 >= 2
    s.close()
    s = System(d)
    s.set_types(2, CHI2)
    bad, bst = workloads.encode_architectures(_molecules(3))
    refused(_abi.SOMA_EINVAL, s.set_topology, bad, bst, np.zeros(d.n_chains, np.uint8))
    s.close()
    s = System(SystemDesc(n_chains=256, N=16, box_Re=(1.0, 1.0, 1.0), grid=(6, 6, 6),
                          grid_dtype=GRID_BF16))
    refused(_abi.SOMA_EINVAL, s.set_types, 3, CHI3)
    s.close()


def test_type_structure_factors_match_oracle(cuda_device):
    """S_ij(q) of the composition n_i - n_j for each pair of three types, and
    the two-type case through the packed grid, against the oracle's DFT."""
    m = [(1, 0, 0), (0, 1, 0), (1, 1, 0), (2, 0, 1), (0, 0, 3), (-1, 2, 1)]
    d, gpu, orc, p = _setup(3, CHI3, 0, n_chains=1024)
    gpu.sweep(5)
    n = gpu.get_type_counts()
    for i, j in ((0, 1), (1, 2), (0, 2), (2, 0)):
        got = gpu.structure_factor_types(i, j, m)
        want = orc.structure_factor(n[i], n[j], m)
        np.testing.assert_allclose(got, want, rtol=1e-9, atol=1e-9)
    gpu.close()
    s = System(SystemDesc(n_chains=1024, N=16, box_Re=(2.0, 2.0, 2.0), grid=(12, 12, 12)))
    s.sweep(3)
    ab = s.structure_factor(m)
    np.testing.assert_array_equal(s.structure_factor_types(0, 1, m), ab)
    np.testing.assert_array_equal(s.structure_factor_types(1, 0, m), ab)
    with pytest.raises(SomaError):
        s.structure_factor_types(0, 0, m)
    s.close()
