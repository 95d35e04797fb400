"""The library's host-side handling of the architecture array (Sec. 3.2.1)
and its set generation (Sec. 3.1.2), through soma_topology_sets on the CPU (no
device): the same sets as the oracle's independent implementation on hand
cases, random trees and random graphs, and every malformed array refused."""
import numpy as np
import pytest

import oracle
from paper_1711_03828_gb300 import SomaError, _abi, topology_sets, workloads


def _lib_sets(mols):
    words, starts = workloads.encode_architectures(mols)
    return topology_sets(words, starts, len(mols[0][0]))


def _oracle_sets(mols):
    words, starts = workloads.encode_architectures(mols)
    out = [oracle.topology_sets(words, int(s)) for s in starts]
    return np.array([o[0] for o in out]), np.array([o[1] for o in out])


def test_library_sets_equal_the_oracle_sets(soma_lib, oracle_lib):
    rng = np.random.default_rng(17)
    cases = [[workloads.star_architecture(3, 5), workloads.comb_architecture(8, 4, 2),
              workloads.ring_architecture(16), workloads.linear_architecture(16)],
             [workloads.ring_architecture(9), workloads.star_architecture(4, 2)],
             workloads.arch_large_molecules()]
    for N in (2, 5, 13, 32, 64):
        trees, graphs = [], []
        for _ in range(20):
            parent = [int(rng.integers(0, i)) for i in range(1, N)]
            perm = rng.permutation(N)     # relabelled: not every particle hangs from an earlier one
            trees.append(([int(t) for t in rng.integers(0, 2, N)],
                          [(int(perm[p]), int(perm[i + 1])) for i, p in enumerate(parent)]))
            pairs = {(int(a), int(b)) for a, b in rng.integers(0, N, (N, 2)) if a != b}
            graphs.append(([0] * N, sorted({(min(a, b), max(a, b)) for a, b in pairs})))
        cases += [trees, [g for g in graphs if _oracle_sets([g])[1][0] <= 8]]
    for mols in cases:
        ls, ln = _lib_sets(mols)
        os_, on = _oracle_sets(mols)
        np.testing.assert_array_equal(ln, on)
        np.testing.assert_array_equal(ls, os_)


def test_malformed_arrays_are_refused(soma_lib):
    ring = workloads.ring_architecture(9)
    good, gst = workloads.encode_architectures([ring])
    topology_sets(good, gst, 9)
    first = int(good[gst[0] + 1] >> 8)

    def refused(w, st, N=9):
        with pytest.raises(SomaError) as e:
            topology_sets(w, st, N)
        assert e.value.status == _abi.SOMA_EINVAL
        return _abi.soma_last_error()

    bad = good.copy()
    bad[gst[0] + 4] = (int(bad[gst[0] + 4]) & 0xFFFFFF00) | 2
    topology_sets(bad, gst, 9)                      # types 0..7: the sets take any of them
    bad[gst[0] + 4] = (int(bad[gst[0] + 4]) & 0xFFFFFF00) | 8
    assert "type" in refused(bad, gst)
    bad = good.copy()
    bad[first] |= 1 << 1
    assert "bond type" in refused(bad, gst)
    bad = good.copy()
    bad[first] = (int(bad[first]) & 0x1F) | (40 << 5)
    assert "outside" in refused(bad, gst)
    bad = good.copy()
    bad[first] = (int(bad[first]) & 0x1F) | (4 << 5)
    assert "one side" in refused(bad, gst)
    past = np.concatenate([good, np.array([9], np.uint32)])   # a block of 9 at the last word
    assert "runs past" in refused(past, np.array([len(past) - 1], np.uint32))
    assert "particles" in refused(good, np.array([len(good) - 2], np.uint32))  # count garbage
    assert "particles" in refused(good, gst, N=8)
    K9 = ([0] * 9, [(i, j) for i in range(9) for j in range(i + 1, 9)])
    w9, s9 = workloads.encode_architectures([K9])
    assert "independent sets" in refused(w9, s9)
    dup, dst = workloads.encode_architectures([([0, 0, 0], [(0, 1), (1, 2), (0, 1)])])
    assert "twice" in refused(dup, dst, N=3)
    last = good.copy()
    last[first] &= ~np.uint32(1)      # particle 0's last bond word loses its end bit
    ends = [k for k in range(first, len(good)) if good[k] & 1]
    last[ends[-1]] &= ~np.uint32(1)    # and the array's final list runs off the end
    refused(last, gst)


def test_sets_of_architectures_shorter_than_N(soma_lib, oracle_lib):
    """Molecules of several lengths: an architecture of n <= N particles fills
    the first n slots; the library's sets equal the oracle's on them and mark
    the absent slots 0xFF; more than N particles, or none, is refused."""
    mols = [workloads.linear_architecture(16), workloads.linear_architecture(8, 0),
            workloads.star_architecture(3, 3), workloads.ring_architecture(12), ([0], [])]
    words, starts = workloads.encode_architectures(mols)
    ls, ln = topology_sets(words, starts, 16)
    for a, (types, _) in enumerate(mols):
        os_, on = oracle.topology_sets(words, int(starts[a]))
        n = len(types)
        assert ln[a] == on
        np.testing.assert_array_equal(ls[a, :n], os_)
        assert np.all(ls[a, n:] == 0xFF)
    with pytest.raises(SomaError) as e:
        topology_sets(words, starts, 12)               # the diblock of 16 does not fit
    assert e.value.status == _abi.SOMA_EINVAL and "particles" in _abi.soma_last_error()
    empty = words.copy()
    empty[starts[4]] = 0                               # an architecture of no particles
    with pytest.raises(SomaError):
        topology_sets(empty, starts, 16)
