"""Pins of the oracle's random numbers against an independent implementation.

The oracle's Philox4x32-10 (SC'11 definition) is compared with the host-side
Philox4x32-10 generator of the CUDA toolkit's cuRAND library, run on the CPU.
That generator emits, for seed s, the blocks Philox(ctr, key=(s lo, s hi)) with
block b at ctr = (b / 65536 as a 64-bit value in words 0-1, b mod 65536, 0);
the generator offset moves b, which reaches counter word 1.
"""
import ctypes
import os

import numpy as np
import pytest

BLOCKS_PER_ROW = 65536


def _curand():
    cands = [os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "lib64", "libcurand.so"),
             "libcurand.so", "libcurand.so.10"]
    for p in cands:
        try:
            return ctypes.CDLL(p)
        except OSError:
            continue
    pytest.skip("libcurand not found on this host")


def curand_host_philox(seed, offset, n_words):
    cr = _curand()
    gen = ctypes.c_void_p()
    assert cr.curandCreateGeneratorHost(ctypes.byref(gen), 161) == 0  # PHILOX4_32_10
    try:
        assert cr.curandSetPseudoRandomGeneratorSeed(gen, ctypes.c_ulonglong(seed)) == 0
        assert cr.curandSetGeneratorOffset(gen, ctypes.c_ulonglong(offset)) == 0
        out = np.zeros(n_words, np.uint32)
        assert cr.curandGenerate(gen, out.ctypes.data_as(ctypes.c_void_p),
                                 ctypes.c_size_t(n_words)) == 0
    finally:
        cr.curandDestroyGenerator(gen)
    return out.reshape(-1, 4)


def check_philox_matches_curand_host_generator(seed, lib=None):
    import oracle
    key = [seed & 0xFFFFFFFF, seed >> 32]
    blocks = curand_host_philox(seed, 0, 4 * 2 * BLOCKS_PER_ROW)
    rng = np.random.default_rng(seed & 0xFFFF)
    pick = np.concatenate([[0, 1, 2, 65535, 65536, 65537, len(blocks) - 1],
                           rng.choice(len(blocks), 400, replace=False)])
    for b in pick:
        ctr = [b // BLOCKS_PER_ROW, 0, b % BLOCKS_PER_ROW, 0]
        np.testing.assert_array_equal(oracle.philox(ctr, key, lib), blocks[b], err_msg=f"block {b}")


@pytest.mark.parametrize("seed", [0, 1, 0x123456789ABCDEF, 2**64 - 1, 0xDEADBEEF00000000])
def test_philox_matches_curand_host_generator(oracle_lib, seed):
    check_philox_matches_curand_host_generator(seed)


def test_philox_high_counter_word_via_offset(oracle_lib):
    oracle = oracle_lib
    seed = 99
    key = [seed, 0]
    # offset 2^50 words = 2^48 blocks = row 2^32: counter word 1 becomes 1
    off = 1 << 50
    blocks = curand_host_philox(seed, off, 4 * 64)
    for b in range(64):
        np.testing.assert_array_equal(oracle.philox([0, 1, b, 0], key), blocks[b])
    # and a row further on: row 2^32 + 20
    blocks = curand_host_philox(seed, off + 20 * 4 * BLOCKS_PER_ROW + 4 * 7, 4)
    np.testing.assert_array_equal(oracle.philox([20, 1, 7, 0], key), blocks[0])


def test_uniform_maps_exact_and_symmetric(oracle_lib):
    oracle = oracle_lib
    rng = np.random.default_rng(5)
    words = np.concatenate([[0, 1, 255, 256, 0x7FFFFFFF, 0x80000000, 0xFFFFFF00, 0xFFFFFFFF],
                            rng.integers(0, 2**32, 2000, dtype=np.uint64)]).astype(np.uint64)
    for r in words:
        r = int(r)
        v = oracle.uniform_sym(r)
        u = oracle.uniform_open(r)
        assert -1.0 < v < 1.0 and v != 0.0
        assert 0.0 < u < 1.0
        # exactly representable in FP32 (the GPU path computes them in FP32)
        assert float(np.float32(v)) == v
        # complementing the 24 leading bits mirrors the symmetric uniform
        assert oracle.uniform_sym(r ^ 0xFFFFFF00) == -v
        # the open uniform is the midpoint of its 2^-24 bin
        assert u * 2**24 - np.floor(u * 2**24) == 0.5
    # all 2^24 bins have mean 0 / mean 1/2: check the extreme bins
    assert oracle.uniform_sym(0) == -1.0 + 2.0**-24
    assert oracle.uniform_sym(0xFFFFFFFF) == 1.0 - 2.0**-24
