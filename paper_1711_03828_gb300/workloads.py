"""Synthetic workloads and seeded input generators.

This module holds no arithmetic of the method: it names the benchmark
configurations (sizes, interaction strengths, seeds) and draws seeded input
configurations with numpy for tests that feed the SAME positions to the CUDA
library and to the CPU oracle.  The paper's workloads are synthetic melts
(Sec. 5: homopolymer and diblock melts of given N, sqrt(Nbar), dL = R_e0/6),
so nothing here stands in for a dataset.
"""
from __future__ import annotations

import math

import numpy as np

from . import SystemDesc


def melt_small(seed=1, **kw):
    """Symmetric A-B diblock melt, 1024 chains of N=32 in a periodic 2x2x2 R_e0
    box, 12^3 grid (dL = R_e0/6), chiN=20, kappaN=50: rho_0 R_e0^3 = 4096,
    sqrt(Nbar) = 128.  32,768 particles."""
    d = dict(n_chains=1024, N=32, f=0.5, box_Re=(2.0, 2.0, 2.0), grid=(12, 12, 12),
             chiN=20.0, kappaN=50.0, seed=seed)
    d.update(kw)
    return SystemDesc(**d)


def melt_large(seed=1, **kw):
    """Lamella-forming diblock melt at scale: 4,194,304 chains of N=32 in a
    periodic 32^3 R_e0 box, 192^3 grid, chiN=30, kappaN=50.  134,217,728
    particles (1.61 GB of FP32 positions)."""
    d = dict(n_chains=4194304, N=32, f=0.5, box_Re=(32.0, 32.0, 32.0), grid=(192, 192, 192),
             chiN=30.0, kappaN=50.0, seed=seed)
    d.update(kw)
    return SystemDesc(**d)


def melt_subbox(seed=1, **kw):
    """4^3 R_e0 sub-box of the large melt (same density and grid spacing):
    8192 chains of N=32, 24^3 grid, chiN=30.  262,144 particles."""
    d = dict(n_chains=8192, N=32, f=0.5, box_Re=(4.0, 4.0, 4.0), grid=(24, 24, 24),
             chiN=30.0, kappaN=50.0, seed=seed)
    d.update(kw)
    return SystemDesc(**d)


def melt_mid(seed=1, **kw):
    """16^3 R_e0 box of the large melt (same density, grid spacing, chiN):
    524,288 chains of N=32, 96^3 grid.  16,777,216 particles (201 MB of
    positions, larger than L2): the profiling case of the sweep kernel."""
    d = dict(n_chains=524288, N=32, f=0.5, box_Re=(16.0, 16.0, 16.0), grid=(96, 96, 96),
             chiN=30.0, kappaN=50.0, seed=seed)
    d.update(kw)
    return SystemDesc(**d)


def melt_tiny(seed=1, **kw):
    """The smallest system of the paper's weak-scaling series (n = 2^7 chains
    of N = 64, sqrt(Nbar) = 128, dL = R_e0/6): 8192 particles in a 1x1x1 R_e0
    box (rho_0 R_e0^3 = 128 N), 6x6x6 grid, homopolymer-like (chiN = 0),
    kappaN = 50."""
    d = dict(n_chains=128, N=64, f=0.5, box_Re=(1.0, 1.0, 1.0), grid=(6, 6, 6), chiN=0.0,
             kappaN=50.0, seed=seed)
    d.update(kw)
    return SystemDesc(**d)


def melt_slow(seed=1, **kw):
    """Slow melt: 1,048,576 chains of N=64 in a 32x32x16 R_e0 box, 192x192x96
    grid, chiN=40, kappaN=50.  67,108,864 particles."""
    d = dict(n_chains=1048576, N=64, f=0.5, box_Re=(32.0, 32.0, 16.0), grid=(192, 192, 96),
             chiN=40.0, kappaN=50.0, seed=seed)
    d.update(kw)
    return SystemDesc(**d)


def batch_replicas(n=64, seed=1, **kw):
    """Independent diblock melts of uneven size for one batched launch: box
    edge L uniform in {2,3,4,6,8} R_e0 (grid 6L, dL = R_e0/6), N in {16,32,64},
    f in {0.3,0.5}, chiN uniform in [10,40], kappaN=50, rho_0 R_e0^3 = 4096
    (n_chains = 4096 L^3 / N), one seed, replica id = index.  The choices are
    drawn with a seeded numpy generator."""
    rng = np.random.default_rng(seed + 7919)
    out = []
    for i in range(n):
        L = int(rng.choice([2, 3, 4, 6, 8]))
        N = int(rng.choice([16, 32, 64]))
        f = float(rng.choice([0.3, 0.5]))
        chiN = float(rng.uniform(10.0, 40.0))
        d = dict(n_chains=4096 * L**3 // N, N=N, f=f, box_Re=(float(L),) * 3, grid=(6 * L,) * 3,
                 chiN=chiN, kappaN=50.0, seed=seed, replica_id=i)
        d.update(kw)
        out.append(SystemDesc(**d))
    return out


def scaled(desc: SystemDesc, box_Re, rho_Re3=4096.0):
    """Same chains and interactions in another box at density rho_0 R_e0^3."""
    cells_per_Re = desc.grid[0] / desc.box_Re[0]
    grid = tuple(int(round(b * cells_per_Re)) for b in box_Re)
    vol = box_Re[0] * box_Re[1] * box_Re[2]
    n_chains = int(round(rho_Re3 * vol / desc.N))
    return SystemDesc(n_chains=n_chains, N=desc.N, f=desc.f, box_Re=tuple(box_Re), grid=grid,
                      chiN=desc.chiN, kappaN=desc.kappaN, a_Re=desc.a_Re, move=desc.move,
                      set_order=desc.set_order, grid_dtype=desc.grid_dtype, seed=desc.seed,
                      replica_id=desc.replica_id, flags=desc.flags)


def random_walk_positions(desc: SystemDesc, seed: int, bond_sigma: float = None,
                          spread: float = 1.0) -> np.ndarray:
    """Seeded synthetic input: chains whose first particle is uniform in the
    box and whose bond components are normal with standard deviation
    ``bond_sigma`` (grid units; default R_e0/sqrt(3(N-1))).  Returns a (3, M)
    float32 array in grid units.  ``spread`` scales the box the first
    particles are drawn from (values > 1 place chains across periodic images)."""
    rng = np.random.default_rng(seed)
    Re = desc.grid[0] / desc.box_Re[0]
    if bond_sigma is None:
        bond_sigma = Re / math.sqrt(3.0 * max(desc.N - 1, 1))
    n, N = desc.n_chains, desc.N
    first = rng.random((3, n, 1)) * np.asarray(desc.grid, dtype=np.float64)[:, None, None] * spread
    steps = rng.normal(0.0, bond_sigma, size=(3, n, N - 1)) if N > 1 else np.zeros((3, n, 0))
    walk = np.concatenate([first, first + np.cumsum(steps, axis=2)], axis=2)
    return walk.reshape(3, n * N).astype(np.float32)


def random_fields(cells: int, seed: int, scale: float = 1.0):
    """Seeded synthetic field planes (omega_A, omega_B) in kT, uniform in
    [-scale, scale), FP64."""
    rng = np.random.default_rng(seed)
    return rng.uniform(-scale, scale, cells), rng.uniform(-scale, scale, cells)


def random_mlp(seed, scale=0.3):
    """Seeded parameters of the learned proposal's network (1604 values,
    layout W1[32][12], b1[32], W2[32][32], b2[32], W3[4][32], b3[4]), uniform
    in [-scale, scale) per fan-in; rounded to BF16-representable values so
    the GPU's BF16 weights hold them exactly."""
    rng = np.random.default_rng(seed)
    parts = []
    for rows, cols in ((32, 12), (32, 1), (32, 32), (32, 1), (4, 32), (4, 1)):
        fan = 12 if rows == 32 and cols == 12 else (32 if cols == 32 else 1)
        parts.append(rng.uniform(-scale, scale, rows * cols) / np.sqrt(max(fan, 1) / 4.0))
    w = np.concatenate(parts).astype(np.float32)
    bits = w.view(np.uint32) & np.uint32(0xFFFF0000)  # truncate to a BF16 value
    return bits.view(np.float32).astype(np.float64)


# ---------------------------------------------------------------------------
# Molecular architectures: a molecule is (types, bonds) with types a list of 0
# (A) / 1 (B) per particle and bonds a list of (i, j) pairs.  encode_architectures
# writes them in the array layout of Sec. 3.2.1 that soma_set_topology reads.

def linear_architecture(N, N_A=None):
    """Linear chain i - (i+1); the first N_A particles are A (default N/2)."""
    N_A = N // 2 if N_A is None else N_A
    return [0 if i < N_A else 1 for i in range(N)], [(i, i + 1) for i in range(N - 1)]


def star_architecture(arms, arm_len, arm_types=None):
    """Star: particle 0 is the centre (type A), then each arm's particles from
    the centre outwards; arm_len is one length for every arm or a list of
    lengths; arm_types[k] is the type of arm k (default alternating A, B)."""
    lens = [arm_len] * arms if isinstance(arm_len, int) else list(arm_len)
    types, bonds = [0], []
    for k in range(arms):
        t = (k % 2) if arm_types is None else arm_types[k]
        prev = 0
        for _ in range(lens[k]):
            i = len(types)
            types.append(t)
            bonds.append((prev, i))
            prev = i
    return types, bonds


def ring_architecture(N, N_A=None):
    """Ring i - (i+1) mod N; the first N_A particles are A (default N/2)."""
    N_A = N // 2 if N_A is None else N_A
    return [0 if i < N_A else 1 for i in range(N)], [(i, (i + 1) % N) for i in range(N)]


def comb_architecture(backbone, teeth, tooth_len):
    """Comb: an A backbone of the given length with `teeth` B side chains of
    tooth_len particles grafted at evenly spaced backbone particles.  Each
    tooth follows its graft point in the particle order."""
    types, bonds = [], []
    graft = set(int(round((k + 0.5) * backbone / teeth)) for k in range(teeth))
    prev_bb = None
    for b in range(backbone):
        i = len(types)
        types.append(0)
        if prev_bb is not None:
            bonds.append((prev_bb, i))
        prev_bb = i
        if b in graft:
            prev = i
            for _ in range(tooth_len):
                j = len(types)
                types.append(1)
                bonds.append((prev, j))
                prev = j
    return types, bonds


def encode_architectures(molecules):
    """Architecture array (uint32) and the first word of each block, for a
    list of (types, bonds).  Block: N; per particle (first bond word << 8) |
    type (0xFFFFFF: no bonds); then per particle its bonds in the order given
    (both directions of every bond), each ((j - i) << 5) | (bond type 0 << 1) |
    last."""
    words, starts = [], []
    for types, bonds in molecules:
        N = len(types)
        partners = [[] for _ in range(N)]
        for i, j in bonds:
            partners[i].append(j)
            partners[j].append(i)
        start = len(words)
        starts.append(start)
        words.append(N)
        mono = len(words)
        words.extend([0] * N)
        for i in range(N):
            if not partners[i]:
                words[mono + i] = (0xFFFFFF << 8) | types[i]
                continue
            words[mono + i] = (len(words) << 8) | types[i]
            for k, j in enumerate(partners[i]):
                last = 1 if k == len(partners[i]) - 1 else 0
                words.append((((j - i) & 0x7FFFFFF) << 5) | last)
    return np.asarray(words, np.uint32), np.asarray(starts, np.uint32)


def architecture_positions(desc: SystemDesc, molecules, arch, seed: int,
                           bond_sigma: float = None, chunk: int = 1 << 18) -> np.ndarray:
    """Seeded synthetic input for molecules of the given architectures
    (arch[k] indexes molecules): particle 0 uniform in the box, every later
    particle at its lowest-index bonded partner plus a normal displacement of
    standard deviation bond_sigma per axis (default R_e0/sqrt(3(N-1))); a
    particle with no earlier partner is placed uniformly in the box, so the
    bonds that close rings start stretched; the absent slots of a molecule of
    fewer than N particles are placed uniformly too.  Molecules are drawn in chunks of
    `chunk` with the generator seeded by (seed, chunk index).  Returns (3, M)
    float32."""
    Re = desc.grid[0] / desc.box_Re[0]
    N = desc.N
    if bond_sigma is None:
        bond_sigma = Re / math.sqrt(3.0 * max(N - 1, 1))
    box = np.asarray(desc.grid, dtype=np.float64)
    parent = []
    for types, bonds in molecules:
        p = [-1] * N
        for i, j in bonds:
            a, b = min(i, j), max(i, j)
            if p[b] < 0 or a < p[b]:
                p[b] = a
        parent.append(p)
    n = desc.n_chains
    arch = np.asarray(arch)
    out = np.empty((3, n, N), np.float32)
    for c, k0 in enumerate(range(0, n, chunk)):
        k1 = min(n, k0 + chunk)
        rng = np.random.default_rng([seed, c])
        part = np.zeros((3, k1 - k0, N))
        free = rng.random((3, k1 - k0, N)) * box[:, None, None]
        steps = rng.normal(0.0, bond_sigma, size=(3, k1 - k0, N))
        ar = arch[k0:k1]
        for a, p in enumerate(parent):
            sel = np.nonzero(ar == a)[0]
            for i in range(N):
                if p[i] < 0:
                    part[:, sel, i] = free[:, sel, i]
                else:
                    part[:, sel, i] = part[:, sel, p[i]] + steps[:, sel, i]
        out[:, k0:k1] = part
    return out.reshape(3, n * N)


def arch_large(seed=1, **kw):
    """The 134M-particle melt of melt_large with molecules of four
    architectures in equal numbers (random per molecule): a three-arm star
    (arms 11, 10, 10; arms alternately A, B), a comb (A backbone of 16 with
    four B teeth of 4), a ring (16 A, 16 B) and the linear diblock; N = 32."""
    return melt_large(seed=seed, **kw)


def arch_mid(seed=1, **kw):
    """arch_large in the 16^3 R_e0 box of melt_mid (16,777,216 particles):
    the profiling case of the architecture sweep."""
    return melt_mid(seed=seed, **kw)


def abc_large(seed=1, **kw):
    """The 134M-particle melt of melt_large with three particle types A, B, C
    (chi_AB N = 30, chi_AC N = 15, chi_BC N = 40, kappaN = 50): molecules of
    abc_molecules(), one drawn per molecule."""
    return melt_large(seed=seed, **kw)


ABC_CHI_N = [[0.0, 30.0, 15.0], [30.0, 0.0, 40.0], [15.0, 40.0, 0.0]]


def abc_molecules():
    """Three architectures of N = 32 with types 0 (A), 1 (B), 2 (C): a linear
    ABC triblock (11, 11, 10), a three-arm star with one arm of each type
    (arms 11, 10, 10; centre A) and a ring of A, B and C blocks (11, 11, 10)."""
    tri = [0] * 11 + [1] * 11 + [2] * 10
    star_types = [0] + [0] * 11 + [1] * 10 + [2] * 10
    return [(tri, linear_architecture(32)[1]),
            (star_types, star_architecture(3, [11, 10, 10])[1]),
            (tri, ring_architecture(32)[1])]


def arch_large_molecules():
    return [star_architecture(3, [11, 10, 10]), comb_architecture(16, 4, 4),
            ring_architecture(32), linear_architecture(32)]
