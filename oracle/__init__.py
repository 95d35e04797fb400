"""FP64 CPU oracle of the SCMF Monte-Carlo cycle (arXiv:1711.03828, Sec. 2, 3.1.2).

TEST INFRASTRUCTURE.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package.  It wraps ``liboracle.so`` (plain C in ``soma_oracle.c``, built by
``oracle.build.build()``) with numpy arrays and shares no code with the CUDA
library in ``paper_1711_03828_gb300``.

Functions and the paper passage each follows:

* ``philox`` / ``draw``          -- Philox4x32-10 (SC'11), the counter RNG that
  replaces the stored-state PCG of Sec. 3.2.3.
* ``System.init_chains``        -- initial Gaussian chains (Sec. 2.1, b0 = sqrt(3/k0)).
* ``System.sort_chains``        -- spatial (Morton) labelling of whole chains (labels are
  arbitrary, Sec. 3.1.1).
* ``System.histogram``          -- occupation numbers, Eq. (density-characteristics).
* ``System.fields``             -- interaction fields, Eq. (omega-fields), option K^0.
* ``System.sweep``              -- one SET Monte-Carlo step (Sec. 2.2, Sec. 3.1.2).
* ``System.observables``        -- E_b (Eq. h-bond), E_nb (Eq. discrete-ham), R_e^2.
* ``System.structure_factor``   -- composition S(q) on the grid (Sec. 5.6).
* ``System.set_topology``       -- molecular architectures in the array layout of
  Sec. 3.2.1 with independent sets (Sec. 3.1.2); ``topology_sets``,
  ``topo_partners``, ``topo_type``, ``System.set_order`` expose the steps.
* ``System.set_types``          -- n_t particle types (Sec. 2.1): ``histogram_types``,
  ``fields_types`` (Eq. omega-fields for n_t types), ``energy_types`` (Eq.
  discrete-ham with Eq. hamil-pair), ``observables_types``.
* ``mlp_forward`` / ``System.set_mlp`` -- the learned proposal's network (no
  counterpart in the paper) in FP64, or with ``bf16=True`` in the BF16 reading
  of the tensor-core evaluators (``mlp_forward_bf16``; ``bf16_slack`` and
  ``System.sweep(want_slack=True)`` measure how near each rounding lies to a
  BF16 rounding boundary).
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lib = None

u32p = ctypes.POINTER(ctypes.c_uint32)
f32p = ctypes.POINTER(ctypes.c_float)
f64p = ctypes.POINTER(ctypes.c_double)
u8p = ctypes.POINTER(ctypes.c_uint8)
i32p = ctypes.POINTER(ctypes.c_int32)

PURPOSE_INIT, PURPOSE_MOVE, PURPOSE_MOVE2, PURPOSE_CONFIG, PURPOSE_TRAIN = 0, 1, 2, 4, 5
PURPOSE_SETS = 6
TOPO_NO_BONDS = 0xFFFFFF
MLP_PARAMS = 1604


def mlp_forward(W, x, L=None):
    """Network outputs (mu_x, mu_y, mu_z, log-scale pre-activation) of features x."""
    Wd = np.ascontiguousarray(W, dtype=np.float64)
    xd = np.ascontiguousarray(x, dtype=np.float64)
    out = np.zeros(4)
    (L or lib()).or_mlp_forward(_ptr(Wd, f64p), _ptr(xd, f64p), _ptr(out, f64p))
    return out


def mlp_forward_bf16(W, x, Tx=None, L=None):
    """Network outputs in the BF16 reading (inputs, weights, biases and hidden
    activations rounded to BF16, sums exact) and the smallest slack of its
    roundings (inf when Tx is None: only the activations count then)."""
    Wd = np.ascontiguousarray(W, dtype=np.float64)
    xd = np.ascontiguousarray(x, dtype=np.float64)
    T = None if Tx is None else np.ascontiguousarray(Tx, dtype=np.float64)
    out = np.zeros(4)
    sl = np.full(1, np.inf)
    (L or lib()).or_mlp_forward_bf16(_ptr(Wd, f64p), _ptr(xd, f64p), _ptr(T, f64p),
                                     _ptr(out, f64p), _ptr(sl, f64p))
    return out, float(sl[0])


def bf16_slack(v, T, L=None):
    """Distance of v from its nearest BF16 rounding boundary, in units of T."""
    return float((L or lib()).or_bf16_slack(float(v), float(T)))


class OrSystem(ctypes.Structure):
    _fields_ = [
        ("n_chains", ctypes.c_uint64),
        ("N", ctypes.c_uint32),
        ("N_A", ctypes.c_uint32),
        ("grid", ctypes.c_uint32 * 3),
        ("Re", ctypes.c_double),
        ("kappaN", ctypes.c_double),
        ("chiN", ctypes.c_double),
        ("a", ctypes.c_double),
        ("a32", ctypes.c_float),
        ("K_b", ctypes.c_double),
        ("rho_cell", ctypes.c_double),
        ("seed", ctypes.c_uint64),
        ("replica", ctypes.c_uint32),
        ("set_order", ctypes.c_int),
        ("move", ctypes.c_int),
        ("mlp", ctypes.c_void_p),
        ("chosen", ctypes.c_void_p),
        ("hamiltonian", ctypes.c_int),
        ("ext", ctypes.c_void_p),
        ("forbidden", ctypes.c_void_p),
        ("seq", ctypes.c_void_p),
        ("arch", ctypes.c_void_p),
        ("topo", ctypes.c_void_p),
        ("topo_start", ctypes.c_void_p),
        ("n_topo", ctypes.c_uint32),
        ("topo_set", ctypes.c_void_p),
        ("topo_nsets", ctypes.c_void_p),
        ("n_types", ctypes.c_uint32),
        ("chi_types", ctypes.c_double * 64),
        ("w_types", ctypes.c_void_p),
        ("mlp_bf16", ctypes.c_int),
        ("mlp_slack", ctypes.c_void_p),
    ]


class OrSweepStats(ctypes.Structure):
    _fields_ = [("attempted", ctypes.c_uint64), ("accepted", ctypes.c_uint64),
                ("near_ties", ctypes.c_uint64)]


class OrObs(ctypes.Structure):
    _fields_ = [("E_b", ctypes.c_double), ("E_nb", ctypes.c_double),
                ("Re2", ctypes.c_double), ("b2", ctypes.c_double), ("E_ext", ctypes.c_double)]


def lib():
    """Load liboracle.so (building it first if it is missing)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(_LIB_PATH):
        from . import build as _b
        _b.build()
    _lib = load(_LIB_PATH)
    return _lib


def load(path):
    """Load an oracle library from ``path`` (tests load mutated builds this way)."""
    L = ctypes.CDLL(path)
    P = ctypes.POINTER(OrSystem)
    L.or_philox4x32_10.argtypes = [u32p, u32p, u32p]
    L.or_draw.argtypes = [P, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_uint32, u32p]
    L.or_uniform_sym.argtypes = [ctypes.c_uint32]
    L.or_uniform_sym.restype = ctypes.c_double
    L.or_uniform_open.argtypes = [ctypes.c_uint32]
    L.or_uniform_open.restype = ctypes.c_double
    L.or_system_init.argtypes = [P, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_double,
                                 f64p, u32p, ctypes.c_double, ctypes.c_double,
                                 ctypes.c_double, ctypes.c_uint64, ctypes.c_uint32,
                                 ctypes.c_int, ctypes.c_int]
    L.or_system_init.restype = ctypes.c_int
    L.or_init_chain_range.argtypes = [P, ctypes.c_uint64, ctypes.c_uint64, f32p, f32p, f32p]
    L.or_histogram.argtypes = [P, f32p, f32p, f32p, u32p, u32p]
    L.or_fields.argtypes = [P, u32p, u32p, f64p, f64p, ctypes.c_int]
    L.or_sweep.argtypes = [P, f32p, f32p, f32p, f64p, f64p, ctypes.c_uint32,
                           ctypes.c_uint64, ctypes.c_uint64, f64p, u8p,
                           ctypes.POINTER(OrSweepStats)]
    L.or_sweep_trial.argtypes = [P, f32p, f32p, f32p, f64p, f64p, ctypes.c_uint32,
                                 ctypes.c_uint64, ctypes.c_uint64, f64p, u8p, f32p,
                                 ctypes.POINTER(OrSweepStats)]
    L.or_observables.argtypes = [P, f32p, f32p, f32p, u32p, u32p, ctypes.POINTER(OrObs)]
    L.or_structure_factor.argtypes = [P, u32p, u32p, i32p, ctypes.c_size_t, f64p]
    L.or_num_threads.restype = ctypes.c_int
    L.or_mlp_forward.argtypes = [f64p, f64p, f64p]
    L.or_set_mlp.argtypes = [P, f64p]
    L.or_mlp_forward_bf16.argtypes = [f64p, f64p, f64p, f64p, f64p]
    L.or_bf16_slack.argtypes = [ctypes.c_double, ctypes.c_double]
    L.or_bf16_slack.restype = ctypes.c_double
    L.or_learned_features.argtypes = [P, f32p, f32p, f32p, f64p, ctypes.c_uint64,
                                      ctypes.c_uint32, f64p, f64p]
    L.or_esjd_sample.argtypes = [P, f64p, f32p, f32p, f32p, f64p, f64p, ctypes.c_uint64,
                                 ctypes.c_uint32, f64p, f64p, f64p]
    L.or_esjd_sample.restype = ctypes.c_double
    L.or_chain_key.argtypes = [P, ctypes.c_float, ctypes.c_float, ctypes.c_float]
    L.or_chain_key.restype = ctypes.c_uint64
    L.or_sort_chains.argtypes = [P, f32p, f32p, f32p, ctypes.POINTER(ctypes.c_uint64)]
    L.or_topo_type.argtypes = [u32p, ctypes.c_uint32, ctypes.c_uint32]
    L.or_topo_type.restype = ctypes.c_uint32
    L.or_topo_partners.argtypes = [u32p, ctypes.c_uint32, ctypes.c_uint32, u32p, ctypes.c_uint32]
    L.or_topo_partners.restype = ctypes.c_uint32
    L.or_topology_sets.argtypes = [u32p, ctypes.c_uint32, u8p]
    L.or_topology_sets.restype = ctypes.c_uint32
    L.or_set_order.argtypes = [P, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32, u32p]
    L.or_type.argtypes = [P, ctypes.c_uint64, ctypes.c_uint32]
    L.or_type.restype = ctypes.c_uint32
    L.or_histogram_types.argtypes = [P, f32p, f32p, f32p, u32p]
    L.or_fields_types.argtypes = [P, u32p, f64p, ctypes.c_int]
    L.or_energy_types.argtypes = [P, u32p]
    L.or_energy_types.restype = ctypes.c_double
    return L


def _ptr(a, t):
    return a.ctypes.data_as(t) if a is not None else None


def philox(ctr, key, L=None):
    """Philox4x32-10 of one 4-word counter and 2-word key."""
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    (L or lib()).or_philox4x32_10(_ptr(c, u32p), _ptr(k, u32p), _ptr(out, u32p))
    return out


def uniform_sym(r, L=None):
    return (L or lib()).or_uniform_sym(int(r))


def uniform_open(r, L=None):
    return (L or lib()).or_uniform_open(int(r))


def topo_type(words, start, i, L=None):
    """Type (0 A, 1 B) of particle i of the architecture block at start."""
    w = np.ascontiguousarray(words, np.uint32)
    return int((L or lib()).or_topo_type(_ptr(w, u32p), int(start), int(i)))


def topo_partners(words, start, i, L=None):
    """Bond partners of particle i of the block at start, in list order."""
    w = np.ascontiguousarray(words, np.uint32)
    out = np.zeros(256, np.uint32)
    k = (L or lib()).or_topo_partners(_ptr(w, u32p), int(start), int(i), _ptr(out, u32p), 256)
    return [int(v) for v in out[:k]]


def topology_sets(words, start, L=None):
    """(set of every particle, number of sets) of the block at start."""
    w = np.ascontiguousarray(words, np.uint32)
    N = int(w[start])
    out = np.zeros(max(N, 1), np.uint8)
    n = (L or lib()).or_topology_sets(_ptr(w, u32p), int(start), _ptr(out, u8p))
    return out[:N], int(n)


def num_threads():
    return int(lib().or_num_threads())


@dataclass
class Positions:
    x: np.ndarray
    y: np.ndarray
    z: np.ndarray

    def copy(self):
        return Positions(self.x.copy(), self.y.copy(), self.z.copy())

    def stacked(self):
        return np.stack([self.x, self.y, self.z])


class System:
    """One oracle system: the parameters of an SCMF simulation of diblock melts."""

    def __init__(self, n_chains, N, f, box_Re, grid, chiN, kappaN, a_Re=0.0, seed=1,
                 replica=0, set_order=0, move=0, L=None):
        self.L = L or lib()
        self.s = OrSystem()
        box = (ctypes.c_double * 3)(*[float(v) for v in box_Re])
        g = (ctypes.c_uint32 * 3)(*[int(v) for v in grid])
        rc = self.L.or_system_init(ctypes.byref(self.s), int(n_chains), int(N), float(f),
                                  ctypes.cast(box, f64p), ctypes.cast(g, u32p),
                                  float(chiN), float(kappaN), float(a_Re), int(seed),
                                  int(replica), int(set_order), int(move))
        if rc != 0:
            raise ValueError("invalid oracle system")
        self.n_chains = int(n_chains)
        self.N = int(N)
        self.M = self.n_chains * self.N
        self.grid = tuple(int(v) for v in grid)
        self.cells = self.grid[0] * self.grid[1] * self.grid[2]

    @property
    def params(self):
        return self.s

    def draw(self, purpose, idx, w):
        out = np.zeros(4, dtype=np.uint32)
        self.L.or_draw(ctypes.byref(self.s), int(purpose), int(idx), int(w), _ptr(out, u32p))
        return out

    def empty_positions(self):
        return Positions(np.zeros(self.M, np.float32), np.zeros(self.M, np.float32),
                         np.zeros(self.M, np.float32))

    def init_chains(self, c0=0, c1=None, pos=None):
        c1 = self.n_chains if c1 is None else c1
        pos = self.empty_positions() if pos is None else pos
        self.L.or_init_chain_range(ctypes.byref(self.s), int(c0), int(c1),
                                  _ptr(pos.x, f32p), _ptr(pos.y, f32p), _ptr(pos.z, f32p))
        return pos

    def set_mlp(self, W, bf16=False):
        """Parameters of the learned proposal (move 2); kept alive here.
        bf16: evaluate the network in the BF16 reading of the tensor-core
        evaluators instead of in FP64."""
        self._mlp = np.ascontiguousarray(W, dtype=np.float64)
        assert self._mlp.size == MLP_PARAMS
        self.L.or_set_mlp(ctypes.byref(self.s), _ptr(self._mlp, f64p))
        self.s.mlp_bf16 = 1 if bf16 else 0

    def learned_features(self, pos, w_t, chain, i, r):
        f = np.zeros(12)
        rr = np.ascontiguousarray(r, dtype=np.float64)
        self.L.or_learned_features(ctypes.byref(self.s), _ptr(pos.x, f32p), _ptr(pos.y, f32p),
                                   _ptr(pos.z, f32p), _ptr(w_t, f64p), int(chain), int(i),
                                   _ptr(rr, f64p), _ptr(f, f64p))
        return f

    def esjd_sample(self, W, pos, wA, wB, chain, i, xi, want_grad=True):
        """(J, dJ/dW or None, log alpha) of one training sample."""
        Wd = np.ascontiguousarray(W, dtype=np.float64)
        g = np.zeros(MLP_PARAMS) if want_grad else None
        la = np.zeros(1)
        xid = np.ascontiguousarray(xi, dtype=np.float64)
        J = self.L.or_esjd_sample(ctypes.byref(self.s), _ptr(Wd, f64p), _ptr(pos.x, f32p),
                                  _ptr(pos.y, f32p), _ptr(pos.z, f32p), _ptr(wA, f64p),
                                  _ptr(wB, f64p), int(chain), int(i), _ptr(xid, f64p),
                                  _ptr(g, f64p), _ptr(la, f64p))
        return J, g, float(la[0])

    def chain_key(self, x0, y0, z0):
        return int(self.L.or_chain_key(ctypes.byref(self.s), float(x0), float(y0), float(z0)))

    def sort_chains(self, pos):
        """Re-label chains in spatial order in place; returns the old label of
        each new label."""
        perm = np.zeros(self.n_chains, np.uint64)
        self.L.or_sort_chains(ctypes.byref(self.s), _ptr(pos.x, f32p), _ptr(pos.y, f32p),
                              _ptr(pos.z, f32p), perm.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)))
        return perm

    def initial_state(self, sort=True):
        """The library's initial configuration: Gaussian chains, then (by
        default) the spatial labelling."""
        pos = self.init_chains()
        if sort:
            self.sort_chains(pos)
        return pos

    def histogram(self, pos):
        nA = np.zeros(self.cells, np.uint32)
        nB = np.zeros(self.cells, np.uint32)
        self.L.or_histogram(ctypes.byref(self.s), _ptr(pos.x, f32p), _ptr(pos.y, f32p),
                           _ptr(pos.z, f32p), _ptr(nA, u32p), _ptr(nB, u32p))
        return nA, nB

    def set_hamiltonian(self, k):
        """0: K^0_inter, 1: K^1_inter (Eq. hamil-pair)."""
        self.s.hamiltonian = int(k)

    def set_external(self, ext=None, forbidden=None):
        """External field per type and cell ((2, cells) kT per particle, added
        to omega) and cells no particle may enter (nonzero entries); None
        removes either.  Kept alive here."""
        self._ext = None if ext is None else np.ascontiguousarray(ext, np.float64).reshape(-1)
        self._forbidden = None if forbidden is None else np.ascontiguousarray(forbidden, np.uint8)
        assert self._ext is None or self._ext.size == 2 * self.cells
        assert self._forbidden is None or self._forbidden.size == self.cells
        self.s.ext = None if self._ext is None else self._ext.ctypes.data
        self.s.forbidden = None if self._forbidden is None else self._forbidden.ctypes.data

    def set_architectures(self, seq=None, arch=None):
        """Mixture of linear architectures: seq (n_arch uint64, bit i = particle
        i is B) and the architecture of every chain (n_chains uint8); None
        restores the diblock of N_A A particles.  Kept alive here."""
        if seq is None:
            self._seq = self._arch = None
            self.s.seq = self.s.arch = None
            return
        self.s.topo = None
        self._seq = np.ascontiguousarray(seq, np.uint64)
        self._arch = np.ascontiguousarray(arch, np.uint8)
        assert self._arch.size == self.n_chains and self._arch.max() < self._seq.size
        self.s.seq = self._seq.ctypes.data
        self.s.arch = self._arch.ctypes.data

    def set_topology(self, words=None, starts=None, arch=None):
        """Molecular architectures in the array layout of Sec. 3.2.1: words
        (uint32), the first word of each architecture's block (starts), and the
        architecture of every molecule (n_chains uint8).  The independent sets
        are generated here by the oracle's own heuristic.  None restores the
        diblock.  Kept alive here."""
        if words is None:
            self._topo = self._topo_start = self._arch = self._topo_set = self._topo_nsets = None
            self.s.topo = self.s.topo_start = self.s.arch = None
            self.s.topo_set = self.s.topo_nsets = None
            self.s.n_topo = 0
            self.s.rho_cell = float(self.M) / self.cells
            return
        # the learned proposal's features are those of a linear chain
        assert int(self.s.move) != 2, "architectures take the uniform or smart Monte Carlo move"
        self._topo = np.ascontiguousarray(words, np.uint32)
        self._topo_start = np.ascontiguousarray(starts, np.uint32)
        self._arch = np.ascontiguousarray(arch, np.uint8)
        na = self._topo_start.size
        assert self._arch.size == self.n_chains and int(self._arch.max()) < na
        # absent slots (past an architecture's n particles) belong to no set
        self._topo_set = np.full(na * self.N, 0xFF, np.uint8)
        self._topo_nsets = np.zeros(na, np.uint8)
        lengths = np.zeros(na, np.int64)
        for a in range(na):
            n_a = int(self._topo[self._topo_start[a]])
            assert 1 <= n_a <= self.N
            lengths[a] = n_a
            sets, n = topology_sets(self._topo, self._topo_start[a], self.L)
            assert 1 <= n <= 8
            self._topo_set[a * self.N:a * self.N + n_a] = sets
            self._topo_nsets[a] = n
        self.s.seq = None
        self._seq = None
        self.s.topo = self._topo.ctypes.data
        self.s.topo_start = self._topo_start.ctypes.data
        self.s.n_topo = na
        self.s.topo_set = self._topo_set.ctypes.data
        self.s.topo_nsets = self._topo_nsets.ctypes.data
        self.s.arch = self._arch.ctypes.data
        # rho_0 dL^3 counts the molecules' particles, absent slots excluded
        self.s.rho_cell = float(lengths[self._arch].sum()) / self.cells

    def set_types(self, n_types=0, chiN=None):
        """n_t particle types (types from the architecture array's type
        bytes): chiN is the n_t x n_t matrix of chi_ij N (symmetric, zero
        diagonal).  n_types 0 returns to the two types A, B."""
        self.s.n_types = int(n_types)
        for k in range(64):
            self.s.chi_types[k] = 0.0
        if n_types:
            c = np.asarray(chiN, np.float64).reshape(n_types, n_types)
            assert 2 <= n_types <= 8 and np.allclose(c, c.T) and np.all(np.diag(c) == 0)
            for i in range(n_types):
                for j in range(n_types):
                    self.s.chi_types[i * 8 + j] = float(c[i, j])

    def type_of(self, chain, i):
        return int(self.L.or_type(ctypes.byref(self.s), int(chain), int(i)))

    def histogram_types(self, pos):
        n = np.zeros((self.s.n_types, self.cells), np.uint32)
        self.L.or_histogram_types(ctypes.byref(self.s), _ptr(pos.x, f32p), _ptr(pos.y, f32p),
                                  _ptr(pos.z, f32p), _ptr(n, u32p))
        return n

    def fields_types(self, n, round_mode=0):
        nn = np.ascontiguousarray(n, np.uint32)
        w = np.zeros((self.s.n_types, self.cells), np.float64)
        self.L.or_fields_types(ctypes.byref(self.s), _ptr(nn, u32p), _ptr(w, f64p), int(round_mode))
        return w

    def energy_types(self, n):
        nn = np.ascontiguousarray(n, np.uint32)
        return float(self.L.or_energy_types(ctypes.byref(self.s), _ptr(nn, u32p)))

    def observables_types(self, pos, n):
        """Observables with n_t types: the bond part as observables(), E_nb of
        the types' energy, no external energy."""
        z = np.zeros(self.cells, np.uint32)
        o = self.observables(pos, z, z)
        o["E_nb"] = self.energy_types(n)
        o["E_ext"] = 0.0
        o["E_tot"] = o["E_b"] + o["E_nb"]
        return o

    def set_order(self, chain, sweep, n_sets):
        """Order in which molecule chain visits its n_sets sets in a sweep."""
        out = np.zeros(8, np.uint32)
        self.L.or_set_order(ctypes.byref(self.s), int(chain), int(sweep), int(n_sets),
                            _ptr(out, u32p))
        return [int(v) for v in out[:n_sets]]

    def fields(self, nA, nB, round_mode=0):
        wA = np.zeros(self.cells, np.float64)
        wB = np.zeros(self.cells, np.float64)
        self.L.or_fields(ctypes.byref(self.s), _ptr(nA, u32p), _ptr(nB, u32p),
                        _ptr(wA, f64p), _ptr(wB, f64p), int(round_mode))
        return wA, wB

    def sweep(self, pos, wA, wB, sweep, c0=0, c1=None, want_margin=False, want_acc=False,
              want_trial=False, want_chosen=False, w_types=None, want_slack=False):
        """One MC step in place; returns (stats, margin or None, accepted or
        None), plus the (3, M) trial positions when want_trial and the chosen
        particle of every attempt when want_chosen (molecule-parallel
        iteration, set_order 2; margin, accepted and trial are then indexed by
        attempt k*N + j instead of by particle)."""
        c1 = self.n_chains if c1 is None else c1
        margin = np.full(self.M, np.nan) if want_margin else None
        acc = np.zeros(self.M, np.uint8) if want_acc else None
        trial = np.full(3 * self.M, np.nan, np.float32) if want_trial else None
        chosen = np.zeros(self.M, np.uint32) if want_chosen else None
        self.s.chosen = chosen.ctypes.data if want_chosen else None
        slack = np.full(self.M, np.inf) if want_slack else None
        self.s.mlp_slack = slack.ctypes.data if want_slack else None
        if w_types is not None:   # the n_t field planes, (n_types, cells)
            planes = [np.ascontiguousarray(w_types[t], np.float64) for t in range(len(w_types))]
            ptrs = (ctypes.c_void_p * len(planes))(*[q.ctypes.data for q in planes])
            self.s.w_types = ctypes.cast(ptrs, ctypes.c_void_p)
            if wA is None:
                wA = wB = planes[0]
        st = OrSweepStats()
        try:
            self.L.or_sweep_trial(ctypes.byref(self.s), _ptr(pos.x, f32p), _ptr(pos.y, f32p),
                                  _ptr(pos.z, f32p), _ptr(wA, f64p), _ptr(wB, f64p), int(sweep),
                                  int(c0), int(c1), _ptr(margin, f64p), _ptr(acc, u8p),
                                  _ptr(trial, f32p), ctypes.byref(st))
        finally:
            self.s.chosen = None
            self.s.w_types = None
            self.s.mlp_slack = None
        out = (st, margin, acc)
        if want_trial:
            out = out + (trial.reshape(3, self.M),)
        if want_chosen:
            out = out + (chosen,)
        if want_slack:
            out = out + (slack,)
        return out

    def observables(self, pos, nA, nB):
        o = OrObs()
        self.L.or_observables(ctypes.byref(self.s), _ptr(pos.x, f32p), _ptr(pos.y, f32p),
                             _ptr(pos.z, f32p), _ptr(nA, u32p), _ptr(nB, u32p),
                             ctypes.byref(o))
        return {"E_b": o.E_b, "E_nb": o.E_nb, "E_ext": o.E_ext,
                "E_tot": o.E_b + o.E_nb + o.E_ext, "Re2": o.Re2, "b2": o.b2}

    def structure_factor(self, nA, nB, m):
        mm = np.ascontiguousarray(np.asarray(m, dtype=np.int32).reshape(-1, 3))
        out = np.zeros(len(mm), np.float64)
        self.L.or_structure_factor(ctypes.byref(self.s), _ptr(nA, u32p), _ptr(nB, u32p),
                                  _ptr(mm, i32p), len(mm), _ptr(out, f64p))
        return out
