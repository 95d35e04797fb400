"""GB300-native SCMF Monte-Carlo for soft coarse-grained diblock melts
(arXiv:1711.03828, "SOMA").

The compute path is ``libsoma.so`` (hand-written sm_103a CUDA behind the C ABI
of ``include/soma.h``); this package holds its ctypes binding (``_abi``, same
names as the C entry points) and ``System``, a thin owner of one handle that
marshals torch tensors and numpy arrays.  PyTorch is used only for device
memory and the CUDA stream.
"""
from __future__ import annotations

import ctypes
from dataclasses import dataclass, field

import numpy as np

from . import _abi
from ._abi import (FLAG_LEARNED_FP32, FLAG_LEARNED_UMMA, FLAG_NO_SORT, GRID_BF16, GRID_F16, GRID_F32, MLP_PARAMS, MOVE_LEARNED,
                   MOVE_SMC, MOVE_UNIFORM, SET_ORDER_FIXED, SET_ORDER_RANDOM, ITERATION_MOLECULE,
                   SomaError)

__all__ = ["SystemDesc", "System", "Batch", "SomaError", "FLAG_NO_SORT", "FLAG_LEARNED_FP32", "FLAG_LEARNED_UMMA", "MOVE_UNIFORM", "MOVE_SMC", "MOVE_LEARNED", "MLP_PARAMS", "SET_ORDER_RANDOM",
           "SET_ORDER_FIXED", "ITERATION_MOLECULE", "GRID_F32", "GRID_BF16", "GRID_F16",
           "topology_sets"]


@dataclass
class SystemDesc:
    """Python mirror of ``soma_system_desc``."""
    n_chains: int
    N: int
    f: float = 0.5
    box_Re: tuple = (2.0, 2.0, 2.0)
    grid: tuple = (12, 12, 12)
    chiN: float = 20.0
    kappaN: float = 50.0
    a_Re: float = 0.0
    move: int = MOVE_UNIFORM
    set_order: int = SET_ORDER_RANDOM
    grid_dtype: int = GRID_F32
    seed: int = 1
    replica_id: int = 0
    flags: int = 0
    hamiltonian: int = 0
    chain_offset: int = 0      # chain sharding: this handle holds chains
    n_chains_total: int = 0    # [chain_offset, chain_offset + n_chains) of n_chains_total

    @property
    def M(self):
        return self.n_chains * self.N

    @property
    def cells(self):
        return int(self.grid[0]) * int(self.grid[1]) * int(self.grid[2])

    def to_c(self, stream=None):
        d = _abi.SomaSystemDesc()
        d.struct_size = ctypes.sizeof(_abi.SomaSystemDesc)
        d.N = int(self.N)
        d.n_chains = int(self.n_chains)
        d.f = float(self.f)
        for k in range(3):
            d.box_Re[k] = float(self.box_Re[k])
            d.grid[k] = int(self.grid[k])
        d.chiN = float(self.chiN)
        d.kappaN = float(self.kappaN)
        d.a_Re = float(self.a_Re)
        d.move = int(self.move)
        d.set_order = int(self.set_order)
        d.grid_dtype = int(self.grid_dtype)
        d.flags = int(self.flags)
        d.hamiltonian = int(self.hamiltonian)
        d.seed = int(self.seed)
        d.replica_id = int(self.replica_id)
        d.stream = stream
        d.chain_offset = int(self.chain_offset)
        d.n_chains_total = int(self.n_chains_total)
        return d


def _torch_stream_handle(stream):
    if stream is None:
        return None
    return ctypes.c_void_p(int(stream.cuda_stream))


def topology_sets(words, starts, N):
    """The library's check and independent sets of an architecture array
    (soma_topology_sets, host only): returns (sets (n_arch, N) uint8, number
    of sets per architecture); raises SomaError for an array soma_set_topology
    would refuse."""
    w = np.ascontiguousarray(words, dtype=np.uint32).reshape(-1)
    st = np.ascontiguousarray(starts, dtype=np.uint32).reshape(-1)
    sets = np.zeros((st.size, N), np.uint8)
    ns = np.zeros(st.size, np.uint8)
    _abi.soma_topology_sets(w.ctypes.data, w.size, st.ctypes.data, st.size, N, sets.ctypes.data,
                            ns.ctypes.data)
    return sets, ns


class System:
    """One SCMF system on the GPU (owns a ``soma_t``, or borrows one from a Batch).

    stream: the torch CUDA stream the handle runs on.  None -- or torch's
    default stream, whose handle is NULL -- gives the handle a stream of its
    own, which torch's operations are not ordered with: synchronise (or pass
    a stream of your own) before torch reads what the handle wrote."""

    def __init__(self, desc: SystemDesc, stream=None, _borrowed=None):
        self.desc = desc
        self._stream_obj = stream
        self.n_types = 0
        if _borrowed is not None:
            self.h = _borrowed
            self._owner = False
            return
        h = ctypes.c_void_p()
        c = desc.to_c(_torch_stream_handle(stream))
        _abi.soma_create(ctypes.byref(c), ctypes.byref(h))
        self.h = h
        self._owner = True

    # -- lifetime ---------------------------------------------------------
    def close(self):
        if getattr(self, "h", None) is not None and self.h.value and getattr(self, "_owner", True):
            _abi.soma_destroy(self.h)
        self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # -- the SCMF cycle ---------------------------------------------------
    def sweep(self, n=1):
        _abi.soma_sweep(self.h, int(n))

    def update_fields(self):
        _abi.soma_update_fields(self.h)

    def sync(self):
        _abi.soma_sync(self.h)

    # -- chain sharding (one exchange of occupation numbers per cycle) -----
    def _counts_arg(self, buf):
        cells = self.desc.cells
        if isinstance(buf, np.ndarray):
            assert buf.dtype == np.uint32 and buf.size == cells and buf.flags.c_contiguous
            return ctypes.c_void_p(buf.ctypes.data), cells
        assert buf.is_contiguous() and buf.numel() == cells and buf.element_size() == 4
        return ctypes.c_void_p(buf.data_ptr()), cells

    def shard_counts(self, buf):
        """Packed occupation numbers of this shard's particles into buf
        (cells uint32/int32: numpy array or tensor); soma_shard_counts."""
        _abi.soma_shard_counts(self.h, *self._counts_arg(buf))

    def shard_sweep(self, buf):
        """MC step of this shard's particles; their packed counts into buf."""
        _abi.soma_shard_sweep(self.h, *self._counts_arg(buf))

    def shard_fields(self, summed):
        """Fields from the counts summed over every shard; ends the cycle."""
        _abi.soma_shard_fields(self.h, *self._counts_arg(summed))

    # -- state access -----------------------------------------------------
    def get_positions(self, out=None):
        """SoA positions (3, M) float32: numpy by default, or into a CUDA tensor."""
        M = self.desc.M
        if out is None:
            a = np.empty(3 * M, np.float32)
            _abi.soma_get_positions(self.h, a.ctypes.data, a.size, 0)
            return a.reshape(3, M)
        _abi.soma_get_positions(self.h, ctypes.c_void_p(out.data_ptr()), out.numel(), 1)
        return out

    def set_positions(self, pos):
        """pos: (3, M) float32 numpy array or CUDA tensor."""
        M = self.desc.M
        if isinstance(pos, np.ndarray):
            a = np.ascontiguousarray(pos, dtype=np.float32).reshape(-1)
            assert a.size == 3 * M
            _abi.soma_set_positions(self.h, a.ctypes.data, a.size, 0)
        else:
            assert pos.is_contiguous() and pos.numel() == 3 * M
            _abi.soma_set_positions(self.h, ctypes.c_void_p(pos.data_ptr()), pos.numel(),
                                    1 if pos.is_cuda else 0)

    def set_external(self, ext=None, forbidden=None):
        """External potential ext ((2, cells) float32: A then B, kT per
        particle) and forbidden cells ((cells,) nonzero = closed); numpy
        arrays or CUDA tensors; None removes that field."""
        cells = self.desc.cells
        keep = []

        def arg(a, dtype, n):
            if a is None:
                return None, 0
            if isinstance(a, np.ndarray):
                b = np.ascontiguousarray(a, dtype=dtype).reshape(-1)
                assert b.size == n
                keep.append(b)
                return ctypes.c_void_p(b.ctypes.data), 0
            assert a.is_contiguous() and a.numel() == n
            return ctypes.c_void_p(a.data_ptr()), 1 if a.is_cuda else 0

        e, on_e = arg(ext, np.float32, 2 * cells)
        f, on_f = arg(forbidden, np.uint8, cells)
        if e is not None and f is not None:
            assert on_e == on_f, "ext and forbidden must both be host or both device arrays"
        _abi.soma_set_external(self.h, e, f, on_e or on_f)

    def set_architectures(self, seq=None, arch=None):
        """Mixture of linear architectures: seq (n_arch uint64, bit i set =
        particle i is B) and the architecture of every chain (n_chains uint8);
        seq None returns to the diblock of the description."""
        if seq is None:
            _abi.soma_set_architectures(self.h, None, 0, None, 0)
            return
        q = np.ascontiguousarray(seq, dtype=np.uint64).reshape(-1)
        a = np.ascontiguousarray(arch, dtype=np.uint8).reshape(-1)
        assert a.size == self.desc.n_chains
        _abi.soma_set_architectures(self.h, q.ctypes.data, q.size, a.ctypes.data, 0)

    def set_topology(self, words=None, starts=None, mol_arch=None):
        """Molecules of any architecture: the architecture array of Sec. 3.2.1
        (words, uint32; see workloads.encode_architectures), the first word
        of each architecture's block (starts) and the architecture of every
        molecule (n_chains uint8); words None returns to the diblock."""
        if words is None:
            _abi.soma_set_topology(self.h, None, 0, None, 0, None, 0)
            return
        w = np.ascontiguousarray(words, dtype=np.uint32).reshape(-1)
        st = np.ascontiguousarray(starts, dtype=np.uint32).reshape(-1)
        a = np.ascontiguousarray(mol_arch, dtype=np.uint8).reshape(-1)
        assert a.size == self.desc.n_chains
        _abi.soma_set_topology(self.h, w.ctypes.data, w.size, st.ctypes.data, st.size,
                               a.ctypes.data, 0)

    def set_types(self, n_types=0, chiN=None):
        """n_t particle types (2..8) with the n_t x n_t matrix chiN of chi_ij N;
        types come from the architecture array.  0 returns to A, B."""
        if not n_types:
            _abi.soma_set_types(self.h, 0, None)
            self.n_types = 0
            return
        c = np.ascontiguousarray(chiN, dtype=np.float64).reshape(n_types, n_types)
        _abi.soma_set_types(self.h, int(n_types), c.ctypes.data)
        self.n_types = int(n_types)

    def structure_factor_types(self, ti, tj, m):
        """S_ij(q) of the composition n_ti - n_tj for wave-vector indices m
        (k x 3)."""
        mm = np.ascontiguousarray(np.asarray(m, dtype=np.int32).reshape(-1, 3))
        out = np.zeros(len(mm), np.float64)
        _abi.soma_structure_factor_types(self.h, int(ti), int(tj), mm.ctypes.data, len(mm),
                                         out.ctypes.data)
        return out

    def get_type_counts(self):
        """Occupation numbers per type, (n_types, cells) uint32."""
        out = np.empty((self.n_types, self.desc.cells), np.uint32)
        _abi.soma_get_type_counts(self.h, out.ctypes.data, out.size, 0)
        return out

    def get_type_fields(self):
        """Fields per type, (n_types, cells) float32."""
        out = np.empty((self.n_types, self.desc.cells), np.float32)
        _abi.soma_get_type_fields(self.h, out.ctypes.data, out.size, 0)
        return out

    def sort_molecules(self):
        """Relabel the molecules in spatial (Morton) order of their particle 0;
        returns the previous label of each new label (n_chains uint64)."""
        perm = np.zeros(self.desc.n_chains, np.uint64)
        _abi.soma_sort_molecules(self.h, perm.ctypes.data)
        return perm

    def get_density(self, out=None):
        """Packed occupation numbers (cells,) uint32: n_A | n_B << 16."""
        cells = self.desc.cells
        if out is None:
            a = np.empty(cells, np.uint32)
            _abi.soma_get_density(self.h, a.ctypes.data, cells, 0)
            return a
        _abi.soma_get_density(self.h, ctypes.c_void_p(out.data_ptr()), cells, 1)
        return out

    def get_density_ab(self):
        n = self.get_density()
        return (n & 0xFFFF).astype(np.uint32), (n >> 16).astype(np.uint32)

    def get_fields(self):
        """omega_A, omega_B as float32 arrays of cells entries."""
        cells = self.desc.cells
        a = np.empty(2 * cells, np.float32)
        _abi.soma_get_fields(self.h, a.ctypes.data, a.size, 0)
        return a[:cells], a[cells:]

    def observables(self):
        o = _abi.SomaObs()
        _abi.soma_observables(self.h, ctypes.byref(o))
        return {k: getattr(o, k) for k, _ in _abi.SomaObs._fields_ if k != "reserved"}

    def parameters(self):
        """Derived parameters (lengths in dL, energies in kT), incl. the SCMF
        accuracy parameter epsilon and sqrt(Nbar)."""
        p = _abi.SomaParams()
        _abi.soma_get_parameters(self.h, ctypes.byref(p))
        return {k: getattr(p, k) for k, _ in _abi.SomaParams._fields_}

    def structure_factor(self, m):
        mm = np.ascontiguousarray(np.asarray(m, dtype=np.int32).reshape(-1, 3))
        out = np.zeros(len(mm), np.float64)
        _abi.soma_structure_factor(self.h, mm.ctypes.data, len(mm), out.ctypes.data)
        return out

    @property
    def sweep_count(self):
        v = ctypes.c_uint64()
        _abi.soma_get_sweep(self.h, ctypes.byref(v))
        return v.value

    def set_sweep(self, s):
        _abi.soma_set_sweep(self.h, int(s))

    def set_timing(self, on=True):
        _abi.soma_set_timing(self.h, 1 if on else 0)

    def timing(self):
        t = _abi.SomaTiming()
        _abi.soma_get_timing(self.h, ctypes.byref(t))
        return {k: getattr(t, k) for k, _ in _abi.SomaTiming._fields_}

    @property
    def stream_handle(self):
        return _abi.soma_stream(self.h)

    # -- learned proposal -------------------------------------------------
    def set_proposal_weights(self, w):
        a = np.ascontiguousarray(w, dtype=np.float32)
        assert a.size == MLP_PARAMS
        _abi.soma_proposal_set_weights(self.h, a.ctypes.data, a.size, 0)

    def get_proposal_weights(self):
        a = np.empty(MLP_PARAMS, np.float32)
        _abi.soma_proposal_get_weights(self.h, a.ctypes.data, a.size, 0)
        return a

    def proposal_grad(self, samples, xi, w=None):
        """(grad sum, J, log_alpha) of given samples (n x 2 uint32 (chain, i))
        and normals (n x 3), as torch CUDA tensors."""
        import torch
        dev = torch.device("cuda")
        s_ = torch.as_tensor(np.ascontiguousarray(samples, dtype=np.uint32).view(np.int32),
                             device=dev).contiguous()
        x_ = torch.as_tensor(np.ascontiguousarray(xi, dtype=np.float32), device=dev).contiguous()
        n = s_.numel() // 2
        g = torch.empty(MLP_PARAMS, dtype=torch.float32, device=dev)
        J = torch.empty(n, dtype=torch.float32, device=dev)
        la = torch.empty(n, dtype=torch.float32, device=dev)
        wp = None
        if w is not None:
            w_ = torch.as_tensor(np.ascontiguousarray(w, dtype=np.float32), device=dev)
            wp = ctypes.c_void_p(w_.data_ptr())
        _abi.soma_proposal_grad(self.h, wp, ctypes.c_void_p(s_.data_ptr()),
                                ctypes.c_void_p(x_.data_ptr()), n, ctypes.c_void_p(g.data_ptr()),
                                ctypes.c_void_p(J.data_ptr()), ctypes.c_void_p(la.data_ptr()))
        self.sync()
        return g.cpu().numpy(), J.cpu().numpy(), la.cpu().numpy()

    def train_proposal(self, steps=200, batch=4096, sweeps_between=1, lr=1e-3, beta1=0.9,
                       beta2=0.999, eps=1e-8):
        c = _abi.SomaTrainCfg(steps, batch, sweeps_between, lr, beta1, beta2, eps)
        lg = _abi.SomaTrainLog()
        _abi.soma_proposal_train(self.h, ctypes.byref(c), ctypes.byref(lg))
        return {"mean_J_first": lg.mean_J_first, "mean_J_last": lg.mean_J_last,
                "mean_alpha_last": lg.mean_alpha_last, "steps": lg.steps_done}


def batch_plan(member_tiles, grid, item_tiles=0):
    """The batched sweep's work items (``soma_batch_plan``, host only): rows
    (member, first tile, end tile); block j takes rows j, j + grid, ..."""
    import numpy as np
    nt = np.ascontiguousarray(member_tiles, dtype=np.uint32)
    n = ctypes.c_size_t()
    _abi.soma_batch_plan(nt.ctypes.data, len(nt), int(grid), int(item_tiles), None, 0, ctypes.byref(n))
    out = np.zeros((n.value, 3), dtype=np.uint32)
    _abi.soma_batch_plan(nt.ctypes.data, len(nt), int(grid), int(item_tiles), out.ctypes.data,
                         n.value, ctypes.byref(n))
    return out


class Batch:
    """Many independent systems advanced by one sweep launch and one field
    launch per cycle (``soma_batch_*``)."""

    def __init__(self, descs, stream=None):
        self.descs = list(descs)
        arr = (_abi.SomaSystemDesc * len(self.descs))(*[d.to_c() for d in self.descs])
        h = ctypes.c_void_p()
        _abi.soma_batch_create(arr, len(self.descs), _torch_stream_handle(stream), ctypes.byref(h))
        self.h = h
        self.members = []
        for i, d in enumerate(self.descs):
            m = ctypes.c_void_p()
            _abi.soma_batch_system(self.h, i, ctypes.byref(m))
            self.members.append(System(d, _borrowed=m))

    def close(self):
        if getattr(self, "h", None) is not None and self.h.value:
            for m in self.members:
                m.h = None
            _abi.soma_batch_destroy(self.h)
        self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def sweep(self, n=1):
        _abi.soma_batch_sweep(self.h, int(n))

    def sync(self):
        _abi.soma_batch_sync(self.h)

    def autotune(self, cycles_per_candidate=3):
        tab = (_abi.SomaTuneEntry * 64)()
        nw = ctypes.c_uint32()
        _abi.soma_batch_autotune(self.h, int(cycles_per_candidate), tab, 64, ctypes.byref(nw))
        return [dict(block=t.block, blocks_per_sm=t.blocks_per_sm, item_tiles=t.item_tiles,
                     ms_per_cycle=t.ms_per_cycle) for t in tab[:nw.value]]

    def set_shape(self, block, blocks_per_sm, item_tiles):
        """Launch shape of the batched sweep (item_tiles 0: one equal
        contiguous range of tiles per block)."""
        t = _abi.SomaTuneEntry(block=int(block), blocks_per_sm=int(blocks_per_sm),
                               item_tiles=int(item_tiles))
        _abi.soma_batch_set_shape(self.h, ctypes.byref(t))

    def shape(self):
        t = _abi.SomaTuneEntry()
        _abi.soma_batch_get_shape(self.h, ctypes.byref(t))
        return dict(block=t.block, blocks_per_sm=t.blocks_per_sm, item_tiles=t.item_tiles)

    def set_timing(self, on=True):
        _abi.soma_batch_set_timing(self.h, 1 if on else 0)

    def timing(self):
        t = _abi.SomaTiming()
        _abi.soma_batch_get_timing(self.h, ctypes.byref(t))
        return {k: getattr(t, k) for k, _ in _abi.SomaTiming._fields_}

    @property
    def M(self):
        return sum(d.M for d in self.descs)
