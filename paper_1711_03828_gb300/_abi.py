"""ctypes binding of libsoma (include/soma.h): argument marshalling only.

Every entry point of the C ABI is exposed under its own name; ``SomaError`` is
raised for any non-zero status with the library's message.  There is no
fallback: if ``libsoma.so`` is missing the import fails loudly.
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libsoma.so")

SOMA_OK, SOMA_EINVAL, SOMA_ENOMEM, SOMA_ECUDA, SOMA_EOVERFLOW, SOMA_ETIMEOUT, SOMA_ESTATE = (
    0, -1, -2, -3, -4, -5, -6)
MOVE_UNIFORM, MOVE_SMC, MOVE_LEARNED = 0, 1, 2
MLP_PARAMS = 1604
SET_ORDER_RANDOM, SET_ORDER_FIXED, ITERATION_MOLECULE = 0, 1, 2
GRID_F32, GRID_BF16, GRID_F16 = 0, 1, 2
FLAG_NO_SORT = 1
FLAG_LEARNED_FP32 = 2
FLAG_LEARNED_UMMA = 4


class SomaSystemDesc(ctypes.Structure):
    _fields_ = [
        ("struct_size", ctypes.c_uint32),
        ("N", ctypes.c_uint32),
        ("n_chains", ctypes.c_uint64),
        ("f", ctypes.c_double),
        ("box_Re", ctypes.c_double * 3),
        ("grid", ctypes.c_uint32 * 3),
        ("hamiltonian", ctypes.c_uint32),
        ("chiN", ctypes.c_double),
        ("kappaN", ctypes.c_double),
        ("a_Re", ctypes.c_double),
        ("move", ctypes.c_int32),
        ("set_order", ctypes.c_int32),
        ("grid_dtype", ctypes.c_int32),
        ("flags", ctypes.c_int32),
        ("seed", ctypes.c_uint64),
        ("replica_id", ctypes.c_uint32),
        ("reserved1", ctypes.c_uint32),
        ("stream", ctypes.c_void_p),
        ("chain_offset", ctypes.c_uint64),
        ("n_chains_total", ctypes.c_uint64),
    ]


class SomaObs(ctypes.Structure):
    _fields_ = [
        ("E_b", ctypes.c_double), ("E_nb", ctypes.c_double), ("E_tot", ctypes.c_double),
        ("Re2", ctypes.c_double), ("Re2_rel", ctypes.c_double), ("b2", ctypes.c_double),
        ("accepted", ctypes.c_uint64), ("attempted", ctypes.c_uint64),
        ("sweeps", ctypes.c_uint64), ("max_cell", ctypes.c_uint32),
        ("reserved", ctypes.c_uint32), ("E_ext", ctypes.c_double),
    ]


class SomaParams(ctypes.Structure):
    _fields_ = [
        ("Re", ctypes.c_double), ("a", ctypes.c_double), ("K_b", ctypes.c_double),
        ("b0", ctypes.c_double), ("rho_cell", ctypes.c_double), ("sqrt_Nbar", ctypes.c_double),
        ("epsilon", ctypes.c_double), ("M", ctypes.c_uint64), ("cells", ctypes.c_uint32),
        ("N_A", ctypes.c_uint32),
    ]


class SomaTiming(ctypes.Structure):
    _fields_ = [
        ("ms_sweep", ctypes.c_double), ("ms_fields", ctypes.c_double),
        ("sweep_launches", ctypes.c_uint64), ("field_launches", ctypes.c_uint64),
        ("kernel_launches", ctypes.c_uint64),
    ]


class SomaTuneEntry(ctypes.Structure):
    _fields_ = [("block", ctypes.c_int32), ("blocks_per_sm", ctypes.c_int32),
                ("item_tiles", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("ms_per_cycle", ctypes.c_double)]


class SomaTrainCfg(ctypes.Structure):
    _fields_ = [("steps", ctypes.c_uint32), ("batch", ctypes.c_uint32),
                ("sweeps_between", ctypes.c_uint32), ("lr", ctypes.c_float),
                ("beta1", ctypes.c_float), ("beta2", ctypes.c_float), ("eps", ctypes.c_float)]


class SomaTrainLog(ctypes.Structure):
    _fields_ = [("mean_J_first", ctypes.c_double), ("mean_J_last", ctypes.c_double),
                ("mean_alpha_last", ctypes.c_double), ("steps_done", ctypes.c_uint32),
                ("reserved", ctypes.c_uint32)]


class SomaError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"soma status {status}: {msg}")
        self.status = status


_lib = None

_c = ctypes
_P = ctypes.c_void_p
_SIGS = {
    "soma_abi_version": ([], _c.c_int),
    "soma_last_error": ([], _c.c_char_p),
    "soma_create": ([_c.POINTER(SomaSystemDesc), _c.POINTER(_P)], _c.c_int),
    "soma_destroy": ([_P], _c.c_int),
    "soma_sweep": ([_P, _c.c_uint32], _c.c_int),
    "soma_update_fields": ([_P], _c.c_int),
    "soma_shard_counts": ([_P, _P, _c.c_size_t], _c.c_int),
    "soma_shard_sweep": ([_P, _P, _c.c_size_t], _c.c_int),
    "soma_shard_fields": ([_P, _P, _c.c_size_t], _c.c_int),
    "soma_get_density": ([_P, _P, _c.c_size_t, _c.c_int], _c.c_int),
    "soma_get_fields": ([_P, _P, _c.c_size_t, _c.c_int], _c.c_int),
    "soma_get_positions": ([_P, _P, _c.c_size_t, _c.c_int], _c.c_int),
    "soma_set_positions": ([_P, _P, _c.c_size_t, _c.c_int], _c.c_int),
    "soma_set_external": ([_P, _P, _P, _c.c_int], _c.c_int),
    "soma_set_architectures": ([_P, _P, _c.c_uint32, _P, _c.c_int], _c.c_int),
    "soma_set_topology": ([_P, _P, _c.c_uint64, _P, _c.c_uint32, _P, _c.c_int], _c.c_int),
    "soma_topology_sets": ([_P, _c.c_uint64, _P, _c.c_uint32, _c.c_uint32, _P, _P], _c.c_int),
    "soma_sort_molecules": ([_P, _P], _c.c_int),
    "soma_set_types": ([_P, _c.c_uint32, _P], _c.c_int),
    "soma_structure_factor_types": ([_P, _c.c_uint32, _c.c_uint32, _P, _c.c_size_t, _P], _c.c_int),
    "soma_get_type_counts": ([_P, _P, _c.c_size_t, _c.c_int], _c.c_int),
    "soma_get_type_fields": ([_P, _P, _c.c_size_t, _c.c_int], _c.c_int),
    "soma_get_parameters": ([_P, _P], _c.c_int),
    "soma_check_bounded_wait": ([_c.c_uint32, _P], _c.c_int),
    "soma_observables": ([_P, _c.POINTER(SomaObs)], _c.c_int),
    "soma_structure_factor": ([_P, _P, _c.c_size_t, _P], _c.c_int),
    "soma_get_sweep": ([_P, _c.POINTER(_c.c_uint64)], _c.c_int),
    "soma_set_sweep": ([_P, _c.c_uint64], _c.c_int),
    "soma_set_timing": ([_P, _c.c_int], _c.c_int),
    "soma_get_timing": ([_P, _c.POINTER(SomaTiming)], _c.c_int),
    "soma_sync": ([_P], _c.c_int),
    "soma_stream": ([_P], _P),
    "soma_philox": ([_P, _P, _P, _c.c_size_t, _P], _c.c_int),
    "soma_smc_draws": ([_P, _P, _c.c_size_t, _P], _c.c_int),
    "soma_structure_factor_noalloc": ([_c.POINTER(SomaSystemDesc), _P, _P, _c.c_size_t, _P, _P],
                                      _c.c_int),
    "soma_proposal_set_weights": ([_P, _P, _c.c_size_t, _c.c_int], _c.c_int),
    "soma_proposal_get_weights": ([_P, _P, _c.c_size_t, _c.c_int], _c.c_int),
    "soma_proposal_grad": ([_P, _P, _P, _P, _c.c_uint32, _P, _P, _P], _c.c_int),
    "soma_proposal_train": ([_P, _c.POINTER(SomaTrainCfg), _c.POINTER(SomaTrainLog)], _c.c_int),
    "soma_batch_create": ([_c.POINTER(SomaSystemDesc), _c.c_uint32, _P, _c.POINTER(_P)], _c.c_int),
    "soma_batch_destroy": ([_P], _c.c_int),
    "soma_batch_sweep": ([_P, _c.c_uint32], _c.c_int),
    "soma_batch_sync": ([_P], _c.c_int),
    "soma_batch_system": ([_P, _c.c_uint32, _c.POINTER(_P)], _c.c_int),
    "soma_batch_autotune": ([_P, _c.c_uint32, _c.POINTER(SomaTuneEntry), _c.c_uint32,
                             _c.POINTER(_c.c_uint32)], _c.c_int),
    "soma_batch_plan": ([_c.c_void_p, _c.c_uint32, _c.c_uint32, _c.c_int32, _c.c_void_p, _c.c_size_t,
                         _c.POINTER(_c.c_size_t)], _c.c_int),
    "soma_batch_set_shape": ([_P, _c.POINTER(SomaTuneEntry)], _c.c_int),
    "soma_batch_get_shape": ([_P, _c.POINTER(SomaTuneEntry)], _c.c_int),
    "soma_batch_set_timing": ([_P, _c.c_int], _c.c_int),
    "soma_batch_get_timing": ([_P, _c.POINTER(SomaTiming)], _c.c_int),
}


def lib():
    """Load libsoma.so (raises if it was not built: no fallback path exists)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"libsoma.so not built at {LIB_PATH}: run __graft_entry__.build()")
        L = ctypes.CDLL(LIB_PATH)
        for name, (args, res) in _SIGS.items():
            fn = getattr(L, name)
            fn.argtypes = args
            fn.restype = res
        _lib = L
    return _lib


def check(status):
    if status != SOMA_OK:
        raise SomaError(status, lib().soma_last_error().decode())
    return status


def _wrap(name):
    def call(*args):
        fn = getattr(lib(), name)
        r = fn(*args)
        if fn.restype is _c.c_int and name != "soma_abi_version":
            check(r)
        return r
    call.__name__ = name
    return call


soma_abi_version = _wrap("soma_abi_version")
soma_create = _wrap("soma_create")
soma_destroy = _wrap("soma_destroy")
soma_sweep = _wrap("soma_sweep")
soma_update_fields = _wrap("soma_update_fields")
soma_shard_counts = _wrap("soma_shard_counts")
soma_shard_sweep = _wrap("soma_shard_sweep")
soma_shard_fields = _wrap("soma_shard_fields")
soma_get_density = _wrap("soma_get_density")
soma_get_fields = _wrap("soma_get_fields")
soma_get_positions = _wrap("soma_get_positions")
soma_set_positions = _wrap("soma_set_positions")
soma_set_external = _wrap("soma_set_external")
soma_set_architectures = _wrap("soma_set_architectures")
soma_set_topology = _wrap("soma_set_topology")
soma_topology_sets = _wrap("soma_topology_sets")
soma_sort_molecules = _wrap("soma_sort_molecules")
soma_set_types = _wrap("soma_set_types")
soma_structure_factor_types = _wrap("soma_structure_factor_types")
soma_get_type_counts = _wrap("soma_get_type_counts")
soma_get_type_fields = _wrap("soma_get_type_fields")
soma_get_parameters = _wrap("soma_get_parameters")
soma_check_bounded_wait = _wrap("soma_check_bounded_wait")
soma_observables = _wrap("soma_observables")
soma_structure_factor = _wrap("soma_structure_factor")
soma_get_sweep = _wrap("soma_get_sweep")
soma_set_sweep = _wrap("soma_set_sweep")
soma_set_timing = _wrap("soma_set_timing")
soma_get_timing = _wrap("soma_get_timing")
soma_sync = _wrap("soma_sync")
soma_stream = _wrap("soma_stream")
soma_philox = _wrap("soma_philox")
soma_smc_draws = _wrap("soma_smc_draws")
soma_structure_factor_noalloc = _wrap("soma_structure_factor_noalloc")
soma_proposal_set_weights = _wrap("soma_proposal_set_weights")
soma_proposal_get_weights = _wrap("soma_proposal_get_weights")
soma_proposal_grad = _wrap("soma_proposal_grad")
soma_proposal_train = _wrap("soma_proposal_train")
soma_batch_create = _wrap("soma_batch_create")
soma_batch_destroy = _wrap("soma_batch_destroy")
soma_batch_sweep = _wrap("soma_batch_sweep")
soma_batch_sync = _wrap("soma_batch_sync")
soma_batch_system = _wrap("soma_batch_system")
soma_batch_autotune = _wrap("soma_batch_autotune")
soma_batch_plan = _wrap("soma_batch_plan")
soma_batch_set_shape = _wrap("soma_batch_set_shape")
soma_batch_get_shape = _wrap("soma_batch_get_shape")
soma_batch_set_timing = _wrap("soma_batch_set_timing")
soma_batch_get_timing = _wrap("soma_batch_get_timing")


def soma_last_error():
    return lib().soma_last_error().decode()


def declared_symbols(header=None):
    """Names of the functions include/soma.h declares (for the export check)."""
    import re
    header = header or os.path.join(os.path.dirname(HERE), "include", "soma.h")
    text = open(header).read()
    return sorted(set(re.findall(r"^\s*(?:[A-Za-z_][\w\s\*]*?)\b(soma_\w+)\s*\(", text, re.M)))
