"""Host-side checks of the C ABI that need no GPU: the library loads, exports
every entry point include/soma.h declares, and rejects invalid descriptions
before touching the device."""
import ctypes

import pytest

from paper_1711_03828_gb300 import SystemDesc, _abi


def test_library_exports_every_declared_symbol(soma_lib):
    names = _abi.declared_symbols()
    assert "soma_create" in names and "soma_sweep" in names and len(names) >= 18
    L = soma_lib.lib()
    missing = [n for n in names if not hasattr(L, n)]
    assert not missing, missing
    assert L.soma_abi_version() == 2


def test_binding_wraps_every_declared_symbol():
    """The Python binding has one function per declared entry point."""
    missing = [n for n in _abi.declared_symbols() if not callable(getattr(_abi, n, None))]
    assert not missing, missing


def _create_status(desc_c):
    h = ctypes.c_void_p()
    st = _abi.lib().soma_create(ctypes.byref(desc_c), ctypes.byref(h))
    return st, h


def _valid():
    return SystemDesc(n_chains=16, N=8, box_Re=(1.0, 1.0, 1.0), grid=(6, 6, 6))


@pytest.mark.parametrize("field,value", [
    ("N", 0), ("N", 257), ("n_chains", 0), ("f", 1.5), ("f", float("nan")),
    ("chiN", float("inf")), ("move", 7), ("set_order", 3), ("grid_dtype", 5),
    ("replica_id", 1 << 24),
])
def test_invalid_description_is_rejected_without_gpu(soma_lib, field, value):
    d = _valid()
    setattr(d, field, value)
    st, h = _create_status(d.to_c())
    assert st == _abi.SOMA_EINVAL
    assert h.value is None
    assert _abi.soma_last_error()


def test_molecule_iteration_takes_uniform_moves_only(soma_lib):
    for move in (1, 2):
        d = _valid()
        d.set_order, d.move = 2, move
        st, h = _create_status(d.to_c())
        assert st == _abi.SOMA_EINVAL and h.value is None


@pytest.mark.parametrize("mutate", ["struct_size", "flags", "box", "grid", "noncubic", "cells"])
def test_invalid_geometry_is_rejected_without_gpu(soma_lib, mutate):
    c = _valid().to_c()
    if mutate == "struct_size":
        c.struct_size = 8
    elif mutate == "flags":
        c.flags = 8
    elif mutate == "box":
        c.box_Re[1] = -1.0
    elif mutate == "grid":
        c.grid[2] = 0
    elif mutate == "noncubic":
        c.grid[0] = 7
    elif mutate == "cells":
        c.grid[0] = c.grid[1] = c.grid[2] = 4096
        c.box_Re[0] = c.box_Re[1] = c.box_Re[2] = 4096.0
    st, h = _create_status(c)
    assert st == _abi.SOMA_EINVAL, _abi.soma_last_error()


def test_null_arguments_are_rejected(soma_lib):
    L = soma_lib.lib()
    assert L.soma_create(None, None) == _abi.SOMA_EINVAL
    assert L.soma_sweep(None, 1) == _abi.SOMA_EINVAL
    assert L.soma_observables(None, None) == _abi.SOMA_EINVAL
    assert L.soma_destroy(None) == _abi.SOMA_OK


def test_struct_layouts_match_header(soma_lib, tmp_path):
    """The ctypes mirrors have the sizes and field offsets of the C structs."""
    import os
    import subprocess
    inc = os.path.join(os.path.dirname(os.path.dirname(_abi.HERE)), "include")
    if not os.path.exists(os.path.join(inc, "soma.h")):
        inc = os.path.join(os.path.dirname(_abi.HERE), "include")
    structs = {"soma_system_desc": _abi.SomaSystemDesc, "soma_obs": _abi.SomaObs,
               "soma_params": _abi.SomaParams,
               "soma_timing": _abi.SomaTiming}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "soma.h"', "int main(void){"]
    for cname, py in structs.items():
        lines.append(f'printf("{cname} %zu\\n", sizeof({cname}));')
        for f, _ in py._fields_:
            lines.append(f'printf("{cname}.{f} %zu\\n", offsetof({cname}, {f}));')
    lines.append("return 0;}")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run(["gcc", f"-I{inc}", str(src), "-o", str(exe)], check=True)
    got = dict(l.split() for l in subprocess.run([str(exe)], capture_output=True, text=True,
                                                 check=True).stdout.splitlines())
    for cname, py in structs.items():
        assert int(got[cname]) == ctypes.sizeof(py), cname
        for f, _ in py._fields_:
            assert int(got[f"{cname}.{f}"]) == getattr(py, f).offset, f"{cname}.{f}"


@pytest.mark.parametrize("bad", ["seed", "odd_N", "long_N", "smc", "dtype", "empty"])
def test_invalid_batch_is_rejected_without_gpu(soma_lib, bad):
    descs = [_valid(), _valid()]
    descs[1].replica_id = 1
    if bad == "seed":
        descs[1].seed = 99
    elif bad == "odd_N":
        descs[1].N = 7
    elif bad == "long_N":
        descs[1].N = 128
    elif bad == "smc":
        descs[1].move = 1
    elif bad == "dtype":
        descs[1].grid_dtype = 1
    arr = (_abi.SomaSystemDesc * 2)(*[d.to_c() for d in descs])
    h = ctypes.c_void_p()
    n = 0 if bad == "empty" else 2
    assert _abi.lib().soma_batch_create(arr, n, None, ctypes.byref(h)) == _abi.SOMA_EINVAL
    assert h.value is None


@pytest.mark.parametrize("offset,count,total", [
    (1, 16, 0),            # an offset without the whole system's chain count
    (10, 16, 20),          # chains beyond the whole system
    (0, 16, 8),            # more chains than the whole system
    (0, 16, 1 << 29),      # a sharded system of 2^32 particles (N = 8)
])
def test_invalid_shard_is_rejected_without_gpu(soma_lib, offset, count, total):
    d = _valid()
    d.chain_offset, d.n_chains, d.n_chains_total = offset, count, total
    st, h = _create_status(d.to_c())
    assert st == _abi.SOMA_EINVAL and h.value is None
    msg = _abi.soma_last_error()
    assert "chain" in msg or "2^32" in msg
