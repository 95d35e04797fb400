"""The allocation-free structure factor (soma_structure_factor_noalloc).

Some callers cannot allocate device memory when they want S(q), for instance
an analysis hook inside an application whose memory pool owns the GPU's free
memory, or code that must not synchronise the device.  This entry point keeps
its scratch in a static device array of libsoma and takes every input and
output from the caller.  Here it is called through the C ABI and compared with
soma_structure_factor, which allocates its own scratch, on two calls in a row
with different wave vectors (the second call must not see the first one's
leftovers).  This file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest

from paper_1711_03828_gb300 import SomaError, System, SystemDesc, _abi, workloads

pytestmark = pytest.mark.gpu


def _noalloc(desc_c, density, ms):
    mm = np.ascontiguousarray(np.asarray(ms, dtype=np.int32).reshape(-1, 3))
    out = np.full(len(mm), np.nan)
    _abi.soma_structure_factor_noalloc(ctypes.byref(desc_c), ctypes.c_void_p(density.data_ptr()),
                                       mm.ctypes.data, len(mm), out.ctypes.data, None)
    return out


def test_noalloc_structure_factor_matches_allocating_entry_point(cuda_device):
    import torch
    d = workloads.melt_small(chiN=30.0)
    s = System(d)
    s.sweep(20)
    dens = torch.empty(d.cells, dtype=torch.int32, device=cuda_device)
    s.get_density(out=dens)
    torch.cuda.synchronize()
    c = d.to_c()
    rng = np.random.default_rng(3)
    first = rng.integers(-12, 13, (32, 3))
    second = [(1, 0, 0), (0, 1, 0), (0, 0, 1), (2, 2, 2), (0, 0, 0), (-3, 5, 7), (6, 6, 6)]
    for ms in (first, second):
        want = s.structure_factor(ms)
        got = _noalloc(c, dens, ms)
        np.testing.assert_allclose(got, want, rtol=1e-9, atol=1e-9)
    s.close()


def test_noalloc_calls_after_the_first_allocate_no_device_memory(cuda_device):
    """The first call on a device loads the scratch array (lazy module
    loading); every later call leaves the device's free memory unchanged."""
    import torch
    d = workloads.melt_small(chiN=30.0)
    s = System(d)
    s.sweep(5)
    dens = torch.empty(d.cells, dtype=torch.int32, device=cuda_device)
    s.get_density(out=dens)
    torch.cuda.synchronize()
    c = d.to_c()
    ms = np.random.default_rng(5).integers(-6, 7, (32, 3))
    first = _noalloc(c, dens, ms)
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(3):
        again = _noalloc(c, dens, ms)
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0, (free0, free1)
    np.testing.assert_array_equal(again, first)
    s.close()


def test_noalloc_rejects_sizes_beyond_its_scratch(cuda_device):
    import torch
    d = workloads.melt_small()
    dens = torch.zeros(d.cells, dtype=torch.int32, device=cuda_device)
    with pytest.raises(SomaError) as e:
        _noalloc(d.to_c(), dens, np.zeros((33, 3)))
    assert e.value.status == _abi.SOMA_EINVAL
    big = SystemDesc(n_chains=1, N=2, box_Re=(64.0, 64.0, 64.0), grid=(384, 384, 384))
    with pytest.raises(SomaError) as e:
        _noalloc(big.to_c(), dens, [(1, 0, 0)])
    assert e.value.status == _abi.SOMA_EINVAL
