"""Failure detection without a GPU fault: a device wait that gives up is
reported as a status with the context still usable, and an allocation the GPU
cannot satisfy is reported as SOMA_ENOMEM with nothing left behind."""
import ctypes

import pytest

from paper_1711_03828_gb300 import SomaError, System, SystemDesc, _abi, workloads

pytestmark = pytest.mark.gpu


def test_bounded_wait_reports_timeout(cuda_device):
    with pytest.raises(SomaError) as e:
        _abi.soma_check_bounded_wait(4096, None)
    assert e.value.status == _abi.SOMA_ETIMEOUT
    # the context still works
    s = System(workloads.melt_small(n_chains=64))
    s.sweep(3)
    assert s.observables()["sweeps"] == 3
    s.close()


def test_out_of_memory_is_reported(cuda_device):
    """25.6 G particles need 307 GB of positions, more than the device holds:
    the first allocation fails, soma_create returns SOMA_ENOMEM and no handle."""
    d = SystemDesc(n_chains=800_000_000, N=32, box_Re=(100.0, 100.0, 100.0),
                   grid=(600, 600, 600))
    h = ctypes.c_void_p()
    st = _abi.lib().soma_create(ctypes.byref(d.to_c()), ctypes.byref(h))
    assert st == _abi.SOMA_ENOMEM, _abi.soma_last_error()
    assert h.value is None
    s = System(workloads.melt_small(n_chains=64))
    s.sweep(1)
    s.close()
