import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: long CPU statistics test")


@pytest.fixture(scope="session")
def oracle_lib():
    import oracle
    from oracle import build as ob
    ob.build()
    return oracle


@pytest.fixture(scope="session")
def soma_lib():
    """The CUDA library, built in-tree if absent (no compute call is made here)."""
    from paper_1711_03828_gb300 import _abi
    if not os.path.exists(_abi.LIB_PATH):
        from paper_1711_03828_gb300 import build
        build.build()
    return _abi


def oracle_system(desc, L=None, **over):
    """An oracle.System with the parameters of a SystemDesc."""
    import oracle
    kw = dict(n_chains=desc.n_chains, N=desc.N, f=desc.f, box_Re=desc.box_Re, grid=desc.grid,
              chiN=desc.chiN, kappaN=desc.kappaN, a_Re=desc.a_Re, seed=desc.seed,
              replica=desc.replica_id, set_order=desc.set_order, move=desc.move)
    kw.update(over)
    s = oracle.System(L=L, **kw)
    s.set_hamiltonian(getattr(desc, "hamiltonian", 0))
    return s


@pytest.fixture(scope="session")
def cuda_device():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1711_03828_gb300 import _abi
    _abi.lib()  # fail loudly if the extension is missing on a GPU machine
    return torch.device("cuda:0")
