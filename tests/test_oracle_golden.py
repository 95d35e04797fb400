"""The oracle's density convention against system sizes the paper prints with
their parameters (tests/golden/paper_systems.txt): for the printed particle
count nN, chain length N and box, the oracle's particles per cell rho_0 dL^3
and R_e0 in cell units give back the printed invariant degree of
polymerization, sqrt(Nbar) = rho_0 R_e0^3 / N (Sec. 2.1), within the printed
digits.  The grid only sets the cell size and drops out."""
import os

import pytest

from paper_1711_03828_gb300 import SystemDesc
from tests.conftest import oracle_system

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_systems.txt")


def _systems():
    out = []
    for line in open(GOLDEN):
        if not line.strip() or line.startswith("#"):
            continue
        name, N, sq, box, nN, _ = [f.strip() for f in line.split("|")]
        out.append((name, int(N), float(sq), [float(b) for b in box.split()], float(nN)))
    return out


def check_printed_systems(lib=None):
    systems = _systems()
    assert len(systems) == 1
    for name, N, sq_nbar, box, nN, in systems:
        n_chains = int(round(nN / N))
        for cells_per_Re in (5, 10):     # two cell sizes (whole cells on every axis)
            grid = tuple(int(round(b * cells_per_Re)) for b in box)
            assert all(abs(g - b * cells_per_Re) < 1e-9 for g, b in zip(grid, box))
            d = SystemDesc(n_chains=n_chains, N=N, f=0.5, box_Re=tuple(box), grid=grid,
                           chiN=0.0, kappaN=0.0)
            prm = oracle_system(d, lib).params
            got = prm.rho_cell * prm.Re**3 / N
            # the printed sqrt(Nbar) carries three significant digits, nN one to three
            assert got == pytest.approx(sq_nbar, rel=2e-3), (name, cells_per_Re, got, sq_nbar)


def test_printed_systems(oracle_lib):
    check_printed_systems()


def test_weak_scaling_workload_has_the_printed_parameters(oracle_lib):
    """melt_tiny is the smallest system of the paper's weak-scaling series
    (Sec. 4.2): n = 2^7 molecules of N = 64, 8192 particles, sqrt(Nbar) ~ 128,
    dL ~ R_e0/6."""
    from paper_1711_03828_gb300 import workloads
    d = workloads.melt_tiny()
    prm = oracle_system(d).params
    assert d.n_chains == 2**7 and d.N == 64 and d.M == 8192
    assert prm.rho_cell * prm.Re**3 / d.N == pytest.approx(128.0, rel=1e-12)
    assert prm.Re == pytest.approx(6.0, rel=1e-12)
