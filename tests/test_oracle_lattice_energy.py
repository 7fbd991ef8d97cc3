"""Pins for the lattice interaction energy (oracle/lattice.py, Sec. 5.3)."""
import math
import os

import numpy as np
import pytest

from oracle import kernel_vectors as kv, lattice, sinc

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "lattice_energy_table.txt")


def _table():
    rows = []
    for line in open(GOLDEN):
        line = line.split("#")[0].split()
        if line:
            rows.append((int(line[0]), float(line[1]), int(line[2]), line[3]))
    return rows


def _sig(x, digits, mode):
    e = math.floor(math.log10(abs(x))) - (digits - 1)
    m = x / 10.0 ** e
    m = math.floor(m) if mode == "trunc" else round(m)
    return m * 10.0 ** e


@pytest.mark.parametrize("L,printed,digits,use", _table())
def test_direct_energy_reproduces_the_printed_table(L, printed, digits, use):
    # charges 2 bohr apart: cell edges 0..L-1 with h = 2
    E = lattice.interaction_energy_direct([np.arange(L)] * 3, 2.0)
    agrees = any(math.isclose(_sig(E, digits, m), printed, rel_tol=1e-12) for m in ("round", "trunc"))
    assert agrees == (use == "pin"), (L, E, printed)


def test_direct_energy_small_configurations():
    D = 1.7
    assert lattice.interaction_energy_direct([[3], [4], [5]], D) == 0.0
    assert math.isclose(lattice.interaction_energy_direct([[0, 1], [0], [0]], D, Z=3.0), 9.0 / D, rel_tol=1e-15)
    # a square: four sides and two diagonals
    E = lattice.interaction_energy_direct([[0, 1], [0, 1], [7]], D)
    assert math.isclose(E, 4.0 / D + 2.0 / (D * math.sqrt(2.0)), rel_tol=1e-14)
    # a cube: 12 edges, 12 face diagonals, 4 body diagonals
    E = lattice.interaction_energy_direct([[0, 1]] * 3, D)
    assert math.isclose(E, (12.0 + 12.0 / math.sqrt(2.0) + 4.0 / math.sqrt(3.0)) / D, rel_tol=1e-14)


def _master(n, b, M):
    t, a = sinc.master_nodes(n, b, M)
    return kv.master_kernel_vectors(n, b, t, a)


def test_tensor_energy_matches_the_direct_sum():
    # 8^3 hydrogen lattice, 2 bohr = 32 cells, R_N = 129 Gaussians: the traced
    # tensor sum (Eq. EnergyLattice) against the direct sum (Eq. EnergyLatSum)
    n, b, M, cells = 512, 16.0, 64, 32
    h = 2 * b / n
    off = (n - 7 * cells) // 2
    edges = [off + cells * np.arange(8)] * 3
    Pm = _master(n, b, M)
    Et = lattice.interaction_energy_tensor(Pm, edges, n, h)
    Ed = lattice.interaction_energy_direct(edges, h)
    assert abs(Et / Ed - 1) < 3e-8
    # a non-cubic, irregular lattice
    edges = [np.array([40, 97, 130]), np.array([60, 100, 200, 333, 400]), np.array([250, 300])]
    Et = lattice.interaction_energy_tensor(Pm, edges, n, h, Z=2.0)
    Ed = lattice.interaction_energy_direct(edges, h, Z=2.0)
    assert abs(Et / Ed - 1) < 5e-8


def test_tensor_energy_improves_with_the_quadrature():
    # the error is set by the sinc quadrature of 1/r, not by h (the 2h cube
    # average of the harmonic 1/r is exact to second order)
    n, b, cells = 1024, 16.0, 64
    h = 2 * b / n
    off = (n - 7 * cells) // 2
    edges = [off + cells * np.arange(8)] * 3
    Ed = lattice.interaction_energy_direct(edges, h)
    errs = [abs(lattice.interaction_energy_tensor(_master(n, b, M), edges, n, h) / Ed - 1) for M in (30, 40, 64)]
    assert errs[0] > errs[1] > errs[2]
    assert errs[2] < 2e-8


def test_tensor_energy_of_one_charge_is_zero():
    n, b, M = 256, 8.0, 20
    Pm = _master(n, b, M)
    assert lattice.interaction_energy_tensor(Pm, [[100], [7], [255]], n, 2 * b / n) == 0.0
