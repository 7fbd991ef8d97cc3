"""Pins for the nuclear potential and its Galerkin matrix (oracle/nuclear.py, Sec. 3.3)."""
import math

import numpy as np

import workloads
from oracle import closed_forms as cf
from oracle import coulomb, kernel_vectors as kv, lattice, nuclear, sinc


def _master(n, b, M):
    t, a = sinc.master_nodes(n, b, M)
    return kv.master_kernel_vectors(n, b, t, a)


def _analytic(basis, items, C, Z):
    """v_km by the Gaussian product theorem and the s-type nuclear attraction integral."""
    first, al, d, X = (basis[k] for k in ("fn_first", "prim_alpha", "prim_d", "fn_centre"))
    out = []
    for mu, nu in items:
        tot = 0.0
        for a in range(first[mu], first[mu + 1]):
            for bb in range(first[nu], first[nu + 1]):
                p = al[a] + al[bb]
                K = math.exp(-al[a] * al[bb] / p * float(np.sum((X[mu] - X[nu]) ** 2)))
                P = (al[a] * X[mu] + al[bb] * X[nu]) / p
                tot += d[a] * d[bb] * K * float(np.sum(Z * cf.nuclear_attraction(p, P, C)))
        out.append(tot)
    return np.array(out)


def test_window_is_the_single_charge_lattice_sum():
    n, b, M = 128, 6.0, 12
    Pm = _master(n, b, M)
    for e in (0, 1, 37, 128):
        assert np.array_equal(nuclear.windowed_factors(Pm, [e], n), lattice.assembled_vectors(Pm, [e], n))


def test_nuclear_matrix_converges_to_analytic_integrals():
    # three contracted s functions, two nuclei on grid-cell edges; the grid
    # error falls as h^2 (collocation of smooth products, Galerkin cells at
    # the singular point)
    basis = workloads.basis_set(3, 2, 3, 0.5, 3.0, 2, 1.0, 11)
    items = coulomb.item_list(3)
    b, M = 8.0, 30
    errs = []
    for n in (64, 128, 256):
        h = 2 * b / n
        edges = np.array([[n // 2 - 3, n // 2 + 5], [n // 2 + 2, n // 2], [n // 2 - 6, n // 2 + 1]])
        C = (-b + edges * h).T  # (2, 3) nucleus positions
        Z = np.array([1.0, 3.0])
        v = nuclear.nuclear_items(n, b, basis, _master(n, b, M), items, edges, Z)
        v0 = _analytic(basis, items, C, Z)
        errs.append(np.max(np.abs(v - v0)) / np.max(np.abs(v0)))
    assert errs[2] < 2e-4
    assert errs[1] / errs[2] > 3.0 and errs[0] / errs[1] > 3.0
    assert np.all(v < 0)  # attraction


def test_nuclear_matrix_is_linear_in_the_charges():
    basis = workloads.basis_set(2, 2, 2, 0.5, 2.0, 2, 1.0, 3)
    items = coulomb.item_list(2)
    n, b, M = 64, 6.0, 16
    Pm = _master(n, b, M)
    edges = np.array([[20, 40], [30, 33], [31, 28]])
    v1 = nuclear.nuclear_items(n, b, basis, Pm, items, edges[:, :1], np.array([2.0]))
    v2 = nuclear.nuclear_items(n, b, basis, Pm, items, edges[:, 1:], np.array([5.0]))
    v12 = nuclear.nuclear_items(n, b, basis, Pm, items, edges, np.array([2.0, 5.0]))
    assert np.allclose(v12, v1 + v2, rtol=1e-13, atol=0)
