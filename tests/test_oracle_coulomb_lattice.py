"""Pins for the Coulomb matrix (oracle/coulomb.py) and lattice sums (oracle/lattice.py)."""
import math

import numpy as np
import pytest

import workloads
from oracle import closed_forms as cf
from oracle import coulomb, cp, kernel_vectors as kv, lattice, sinc


def _basis(seed, nb=4, lo=2, hi=3, a_lo=0.5, a_hi=2.0, centres=3, half=1.2):
    return workloads.basis_set(nb, lo, hi, a_lo, a_hi, centres, half, seed)


def _kernel(n, b, M):
    t, a = sinc.conv_nodes(n, b, M)
    return kv.conv_kernel_vectors(n, b, t, a)


def _analytic_J(basis, items):
    """Sum over primitives of (ab|cd) with the Gaussian product theorem."""
    first, al, d, X, w = (basis[k] for k in ("fn_first", "prim_alpha", "prim_d", "fn_centre", "w"))
    nb = len(first) - 1

    def pairs(mu, nu):
        out = []
        for a in range(first[mu], first[mu + 1]):
            for b in range(first[nu], first[nu + 1]):
                p = al[a] + al[b]
                K = math.exp(-al[a] * al[b] / p * float(np.sum((X[mu] - X[nu]) ** 2)))
                P = (al[a] * X[mu] + al[b] * X[nu]) / p
                out.append((d[a] * d[b] * K, p, P))
        return out

    rho = [(w[k] * cK, p, P) for k in range(nb) for (cK, p, P) in pairs(k, k)]
    J = []
    for mu, nu in items:
        tot = 0.0
        for (c1, p1, P1) in pairs(mu, nu):
            for (c2, p2, P2) in rho:
                tot += c1 * c2 * float(cf.coulomb_pair(p1, P1, p2, P2))
        J.append(tot)
    return np.array(J)


def test_coulomb_matrix_against_dense_tensors():
    n, b, M = 10, 3.0, 6
    h = 2 * b / n
    basis = _basis(7, nb=3, half=0.8)
    P = _kernel(n, b, M)
    items = coulomb.item_list(3)
    J, _ = coulomb.coulomb_items(n, b, basis, P, items)
    # dense: g_mu on the grid, rho = sum w g^2, V = rho * P (3D), J = h^3 sum g g V
    Gp = coulomb.primitive_factors(n, b, basis)
    first = basis["fn_first"]
    g = []
    for mu in range(3):
        s = slice(first[mu], first[mu + 1])
        g.append(cp.full_tensor(Gp[:, s, :], basis["prim_d"][s]))
    rho = sum(basis["w"][mu] * g[mu] ** 2 for mu in range(3))
    off = np.abs(np.arange(-(n - 1), n))
    Pd = np.einsum("qi,qj,qk->ijk", P[:, off], P[:, off], P[:, off])
    V = np.zeros((n, n, n))
    r = np.arange(n)
    for i in range(n):
        for j in range(n):
            for k in range(n):
                V[i, j, k] = np.sum(rho * Pd[np.ix_(i - r + n - 1, j - r + n - 1, k - r + n - 1)])
    Jd = np.array([h ** 3 * np.sum(g[mu] * g[nu] * V) for mu, nu in items])
    assert np.max(np.abs(J - Jd)) < 1e-12 * np.max(np.abs(Jd))


def test_coulomb_matrix_symmetry_and_energy():
    n, b, M = 40, 6.0, 16
    h = 2 * b / n
    basis = _basis(9)
    P = _kernel(n, b, M)
    items = [(0, 1), (1, 0), (2, 3), (3, 2), (0, 0), (1, 1), (2, 2), (3, 3)]
    J, W = coulomb.coulomb_items(n, b, basis, P, items)
    assert abs(J[0] - J[1]) < 1e-13 * abs(J[0]) and abs(J[2] - J[3]) < 1e-13 * abs(J[2])
    E = float(basis["w"] @ J[4:])
    U_rho, c_rho = coulomb.density_cp(n, b, basis)
    E2 = cp.hartree_energy(U_rho, c_rho, P, h)
    assert abs(E / E2 - 1) < 1e-13


def test_coulomb_matrix_converges_to_analytic_integrals():
    b, M = 8.0, 40
    basis = _basis(13)
    items = coulomb.item_list(4)
    ex = _analytic_J(basis, items)
    J = {}
    for n in (64, 128):
        J[n], _ = coulomb.coulomb_items(n, b, basis, _kernel(n, b, M), items)
    rich = (4 * J[128] - J[64]) / 3
    assert np.max(np.abs(rich - ex)) < 5e-5 * np.max(np.abs(ex)), np.max(np.abs(rich - ex)) / np.max(np.abs(ex))
    assert np.max(np.abs(J[128] - ex)) < 5e-3 * np.max(np.abs(ex))


def _master(n, b, M):
    t, a = sinc.master_nodes(n, b, M)
    return kv.master_kernel_vectors(n, b, t, a)


def test_assembled_lattice_equals_per_charge_sum():
    n, b, M, L = 64, 8.0, 14, 4
    h = 2 * b / n
    geo = workloads.lattice_geometry(n, L, 8)
    Pm = _master(n, b, M)
    S = [lattice.assembled_vectors(Pm, geo["edges"], n) for _ in range(3)]
    idx = np.array(np.meshgrid(geo["sub_idx"], geo["sub_idx"], geo["sub_idx"], indexing="ij")).reshape(3, -1).T
    V = lattice.potential_on_points(S, h, idx)
    Vd = lattice.per_charge_sum(Pm, [geo["edges"]] * 3, n, h, idx)
    assert np.max(np.abs(V / Vd - 1)) < 1e-13
    # rank of the assembled sum stays R_N (Sec. 5.1): the sub-grid tensor equals
    # the CP reconstruction from R_N assembled vectors per axis
    Vsub = lattice.potential_subgrid(S, h, [geo["sub_idx"]] * 3)
    assert np.allclose(Vsub.reshape(-1), V, rtol=1e-14, atol=0)


def test_lattice_potential_against_direct_coulomb_sum():
    # h^-3 P_cL approximates sum_k 1/|x - x_k| (Sec. 5.2, accuracy O(h^2); the
    # h^2 term of a cell average of a harmonic function vanishes)
    L, spacing, n0, M = 8, 4.0, 128, 30
    n = L * n0
    b = L * spacing / 2
    h = 2 * b / n
    geo = workloads.lattice_geometry(n, L, 32)
    Pm = _master(n, b, M)
    S = [lattice.assembled_vectors(Pm, geo["edges"], n) for _ in range(3)]
    pts = workloads.check_points(32, 200, seed=3)
    idx = geo["sub_idx"][pts]
    V = lattice.potential_on_points(S, h, idx)
    x = -b + (idx + 0.5) * h
    q = -b + (geo["edges"] * h)  # charge coordinates per axis (cell edges)
    Q = np.array(np.meshgrid(q, q, q, indexing="ij")).reshape(3, -1).T
    ref = np.array([np.sum(1.0 / np.linalg.norm(Q - xi, axis=1)) for xi in x])
    assert np.max(np.abs(V / ref - 1)) < 5e-5, np.max(np.abs(V / ref - 1))
    # charges sit at unit-cell centres
    assert np.allclose(q, -b + spacing * (np.arange(L) + 0.5))
