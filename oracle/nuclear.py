"""Nuclear potential of a molecule and its Galerkin matrix (Sec. 3.3).

TEST INFRASTRUCTURE ONLY (see the package docstring).

The nuclear potential V_c(x) = -sum_alpha Z_alpha / |x - a_alpha| is the
reference Newton kernel of the 2n master grid (Sec. 5.1, Eq. refTensor)
shifted onto each nucleus by the rank-1 windowing operator and summed with
the charges (Sec. 3.3):

    P_c = sum_alpha Z_alpha sum_q f_{alpha q}^(1) (x) f_{alpha q}^(2) (x) f_{alpha q}^(3),
    f_{alpha q}^(l)[i] = p~_q[i - e_alpha^(l)],  i = 0..n-1,

a nucleus sitting at the grid-cell edge e_alpha^(l) of each axis, so that
cell i holds the Galerkin integral over the master cell i - e, whose centre
is (i - e + 1/2) h away (the same windowing as the lattice sums).  P_c is
h^3 times the potential at the cell centres, and the Galerkin matrix of V_c
over product functions is

    v_km = -<G_k . G_m, P_c>
         = -sum_{(a,b) in km} d_a d_b sum_alpha Z_alpha sum_q prod_l <g_a^(l) . g_b^(l), f_{alpha q}^(l)>

(1D scalar products as for the Coulomb matrix).
"""
from __future__ import annotations

import numpy as np

from . import coulomb


def windowed_factors(Pm: np.ndarray, edges: np.ndarray, n: int) -> np.ndarray:
    """(len(edges) R_N, n): row alpha R_N + q holds p~_q[i - edges[alpha]]."""
    R_N = Pm.shape[0]
    i = np.arange(n)
    F = np.empty((len(edges) * R_N, n))
    for a, e in enumerate(edges):
        F[a * R_N:(a + 1) * R_N] = Pm[:, i - int(e) + n]
    return F


def nuclear_items(n: int, b: float, basis: dict, Pm: np.ndarray, items, nuc_edges: np.ndarray,
                  Z: np.ndarray) -> np.ndarray:
    """v for the listed items (mu, nu); nuc_edges (3, N_nuc) grid-cell edges,
    Z (N_nuc,) charges."""
    R_N = Pm.shape[0]
    F = [windowed_factors(Pm, nuc_edges[l], n) for l in range(3)]
    Gp = coulomb.primitive_factors(n, b, basis)
    pa, pb, coef, off = coulomb.item_pairs(basis, items)
    Ui = coulomb.hadamard(Gp, pa, pb)
    z_aq = np.repeat(np.asarray(Z, dtype=np.float64), R_N)  # charge of column alpha R_N + q
    v = np.empty(len(items))
    for it in range(len(items)):
        s = slice(off[it], off[it + 1])
        prod = np.ones((off[it + 1] - off[it], F[0].shape[0]))
        for l in range(3):
            prod *= Ui[l, s] @ F[l].T
        v[it] = -float(coef[s] @ (prod @ z_aq))
    return v
