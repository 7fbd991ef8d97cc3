"""Assembled lattice sums of Newton potentials (Sec. 5.1).

TEST INFRASTRUCTURE ONLY (see the package docstring).

Charges sit on an L x L x L lattice inside an n-cell box; the master kernel
p~_q lives on 2n cells [j h, (j+1) h], j = -n..n-1 (Eq. refTensor).  A charge at
the grid-cell edge e contributes to cell centre i through master cell i - e,
whose centre is (i - e + 1/2) h away.  Shifting and windowing the master vector
onto the box and summing over the lattice positions per axis gives the
assembled vectors (Eq. CoulombLatTensCan)

    s_q^(l)[i] = sum_{k=0}^{L-1} p~_q[i - e_k^(l)],   i = 0..n-1,

and the lattice potential at cell centres is h^{-3} sum_q prod_l s_q^(l)[i_l]
(the h^{-3} scaling of Sec. 5.2, Eq. EnergyLattice).  The CP rank stays R_N.
"""
from __future__ import annotations

import numpy as np


def assembled_vectors(Pm: np.ndarray, edges: np.ndarray, n: int) -> np.ndarray:
    """s[q, i] = sum_k Pm[q, (i - edges[k]) + n]  (Pm column j+n holds offset j)."""
    R = Pm.shape[0]
    s = np.zeros((R, n))
    i = np.arange(n)
    for e in edges:
        s += Pm[:, i - int(e) + n]
    return s


def potential_on_points(S: list, h: float, idx: np.ndarray) -> np.ndarray:
    """V at points idx (npts, 3) of grid indices: h^-3 sum_q prod_l S[l][q, idx[:, l]]."""
    prod = S[0][:, idx[:, 0]] * S[1][:, idx[:, 1]] * S[2][:, idx[:, 2]]
    return prod.sum(axis=0) / h ** 3


def potential_subgrid(S: list, h: float, sub_idx: list) -> np.ndarray:
    """V on the tensor sub-grid sub_idx[0] x sub_idx[1] x sub_idx[2] (small sizes)."""
    A = [S[l][:, sub_idx[l]] for l in range(3)]
    return np.einsum("qi,qj,qk->ijk", A[0], A[1], A[2]) / h ** 3


def per_charge_sum(Pm: np.ndarray, edges: list, n: int, h: float, idx: np.ndarray) -> np.ndarray:
    """The same discrete potential summed charge by charge (no assembly):
    h^-3 sum_{k1,k2,k3} sum_q prod_l Pm[q, idx_l - e_{k_l} + n]."""
    out = np.zeros(len(idx))
    for e1 in edges[0]:
        A1 = Pm[:, idx[:, 0] - int(e1) + n]
        for e2 in edges[1]:
            A12 = A1 * Pm[:, idx[:, 1] - int(e2) + n]
            for e3 in edges[2]:
                out += (A12 * Pm[:, idx[:, 2] - int(e3) + n]).sum(axis=0)
    return out / h ** 3
