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

The interaction energy of the lattice charges (Sec. 5.3, Eqs. EnergyLatSum and
EnergyLattice) is given both by brute force and by the tensor lattice sum
traced at the lattice points with the singular-point correction.
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


# ---- interaction energy of the lattice charges (Sec. 5.3) ----------------------

def interaction_energy_direct(edges: list, h: float, Z: float = 1.0) -> float:
    """E_L = 1/2 sum_{k != j} Z^2 / |x_k - x_j| (Eq. EnergyLatSum) for equal
    charges Z at x = e h on the tensor lattice edges[0] x edges[1] x edges[2].

    Brute force over distinct displacement vectors: per axis the differences
    d = e_j - e_k with their multiplicities, then the double sum as
    sum_{d != 0} c1(d1) c2(d2) c3(d3) / (h |d|)."""
    ds, cs = [], []
    for e in edges:
        e = np.asarray(e, dtype=np.int64)
        d, c = np.unique(np.subtract.outer(e, e).ravel(), return_counts=True)
        ds.append(d.astype(np.float64))
        cs.append(c.astype(np.float64))
    d23 = ds[1][:, None] ** 2 + ds[2][None, :] ** 2
    c23 = cs[1][:, None] * cs[2][None, :]
    tot = 0.0
    for d1, c1 in zip(ds[0], cs[0]):
        r = h * np.sqrt(d1 * d1 + d23)
        w = c1 * c23
        m = r > 0
        tot += float(np.sum(w[m] / r[m]))
    return 0.5 * Z * Z * tot


def interaction_energy_tensor(Pm: np.ndarray, edges: list, n: int, h: float, Z: float = 1.0) -> float:
    """E_L by the rank-R_N lattice sum traced at the lattice points (Sec. 5.3,
    Eq. EnergyLattice): Z^2 h^-3 / 2 (<P^_cL, 1> - <P_0L, 1>).

    A charge sits at a grid-cell edge, the corner shared by the cells e-1 and e
    of each axis; the tensor entry at a lattice point is read as the mean of the
    8 cells around it (the doubled 2L lattice of the traced sub-tensor), so that
    per axis
        T_q = sum_{j in K} (s_q[e_j - 1] + s_q[e_j]) / 2,
        t0_q = (p~_q[-1] + p~_q[0]) / 2           (the singular point x = 0),
    with s_q the assembled vectors, and
        <P^_cL, 1> = sum_q prod_l T_q^(l),   <P_0L, 1> = L1 L2 L3 sum_q prod_l t0_q."""
    T = []
    for e in edges:
        e = np.asarray(e, dtype=np.int64)
        # the assembled vectors traced at the 2L cells around the points
        # (the same sums over k as assembled_vectors, at those cells only)
        cells = np.concatenate([e - 1, e])
        s = np.zeros((Pm.shape[0], len(cells)))
        for ek in e:
            s += Pm[:, cells - ek + n]
        T.append(0.5 * s.sum(axis=1))
    t0 = 0.5 * (Pm[:, n - 1] + Pm[:, n])
    count = float(len(edges[0]) * len(edges[1]) * len(edges[2]))
    lattice_sum = float(np.sum(T[0] * T[1] * T[2]))
    singular = count * float(np.sum(t0 * t0 * t0))
    return 0.5 * Z * Z / h ** 3 * (lattice_sum - singular)
