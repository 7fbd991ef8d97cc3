"""Coulomb matrix over product functions (Sec. 3.1, J_km = <G_k . G_m, V_H>).

TEST INFRASTRUCTURE ONLY (see the package docstring).

A contracted s-type basis g_mu = sum_{p in mu} d_p exp(-alpha_p |x - X_mu|^2) is
sampled at cell centres; every primitive is rank 1 (Sec. 3.1, Eq. disc_GTO).
Products of two basis functions are formed by 1D Hadamard products of the
primitive factors (Sec. 2.5, Eq. had): the item (mu, nu) has CP rank
n_mu * n_nu with factors g_a^(l) . g_b^(l) and coefficients d_a d_b.

The density is the diagonal one rho = sum_mu w_mu g_mu^2: its CP factors are the
products g_a . g_b for a <= b inside one function, with coefficient
w_mu d_a d_b, doubled when a != b (the (a,b) and (b,a) terms are equal).
V_H = rho * P_R has the factors W = u_m * p_q (Sec. 3.1), and

    J_{mu nu} = h^3 sum_{(a,b) in mu nu} d_a d_b sum_m c_m sum_q
                prod_l <g_a^(l) . g_b^(l), W^(l)[:, m R_N + q]>

(the 1D scalar products of Sec. 3.1).  With D = diag(w) the energy is
E_H = sum_mu w_mu J_{mu mu} = h^3 <rho, P_R * rho>  (App. 2, J(D)).
"""
from __future__ import annotations

import numpy as np

from . import cp


def primitive_factors(n: int, b: float, basis: dict) -> np.ndarray:
    """(3, P, n) sampled primitives exp(-alpha_p (x_i - X_mu(p),l)^2)."""
    first = basis["fn_first"]
    nb = len(first) - 1
    centre = np.empty((first[-1], 3))
    for mu in range(nb):
        centre[first[mu]:first[mu + 1]] = basis["fn_centre"][mu]
    return cp.sample_gaussians(n, b, basis["prim_alpha"], centre)


def density_pairs(basis: dict):
    """Primitive pairs (a, b), a <= b within each function, and their CP
    coefficients w_mu d_a d_b (x2 when a != b) for rho = sum w_mu g_mu^2."""
    first, d, w = basis["fn_first"], basis["prim_d"], basis["w"]
    pa, pb, coef = [], [], []
    for mu in range(len(first) - 1):
        for a in range(first[mu], first[mu + 1]):
            for bb in range(a, first[mu + 1]):
                pa.append(a)
                pb.append(bb)
                coef.append(w[mu] * d[a] * d[bb] * (1.0 if a == bb else 2.0))
    return np.array(pa), np.array(pb), np.array(coef)


def item_list(nb: int):
    """Items (mu, nu), mu <= nu, in row-major order of the upper triangle."""
    return [(mu, nu) for mu in range(nb) for nu in range(mu, nb)]


def item_pairs(basis: dict, items):
    """For each item, its primitive pairs (a in mu, b in nu) and coefficients d_a d_b.
    Returns concatenated pair arrays and offsets (len(items)+1)."""
    first, d = basis["fn_first"], basis["prim_d"]
    pa, pb, coef, off = [], [], [], [0]
    for mu, nu in items:
        for a in range(first[mu], first[mu + 1]):
            for bb in range(first[nu], first[nu + 1]):
                pa.append(a)
                pb.append(bb)
                coef.append(d[a] * d[bb])
        off.append(len(pa))
    return np.array(pa), np.array(pb), np.array(coef), np.array(off)


def hadamard(Gp: np.ndarray, pa: np.ndarray, pb: np.ndarray) -> np.ndarray:
    """(3, len(pa), n) factors g_a^(l) . g_b^(l) (Sec. 2.5, Eq. had)."""
    return Gp[:, pa, :] * Gp[:, pb, :]


def density_cp(n: int, b: float, basis: dict):
    Gp = primitive_factors(n, b, basis)
    pa, pb, coef = density_pairs(basis)
    return hadamard(Gp, pa, pb), coef


def coulomb_items(n: int, b: float, basis: dict, P: np.ndarray, items,
                  W_rho: np.ndarray | None = None, rho=None):
    """J for the listed items by direct 1D scalar products against V_H's factors.
    Returns (J array, W_rho) so callers can reuse the V_H factors."""
    h = 2.0 * b / n
    R_N = P.shape[0]
    if rho is None:
        rho = density_cp(n, b, basis)
    U_rho, c_rho = rho
    if W_rho is None:
        W_rho = cp.convolve_factors(U_rho, P)
    Gp = primitive_factors(n, b, basis)
    pa, pb, coef, off = item_pairs(basis, items)
    Ui = hadamard(Gp, pa, pb)
    c_mq = np.repeat(c_rho, R_N)          # coefficient of column m*R_N + q
    J = np.empty(len(items))
    for it in range(len(items)):
        s = slice(off[it], off[it + 1])
        prod = np.ones((off[it + 1] - off[it], W_rho.shape[1]))
        for l in range(3):
            prod *= Ui[l, s] @ W_rho[l].T     # <u_a^(l), W^(l)[:, mq]>
        J[it] = h ** 3 * float(coef[s] @ (prod @ c_mq))
    return J, W_rho
