"""CP (canonical) Coulomb convolution by direct summation in float64.

TEST INFRASTRUCTURE ONLY (see the package docstring).

Grid: box [-b, b]^3, n cells per axis of width h = 2b/n, cell centres
x_i = -b + (i + 1/2) h, i = 0..n-1 (the piecewise-constant sampling at cell
centres of Sec. 3.1).  A function in CP format (Sec. 2.1, Eq. CP_form) is
f = sum_k c_k u_k^(1) (x) u_k^(2) (x) u_k^(3); its side matrices are stored here
as arrays U of shape (3, R, n): U[l, k] is the k-th canonical vector of axis l.

Names follow the paper: p_q are the Newton-kernel vectors (Appendix 3), W are
the convolved factors u_k * p_q (Sec. 2.5, Eq. conv and the V_H formula of
Sec. 3.1), G_q^(l) = U^(l)T (p_q * U^(l)) are the convolution matrices M_k^(l)
of Sec. 3.2 (Eq. Factor_Mk_Conv), and E_H = h^3 <f, P_R * f> uses the CP scalar
product (Sec. 2.5, Eq. scal).
"""
from __future__ import annotations

import numpy as np


def cell_centres(n: int, b: float) -> np.ndarray:
    h = 2.0 * b / n
    return -b + (np.arange(n, dtype=np.float64) + 0.5) * h


def sample_gaussians(n: int, b: float, a: np.ndarray, X: np.ndarray) -> np.ndarray:
    """U[l, k, i] = exp(-a_k (x_i - X_{k,l})^2): the rank-1 factors of each
    Gaussian exp(-a_k |x - X_k|^2) sampled at cell centres (Sec. 3.1, Eq. disc_GTO)."""
    x = cell_centres(n, b)
    U = np.empty((3, len(a), n))
    for l in range(3):
        U[l] = np.exp(-a[:, None] * np.square(x[None, :] - X[:, l][:, None]))
    return U


def toeplitz_from_even(p: np.ndarray) -> np.ndarray:
    """n x n matrix T[i, j] = p[|i - j|] for an even kernel given at offsets 0..n-1."""
    n = p.shape[0]
    idx = np.abs(np.arange(n)[:, None] - np.arange(n)[None, :])
    return p[idx]


def conv1d(u: np.ndarray, p: np.ndarray) -> np.ndarray:
    """w[i] = sum_{j=0}^{n-1} u[j] p[i - j], i = 0..n-1 (the univariate convolution
    of Sec. 2.5, restricted to the grid); p is even and given at offsets 0..n-1.
    ``u`` may be (n,) or (n, cols)."""
    return toeplitz_from_even(p) @ u


def conv1d_direct(u: np.ndarray, p: np.ndarray) -> np.ndarray:
    """The same w = u * p for one column by numpy's direct (O(n^2)) linear
    convolution with the kernel spread over offsets -(n-1)..n-1: output index
    i + n - 1 of the full convolution is w[i]."""
    n = u.shape[0]
    p_sym = np.concatenate([p[:0:-1], p])  # offsets -(n-1)..n-1
    return np.convolve(u, p_sym)[n - 1:2 * n - 1]


def convolve_factors(U: np.ndarray, P: np.ndarray) -> np.ndarray:
    """W[l, k*R_N + q, :] = U[l, k] * p_q for every axis l, rank k and kernel term q.

    These are the factors of V_H = f * P_R (Sec. 3.1): column k*R_N + q of axis l
    holds the 1D convolution of u_k^(l) with p_q."""
    L, R_f, n = U.shape
    R_N = P.shape[0]
    W = np.empty((L, R_f * R_N, n))
    for l in range(L):
        for q in range(R_N):
            Wq = conv1d(U[l].T, P[q]).T  # (R_f, n)
            W[l, q::R_N] = Wq
    return W


def conv_matrices(U: np.ndarray, W: np.ndarray, R_N: int) -> np.ndarray:
    """G[l, q] = U^(l)T (p_q * U^(l)), shape (3, R_N, R_f, R_f) (Sec. 3.2, Eq. Factor_Mk_Conv)."""
    L, R_f, n = U.shape
    G = np.empty((L, R_N, R_f, R_f))
    for l in range(L):
        for q in range(R_N):
            G[l, q] = U[l] @ W[l, q::R_N].T
    return G


def hartree_energy_from_G(G: np.ndarray, c: np.ndarray, h: float) -> float:
    """E_H = h^3 sum_q sum_{k,k'} c_k c_k' prod_l G[l, q, k, k'] (Sec. 2.5, Eq. scal
    applied to <f, P_R * f>).  The double sum is taken pairwise (numpy's sum)."""
    prod = G[0] * G[1] * G[2]  # (R_N, R_f, R_f)
    cc = np.outer(c, c)
    return float(h ** 3 * np.sum(prod * cc[None, :, :]))


def hartree_energy(U: np.ndarray, c: np.ndarray, P: np.ndarray, h: float) -> float:
    W = convolve_factors(U, P)
    return hartree_energy_from_G(conv_matrices(U, W, P.shape[0]), c, h)


def hartree_energy_adjoint(U: np.ndarray, c: np.ndarray, P: np.ndarray, h: float):
    """Gradients of E_H (Sec. 2.5 Eq. scal with Eq. conv; each T_q is symmetric):

      dE/dU^(l)[:, m] = 2 h^3 c_m sum_q sum_k' c_k' H_q^(l)[m, k'] W_q^(l)[:, k'],
      H_q^(l) = prod_{l' != l} G_q^(l')  (elementwise),
      dE/dc_m        = 2 h^3 sum_q sum_k' c_k' prod_l G_q^(l)[m, k'].

    Returns (dU with U's shape, dc)."""
    L, R_f, n = U.shape
    R_N = P.shape[0]
    W = convolve_factors(U, P)
    G = conv_matrices(U, W, R_N)
    dU = np.zeros_like(U)
    for l in range(L):
        others = [m for m in range(L) if m != l]
        for q in range(R_N):
            H = G[others[0], q] * G[others[1], q]
            B = H * c[None, :]               # B[m, k'] = H[m, k'] c_k'
            dU[l] += 2.0 * h ** 3 * c[:, None] * (B @ W[l, q::R_N])
    prod = G[0] * G[1] * G[2]
    dc = 2.0 * h ** 3 * np.einsum("qmk,k->m", prod, c)
    return dU, dc


def gaussian_param_grad(n: int, b: float, a: np.ndarray, X: np.ndarray,
                        U: np.ndarray, dU: np.ndarray):
    """Chain rule from dE/dU to the Gaussian exponents and centres:
    dU[l,k,i]/da_k = -(x_i - X_kl)^2 U[l,k,i],  dU[l,k,i]/dX_kl = 2 a_k (x_i - X_kl) U[l,k,i]."""
    x = cell_centres(n, b)
    da = np.zeros_like(a)
    dX = np.zeros_like(X)
    for l in range(3):
        d = x[None, :] - X[:, l][:, None]
        da += np.sum(dU[l] * (-(d * d)) * U[l], axis=1)
        dX[:, l] = np.sum(dU[l] * (2.0 * a[:, None] * d) * U[l], axis=1)
    return da, dX


def full_tensor(U: np.ndarray, c: np.ndarray) -> np.ndarray:
    """Dense n^3 tensor sum_k c_k u_k^(1) (x) u_k^(2) (x) u_k^(3) (small n only)."""
    return np.einsum("k,ki,kj,kl->ijl", c, U[0], U[1], U[2])
