"""Two-electron integrals by 1D density fitting and a low-rank Cholesky
factorisation (Sec. 3.2).

TEST INFRASTRUCTURE ONLY (see the package docstring).

For a basis of N_b s-type primitive Gaussians g_mu (each rank 1), the pair
products g_mu g_nu (mu <= nu, N_P = N_b (N_b + 1)/2 of them) have, per axis l,
the side matrix G^(l) = [g_mu^(l) . g_nu^(l)] of size n x N_P (Sec. 3.2).
The steps follow the paper's order:

1. 1D density fitting (Eq. 1DDensFit): G^(l) ~ U^(l) V^(l)T from the truncated
   Cholesky factorisation of A = G^(l) G^(l)T.  Reading: diagonal pivoting,
   stopped when the largest remaining diagonal falls to tol times the largest
   diagonal of A; with pivots I and A ~ L L^T,
       U = A[:, I] A[I, I]^{-1} = L L[I, :]^{-1},   V = G[I, :]^T,
   i.e. each grid row of G is projected on the span of the pivot rows.
2. Convolution matrices (Eq. Factor_Mk_Conv): M_k^(l) = U^(l)T (p_k * U^(l)).
3. The TEI matrix B = h^3 sum_k (.)_l V^(l) M_k^(l) V^(l)T (Hadamard product
   over the axes), entries b_{mu nu, kappa lambda} = <G_mu . G_nu, P_R * (G_kappa . G_lambda)>
   (Eq. TEI_tens); h^3 is the quadrature weight of the discrete scalar product
   (as in E_H).  Its diagonal and selected columns are formed from the
   factors only, and the truncated Cholesky factorisation B ~ L L^T is built
   from them (same pivoting and stopping rule).
4. The Coulomb matrix of a density matrix D (symmetric, N_b x N_b):
   J_{mu nu} = sum_{kappa, lambda} b_{mu nu, kappa lambda} D_{kappa lambda}
             = (L (L^T d))_{mu nu},  d_{kappa lambda} = (2 - delta_{kappa lambda}) D_{kappa lambda}
   over the pairs kappa <= lambda.
5. The exchange matrix: the exchange operator of Sec. 3.1,
   K_km,a = <G_k . phi_a, (G_m . phi_a) * P_R> with phi_a = sum_mu c_{mu a} G_mu,
   summed over the orbitals a with D = sum_a c_a c_a^T, is
   K_km = sum_{mu nu} D_{mu nu} b_{k mu, m nu}; with B ~ L L^T,
   K = sum_s X_s D X_s^T, X_s[k, mu] = L[(k mu), s] (the pair of g_k g_mu).
"""
from __future__ import annotations

import numpy as np

from . import cp


def pair_list(nb: int):
    """Pairs (mu, nu), mu <= nu, in row-major order of the upper triangle."""
    pa, pb = np.triu_indices(nb)
    return pa, pb


def side_matrix(U_l: np.ndarray, pa: np.ndarray, pb: np.ndarray) -> np.ndarray:
    """G^(l)[i, p] = g_{pa[p]}^(l)[i] g_{pb[p]}^(l)[i]; U_l is (N_b, n)."""
    return (U_l[pa] * U_l[pb]).T


def pivoted_cholesky(diag: np.ndarray, column, tol: float, max_rank: int):
    """Truncated Cholesky factorisation with diagonal pivoting of an SPD matrix
    given by its diagonal and a column function.  Stops when the largest
    remaining diagonal is <= tol times the largest initial diagonal, or at
    max_rank.  Returns L (N x r) and the pivots (r,)."""
    d = np.array(diag, dtype=np.float64)
    N = d.shape[0]
    stop = tol * float(np.max(d))
    L = np.zeros((N, max_rank))
    piv = []
    for s in range(max_rank):
        p = int(np.argmax(d))
        if d[p] <= stop:
            break
        c = column(p) - L[:, :s] @ L[p, :s]
        L[:, s] = c / np.sqrt(d[p])
        d = d - L[:, s] ** 2
        piv.append(p)
    r = len(piv)
    return L[:, :r], np.array(piv, dtype=np.int64)


def density_fit(G: np.ndarray, tol: float, max_rank: int):
    """G (n x N_P) ~ U V^T by the truncated Cholesky of A = G G^T (step 1)."""
    A = G @ G.T
    L, I = pivoted_cholesky(np.diag(A).copy(), lambda p: A[:, p], tol, max_rank)
    U = np.linalg.solve(L[I, :].T, L.T).T  # L L[I, :]^{-1}
    V = G[I, :].T
    return U, V, I


def conv_matrices_axis(U: np.ndarray, P: np.ndarray) -> np.ndarray:
    """M_k = U^T (p_k * U) for one axis, shape (R_N, R, R) (step 2)."""
    W = cp.convolve_factors(U.T[None], P)  # (1, R R_N, n), column k R_N + q
    R, R_N = U.shape[1], P.shape[0]
    M = np.empty((R_N, R, R))
    for q in range(R_N):
        M[q] = U.T @ W[0, q::R_N].T
    return M


def tei_column(V: list, M: list, h: float, j: int) -> np.ndarray:
    """B[:, j] = h^3 sum_k prod_l V^(l) (M_k^(l) V^(l)[j, :]^T) (step 3)."""
    out = np.zeros(V[0].shape[0])
    for k in range(M[0].shape[0]):
        prod = np.ones(V[0].shape[0])
        for l in range(3):
            prod *= V[l] @ (M[l][k] @ V[l][j])
        out += prod
    return h ** 3 * out


def tei_diagonal(V: list, M: list, h: float) -> np.ndarray:
    """B[i, i] = h^3 sum_k prod_l V^(l)[i, :] M_k^(l) V^(l)[i, :]^T (step 3)."""
    out = np.zeros(V[0].shape[0])
    for k in range(M[0].shape[0]):
        prod = np.ones(V[0].shape[0])
        for l in range(3):
            prod *= np.einsum("ir,rs,is->i", V[l], M[l][k], V[l])
        out += prod
    return h ** 3 * out


def tei_matrix_direct(U_prims: np.ndarray, P: np.ndarray, h: float, pa, pb) -> np.ndarray:
    """B without density fitting: h^3 sum_k prod_l G^(l)T (p_k * G^(l)) (Eq. TEI_tens
    with the full side matrices); small N_b only."""
    B = np.zeros((len(pa), len(pa)))
    for k in range(P.shape[0]):
        prod = np.ones_like(B)
        for l in range(3):
            G = side_matrix(U_prims[l], pa, pb)
            prod *= G.T @ cp.conv1d(G, P[k])
        B += prod
    return h ** 3 * B


def tei_cholesky(U_prims: np.ndarray, P: np.ndarray, h: float, pa, pb, tol_df: float, tol_b: float,
                 max_rank_df: int, max_rank_b: int):
    """Steps 1-3: the factor L of B ~ L L^T, with the fitted factors."""
    U, V, M = [], [], []
    for l in range(3):
        Ul, Vl, _ = density_fit(side_matrix(U_prims[l], pa, pb), tol_df, max_rank_df)
        U.append(Ul)
        V.append(Vl)
        M.append(conv_matrices_axis(Ul, P))
    L, piv = pivoted_cholesky(tei_diagonal(V, M, h), lambda j: tei_column(V, M, h, j), tol_b, max_rank_b)
    return L, piv, U, V, M


def coulomb_from_cholesky(L: np.ndarray, D: np.ndarray, pa, pb) -> np.ndarray:
    """J over the pairs (step 4)."""
    d = np.where(pa == pb, 1.0, 2.0) * D[pa, pb]
    return L @ (L.T @ d)


def pair_index(nb: int, pa: np.ndarray, pb: np.ndarray) -> np.ndarray:
    """(nb, nb) map of (kappa, lambda) to the pair holding g_kappa g_lambda (either order), -1 if none."""
    idx = -np.ones((nb, nb), dtype=np.int64)
    idx[pa, pb] = np.arange(len(pa))
    idx[pb, pa] = np.arange(len(pa))
    return idx


def exchange_from_tei(B: np.ndarray, D: np.ndarray, pa, pb) -> np.ndarray:
    """Exchange matrix K_km = sum_a K_km,a = sum_{mu nu} D_{mu nu} (k mu | m nu) (Sec. 3.1, the
    exchange operator K_km,a with the orbitals summed into D = sum_a c_a c_a^T), from a TEI
    matrix B over the pairs."""
    nb = D.shape[0]
    idx = pair_index(nb, pa, pb)
    K = np.zeros((nb, nb))
    for k in range(nb):
        for m in range(nb):
            K[k, m] = float(np.sum(B[np.ix_(idx[k], idx[m])] * D))
    return K


def exchange_from_cholesky(L: np.ndarray, D: np.ndarray, pa, pb) -> np.ndarray:
    """The same from B ~ L L^T: K = sum_s X_s D X_s^T with X_s[k, mu] = L[(k mu), s]."""
    nb = D.shape[0]
    idx = pair_index(nb, pa, pb)
    K = np.zeros((nb, nb))
    for s in range(L.shape[1]):
        X = L[idx, s]
        K += X @ D @ X.T
    return K
