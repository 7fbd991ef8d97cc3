"""Pins for the TEI oracle (oracle/tei.py, Sec. 3.2): 1D density fitting,
the TEI matrix from its factors, and its truncated Cholesky factorisation."""
import math

import numpy as np

import workloads
from oracle import closed_forms as cf
from oracle import coulomb, cp, kernel_vectors as kv, sinc, tei


def _kernel(n, b, M):
    t, a = sinc.conv_nodes(n, b, M)
    return kv.conv_kernel_vectors(n, b, t, a)


def _prims(nb, seed, a_lo=0.4, a_hi=3.0, half=1.0):
    g = workloads.gaussian_mixture(nb, a_lo, a_hi, seed, centre_half=half)
    return g["a"], g["X"]


def test_pivoted_cholesky_reproduces_spd_and_low_rank_matrices():
    rng = np.random.default_rng(0)
    X = rng.standard_normal((30, 30))
    A = X @ X.T + 30 * np.eye(30)
    L, piv = tei.pivoted_cholesky(np.diag(A).copy(), lambda p: A[:, p], 0.0, 30)
    assert L.shape == (30, 30) and len(set(piv.tolist())) == 30
    assert np.max(np.abs(L @ L.T - A)) < 1e-12 * np.max(np.abs(A))
    # lower triangular in pivot order, as numpy's Cholesky of the permuted matrix
    Lc = np.linalg.cholesky(A[np.ix_(piv, piv)])
    assert np.allclose(L[piv], Lc, rtol=0, atol=1e-12 * np.max(np.abs(Lc)))
    Y = rng.standard_normal((40, 7))
    A7 = Y @ Y.T
    L7, piv7 = tei.pivoted_cholesky(np.diag(A7).copy(), lambda p: A7[:, p], 1e-12, 40)
    assert L7.shape[1] == 7
    assert np.max(np.abs(L7 @ L7.T - A7)) < 1e-10 * np.max(np.abs(A7))


def test_density_fit_error_follows_the_tolerance():
    n, b = 128, 5.0
    a, X = _prims(6, 2)
    U = cp.sample_gaussians(n, b, a, X)
    pa, pb = tei.pair_list(6)
    G = tei.side_matrix(U[0], pa, pb)
    errs = []
    for tol in (1e-4, 1e-8, 1e-12):
        Uf, Vf, I = tei.density_fit(G, tol, 128)
        errs.append(np.linalg.norm(Uf @ Vf.T - G) / np.linalg.norm(G))
        assert Uf.shape[1] == len(I) <= len(pa)
    assert errs[0] > errs[1] > errs[2]
    assert errs[2] < 1e-5


def test_direct_tei_converges_to_analytic_integrals():
    # (mu nu | kappa lambda) of s primitives by the Gaussian product theorem
    b, M = 6.0, 20
    a, X = _prims(3, 5)
    pa, pb = tei.pair_list(3)
    def prod(mu, nu):
        p = a[mu] + a[nu]
        K = math.exp(-a[mu] * a[nu] / p * float(np.sum((X[mu] - X[nu]) ** 2)))
        return K, p, (a[mu] * X[mu] + a[nu] * X[nu]) / p
    B0 = np.zeros((len(pa), len(pa)))
    for i in range(len(pa)):
        K1, p1, P1 = prod(pa[i], pb[i])
        for j in range(len(pa)):
            K2, p2, P2 = prod(pa[j], pb[j])
            B0[i, j] = K1 * K2 * float(cf.coulomb_pair(p1, P1, p2, P2))
    errs = []
    for n in (64, 128, 256):
        U = cp.sample_gaussians(n, b, a, X)
        B = tei.tei_matrix_direct(U, _kernel(n, b, M), 2 * b / n, pa, pb)
        errs.append(np.max(np.abs(B - B0)) / np.max(np.abs(B0)))
    assert errs[2] < 3e-4
    assert errs[0] / errs[1] > 3.0 and errs[1] / errs[2] > 3.0


def test_tei_from_fitted_factors_and_its_cholesky():
    n, b, M = 128, 6.0, 16
    h = 2 * b / n
    a, X = _prims(5, 7)
    U = cp.sample_gaussians(n, b, a, X)
    P = _kernel(n, b, M)
    pa, pb = tei.pair_list(5)
    B0 = tei.tei_matrix_direct(U, P, h, pa, pb)
    L, piv, Uf, Vf, Mf = tei.tei_cholesky(U, P, h, pa, pb, 1e-13, 1e-12, 128, 64)
    B = np.stack([tei.tei_column(Vf, Mf, h, j) for j in range(len(pa))], axis=1)
    assert np.max(np.abs(B - B0)) < 1e-7 * np.max(np.abs(B0))
    assert np.allclose(np.diag(B), tei.tei_diagonal(Vf, Mf, h), rtol=1e-12, atol=0)
    assert np.max(np.abs(L @ L.T - B)) < 1e-10 * np.max(np.abs(B))
    assert L.shape[1] <= len(pa)


def test_coulomb_matrix_of_a_diagonal_density_agrees_with_the_product_form():
    # J(D) for D = diag(w) through B ~ L L^T equals the Coulomb matrix of
    # rho = sum w_mu g_mu^2 computed from the V_H factors (Sec. 3.1)
    n, b, M = 128, 6.0, 16
    h = 2 * b / n
    nb = 5
    a, X = _prims(nb, 9)
    w = np.linspace(0.5, 1.5, nb)
    U = cp.sample_gaussians(n, b, a, X)
    P = _kernel(n, b, M)
    pa, pb = tei.pair_list(nb)
    L, *_ = tei.tei_cholesky(U, P, h, pa, pb, 1e-13, 1e-12, 128, 64)
    J = tei.coulomb_from_cholesky(L, np.diag(w), pa, pb)
    basis = dict(fn_first=np.arange(nb + 1), prim_alpha=a, prim_d=np.ones(nb), fn_centre=X, w=w)
    items = list(zip(pa.tolist(), pb.tolist()))
    J0, _ = coulomb.coulomb_items(n, b, basis, P, items)
    assert np.max(np.abs(J - J0)) < 1e-7 * np.max(np.abs(J0))


def test_exchange_matrix_against_analytic_integrals_and_the_factor():
    # K_km = sum_{mu nu} D_{mu nu} (k mu | m nu): from the direct TEI matrix
    # (converging to the analytic integrals) and from B ~ L L^T
    b, M, nb = 6.0, 20, 4
    a, X = _prims(nb, 13)
    pa, pb = tei.pair_list(nb)
    rng = np.random.default_rng(1)
    C = rng.standard_normal((nb, 2))
    D = C @ C.T  # two orbitals
    def eri(k, mu, m, nu):
        p, q = a[k] + a[mu], a[m] + a[nu]
        K1 = math.exp(-a[k] * a[mu] / p * float(np.sum((X[k] - X[mu]) ** 2)))
        K2 = math.exp(-a[m] * a[nu] / q * float(np.sum((X[m] - X[nu]) ** 2)))
        P1, P2 = (a[k] * X[k] + a[mu] * X[mu]) / p, (a[m] * X[m] + a[nu] * X[nu]) / q
        return K1 * K2 * float(cf.coulomb_pair(p, P1, q, P2))
    K0 = np.array([[sum(D[mu, nu] * eri(k, mu, m, nu) for mu in range(nb) for nu in range(nb))
                    for m in range(nb)] for k in range(nb)])
    errs = []
    for n in (64, 128):
        h = 2 * b / n
        U = cp.sample_gaussians(n, b, a, X)
        P = _kernel(n, b, M)
        Bd = tei.tei_matrix_direct(U, P, h, pa, pb)
        K = tei.exchange_from_tei(Bd, D, pa, pb)
        errs.append(np.max(np.abs(K - K0)) / np.max(np.abs(K0)))
        L, *_ = tei.tei_cholesky(U, P, h, pa, pb, 1e-13, 1e-13, 128, len(pa))
        Kc = tei.exchange_from_cholesky(L, D, pa, pb)
        assert np.max(np.abs(Kc - K)) < 1e-7 * np.max(np.abs(K))
        assert np.allclose(Kc, Kc.T, rtol=0, atol=1e-12 * np.max(np.abs(Kc)))
    assert errs[1] < 2e-3 and errs[0] / errs[1] > 3.0
