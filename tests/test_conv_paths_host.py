"""The host choice of how each kernel term is convolved (no GPU): banded
direct sums for narrow terms, the separable Chebyshev form for smooth terms,
the FFT for the rest (Sec. 2.5, Eq. conv: every path evaluates the same
univariate convolution p_q * u).  The library's choice and its Chebyshev
coefficients are checked against the oracle's own kernel vectors, and the
separable evaluation W = T^T (C (T u)) against the oracle's Toeplitz product."""
import numpy as np
import pytest

from oracle import cp as ocp
from tests.gpu_util import oracle_conv_kernel

CONFIGS = [(256, 6.0, 12), (1024, 8.0, 16), (4096, 16.0, 25), (8192, 20.0, 30)]
# bounds of each W type: band tails (fraction of |p_q|_1), Chebyshev error
# (fraction of p_q[0]; the host checks a quarter of it on a lattice)
TAU = {0: 2.0 ** -32, 1: 2.0 ** -60}
EPS = {0: 2.0 ** -32, 1: 2.0 ** -44}


@pytest.fixture(scope="module")
def cpc():
    import paper_1504_06289_gb300 as m
    from paper_1504_06289_gb300 import build
    build.build()
    return m


def tail_fraction(p, H):
    a = np.abs(p)
    return 2.0 * a[H + 1:].sum() / (a[0] + 2.0 * a[1:].sum())


def cheb_table(n, K=16):
    """T_k(x_i / b) at the cell centres x_i = -b + (i + 1/2) h, from numpy's Chebyshev basis."""
    xh = -1.0 + (2.0 * np.arange(n) + 1.0) / n
    return np.stack([np.polynomial.chebyshev.Chebyshev.basis(k)(xh) for k in range(K)])


def sample_pairs(n, rng, count=4000):
    """Cell pairs (i, j): both ends, the middle and random pairs."""
    ends = np.array([0, 1, n // 2, n - 2, n - 1])
    i = np.concatenate([np.repeat(ends, len(ends)), rng.integers(0, n, count)])
    j = np.concatenate([np.tile(ends, len(ends)), rng.integers(0, n, count)])
    return i, j


@pytest.mark.parametrize("n,b,M", CONFIGS)
def test_paths_partition_terms_and_meet_bounds(cpc, n, b, M):
    hw, rk, cheb = cpc.make_newton_kernel_paths(n, b, M)
    _, _, P0 = oracle_conv_kernel(n, b, M)
    R_N = 2 * M + 1
    assert hw.shape == rk.shape == (2, R_N)
    T = cheb_table(n)
    rng = np.random.default_rng(n)
    ii, jj = sample_pairs(n, rng)
    for cls, hmax in ((0, 20), (1, 24)):
        band, smooth = hw[cls] >= 0, rk[cls] > 0
        assert not (band & smooth).any()
        assert band.any() and smooth.any()
        # narrow terms are the large exponents (the last terms), smooth ones the small
        assert np.all(np.nonzero(smooth)[0] < np.nonzero(band)[0].min())
        for q in np.nonzero(band)[0]:
            assert hw[cls, q] <= hmax and tail_fraction(P0[q], hw[cls, q]) <= TAU[cls]
        for q in np.nonzero(smooth)[0]:
            K = rk[cls, q]
            assert K in (4, 8, 12, 16)
            C = cheb[q, :K, :K]
            # the expansion sum_kl C_kl T_k(x_i) T_l(x_j) against p_q[|i - j|]
            approx = np.einsum("ks,kl,ls->s", T[:K][:, ii], C, T[:K][:, jj])
            err = np.max(np.abs(approx - P0[q][np.abs(ii - jj)]))
            assert err <= EPS[cls] * abs(P0[q][0]), (cls, q, K, err / P0[q][0])
        if n <= 1024:  # every pair of cells for the small grids
            for q in np.nonzero(smooth)[0]:
                K = rk[cls, q]
                A = T[:K].T @ cheb[q, :K, :K] @ T[:K]
                full = ocp.toeplitz_from_even(P0[q])
                assert np.max(np.abs(A - full)) <= EPS[cls] * abs(P0[q][0])


@pytest.mark.parametrize("n,b,M", CONFIGS[:2])
def test_chebyshev_convolution_matches_oracle(cpc, n, b, M):
    """W = sum_k d_k T_k, d = C m, m = T u (the moments): the algebra of the
    device's Chebyshev kernels, against the oracle's direct Toeplitz product."""
    hw, rk, cheb = cpc.make_newton_kernel_paths(n, b, M)
    _, _, P0 = oracle_conv_kernel(n, b, M)
    T = cheb_table(n)
    rng = np.random.default_rng(7)
    x = -b + (np.arange(n) + 0.5) * (2 * b / n)
    U = np.stack([np.exp(-a * (x - c) ** 2) for a, c in zip(10 ** rng.uniform(-1, 1.5, 6), rng.uniform(-1, 1, 6))])
    for cls in (0, 1):
        for q in np.nonzero(rk[cls] > 0)[0]:
            K = rk[cls, q]
            m = T[:K] @ U.T                      # moments, (K, cols)
            d = cheb[q, :K, :K] @ m              # coefficients
            W = (T[:K].T @ d).T                  # (cols, n)
            W0 = np.stack([ocp.conv1d(u, P0[q]) for u in U])
            # |dW| <= eps p_q[0] sum_j |u_j| per output
            bound = EPS[cls] * abs(P0[q][0]) * np.abs(U).sum(axis=1, keepdims=True)
            assert np.all(np.abs(W - W0) <= bound), (cls, q)


def test_limits_switch_paths_off(cpc):
    hw, rk, _ = cpc.make_newton_kernel_paths(256, 6.0, 12, -1, -1, -1, -1)
    assert (hw < 0).all() and (rk < 0).all()
    hw, rk, _ = cpc.make_newton_kernel_paths(256, 6.0, 12, 20, 24, -1, -1)
    assert (hw >= 0).any() and (rk < 0).all()
    hw, rk, _ = cpc.make_newton_kernel_paths(256, 6.0, 12, -1, -1, 16, 16)
    assert (hw < 0).all() and (rk > 0).any()
    from paper_1504_06289_gb300 import CpcError
    for bad in ((33, 24, 16, 16), (20, -2, 16, 16), (20, 24, 17, 16), (20, 24, 16, -2)):
        with pytest.raises(CpcError):
            cpc.make_newton_kernel_paths(256, 6.0, 12, *bad)


@pytest.mark.parametrize("n,b,M", [(8192, 20.0, 30), (4096, 20.0, 25), (256, 6.0, 12), (1024, 8.0, 16)])
def test_energy_path_lag_plan(cpc, n, b, M):
    # the energy paths take the banded terms with half-width H < L from L lag
    # Gram matrices S_m = U^T (U shifted by +-m), m < L (G_q = sum_{m<=H}
    # p_q[m] S_m, exact algebra of the banded sum): L must minimise the rows
    # contracted over the cells, L + #(banded terms with H >= L), over
    # 0 <= L <= 8 with at least L covered terms (their slice slots hold the
    # lag rows), and the row count must add up with the FFT terms
    hw, rk, _ = cpc.make_newton_kernel_paths(n, b, M)
    plan = cpc.make_newton_kernel_eh_plan(n, b, M)
    R_N = 2 * M + 1
    for cls in (0, 1):
        h = [int(x) for x in hw[cls] if x >= 0]
        n_smooth = int((rk[cls] > 0).sum())
        n_fft = R_N - len(h) - n_smooth
        L, n_cov, n_eh = (int(x) for x in plan[cls])
        feasible = [t for t in range(0, 9) if sum(x < t for x in h) >= t]
        best = min(t + sum(x >= t for x in h) for t in feasible)
        assert L in feasible and L + sum(x >= L for x in h) == best
        # ties go to the smallest L (no lag rows unless they save a row)
        assert all(t + sum(x >= t for x in h) > best for t in feasible if t < L)
        assert n_cov == sum(x < L for x in h)
        assert n_eh == (len(h) - n_cov) + n_fft + L
    # the float32 class of the headline workload: half-widths 14, 10, 6, 4, 2,
    # 2, 1, 1 and eight 0: three lags cover twelve terms, 24 rows
    if (n, b, M) == (8192, 20.0, 30):
        assert tuple(plan[0]) == (3, 12, 24)
        assert tuple(plan[1]) == (2, 10, 26)


def _gaussian_columns(n, b, count, seed):
    rng = np.random.default_rng(seed)
    x = -b + (np.arange(n) + 0.5) * (2 * b / n)
    return np.stack([np.exp(-a * (x - c) ** 2)
                     for a, c in zip(10 ** rng.uniform(-1, 1.5, count), rng.uniform(-1, 1, count))])


@pytest.mark.parametrize("n,b,M", CONFIGS[:2])
def test_gram_from_moments_matches_oracle(cpc, n, b, M):
    """The energy paths' Gram matrices of smooth terms: G = m^T d with the K
    moments m = T u of every column and d = C_q m (Sec. 3.2 Eq.
    Factor_Mk_Conv on the separable form), against the oracle's U^T (p_q * U):
    |dG[r][s]| <= eps p_q[0] sum|u_r| sum|u_s| (the fit bound, both sides)."""
    hw, rk, cheb = cpc.make_newton_kernel_paths(n, b, M)
    _, _, P0 = oracle_conv_kernel(n, b, M)
    T = cheb_table(n)
    U = _gaussian_columns(n, b, 8, 11)
    s1 = np.abs(U).sum(axis=1)
    for cls in (0, 1):
        for q in np.nonzero(rk[cls] > 0)[0]:
            K = rk[cls, q]
            m = T[:K] @ U.T                      # (K, cols)
            G = m.T @ (cheb[q, :K, :K] @ m)      # (cols, cols)
            G0 = U @ ocp.conv1d(U.T, P0[q])      # U^T (p_q * U) with cols as rows of U
            bound = EPS[cls] * abs(P0[q][0]) * np.outer(s1, s1)
            assert np.all(np.abs(G - G0) <= bound), (cls, q)
            assert np.allclose(G, G.T, rtol=0, atol=1e-15 * np.abs(G).max())


@pytest.mark.parametrize("n,b,M", CONFIGS[:2])
def test_gram_from_lags_matches_oracle(cpc, n, b, M):
    """The energy paths' Gram matrices of narrow terms: G_q = sum_{m <= H}
    p_q[m] S_m with S_0 = U U^T, S_m = U (U shifted by +m plus U shifted by
    -m)^T (zero outside the grid), for the terms the plan covers (H < L),
    against the oracle's U^T (p_q * U) with p_q cut at H: the same sums in
    another order (float64 rounding apart), and within the banded tail bound
    of the untruncated p_q."""
    hw, _, _ = cpc.make_newton_kernel_paths(n, b, M)
    plan = cpc.make_newton_kernel_eh_plan(n, b, M)
    _, _, P0 = oracle_conv_kernel(n, b, M)
    U = _gaussian_columns(n, b, 8, 13)
    for cls in (0, 1):
        L = int(plan[cls][0])
        assert L >= 1
        S = []
        for m in range(L):
            V = U.copy() if m == 0 else np.zeros_like(U)
            if m:
                V[:, m:] += U[:, :-m]
                V[:, :-m] += U[:, m:]
            S.append(U @ V.T)
        covered = [q for q in range(2 * M + 1) if 0 <= hw[cls, q] < L]
        assert len(covered) == int(plan[cls][1])
        for q in covered:
            H = int(hw[cls, q])
            G = sum(P0[q][m] * S[m] for m in range(H + 1))
            p_cut = np.where(np.arange(n) <= H, P0[q], 0.0)
            Gcut = U @ ocp.conv1d(U.T, p_cut)
            assert np.max(np.abs(G - Gcut)) <= 1e-13 * np.max(np.abs(Gcut))
            G0 = U @ ocp.conv1d(U.T, P0[q])
            tail = TAU[cls] * (abs(P0[q][0]) + 2 * np.abs(P0[q][1:]).sum())
            assert np.max(np.abs(G - G0)) <= tail * np.abs(U).sum(axis=1).max() * np.abs(U).max() + \
                1e-13 * np.max(np.abs(G0))
