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
