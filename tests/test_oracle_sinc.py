"""Pins for the sinc quadrature (Appendix 3, Eq. sinc_Newt) against 1/r itself."""
import math

import numpy as np
import pytest

from oracle import sinc

# (n, b, M, master, bound on max |r * sum - 1| over r in [h, 2 sqrt(3) b])
CASES = {
    "conv n=128 b=10 M=20": (128, 10.0, 20, False, 3e-4),
    "conv n=8192 b=20 M=30": (8192, 20.0, 30, False, 1e-4),
    "conv n=4096 b=20 M=25": (4096, 20.0, 25, False, 2e-4),
    "conv n=4096 b=16 M=25": (4096, 16.0, 25, False, 2e-4),
    "master n=16384 b=64 M=30": (16384, 64.0, 30, True, 1e-4),
}


def _max_rel(n, b, M, master):
    h = 2 * b / n
    t, a = sinc.sinc_nodes(M, h, 2 * math.sqrt(3) * b, master)
    r = np.exp(np.linspace(math.log(h), math.log(2 * math.sqrt(3) * b), 20000))
    return np.max(np.abs(r * sinc.gauss_sum(t, a, r) - 1.0))


@pytest.mark.parametrize("name", list(CASES))
def test_sum_approximates_inverse_r(name):
    n, b, M, master, bound = CASES[name]
    err = _max_rel(n, b, M, master)
    assert err < bound, (name, err)


@pytest.mark.parametrize("name", list(CASES))
def test_error_decreases_with_M(name):
    # exponential convergence in M (Appendix 3, the bound C/a exp(-beta sqrt(M)))
    n, b, M, master, _ = CASES[name]
    errs = [_max_rel(n, b, m, master) for m in (M - 8, M, M + 8)]
    assert errs[0] > errs[1] > errs[2], errs
    assert errs[2] < 0.5 * errs[1]


def test_nodes_are_distinct_positive_and_rank_2M_plus_1():
    t, a = sinc.conv_nodes(128, 10.0, 20)
    assert len(t) == 41 and len(a) == 41
    assert np.all(np.diff(t) > 0) and np.all(a > 0)
    hs = np.log(t[1:] / t[:-1])
    assert np.allclose(hs, hs[0], rtol=1e-12)
    assert np.allclose(a, 2 / math.sqrt(math.pi) * hs[0] * t, rtol=1e-13)


def test_literal_uniform_nodes_double_count():
    # The printed rule t_k = k h_M, a_k = 2 h_M/sqrt(pi), k = -M..M sums the
    # symmetric trapezoid over R (twice the half-line integral): ~2/r at r = 1.
    M = 20
    hM = 3 * math.log(M) / M
    k = np.arange(-M, M + 1)
    s = np.sum(2 / math.sqrt(math.pi) * hM * np.exp(-(k * hM) ** 2))
    assert abs(s - 2.0) < 1e-3


def test_kappa_unit_cube():
    # int_{[0,1]^3} dx/|x| by nested Gauss-Legendre in spherical-like splitting:
    # integrate 1/|x| over the cube as 3 pyramids (x >= y,z etc.) in closed
    # radial form: int_pyramid = int_0^1 dx int_0^1 int_0^1 x^2 dv dw / (x sqrt(1+v^2+w^2))
    #             = 1/2 * int_0^1 int_0^1 dv dw / sqrt(1+v^2+w^2)
    xg, wg = np.polynomial.legendre.leggauss(60)
    v = 0.5 * (xg + 1)
    w = 0.5 * wg
    inner = np.sum(w[:, None] * w[None, :] / np.sqrt(1 + v[:, None] ** 2 + v[None, :] ** 2))
    assert abs(3 * 0.5 * inner - sinc.KAPPA_UNIT_CUBE) < 1e-13


def test_mpmath_integral_identity():
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 40
    # (2/sqrt(pi)) int_0^inf exp(-t^2 r^2) dt = 1/r: pins the prefactor of the weights
    for r in (0.01, 1.0, 37.0):
        v = 2 / mp.sqrt(mp.pi) * mp.quad(lambda t: mp.e ** (-(t * r) ** 2), [0, mp.inf])
        assert abs(v * r - 1) < 1e-30
