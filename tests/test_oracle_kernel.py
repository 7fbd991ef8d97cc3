"""Pins for the Galerkin kernel vectors p_q (Appendix 3, Eq. galten) and P_R."""
import math

import numpy as np
import pytest

from oracle import kernel_vectors as kv
from oracle import sinc
from tests import prism


def test_prism_formula_unit_cube_and_quadrature():
    assert abs(prism.box_nonneg(0, 1, 0, 1, 0, 1) - sinc.KAPPA_UNIT_CUBE) < 1e-14
    # an offset box against tensor Gauss-Legendre (smooth integrand there)
    xg, wg = np.polynomial.legendre.leggauss(30)
    lo, hi = np.array([1.0, -0.5, 2.0]), np.array([1.7, 0.25, 2.4])
    pts = [0.5 * (hi[l] - lo[l]) * xg + 0.5 * (hi[l] + lo[l]) for l in range(3)]
    ws = [0.5 * (hi[l] - lo[l]) * wg for l in range(3)]
    X, Y, Z = np.meshgrid(*pts, indexing="ij")
    Wt = ws[0][:, None, None] * ws[1][None, :, None] * ws[2][None, None, :]
    ref = np.sum(Wt / np.sqrt(X * X + Y * Y + Z * Z))
    assert abs(prism.box(lo, hi) / ref - 1) < 1e-13


def test_cell_integrals_against_mpmath():
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 50
    n, b, M = 128, 10.0, 20
    h = 2 * b / n
    t, a = sinc.conv_nodes(n, b, M)
    rng = np.random.default_rng(5)
    P = kv.conv_kernel_vectors(n, b, t, a)
    Pm = kv.master_kernel_vectors(n, b, t, a)
    checked = 0
    for q in range(len(t)):
        tq = mp.mpf(t[q])
        for m in sorted(set([0, 1, 2, n - 1] + list(rng.integers(0, n, 4)))):
            exact = mp.cbrt(mp.mpf(a[q])) * mp.sqrt(mp.pi) / (2 * tq) * (
                mp.erf(tq * (m + 0.5) * h) - mp.erf(tq * (m - 0.5) * h))
            # relative 1e-13 where the entry matters (>= 1e-12 of the vector's peak),
            # absolute 1e-13 of the peak in the far tail
            peak = P[q, 0]
            if float(exact) >= 1e-12 * peak:
                assert abs(P[q, m] / float(exact) - 1) < 1e-13, (q, m)
            else:
                assert abs(P[q, m] - float(exact)) < 1e-13 * peak, (q, m)
            checked += 1
        for j in [-n, -1, 0, 5, n - 1]:
            exact = mp.cbrt(mp.mpf(a[q])) * mp.sqrt(mp.pi) / (2 * tq) * (
                mp.erf(tq * (j + 1) * h) - mp.erf(tq * j * h))
            peak = Pm[q, n]
            if float(exact) >= 1e-12 * peak:
                assert abs(Pm[q, j + n] / float(exact) - 1) < 1e-13, (q, j)
            else:
                assert abs(Pm[q, j + n] - float(exact)) < 1e-13 * peak, (q, j)
            checked += 1
    assert checked > 300


def test_cell_integrals_telescope_to_gaussian_integral():
    # sum over all cells of int exp(-t^2 x^2) = the integral over the covered interval
    n, b = 128, 10.0
    h = 2 * b / n
    t, a = sinc.conv_nodes(n, b, 20)
    P = kv.conv_kernel_vectors(n, b, t, a)
    total = P[:, 0] + 2 * P[:, 1:].sum(axis=1)
    from scipy.special import erf
    ref = np.cbrt(a) * math.sqrt(math.pi) / t * erf(t * (n - 0.5) * h)
    assert np.max(np.abs(total / ref - 1)) < 1e-13


@pytest.mark.parametrize("n,b,M,bound", [(128, 10.0, 20, 3e-4), (4096, 20.0, 25, 2e-4),
                                          (8192, 20.0, 30, 1e-4)])
def test_PR_matches_exact_galerkin_entries(n, b, M, bound):
    # P_R entries sum_q p_q[i] p_q[j] p_q[k] against the exact cell integral of 1/|x|
    # (the max-norm criterion of Appendix 3); offsets near and far from the origin.
    h = 2 * b / n
    t, a = sinc.conv_nodes(n, b, M)
    offs = [(0, 0, 0), (1, 0, 0), (1, 1, 1), (2, 1, 0), (3, 2, 1), (7, 7, 0), (40, 3, 1),
            (n - 1, 0, 0), (n // 2, n // 3, n // 5), (n - 1, n - 1, n - 1)]
    need = sorted(set(v for o in offs for v in o))
    sub = np.array(need)
    lo, hi = (sub - 0.5) * h, (sub + 0.5) * h
    vec = np.stack([np.cbrt(a[q]) * kv.gauss_cell_integral(float(t[q]), lo, hi)
                    for q in range(len(t))])
    col = {m: i for i, m in enumerate(need)}
    for o in offs:
        PR = float(np.sum(vec[:, col[o[0]]] * vec[:, col[o[1]]] * vec[:, col[o[2]]]))
        ex = prism.cell([(o[l] - 0.5) * h for l in range(3)], [(o[l] + 0.5) * h for l in range(3)])
        assert abs(PR / ex - 1) < bound, (o, PR / ex - 1)


def test_master_corner_cells_match_exact():
    n, b, M = 16384, 64.0, 30
    h = 2 * b / n
    t, a = sinc.master_nodes(n, b, M)
    for j in [(0, 0, 0), (-1, 0, 0), (-1, -1, -1), (3, -2, 1), (100, 50, -70), (n - 1, -n, 0)]:
        v = 1.0
        PR = 0.0
        for q in range(len(t)):
            pr = a[q]
            for l in range(3):
                pr *= kv.gauss_cell_integral(float(t[q]), np.array([j[l] * h]), np.array([(j[l] + 1) * h]))[0]
            PR += pr
        ex = prism.cell([j[l] * h for l in range(3)], [(j[l] + 1) * h for l in range(3)])
        assert abs(PR / ex - 1) < 1e-4, (j, PR / ex - 1)
