"""Galerkin cell integrals of the sinc-quadrature Newton kernel (Appendix 3).

TEST INFRASTRUCTURE ONLY (see the package docstring).

With piecewise-constant basis functions on cells of width h, the canonical
vectors of P_R are p_q = a_q^{1/3} [ int_{cell} exp(-t_q^2 x^2) dx ] over the
cells (Appendix 3, Eq. galten and the definition of p_q^(l)), and P_R is the
sum over q of p_q (x) p_q (x) p_q, the same vector on all three axes.

Two index sets are used:

* convolution kernel (Sec. 3.1): cells centred at m*h, m = -(n-1)..n-1, i.e.
  the offsets between two cell centres of the n-cell grid.  The vector is even
  in m, so it is returned for m = 0..n-1 only (shape (R, n)).
* master kernel for lattice sums (Sec. 5.1, Eq. refTensor): 2n cells
  [j h, (j+1) h], j = -n..n-1, with the origin on a cell edge.  Returned for
  j = -n..n-1 (shape (R, 2n), column 0 is j = -n).

The integral of exp(-t^2 x^2) over [x0, x1]:
* t*h < 0.05: 20-point Gauss-Legendre on the cell (the integrand varies slowly
  across the cell, and erf differences would cancel);
* 0.5 <= t*min(|x0|,|x1|) on one side of 0: difference of erfc values;
* otherwise: difference of erf values;
both closed forms carry the factor sqrt(pi)/(2t).
"""
from __future__ import annotations

import math

import numpy as np
from scipy.special import erf, erfc

_GL_X, _GL_W = np.polynomial.legendre.leggauss(20)


def gauss_cell_integral(t: float, x0: np.ndarray, x1: np.ndarray) -> np.ndarray:
    """int_{x0}^{x1} exp(-t^2 x^2) dx elementwise, x0 < x1 (float64)."""
    x0 = np.asarray(x0, dtype=np.float64)
    x1 = np.asarray(x1, dtype=np.float64)
    width = x1 - x0
    out = np.empty(np.broadcast(x0, x1).shape)
    if t * float(np.max(width)) < 0.05:
        mid = 0.5 * (x0 + x1)
        half = 0.5 * width
        xs = mid[..., None] + half[..., None] * _GL_X
        out[...] = half * (np.exp(-np.square(t * xs)) @ _GL_W)
        return out
    scale = math.sqrt(math.pi) / (2.0 * t)
    # reflect cells lying in x < 0 to x > 0 (the integrand is even)
    neg = x1 <= 0.0
    lo = np.where(neg, -x1, x0)
    hi = np.where(neg, -x0, x1)
    use_erfc = (lo * t >= 0.5)
    out[...] = np.where(use_erfc,
                        scale * (erfc(t * lo) - erfc(t * hi)),
                        scale * (erf(t * hi) - erf(t * lo)))
    return out


def conv_kernel_vectors(n: int, b: float, t: np.ndarray, a: np.ndarray) -> np.ndarray:
    """p_q[m], m = 0..n-1, q = 0..R-1: a_q^{1/3} * int_{(m-1/2)h}^{(m+1/2)h} exp(-t_q^2 x^2) dx."""
    h = 2.0 * b / n
    m = np.arange(n, dtype=np.float64)
    x0, x1 = (m - 0.5) * h, (m + 0.5) * h
    P = np.empty((len(t), n))
    for q in range(len(t)):
        P[q] = np.cbrt(a[q]) * gauss_cell_integral(float(t[q]), x0, x1)
    return P


def master_kernel_vectors(n: int, b: float, t: np.ndarray, a: np.ndarray) -> np.ndarray:
    """p~_q[j], j = -n..n-1 stored at column j+n: a_q^{1/3} int_{jh}^{(j+1)h} exp(-t_q^2 x^2) dx."""
    h = 2.0 * b / n
    j = np.arange(-n, n, dtype=np.float64)
    x0, x1 = j * h, (j + 1.0) * h
    P = np.empty((len(t), 2 * n))
    for q in range(len(t)):
        P[q] = np.cbrt(a[q]) * gauss_cell_integral(float(t[q]), x0, x1)
    return P
