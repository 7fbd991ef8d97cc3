"""Sinc quadrature of the Laplace-Gauss transform of 1/r (Appendix 3, Eq. sinc_Newt).

TEST INFRASTRUCTURE ONLY (see the package docstring).

The paper writes 1/r = (2/sqrt(pi)) * int_0^inf exp(-t^2 r^2) dt and replaces the
integral by a (2M+1)-point sinc (trapezoidal) rule.  Taken literally, its nodes
t_k = k*h_M with equal weights sum the symmetric rule over the whole real line
(twice the half-line integral) and repeat each Gaussian for +k and -k.  The
reading used here substitutes t = exp(u), which turns the half-line integral
into a whole-line one with a doubly exponentially decaying integrand:

    1/r = (2/sqrt(pi)) * int_R exp(-exp(2u) r^2) exp(u) du
        ~ sum_{k=-M..M} a_k exp(-t_k^2 r^2),
    t_k = exp(u0 + k*hs),   a_k = (2/sqrt(pi)) * hs * t_k,

so there are 2M+1 distinct positive terms, R = 2M+1, renumbered q = k+M+1.
The step has the paper's form hs = C0 log(M)/M with the constant C0 left open;
hs and the shift u0 are fixed by balancing three error estimates of the
Galerkin tensor P_R against P in the max norm the paper uses for choosing M:

* discretisation, relative, any r:  E_d = 2 sqrt(2) exp(-pi^2/(2 hs))  (the
  Fourier transform of the integrand in u is Gamma(1/2 - i w/2)/sqrt(pi));
* lower truncation (terms k < -M, where t r << 1), relative at r = r_max:
  E_lo = (2/sqrt(pi)) hs r_max exp(u0 - M hs) e^{-hs} / (1 - e^{-hs});
* upper truncation (terms k > M): the dropped Gaussians are narrower than a
  cell, so they lose their whole integral 2 pi hs / t^2 each from the cell(s)
  touching the origin.  Relative to that cell's entry
  P_0 = kappa h^2 * (8 for the convolution kernel, whose central cell
  [-h/2, h/2]^3 holds the origin; 1 for the master kernel, whose origin is a
  cell corner shared by 8 cells, each receiving 1/8):
  E_hi = 2 pi hs exp(-2 (u0 + M hs + hs)) / (1 - e^{-2 hs}) / (share * P_0),
  kappa = int_{[0,1]^3} dx/|x| = 3 ln((1 + sqrt 3)/sqrt 2) - pi/4.

u0 solves E_lo = E_hi for a given hs (bisection); hs solves E_d = E_lo
(bisection).  Both are continuous in (M, h, r_max) and monotone where solved.
"""
from __future__ import annotations

import math

import numpy as np

_TWO_OVER_SQRTPI = 2.0 / math.sqrt(math.pi)
KAPPA_UNIT_CUBE = 3.0 * math.log((1.0 + math.sqrt(3.0)) / math.sqrt(2.0)) - math.pi / 4.0


def _log_errors(M: int, hs: float, u0: float, h: float, r_max: float, master: bool):
    log_lo = (math.log(_TWO_OVER_SQRTPI * hs * r_max) + (u0 - M * hs) - hs
              - math.log(-math.expm1(-hs)))
    # convolution: the central cell [-h/2,h/2]^3 holds the whole Gaussian, entry 8 kappa (h/2)^2;
    # master: each of the 8 corner cells [0,h]^3 holds 1/8 of it, entry kappa h^2.
    cell = 2.0 * KAPPA_UNIT_CUBE * h * h if not master else 8.0 * KAPPA_UNIT_CUBE * h * h
    log_hi = (math.log(2.0 * math.pi * hs / -math.expm1(-2.0 * hs) / cell)
              - 2.0 * (u0 + M * hs + hs))
    log_d = math.log(2.0 * math.sqrt(2.0)) - math.pi ** 2 / (2.0 * hs)
    return log_lo, log_hi, log_d


def _balance_shift(M, hs, h, r_max, master):
    lo, hi = -200.0, 200.0
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        e_lo, e_hi, _ = _log_errors(M, hs, mid, h, r_max, master)
        if e_lo > e_hi:
            hi = mid
        else:
            lo = mid
    return 0.5 * (lo + hi)


def sinc_step_and_shift(M: int, h: float, r_max: float, master: bool = False):
    """(hs, u0) of the balanced rule described in the module docstring."""
    if M < 1 or not (0.0 < h < r_max):
        raise ValueError("need M >= 1 and 0 < h < r_max")
    lo, hi = 0.02, 3.0
    for _ in range(200):
        hs = 0.5 * (lo + hi)
        u0 = _balance_shift(M, hs, h, r_max, master)
        e_lo, _, e_d = _log_errors(M, hs, u0, h, r_max, master)
        if e_d > e_lo:
            hi = hs
        else:
            lo = hs
    hs = 0.5 * (lo + hi)
    return hs, _balance_shift(M, hs, h, r_max, master)


def sinc_nodes(M: int, h: float, r_max: float, master: bool = False):
    """Nodes t_q and weights a_q, q = 1..2M+1 in increasing t (Appendix 3)."""
    hs, u0 = sinc_step_and_shift(M, h, r_max, master)
    k = np.arange(-M, M + 1, dtype=np.float64)
    t = np.exp(u0 + k * hs)
    a = _TWO_OVER_SQRTPI * hs * t
    return t, a


def conv_nodes(n: int, b: float, M: int):
    """Nodes of the convolution kernel on [-b,b]^3, h = 2b/n: distances up to the
    box diagonal 2 sqrt(3) b."""
    return sinc_nodes(M, 2.0 * b / n, 2.0 * math.sqrt(3.0) * b, master=False)


def master_nodes(n: int, b: float, M: int):
    """Nodes of the 2n master kernel for lattice sums (Sec. 5.1): charges and
    evaluation points share the n-cell box of edge 2b, distances up to 2 sqrt(3) b."""
    return sinc_nodes(M, 2.0 * b / n, 2.0 * math.sqrt(3.0) * b, master=True)


def gauss_sum(t: np.ndarray, a: np.ndarray, r: np.ndarray) -> np.ndarray:
    """sum_q a_q exp(-t_q^2 r^2) at each r (the right side of Eq. sinc_Newt)."""
    r = np.asarray(r, dtype=np.float64)
    return (a[None, :] * np.exp(-np.square(np.outer(r, t)))).sum(axis=1)
