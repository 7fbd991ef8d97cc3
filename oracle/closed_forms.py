"""Analytic Gaussian Coulomb results used to pin the oracle.

TEST INFRASTRUCTURE ONLY (see the package docstring).  None of this is the
method; these are textbook integrals the discrete method must approach as the
grid is refined and M grows.

* potential of exp(-a |y - A|^2):  (pi/a)^{3/2} erf(sqrt(a) r) / r,  r = |x - A|
* nuclear attraction of exp(-a|x-A|^2) by a unit charge at C:
  -(2 pi / a) F0(a |A - C|^2)
* Coulomb integral of exp(-a|x-A|^2) and exp(-b|y-B|^2):
  2 pi^{5/2} / (a b sqrt(a+b)) * F0(a b/(a+b) |A - B|^2),
  F0(T) = (1/2) sqrt(pi/T) erf(sqrt(T)), F0(0) = 1  (the s-type Boys function).
"""
from __future__ import annotations

import math

import numpy as np
from scipy.special import erf


def boys0(T):
    T = np.asarray(T, dtype=np.float64)
    out = np.ones_like(T)
    big = T > 1e-12
    out[big] = 0.5 * np.sqrt(math.pi / T[big]) * erf(np.sqrt(T[big]))
    small = ~big
    out[small] = 1.0 - T[small] / 3.0
    return out


def gaussian_potential(a: float, A: np.ndarray, x: np.ndarray) -> np.ndarray:
    r = np.linalg.norm(np.asarray(x) - np.asarray(A), axis=-1)
    return (math.pi / a) ** 1.5 * erf(math.sqrt(a) * r) / r


def coulomb_pair(a, A, b, B):
    """(a|b) Coulomb integral of two unnormalised s Gaussians (arrays broadcast)."""
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    d2 = np.sum(np.square(np.asarray(A) - np.asarray(B)), axis=-1)
    return 2.0 * math.pi ** 2.5 / (a * b * np.sqrt(a + b)) * boys0(a * b / (a + b) * d2)


def mixture_energy(a, X, c) -> float:
    """<f, 1/r * f> for f = sum_k c_k exp(-a_k |x - X_k|^2)."""
    M = coulomb_pair(a[:, None], X[:, None, :], a[None, :], X[None, :, :])
    return float(c @ M @ c)


def mixture_energy_grad(a, X, c):
    """Closed-form gradients of mixture_energy with respect to a_k, X_k, c_k."""
    a = np.asarray(a, dtype=np.float64)
    A = a[:, None]
    B = a[None, :]
    D = X[:, None, :] - X[None, :, :]
    d2 = np.sum(D * D, axis=-1)
    s = A + B
    mu = A * B / s
    T = mu * d2
    F0 = boys0(T)
    # F0'(T) = (exp(-T) - F0)/(2T), limit -1/3 at T -> 0
    dF = np.where(T > 1e-8, (np.exp(-T) - F0) / (2.0 * np.where(T > 1e-8, T, 1.0)), -1.0 / 3.0 + T / 5.0)
    pref = 2.0 * math.pi ** 2.5 / (A * B * np.sqrt(s))
    # d/dA of pref: pref * (-1/A - 1/(2 s)); d/dA of T: d2 * B^2 / s^2
    dpref_dA = pref * (-1.0 / A - 0.5 / s)
    dT_dA = d2 * (B * B) / (s * s)
    dM_dA = dpref_dA * F0 + pref * dF * dT_dA
    cc = np.outer(c, c)
    # E = sum_kl c_k c_l M_kl; a_k appears as A in row k and as B in column k (symmetric)
    da = 2.0 * np.sum(cc * dM_dA, axis=1)
    # dT/dX_k = 2 mu (X_k - X_l)
    dM_dX = (pref * dF * 2.0 * mu)[:, :, None] * D
    dX = 2.0 * np.einsum("kl,kld->kd", cc, dM_dX)
    Mfull = pref * F0
    dc = 2.0 * Mfull @ c
    return da, dX, dc


def nuclear_attraction(a, A, C) -> np.ndarray:
    """-(a|C): integral of exp(-a |x - A|^2) / |x - C| over R^3, negated
    (attraction by a unit charge at C): -(2 pi / a) F0(a |A - C|^2)."""
    a = np.asarray(a, dtype=np.float64)
    d2 = np.sum(np.square(np.asarray(A) - np.asarray(C)), axis=-1)
    return -2.0 * math.pi / a * boys0(a * d2)
