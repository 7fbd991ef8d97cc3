"""Helpers shared by the GPU tests: oracle-side references and error measures."""
import numpy as np

from oracle import kernel_vectors as kv
from oracle import sinc


def oracle_conv_kernel(n, b, M):
    t, a = sinc.conv_nodes(n, b, M)
    return t, a, kv.conv_kernel_vectors(n, b, t, a)


def oracle_master_kernel(n, b, M):
    t, a = sinc.master_nodes(n, b, M)
    return t, a, kv.master_kernel_vectors(n, b, t, a)


def col_rel_err(A, B):
    """max over columns of ||A - B||_2 / ||B||_2 for arrays (..., cols, n)."""
    A = np.asarray(A, dtype=np.float64).reshape(-1, np.shape(A)[-1])
    B = np.asarray(B, dtype=np.float64).reshape(-1, np.shape(B)[-1])
    num = np.linalg.norm(A - B, axis=1)
    den = np.linalg.norm(B, axis=1)
    return float(np.max(num / np.where(den > 0, den, 1.0)))


def rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def cancellation(G0, c, h):
    """kappa = sum_kk' |c_k c_k' J_kk'| / |E_H| with J_kk' = h^3 sum_q prod_l G0[l, q, k, k']
    (G0: the oracle's convolution matrices, shape (3, R_N, R_f, R_f)): how much the
    terms of E_H = sum_kk' c_k c_k' J_kk' cancel.  It is 1 for a density with
    non-negative coefficients (all J_kk' > 0) and grows when coefficients of both
    signs cancel; a float32 rounding of the terms moves E_H by up to kappa times
    its relative size."""
    J = h ** 3 * np.sum(np.prod(G0, axis=0), axis=0)
    c = np.asarray(c, dtype=np.float64)
    E = float(c @ J @ c)
    return float(np.sum(np.abs(np.outer(c, c) * J)) / abs(E))
