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
