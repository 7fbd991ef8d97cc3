"""cp_hartree_energy_noalloc against cp_hartree_energy, through the C ABI.

The allocation-free entry point exists for callers that cannot allocate
device memory (a program that owns a fixed device pool, a plug-in inside
another runtime's allocator, a loop that must not call cudaMalloc).  It takes
its scratch from the library's fixed 32 MiB device array instead of a
caller workspace.  Here it must reproduce the workspace entry point on two
calls in a row (with different inputs, so stale scratch would show), in all
three precision forms (SPLIT keeps a different scratch layout: float64
spectra and CUDA-core partial sums, no tensor-core slices), reject a size
whose scratch exceeds the array, and report an invalid argument as invalid
even when the size would also be too large.

This file is collected last so a run that stops at the first failure has
already run every other test; it also passes on its own in a fresh process.
"""
import ctypes as C

import numpy as np
import pytest
import torch

import workloads

pytestmark = pytest.mark.gpu

# the same kernels on the same inputs: agreement to rounding of the final sums
TOL = {"fp64": 1e-10, "fp32": 1e-10, "split": 1e-10}


@pytest.fixture(scope="module")
def cpc():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1504_06289_gb300 as m
    from paper_1504_06289_gb300 import build
    build.build()
    return m


def _inputs(cpc, seed, n, b, R_f):
    g = workloads.gaussian_mixture(R_f, 0.5, 50.0, seed, centre_half=3.0)
    a = torch.tensor(g["a"], device="cuda")
    X = torch.tensor(g["X"], device="cuda")
    c = torch.tensor(g["c"], device="cuda")
    return cpc.cp_sample_gaussians(n, b, a, X), c


@pytest.mark.parametrize("precision", ["fp64", "fp32", "split"])
def test_noalloc_matches_workspace_entry_on_consecutive_calls(cpc, precision):
    lib = cpc.load()
    n, b, M, R_f = 128, 10.0, 20, 8
    P = cpc.make_newton_kernel(n, b, M)
    dt = torch.float32 if precision == "fp32" else torch.float64
    pr = cpc._prec(precision)
    stream = cpc._stream()
    for seed in (11, 12):  # two calls in a row, different densities
        U, c = _inputs(cpc, seed, n, b, R_f)
        # existing entry point with a caller workspace
        E_ref, W_ref, G_ref = cpc.cp_hartree_energy(P, U, c, precision, want_G=True)
        # allocation-free entry point, called directly through the C ABI
        W = torch.empty((3, R_f * P.R_N, n), dtype=dt, device="cuda")
        G = torch.empty((3, P.R_N, R_f, R_f), dtype=torch.float64, device="cuda")
        E = torch.empty((), dtype=torch.float64, device="cuda")
        st = lib.cp_hartree_energy_noalloc(P.handle, R_f, C.c_void_p(U.data_ptr()), C.c_void_p(c.data_ptr()),
                                           C.c_void_p(W.data_ptr()), C.c_void_p(G.data_ptr()),
                                           C.c_void_p(E.data_ptr()), pr, stream)
        assert st == 0, lib.cpc_last_error().decode()
        torch.cuda.synchronize()
        tol = TOL[precision]
        assert abs(E.item() / E_ref.item() - 1) < tol
        Wn, Wr = W.double().cpu().numpy(), W_ref.double().cpu().numpy()
        assert np.max(np.linalg.norm(Wn - Wr, axis=-1) / np.linalg.norm(Wr, axis=-1)) < tol
        assert np.linalg.norm((G - G_ref).cpu().numpy()) < tol * np.linalg.norm(G_ref.cpu().numpy())


def test_noalloc_rejects_sizes_beyond_its_scratch(cpc):
    lib = cpc.load()
    n, b, M = 4096, 16.0, 25
    P = cpc.make_newton_kernel(n, b, M)
    R_f = 400  # 3 * 400 * 4097 spectra bins of 16 bytes = 79 MB > 32 MiB
    need = lib.cp_hartree_energy_workspace(P.handle, R_f, 0)
    assert need > (32 << 20)
    dummy = torch.empty(16, dtype=torch.float64, device="cuda")
    p = C.c_void_p(dummy.data_ptr())
    st = lib.cp_hartree_energy_noalloc(P.handle, R_f, p, p, p, None, p, 0, cpc._stream())
    assert st == -5
    msg = lib.cpc_last_error().decode()
    assert "32 MiB" in msg and str(need) in msg


def test_noalloc_reports_invalid_arguments_before_the_size_limit(cpc):
    lib = cpc.load()
    n, b, M = 4096, 16.0, 25
    R_f = 400  # too large for the scratch array, but the arguments are wrong first
    P = cpc.make_newton_kernel(n, b, M)
    Pm = cpc.make_newton_kernel(256, 8.0, 12, "master")
    dummy = torch.empty(16, dtype=torch.float64, device="cuda")
    p = C.c_void_p(dummy.data_ptr())
    # a MASTER kernel, an unknown precision, a NULL factor pointer
    assert lib.cp_hartree_energy_noalloc(Pm.handle, R_f, p, p, p, None, p, 0, cpc._stream()) == -1
    assert "CONV" in lib.cpc_last_error().decode()
    assert lib.cp_hartree_energy_noalloc(P.handle, R_f, p, p, p, None, p, 7, cpc._stream()) == -5
    assert "precision" in lib.cpc_last_error().decode()
    assert lib.cp_hartree_energy_noalloc(P.handle, R_f, None, p, p, None, p, 0, cpc._stream()) == -1
    assert "NULL" in lib.cpc_last_error().decode()
