"""GB300 (sm_103a) rank-structured 3D Coulomb convolution.

Thin Python binding over the C ABI in include/cpc.h (libcpc.so).  Every
function here only marshals torch CUDA tensors into pointers and sizes; all
arithmetic runs in the library's CUDA kernels (and its float64 host set-up of
the kernel tables).  There is no CPU fallback: without libcpc.so or a CUDA
device the calls raise.

Method: Khoromskaia & Khoromskij, "Tensor numerical methods in quantum
chemistry" (arXiv:1504.06289) -- CP convolution with the sinc-quadrature
Newton kernel (Sec. 2.5, Sec. 3.1, Appendix 3), convolution matrices
(Sec. 3.2), assembled lattice sums (Sec. 5.1).
"""
from __future__ import annotations

import ctypes as C

import numpy as np
import torch

from ._abi import KIND, PRECISION, CpcError, check, load

__all__ = [
    "NewtonKernel", "make_newton_kernel", "make_newton_kernel_tables", "cp_sample_gaussians", "cp_hadamard_pairs",
    "cp_convolve", "cp_hartree_energy", "cp_hartree_energy_from_factors",
    "cp_factor_spectra", "cp_convolve_from_spectra", "cp_hartree_energy_from_spectra",
    "cp_hartree_energy_noalloc", "cp_hartree_energy_adjoint", "cp_gaussian_param_grad",
    "coulomb_matrix", "nuclear_matrix", "tei_cholesky", "tei_coulomb", "tei_exchange", "lattice_potential_sum", "lattice_interaction_energy", "CPHartreeEnergy", "CpcError",
    "make_newton_kernel_paths", "make_newton_kernel_eh_plan",
]


def _stream(stream=None) -> C.c_void_p:
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


def _ptr(t: torch.Tensor | None) -> C.c_void_p:
    if t is None:
        return C.c_void_p(None)
    if not t.is_cuda or not t.is_contiguous():
        raise CpcError("expected a contiguous CUDA tensor")
    return C.c_void_p(t.data_ptr())


def _prec(p: str) -> int:
    try:
        return PRECISION[p]
    except KeyError:
        raise CpcError(f"unknown precision {p!r}; use one of {sorted(PRECISION)}")


def _out_dtype(precision: str):
    """Storage type of V_H factors and spectra: float32 only for the fp32 form."""
    return torch.float32 if precision == "fp32" else torch.float64


def _workspace(nbytes: int, device) -> torch.Tensor:
    return torch.empty(max(int(nbytes), 256), dtype=torch.uint8, device=device)


class NewtonKernel:
    """Handle to a CP Newton kernel built by make_newton_kernel (owns device tables)."""

    def __init__(self, handle: C.c_void_p, device):
        self._h = handle
        self.device = device
        n, M, R_N, kind = C.c_int(), C.c_int(), C.c_int(), C.c_int()
        b, hs, u0 = C.c_double(), C.c_double(), C.c_double()
        check(load().cpc_kernel_info(handle, C.byref(n), C.byref(b), C.byref(M), C.byref(R_N),
                                     C.byref(kind), C.byref(hs), C.byref(u0)), "cpc_kernel_info")
        self.n, self.b, self.M, self.R_N = n.value, b.value, M.value, R_N.value
        self.kind, self.hs, self.u0 = kind.value, hs.value, u0.value
        self.h = 2.0 * self.b / self.n

    @property
    def handle(self) -> C.c_void_p:
        return self._h

    def tables(self):
        """Host float64 copies (t, a, p) of the nodes, weights and kernel vectors."""
        length = self.n if self.kind == KIND["conv"] else 2 * self.n
        t = np.empty(self.R_N)
        a = np.empty(self.R_N)
        p = np.empty((self.R_N, length))
        check(load().cpc_kernel_tables(self._h, t.ctypes.data, a.ctypes.data, p.ctypes.data),
              "cpc_kernel_tables")
        return t, a, p

    def set_conv_paths(self, max_half_width32: int = 20, max_half_width64: int = 24, max_rank32: int = 16,
                       max_rank64: int = 16, stream=None):
        """Largest half-width of the banded terms and largest rank of the smooth
        (Chebyshev) terms, per W type (-1 disables the path; the FFT takes the rest)."""
        with torch.cuda.device(self.device):
            check(load().cpc_kernel_set_conv_paths(self._h, int(max_half_width32), int(max_half_width64),
                                                   int(max_rank32), int(max_rank64), _stream(stream)),
                  "cpc_kernel_set_conv_paths")

    def conv_paths(self, precision: str = "fp32"):
        """(half_width, rank) of every kernel term for the W type of `precision`:
        banded terms have half_width >= 0, smooth terms rank > 0, the rest -1, -1 (FFT)."""
        hw = np.empty(self.R_N, dtype=np.int32)
        rk = np.empty(self.R_N, dtype=np.int32)
        check(load().cpc_kernel_conv_paths(self._h, _prec(precision), hw.ctypes.data, rk.ctypes.data),
              "cpc_kernel_conv_paths")
        return hw, rk

    def close(self):
        if self._h is not None:
            load().cpc_kernel_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def make_newton_kernel_tables(n: int, b: float, M: int, kind: str = "conv"):
    """Host float64 tables (t, a, p, hs, u0) of the CP Newton kernel, no GPU needed."""
    R_N = 2 * M + 1
    length = n if kind == "conv" else 2 * n
    t, a, p = np.empty(R_N), np.empty(R_N), np.empty((R_N, length))
    hs, u0 = C.c_double(), C.c_double()
    check(load().make_newton_kernel_tables(int(n), float(b), int(M), KIND[kind], t.ctypes.data, a.ctypes.data,
                                           p.ctypes.data, C.byref(hs), C.byref(u0)), "make_newton_kernel_tables")
    return t, a, p, hs.value, u0.value


def make_newton_kernel_eh_plan(n: int, b: float, M: int, max_half_width32: int = 20, max_half_width64: int = 24,
                               max_rank32: int = 16, max_rank64: int = 16):
    """Host-only contraction plan of the energy paths: an int array (2, 3), per W type
    (row 0 float32, row 1 float64) the lag count L, the banded terms it covers and the
    rows the tensor-core contraction takes over the cells."""
    plan = np.empty((2, 3), dtype=np.int32)
    check(load().make_newton_kernel_eh_plan(int(n), float(b), int(M), int(max_half_width32), int(max_half_width64),
                                            int(max_rank32), int(max_rank64), plan.ctypes.data),
          "make_newton_kernel_eh_plan")
    return plan


def make_newton_kernel_paths(n: int, b: float, M: int, max_half_width32: int = 20, max_half_width64: int = 24,
                             max_rank32: int = 16, max_rank64: int = 16):
    """Host-only path choice of a CONV kernel's terms, no GPU needed: (half_width,
    rank, cheb) with half_width and rank of shape (2, R_N) (row 0 float32 W, row 1
    float64 W; -1 where the path is not taken) and cheb (R_N, 16, 16)."""
    R_N = 2 * M + 1
    hw = np.empty((2, R_N), dtype=np.int32)
    rk = np.empty((2, R_N), dtype=np.int32)
    cheb = np.empty((R_N, 16, 16))
    check(load().make_newton_kernel_paths(int(n), float(b), int(M), int(max_half_width32), int(max_half_width64),
                                          int(max_rank32), int(max_rank64), hw.ctypes.data, rk.ctypes.data,
                                          cheb.ctypes.data), "make_newton_kernel_paths")
    return hw, rk, cheb


def make_newton_kernel(n: int, b: float, M: int, kind: str = "conv", device="cuda",
                       stream=None) -> NewtonKernel:
    """Build the R_N = 2M+1 term CP Newton kernel on the n-cell grid of [-b,b]^3."""
    lib = load()
    dev = torch.device(device)
    with torch.cuda.device(dev):
        h = C.c_void_p()
        check(lib.make_newton_kernel(int(n), float(b), int(M), KIND[kind], _stream(stream),
                                     C.byref(h)), "make_newton_kernel")
    return NewtonKernel(h, dev)


def cp_sample_gaussians(n: int, b: float, a: torch.Tensor, X: torch.Tensor, stream=None) -> torch.Tensor:
    """U[l][k][i] = exp(-a_k (x_i - X_kl)^2) on the cell centres, shape (3, R, n)."""
    R = a.numel()
    U = torch.empty((3, R, n), dtype=torch.float64, device=a.device)
    check(load().cp_sample_gaussians(int(n), float(b), R, _ptr(a), _ptr(X), _ptr(U), _stream(stream)),
          "cp_sample_gaussians")
    return U


def cp_hadamard_pairs(F: torch.Tensor, pa: torch.Tensor, pb: torch.Tensor, d: torch.Tensor | None = None,
                      scale: torch.Tensor | None = None, stream=None):
    """Factors F[l][pa[r]] * F[l][pb[r]] (and coefficients scale*d[pa]*d[pb] if d is given)."""
    _, n_in, n = F.shape
    n_pairs = pa.numel()
    out = torch.empty((3, n_pairs, n), dtype=torch.float64, device=F.device)
    c_out = torch.empty(n_pairs, dtype=torch.float64, device=F.device) if d is not None else None
    check(load().cp_hadamard_pairs(n, n_in, n_pairs, _ptr(pa), _ptr(pb), _ptr(F), _ptr(d), _ptr(scale),
                                   _ptr(out), _ptr(c_out), _stream(stream)), "cp_hadamard_pairs")
    return out, c_out


def cp_convolve(P: NewtonKernel, U: torch.Tensor, precision: str = "fp64", W: torch.Tensor | None = None,
                stream=None) -> torch.Tensor:
    """V_H factors W[l][k*R_N+q] = U[l][k] * p_q, shape (3, R_f*R_N, n)."""
    lib = load()
    R_f = U.shape[1]
    pr = _prec(precision)
    if W is None:
        W = torch.empty((3, R_f * P.R_N, P.n), dtype=_out_dtype(precision), device=U.device)
    nb = lib.cp_convolve_workspace(P.handle, R_f, pr)
    ws = _workspace(nb, U.device)
    check(lib.cp_convolve(P.handle, R_f, _ptr(U), _ptr(W), pr, _ptr(ws), ws.numel(), _stream(stream)),
          "cp_convolve")
    return W


def cp_factor_spectra(P: NewtonKernel, U: torch.Tensor, precision: str = "fp64", spec: torch.Tensor | None = None,
                      stream=None) -> torch.Tensor:
    """Spectra of the zero-padded factor columns, (3, R_f, n+1, 2) as (re, im)."""
    R_f = U.shape[1]
    if spec is None:
        spec = torch.empty((3, R_f, P.n + 1, 2), dtype=_out_dtype(precision), device=U.device)
    check(load().cp_factor_spectra(P.handle, R_f, _ptr(U), _ptr(spec), _prec(precision), _stream(stream)),
          "cp_factor_spectra")
    return spec


def cp_convolve_from_spectra(P: NewtonKernel, spec: torch.Tensor, precision: str = "fp64",
                             W: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """V_H factors from factor spectra (the second half of cp_convolve)."""
    R_f = spec.shape[1]
    if W is None:
        W = torch.empty((3, R_f * P.R_N, P.n), dtype=_out_dtype(precision), device=spec.device)
    check(load().cp_convolve_from_spectra(P.handle, R_f, _ptr(spec), _ptr(W), _prec(precision), _stream(stream)),
          "cp_convolve_from_spectra")
    return W


def cp_hartree_energy_from_spectra(P: NewtonKernel, spec: torch.Tensor, c: torch.Tensor, want_G: bool = False,
                                   ws: torch.Tensor | None = None, E: torch.Tensor | None = None, stream=None):
    """float32 form: E_H (device scalar) and optionally G from float32 spectra (Parseval)."""
    lib = load()
    R_f = spec.shape[1]
    G = torch.empty((3, P.R_N, R_f, R_f), dtype=torch.float64, device=spec.device) if want_G else None
    if E is None:
        E = torch.empty((), dtype=torch.float64, device=spec.device)
    nb = lib.cp_hartree_energy_from_spectra_workspace(P.handle, R_f)
    if ws is None or ws.numel() < nb:
        ws = _workspace(nb, spec.device)
    check(lib.cp_hartree_energy_from_spectra(P.handle, R_f, _ptr(spec), _ptr(c), _ptr(G), _ptr(E), PRECISION["fp32"],
                                             _ptr(ws), ws.numel(), _stream(stream)), "cp_hartree_energy_from_spectra")
    return E, G


def cp_hartree_energy(P: NewtonKernel, U: torch.Tensor, c: torch.Tensor, precision: str = "fp64",
                      want_G: bool = False, W: torch.Tensor | None = None, ws: torch.Tensor | None = None,
                      stream=None):
    """E_H = h^3 <f, P_R * f> as a device scalar, with the V_H factors W and
    (optionally) the convolution matrices G[l][q] = U^T (p_q * U)."""
    lib = load()
    R_f = U.shape[1]
    pr = _prec(precision)
    if W is None:
        W = torch.empty((3, R_f * P.R_N, P.n), dtype=_out_dtype(precision), device=U.device)
    G = torch.empty((3, P.R_N, R_f, R_f), dtype=torch.float64, device=U.device) if want_G else None
    E = torch.empty((), dtype=torch.float64, device=U.device)
    nb = lib.cp_hartree_energy_workspace(P.handle, R_f, pr)
    if ws is None or ws.numel() < nb:
        ws = _workspace(nb, U.device)
    check(lib.cp_hartree_energy(P.handle, R_f, _ptr(U), _ptr(c), _ptr(W), _ptr(G), _ptr(E), pr, _ptr(ws),
                                ws.numel(), _stream(stream)), "cp_hartree_energy")
    return E, W, G


def cp_hartree_energy_from_factors(P: NewtonKernel, U: torch.Tensor, c: torch.Tensor, W: torch.Tensor,
                                   precision: str = "fp64", want_G: bool = False, ws: torch.Tensor | None = None,
                                   E: torch.Tensor | None = None, stream=None):
    """E_H (device scalar) and optionally G from existing V_H factors W."""
    lib = load()
    R_f = U.shape[1]
    G = torch.empty((3, P.R_N, R_f, R_f), dtype=torch.float64, device=U.device) if want_G else None
    if E is None:
        E = torch.empty((), dtype=torch.float64, device=U.device)
    nb = lib.cp_hartree_energy_from_factors_workspace(P.handle, R_f, _prec(precision))
    if ws is None or ws.numel() < nb:
        ws = _workspace(nb, U.device)
    check(lib.cp_hartree_energy_from_factors(P.handle, R_f, _ptr(U), _ptr(c), _ptr(W), _ptr(G), _ptr(E),
                                             _prec(precision), _ptr(ws), ws.numel(), _stream(stream)),
          "cp_hartree_energy_from_factors")
    return E, G


def cp_hartree_energy_noalloc(P: NewtonKernel, U: torch.Tensor, c: torch.Tensor, W: torch.Tensor,
                              G: torch.Tensor | None = None, E: torch.Tensor | None = None,
                              precision: str = "fp64", stream=None) -> torch.Tensor:
    """cp_hartree_energy for callers that cannot allocate: the caller provides
    W (and G, E if wanted); the library's fixed 32 MiB device scratch replaces
    the workspace.  Returns the device scalar E."""
    if E is None:
        E = torch.empty((), dtype=torch.float64, device=U.device)
    check(load().cp_hartree_energy_noalloc(P.handle, U.shape[1], _ptr(U), _ptr(c), _ptr(W), _ptr(G), _ptr(E),
                                           _prec(precision), _stream(stream)), "cp_hartree_energy_noalloc")
    return E


def cp_hartree_energy_adjoint(P: NewtonKernel, c: torch.Tensor, W: torch.Tensor, G: torch.Tensor,
                              precision: str = "fp64", want_dc: bool = True, stream=None):
    """dE_H/dU (3, R_f, n) and dE_H/dc (R_f,) from the forward's W and G."""
    R_f = c.numel()
    dU = torch.empty((3, R_f, P.n), dtype=torch.float64, device=c.device)
    dc = torch.empty(R_f, dtype=torch.float64, device=c.device) if want_dc else None
    check(load().cp_hartree_energy_adjoint(P.handle, R_f, _ptr(c), _ptr(W), _ptr(G), _ptr(dU), _ptr(dc),
                                           _prec(precision), _stream(stream)), "cp_hartree_energy_adjoint")
    return dU, dc


def cp_gaussian_param_grad(n: int, b: float, a: torch.Tensor, X: torch.Tensor, U: torch.Tensor,
                           dU: torch.Tensor, stream=None):
    """Chain rule dE/da (R,), dE/dX (R, 3) from dE/dU."""
    R = a.numel()
    da = torch.empty(R, dtype=torch.float64, device=a.device)
    dX = torch.empty((R, 3), dtype=torch.float64, device=a.device)
    check(load().cp_gaussian_param_grad(int(n), float(b), R, _ptr(a), _ptr(X), _ptr(U), _ptr(dU), _ptr(da),
                                        _ptr(dX), _stream(stream)), "cp_gaussian_param_grad")
    return da, dX


_TUNE_CACHE = None


def _tune_cache_path():
    import os
    return os.environ.get("CPC_TUNE_CACHE", os.path.join(os.path.expanduser("~"), ".cache", "cpc_tune.json"))


def _tune_key(P, n_factors, R_rho, precision, device):
    props = torch.cuda.get_device_properties(device)
    return f"{props.name}|sm{props.multi_processor_count}|n{P.n}|RN{P.R_N}|F{n_factors}|R{R_rho}|{precision}"


def _tune_lookup(key):
    global _TUNE_CACHE
    import json
    import os
    if _TUNE_CACHE is None:
        try:
            with open(_tune_cache_path()) as f:
                _TUNE_CACHE = json.load(f)
        except (OSError, ValueError):
            _TUNE_CACHE = {}
    return _TUNE_CACHE.get(key)


def _tune_store(key, value):
    import json
    import os
    _tune_lookup(key)  # loads the cache file on first use
    _TUNE_CACHE[key] = value
    path = _tune_cache_path()
    try:
        os.makedirs(os.path.dirname(path), exist_ok=True)
        tmp = path + ".tmp"
        with open(tmp, "w") as f:
            json.dump(_TUNE_CACHE, f, indent=1, sort_keys=True)
        os.replace(tmp, path)
    except OSError:
        pass


def coulomb_matrix(P: NewtonKernel, off: torch.Tensor, U_items: torch.Tensor, c_items: torch.Tensor,
                   U_rho: torch.Tensor, c_rho: torch.Tensor, precision: str = "fp64",
                   W_rho: torch.Tensor | None = None, ws: torch.Tensor | None = None, tiles_per_cta=None,
                   stream=None):
    """J[t] = <item_t, V_H(rho)> for items in CP form (factor offsets `off`, int32).

    tiles_per_cta: schedule of the persistent contraction; None looks it up in
    the tuning cache (file CPC_TUNE_CACHE, default ~/.cache/cpc_tune.json) and
    runs coulomb_matrix_tune on a miss; "tune" forces a new tuning; an int is
    used as given (0 = library default)."""
    lib = load()
    n_items = off.numel() - 1
    n_factors = U_items.shape[1]
    R_rho = U_rho.shape[1]
    pr = _prec(precision)
    if W_rho is None:
        W_rho = torch.empty((3, R_rho * P.R_N, P.n), dtype=_out_dtype(precision), device=U_rho.device)
    J = torch.empty(n_items, dtype=torch.float64, device=U_rho.device)
    nb = lib.coulomb_matrix_workspace(P.handle, n_items, n_factors, R_rho, pr)
    if ws is None or ws.numel() < nb:
        ws = _workspace(nb, U_rho.device)
    args = (P.handle, n_items, _ptr(off), n_factors, _ptr(U_items), _ptr(c_items), R_rho, _ptr(U_rho), _ptr(c_rho),
            _ptr(W_rho), _ptr(J), pr)
    key = None
    if tiles_per_cta is None or tiles_per_cta == "tune":
        key = _tune_key(P, n_factors, R_rho, precision, U_rho.device)
        cached = _tune_lookup(key) if tiles_per_cta is None else None
        if cached is not None:
            tiles_per_cta = int(cached["tiles_per_cta"])
        else:
            best, ms = C.c_int(), C.c_float()
            times = (C.c_float * 8)()
            check(lib.coulomb_matrix_tune(*args, _ptr(ws), ws.numel(), _stream(stream), C.byref(best), C.byref(ms),
                                          times), "coulomb_matrix_tune")
            cands = {str(1 << k): float(times[k]) for k in range(8) if times[k] == times[k]}
            _tune_store(key, {"tiles_per_cta": best.value, "ms": ms.value, "candidates_ms": cands})
            return J, W_rho
    check(lib.coulomb_matrix(*args, int(tiles_per_cta), _ptr(ws), ws.numel(), _stream(stream)), "coulomb_matrix")
    return J, W_rho


def nuclear_matrix(P: NewtonKernel, off: torch.Tensor, U_items: torch.Tensor, c_items: torch.Tensor, nuc_edges,
                   Z: torch.Tensor, precision: str = "fp64", F: torch.Tensor | None = None,
                   ws: torch.Tensor | None = None, stream=None):
    """V[t] = -<item_t, P_c> with P_c the master kernel P shifted onto nuclei at
    the grid-cell edges `nuc_edges` (3, n_nuc) with charges Z (Sec. 3.3).
    Returns (V, F), F the windowed nuclear factors (3, n_nuc R_N, n)."""
    lib = load()
    n_items = off.numel() - 1
    n_factors = U_items.shape[1]
    e = np.ascontiguousarray(np.asarray(nuc_edges, dtype=np.int32).reshape(3, -1))
    n_nuc = e.shape[1]
    pr = _prec(precision)
    if F is None:
        F = torch.empty((3, n_nuc * P.R_N, P.n), dtype=_out_dtype(precision), device=U_items.device)
    V = torch.empty(n_items, dtype=torch.float64, device=U_items.device)
    nb = lib.nuclear_matrix_workspace(P.handle, n_items, n_factors, n_nuc, pr)
    if ws is None or ws.numel() < nb:
        ws = _workspace(nb, U_items.device)
    check(lib.nuclear_matrix(P.handle, n_items, _ptr(off), n_factors, _ptr(U_items), _ptr(c_items), n_nuc,
                             e.ctypes.data, _ptr(Z), _ptr(F), _ptr(V), pr, _ptr(ws), ws.numel(), _stream(stream)),
          "nuclear_matrix")
    return V, F


def tei_cholesky(P: NewtonKernel, U_prims: torch.Tensor, pa: torch.Tensor, pb: torch.Tensor, tol_df: float = 1e-12,
                 tol_b: float = 1e-10, max_rank_df: int = 128, max_rank_b: int | None = None, stream=None):
    """Truncated Cholesky factor of the TEI matrix over the pairs (pa, pb) of
    primitive Gaussians with sampled factors U_prims (3, n_b, n), via 1D
    density fitting (Sec. 3.2).  Returns (L (max_rank_b, n_pairs), ranks
    (4,) int32 device: the fitted ranks of the three axes and the rank of L)."""
    lib = load()
    n_b, n_pairs = U_prims.shape[1], pa.numel()
    if max_rank_b is None:
        max_rank_b = n_pairs
    L = torch.empty((max_rank_b, n_pairs), dtype=torch.float64, device=U_prims.device)
    ranks = torch.zeros(4, dtype=torch.int32, device=U_prims.device)
    ws = _workspace(lib.tei_cholesky_workspace(P.handle, n_pairs, max_rank_b), U_prims.device)
    check(lib.tei_cholesky(P.handle, n_b, _ptr(U_prims), n_pairs, _ptr(pa), _ptr(pb), float(tol_df), float(tol_b),
                           int(max_rank_df), int(max_rank_b), _ptr(L), _ptr(ranks), _ptr(ws), ws.numel(),
                           _stream(stream)), "tei_cholesky")
    return L, ranks


def tei_coulomb(L: torch.Tensor, ranks: torch.Tensor, pa: torch.Tensor, pb: torch.Tensor, D: torch.Tensor,
                stream=None) -> torch.Tensor:
    """J over the pairs for the density matrix D (n_b, n_b) from tei_cholesky's factor."""
    lib = load()
    n_b, n_pairs, max_rank_b = D.shape[0], pa.numel(), L.shape[0]
    J = torch.empty(n_pairs, dtype=torch.float64, device=L.device)
    ws = _workspace(((8 * n_pairs + 255) // 256) * 256 + 8 * max_rank_b, L.device)
    check(lib.tei_coulomb(n_b, n_pairs, _ptr(pa), _ptr(pb), max_rank_b, _ptr(L), _ptr(ranks), _ptr(D), _ptr(J),
                          _ptr(ws), ws.numel(), _stream(stream)), "tei_coulomb")
    return J


def tei_exchange(L: torch.Tensor, ranks: torch.Tensor, pa: torch.Tensor, pb: torch.Tensor, D: torch.Tensor,
                 stream=None) -> torch.Tensor:
    """Exchange matrix K (n_b, n_b) of the density matrix D from tei_cholesky's factor."""
    lib = load()
    n_b, n_pairs, max_rank_b = D.shape[0], pa.numel(), L.shape[0]
    K = torch.empty((n_b, n_b), dtype=torch.float64, device=L.device)
    ws = _workspace(lib.tei_exchange_workspace(n_b, max_rank_b), L.device)
    check(lib.tei_exchange(n_b, n_pairs, _ptr(pa), _ptr(pb), max_rank_b, _ptr(L), _ptr(ranks), _ptr(D), _ptr(K),
                           _ptr(ws), ws.numel(), _stream(stream)), "tei_exchange")
    return K


def lattice_potential_sum(P: NewtonKernel, edges, sub: torch.Tensor | None = None, precision: str = "fp64",
                          stream=None):
    """Assembled vectors S (3, R_N, n) for charges at grid-cell edges `edges`
    (a list of three int arrays) and, if `sub` (3, n_sub) int32 is given, the
    potential on the sub-grid (n_sub, n_sub, n_sub)."""
    lib = load()
    L = (C.c_int * 3)(*[len(e) for e in edges])
    flat = np.ascontiguousarray(np.concatenate([np.asarray(e, dtype=np.int32) for e in edges]))
    S = torch.empty((3, P.R_N, P.n), dtype=torch.float64, device=P.device)
    V = None
    n_sub = 0
    if sub is not None:
        n_sub = sub.shape[1]
        V = torch.empty((n_sub, n_sub, n_sub), dtype=_out_dtype(precision), device=P.device)
    check(lib.lattice_potential_sum(P.handle, L, flat.ctypes.data, _ptr(S), n_sub, _ptr(sub), _ptr(V),
                                    _prec(precision), _stream(stream)), "lattice_potential_sum")
    return S, V


def lattice_interaction_energy(P: NewtonKernel, edges, Z: float = 1.0, stream=None) -> torch.Tensor:
    """Interaction energy E_L of equal charges Z at the grid-cell edges `edges`
    (three int arrays, each entry in [1, n-1]) of a MASTER kernel (Sec. 5.3,
    Eq. EnergyLattice): a 0-d float64 device tensor."""
    lib = load()
    L = (C.c_int * 3)(*[len(e) for e in edges])
    flat = np.ascontiguousarray(np.concatenate([np.asarray(e, dtype=np.int32) for e in edges]))
    E = torch.empty((), dtype=torch.float64, device=P.device)
    check(lib.lattice_interaction_energy(P.handle, L, flat.ctypes.data, float(Z), _ptr(E), _stream(stream)),
          "lattice_interaction_energy")
    return E


class CPHartreeEnergy(torch.autograd.Function):
    """E_H of a Gaussian mixture f = sum c_k exp(-a_k|x - X_k|^2) with gradients
    in a, X and c through the hand-written adjoint kernels."""

    @staticmethod
    def forward(ctx, a, X, c, P: NewtonKernel, precision: str = "fp64"):
        U = cp_sample_gaussians(P.n, P.b, a.detach(), X.detach())
        E, W, G = cp_hartree_energy(P, U, c.detach(), precision, want_G=True)
        ctx.save_for_backward(a.detach(), X.detach(), c.detach())
        ctx.P, ctx.precision, ctx.U, ctx.W, ctx.G = P, precision, U, W, G
        return E

    @staticmethod
    def backward(ctx, gE):
        a, X, c = ctx.saved_tensors
        P = ctx.P
        dU, dc = cp_hartree_energy_adjoint(P, c, ctx.W, ctx.G, ctx.precision)
        da, dX = cp_gaussian_param_grad(P.n, P.b, a, X, ctx.U, dU)
        return gE * da, gE * dX, gE * dc, None, None


def kernel_timing(enable: bool) -> None:
    """Start (clearing earlier records) or stop CUDA-event timing of the
    library's main kernels (spectra_kernel, conv_kernel, slice_rows_kernel,
    gemm3_tc_kernel)."""
    check(load().cpc_kernel_timing(1 if enable else 0), "cpc_kernel_timing")


def kernel_timing_read(kernel: str):
    """(total device ms, launches) recorded for `kernel` since timing was enabled."""
    ms, cnt = C.c_double(), C.c_int()
    check(load().cpc_kernel_timing_read(kernel.encode(), C.byref(ms), C.byref(cnt)), "cpc_kernel_timing_read")
    return ms.value, cnt.value
