"""Seeded synthetic inputs for the rank-structured 3D Coulomb convolution.

This module holds random draws and fixed geometry only: exponents, centres and
coefficients of Gaussian mixtures, contracted s-type basis sets, lattice
geometry and sample points.  It does none of the method's arithmetic (no grid
sampling, no quadrature, no convolution, no contraction), so the CPU oracle and
the CUDA path can start from the same numbers without sharing any of the
computation.  Every draw uses numpy's Philox bit generator with an explicit seed.

The workloads stand in for the paper's molecules (H2O, glycine, alanine in
cc-pVDZ, which are not available here) with the paper's box sizes and grid
scales: box [-20,20]^3 for molecules (Sec. 3.2, Table 2), grids up to n=8192 per
axis, and a cubic lattice of unit charges (Sec. 5.1).
"""
from __future__ import annotations

import math

import numpy as np

# name -> sizes.  n: cells per axis; b: half box edge (box [-b,b]^3, h=2b/n);
# M: sinc quadrature half-count (R_N = 2M+1 Gaussian terms).
CONFIGS = {
    # 8 Gaussians on a 128^3 grid; parity-sized.
    "gauss8_n128": dict(n=128, b=10.0, M=20, R_f=8, a_lo=0.5, a_hi=50.0,
                        centre_half=3.0, centres=None),
    # molecule-like density of 600 Gaussians at 12 centres, 8192^3 grid.
    "density600_n8192": dict(n=8192, b=20.0, M=30, R_f=600, a_lo=0.1, a_hi=5000.0,
                             cluster_radius=3.0, centres=12),
    # 80 contracted s-type functions (3-6 primitives) at 10 centres, 4096^3 grid.
    "basis80_n4096": dict(n=4096, b=20.0, M=25, n_basis=80, prim_lo=3, prim_hi=6,
                          a_lo=0.05, a_hi=2000.0, centres=10, centre_half=3.0),
    # 200 Gaussians for the gradient workload, 4096^3 grid.
    "density200_n4096": dict(n=4096, b=16.0, M=25, R_f=200, a_lo=0.2, a_hi=200.0,
                             centre_half=4.0, centres=None),
    # 32^3 lattice of unit charges with spacing 4 bohr, 16384^3 grid, 512^3 sub-grid.
    "lattice32_n16384": dict(n=16384, b=64.0, M=30, L=32, spacing=4.0, sub=512,
                             n_check=1000),
    # nuclear-attraction matrix over the basis80_n4096 products: nuclei at the
    # 10 basis centres (rounded to grid-cell edges), charges 1..8, master kernel M=25
    "nuclear80_n4096": dict(n=4096, b=20.0, M=25, n_basis=80, prim_lo=3, prim_hi=6,
                            a_lo=0.05, a_hi=2000.0, centres=10, centre_half=3.0),
    # two-electron integrals of 80 s primitives at 10 centres (1D density
    # fitting + truncated Cholesky of the TEI matrix)
    "tei80_n4096": dict(n=4096, b=20.0, M=25, n_prims=80, a_lo=0.3, a_hi=30.0, centres=10,
                        cluster_radius=3.0, tol_df=1e-14, tol_b=1e-10, max_rank_b=512),
    # interaction energy of hydrogen lattices, 2 bohr apart (128 or 64 cells)
    "lattice_energy24_n4096": dict(n=4096, b=32.0, M=64, L=24, cells=128),
    "lattice_energy256_n16384": dict(n=16384, b=256.0, M=64, L=256, cells=64),
}


def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.Philox(seed))


def grid_step(n: int, b: float) -> float:
    """Cell width of the cell-centred grid on [-b, b]: h = 2b/n."""
    return 2.0 * b / n


def gaussian_mixture(R_f: int, a_lo: float, a_hi: float, seed: int,
                     centre_half: float | None = None, centres: int | None = None,
                     cluster_radius: float | None = None) -> dict:
    """Random parameters of f(x) = sum_k c_k exp(-a_k |x - X_k|^2).

    a_k log-uniform in [a_lo, a_hi]; c_k ~ N(0,1).  Centres are either uniform in
    [-centre_half, centre_half]^3 (one per Gaussian) or, when ``centres`` is
    given, a set of that many points uniform in a ball of ``cluster_radius``
    with each Gaussian assigned to one of them in turn.
    Returns float64 arrays a (R_f,), X (R_f, 3), c (R_f,).
    """
    g = rng(seed)
    a = np.exp(g.uniform(math.log(a_lo), math.log(a_hi), size=R_f))
    if centres:
        pts = []
        while len(pts) < centres:
            p = g.uniform(-cluster_radius, cluster_radius, size=3)
            if p @ p <= cluster_radius ** 2:
                pts.append(p)
        pts = np.asarray(pts)
        X = pts[np.arange(R_f) % centres].copy()
    else:
        X = g.uniform(-centre_half, centre_half, size=(R_f, 3))
    c = g.standard_normal(R_f)
    return dict(a=a.astype(np.float64), X=np.ascontiguousarray(X, dtype=np.float64),
                c=c.astype(np.float64))


def mixture_for(name: str, seed: int) -> dict:
    cfg = CONFIGS[name]
    return gaussian_mixture(cfg["R_f"], cfg["a_lo"], cfg["a_hi"], seed,
                            centre_half=cfg.get("centre_half"), centres=cfg.get("centres"),
                            cluster_radius=cfg.get("cluster_radius"))


def basis_set(n_basis: int, prim_lo: int, prim_hi: int, a_lo: float, a_hi: float,
              centres: int, centre_half: float, seed: int) -> dict:
    """Random contracted s-type basis g_mu(x) = sum_{p in mu} d_p exp(-alpha_p |x - X_mu|^2).

    Each function has U{prim_lo..prim_hi} primitives with exponents log-uniform in
    [a_lo, a_hi] and coefficients N(0,1) scaled to unit 2-norm per function;
    its centre is one of ``centres`` points uniform in [-centre_half, centre_half]^3.
    Density weights w_mu ~ U(0, 2) define the diagonal density rho = sum w_mu g_mu^2.

    Returns prim_alpha (P,), prim_d (P,), fn_first (n_basis+1,) offsets into the
    primitive arrays, fn_centre (n_basis, 3), w (n_basis,).
    """
    g = rng(seed)
    pts = g.uniform(-centre_half, centre_half, size=(centres, 3))
    counts = g.integers(prim_lo, prim_hi + 1, size=n_basis)
    which = g.integers(0, centres, size=n_basis)
    alpha, d = [], []
    for m in range(n_basis):
        al = np.exp(g.uniform(math.log(a_lo), math.log(a_hi), size=counts[m]))
        co = g.standard_normal(counts[m])
        co = co / np.sqrt(co @ co)
        alpha.append(al)
        d.append(co)
    fn_first = np.zeros(n_basis + 1, dtype=np.int64)
    fn_first[1:] = np.cumsum(counts)
    w = g.uniform(0.0, 2.0, size=n_basis)
    return dict(prim_alpha=np.concatenate(alpha), prim_d=np.concatenate(d),
                fn_first=fn_first, fn_centre=np.ascontiguousarray(pts[which]),
                w=w)


def basis_for(name: str, seed: int) -> dict:
    cfg = CONFIGS[name]
    return basis_set(cfg["n_basis"], cfg["prim_lo"], cfg["prim_hi"], cfg["a_lo"], cfg["a_hi"],
                     cfg["centres"], cfg["centre_half"], seed)


def lattice_geometry(n: int, L: int, sub: int) -> dict:
    """Lattice of L unit charges per axis in a box of n cells, one per unit cell.

    The box holds L unit cells of n0 = n/L grid cells each; each charge sits at
    its unit cell's centre, which is the grid-cell EDGE with index
    e_k = n0*k + n0/2 (n0 even), k = 0..L-1.  The sub-grid takes every
    (n/sub)-th cell centre, i_s = n/(2 sub) + (n/sub) s, s = 0..sub-1.
    """
    if n % L or (n // L) % 2 or n % sub or (n // sub) % 2:
        raise ValueError("need n/L even and n/sub even")
    n0 = n // L
    edges = (n0 * np.arange(L) + n0 // 2).astype(np.int32)
    stride = n // sub
    sub_idx = (stride // 2 + stride * np.arange(sub)).astype(np.int32)
    return dict(edges=edges, sub_idx=sub_idx)


def nuclei_for(basis: dict, n: int, b: float, seed: int):
    """Nuclei at the distinct basis centres, each moved to the nearest grid-cell
    edge (x = -b + e h): edges (3, N) int32 and charges Z (N,) in 1..8."""
    C = np.unique(np.asarray(basis["fn_centre"]), axis=0)
    h = 2.0 * b / n
    e = np.clip(np.rint((C + b) / h), 0, n).astype(np.int32).T
    Z = rng(seed).integers(1, 9, size=C.shape[0]).astype(np.float64)
    return np.ascontiguousarray(e), Z


def lattice_energy_edges(n: int, L: int, cells: int) -> np.ndarray:
    """Grid-cell edges of L charges ``cells`` cells apart, centred in the n-cell box."""
    off = (n - (L - 1) * cells) // 2
    if off < 1:
        raise ValueError("lattice does not fit the box")
    return (off + cells * np.arange(L)).astype(np.int32)


def check_points(sub: int, count: int, seed: int) -> np.ndarray:
    """``count`` random sub-grid points as (count, 3) int64 indices in [0, sub)."""
    return rng(seed).integers(0, sub, size=(count, 3))


# ---- index bookkeeping of product functions (no arithmetic of the method) ----

def upper_pairs(nb: int):
    """Pairs (mu, nu), mu <= nu, in row-major order of the upper triangle."""
    pa, pb = np.triu_indices(nb)
    return pa, pb


def basis_density_pairs(basis: dict):
    """Primitive pairs (a, b), a <= b inside each function, of the diagonal
    density rho = sum_mu w_mu g_mu^2, and each pair's weight: w_mu, doubled when
    a != b (the (a, b) and (b, a) terms are equal).  The contraction
    coefficients d_a d_b are not included."""
    first, w = basis["fn_first"], basis["w"]
    pa, pb, wt = [], [], []
    for mu in range(len(first) - 1):
        for a in range(first[mu], first[mu + 1]):
            for b in range(a, first[mu + 1]):
                pa.append(a)
                pb.append(b)
                wt.append(w[mu] * (1.0 if a == b else 2.0))
    return np.array(pa), np.array(pb), np.array(wt)


def basis_item_pairs(basis: dict):
    """Items (mu, nu), mu <= nu, in row-major order of the upper triangle; for
    each item its primitive pairs (a in mu, b in nu), concatenated, and the
    offsets of each item's pairs (len(items) + 1 entries)."""
    first = basis["fn_first"]
    nb = len(first) - 1
    items = [(mu, nu) for mu in range(nb) for nu in range(mu, nb)]
    pa, pb, off = [], [], [0]
    for mu, nu in items:
        for a in range(first[mu], first[mu + 1]):
            for b in range(first[nu], first[nu + 1]):
                pa.append(a)
                pb.append(b)
        off.append(len(pa))
    return items, np.array(pa), np.array(pb), np.array(off)
