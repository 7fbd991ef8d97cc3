"""Parity at the full workload sizes, in the launch configuration bench.py uses.

Where the oracle cannot finish the whole problem in seconds it computes
sampled outputs one by one (single convolution columns, Gram columns, single
Coulomb-matrix items, lattice check points); the rest is checked through
properties that hold at any size (the fused E_H reduction against a host
reduction of the full convolution matrices; E_H = sum_mu w_mu J_mu,mu)."""
import math

import numpy as np
import pytest
import torch

import workloads
from oracle import closed_forms as ocf
from oracle import coulomb as ocoul
from oracle import cp as ocp
from oracle import lattice as olat
from tests.gpu_util import col_rel_err, oracle_conv_kernel, oracle_master_kernel, rel

pytestmark = pytest.mark.gpu
TOL64 = 1e-10


@pytest.fixture(scope="module")
def cpc():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1504_06289_gb300 as m
    return m


def dev(x, dtype=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(x), dtype=dtype, device="cuda")


def test_density600_n8192(cpc):
    name = "density600_n8192"
    cfg = workloads.CONFIGS[name]
    n, b, M = cfg["n"], cfg["b"], cfg["M"]
    h = 2 * b / n
    g = workloads.mixture_for(name, 100)
    P = cpc.make_newton_kernel(n, b, M)
    R_N, R_f = P.R_N, cfg["R_f"]
    U = cpc.cp_sample_gaussians(n, b, dev(g["a"]), dev(g["X"]))
    c = dev(g["c"])
    E64, W64, G64 = cpc.cp_hartree_energy(P, U, c, "fp64", want_G=True)
    torch.cuda.synchronize()
    _, _, P0 = oracle_conv_kernel(n, b, M)
    U0 = ocp.sample_gaussians(n, b, g["a"], g["X"])
    rng = np.random.default_rng(0)
    picks = [(int(rng.integers(3)), int(rng.integers(R_f)), int(rng.integers(R_N))) for _ in range(16)]
    picks += [(0, 0, 0), (2, R_f - 1, R_N - 1), (1, 17, R_N // 2)]
    Wcols, Wref, Gcols, Gref = [], [], [], []
    for l, k, q in picks:
        w0 = ocp.conv1d_direct(U0[l, k], P0[q])
        Wcols.append(W64[l, k * R_N + q].cpu().numpy())
        Wref.append(w0)
        Gcols.append(G64[l, q, :, k].cpu().numpy())
        Gref.append(U0[l] @ w0)
    assert col_rel_err(np.array(Wcols), np.array(Wref)) < TOL64
    assert col_rel_err(np.array(Gcols), np.array(Gref)) < TOL64
    # fused reduction vs host reduction of the full convolution matrices
    Gh = G64.cpu().numpy()
    E_host = h ** 3 * np.sum(Gh[0] * Gh[1] * Gh[2] * np.outer(g["c"], g["c"])[None])
    assert abs(E64.item() / E_host - 1) < 1e-12
    del W64, G64
    torch.cuda.empty_cache()
    # float32 and split forms in the bench's configuration
    E32, W32, _ = cpc.cp_hartree_energy(P, U, c, "fp32")
    cols32 = np.array([W32[l, k * R_N + q].double().cpu().numpy() for l, k, q in picks])
    assert col_rel_err(cols32, np.array(Wref)) < 2e-6
    # the stated bound of the float32 form (compensated float32 FFT, exact
    # tensor-core contraction): 1e-7 relative on E_H
    assert abs(E32.item() / E64.item() - 1) < 1e-7
    del W32
    torch.cuda.empty_cache()
    Es, Ws, _ = cpc.cp_hartree_energy(P, U, c, "split")
    assert abs(Es.item() / E64.item() - 1) < 1e-7
    del Ws
    torch.cuda.empty_cache()
    # the float64-accurate tensor-core form: the float64 bar, and the sampled
    # convolution-matrix columns against the oracle
    Et, Wt, Gt = cpc.cp_hartree_energy(P, U, c, "fp64tc", want_G=True)
    assert abs(Et.item() / E64.item() - 1) < TOL64
    Gtc = np.array([Gt[l, q, :, k].cpu().numpy() for l, k, q in picks])
    assert col_rel_err(Gtc, np.array(Gref)) < TOL64


def test_density200_n4096_adjoint(cpc):
    name = "density200_n4096"
    cfg = workloads.CONFIGS[name]
    n, b, M = cfg["n"], cfg["b"], cfg["M"]
    h = 2 * b / n
    g = workloads.mixture_for(name, 5)
    P = cpc.make_newton_kernel(n, b, M)
    a, X, c = dev(g["a"]), dev(g["X"]), dev(g["c"])
    U = cpc.cp_sample_gaussians(n, b, a, X)
    E, W, G = cpc.cp_hartree_energy(P, U, c, "fp64", want_G=True)
    dU, dc = cpc.cp_hartree_energy_adjoint(P, c, W, G, "fp64")
    da, dX = cpc.cp_gaussian_param_grad(n, b, a, X, U, dU)
    _, _, P0 = oracle_conv_kernel(n, b, M)
    U0 = ocp.sample_gaussians(n, b, g["a"], g["X"])
    dU0, dc0 = ocp.hartree_energy_adjoint(U0, g["c"], P0, h)
    da0, dX0 = ocp.gaussian_param_grad(n, b, g["a"], g["X"], U0, dU0)
    assert rel(dU.cpu().numpy(), dU0) < TOL64
    assert rel(dc.cpu().numpy(), dc0) < TOL64
    assert rel(da.cpu().numpy(), da0) < TOL64
    assert rel(dX.cpu().numpy(), dX0) < TOL64
    # central differences (step 1e-5) of the library's own energy in a few parameters
    rng = np.random.default_rng(1)
    for _ in range(4):
        k = int(rng.integers(cfg["R_f"]))
        for which in ("a", "X"):
            vals = []
            for sgn in (1, -1):
                aa, XX = g["a"].copy(), g["X"].copy()
                if which == "a":
                    aa[k] += sgn * 1e-5
                else:
                    XX[k, 1] += sgn * 1e-5
                Ud = cpc.cp_sample_gaussians(n, b, dev(aa), dev(XX))
                vals.append(cpc.cp_hartree_energy(P, Ud, c, "fp64")[0].item())
            fd = (vals[0] - vals[1]) / 2e-5
            ref = da0[k] if which == "a" else dX0[k, 1]
            scale = np.max(np.abs(da0)) if which == "a" else np.max(np.abs(dX0))
            assert abs(fd - ref) < 1e-6 * scale, (which, k, fd, ref)
    # float32 form of the adjoint
    E32, W32, G32 = cpc.cp_hartree_energy(P, U, c, "fp32", want_G=True)
    assert abs(E32.item() / E.item() - 1) < 1e-7
    dU32, dc32 = cpc.cp_hartree_energy_adjoint(P, c, W32, G32, "fp32")
    assert rel(dU32.cpu().numpy(), dU0) < 1e-5
    assert rel(dc32.cpu().numpy(), dc0) < 1e-5


def _coulomb_inputs(cpc, n, b, basis, items):
    first = basis["fn_first"]
    nb = len(first) - 1
    centre = np.repeat(basis["fn_centre"], np.diff(first), axis=0)
    F = cpc.cp_sample_gaussians(n, b, dev(basis["prim_alpha"]), dev(centre))
    d = dev(basis["prim_d"])
    pa, pb, coef = ocoul.density_pairs(basis)
    sc = [basis["w"][mu] * (1.0 if x == y else 2.0)
          for mu in range(nb) for x in range(first[mu], first[mu + 1]) for y in range(x, first[mu + 1])]
    U_rho, c_rho = cpc.cp_hadamard_pairs(F, dev(pa, torch.int32), dev(pb, torch.int32), d, dev(sc))
    ia, ib, _, off = ocoul.item_pairs(basis, items)
    U_it, c_it = cpc.cp_hadamard_pairs(F, dev(ia, torch.int32), dev(ib, torch.int32), d)
    return U_rho, c_rho, U_it, c_it, dev(off, torch.int32)


def _oracle_items_streamed(n, b, basis, P0, items):
    """Oracle J for a few items, summing over q outside so memory stays per-q."""
    h = 2 * b / n
    U_rho, c_rho = ocoul.density_cp(n, b, basis)
    Gp = ocoul.primitive_factors(n, b, basis)
    pa, pb, coef, off = ocoul.item_pairs(basis, items)
    Ui = ocoul.hadamard(Gp, pa, pb)
    acc = np.zeros(len(pa))
    for q in range(P0.shape[0]):
        T = ocp.toeplitz_from_even(P0[q])
        prod = np.ones((len(pa), U_rho.shape[1]))
        for l in range(3):
            prod *= Ui[l] @ (T @ U_rho[l].T)
        acc += prod @ c_rho
    return np.array([h ** 3 * coef[off[t]:off[t + 1]] @ acc[off[t]:off[t + 1]] for t in range(len(items))])


def test_basis80_n4096_coulomb_matrix(cpc):
    name = "basis80_n4096"
    cfg = workloads.CONFIGS[name]
    n, b, M = cfg["n"], cfg["b"], cfg["M"]
    basis = workloads.basis_for(name, 3)
    nb = cfg["n_basis"]
    P = cpc.make_newton_kernel(n, b, M)
    rng = np.random.default_rng(2)
    all_items = ocoul.item_list(nb)
    sample = [all_items[int(i)] for i in rng.choice(len(all_items), 10, replace=False)] + [(0, 0), (nb - 1, nb - 1)]
    U_rho, c_rho, U_it, c_it, off = _coulomb_inputs(cpc, n, b, basis, sample)
    J64, _ = cpc.coulomb_matrix(P, off, U_it, c_it, U_rho, c_rho, "fp64", tiles_per_cta=0)
    _, _, P0 = oracle_conv_kernel(n, b, M)
    J0 = _oracle_items_streamed(n, b, basis, P0, sample)
    assert np.max(np.abs(J64.cpu().numpy() - J0)) < TOL64 * np.max(np.abs(J0))
    # E_H = sum_mu w_mu J_mu,mu over all diagonal items = h^3 <rho, P rho>
    diag = [(mu, mu) for mu in range(nb)]
    U_rho, c_rho, U_d, c_d, off_d = _coulomb_inputs(cpc, n, b, basis, diag)
    Jd, _ = cpc.coulomb_matrix(P, off_d, U_d, c_d, U_rho, c_rho, "fp64", tiles_per_cta=0)
    E_items = float(np.dot(basis["w"], Jd.cpu().numpy()))
    E_direct = cpc.cp_hartree_energy(P, U_rho, c_rho, "fp64")[0].item()
    assert abs(E_items / E_direct - 1) < 1e-10
    # the full matrix (3240 items) in the float32 form, one launch; checked on the sample
    U_rho, c_rho, U_all, c_all, off_all = _coulomb_inputs(cpc, n, b, basis, all_items)
    J32, _ = cpc.coulomb_matrix(P, off_all, U_all, c_all, U_rho, c_rho, "fp32", tiles_per_cta=0)
    J32 = J32.cpu().numpy()
    idx = [all_items.index(it) for it in sample]
    assert np.max(np.abs(J32[idx] - J0)) < 1e-5 * np.max(np.abs(J0))
    # and the float64 diagonal against the float32 full run
    didx = [all_items.index(it) for it in diag]
    assert np.max(np.abs(J32[didx] - Jd.cpu().numpy())) < 1e-5 * np.max(np.abs(Jd.cpu().numpy()))
    # the batched reduced-precision forms' energy E_H = sum_mu w_mu J_mu,mu against
    # the float64 form: the stated 1e-7 (the terms w_mu J_mu,mu are all positive)
    E32 = float(np.dot(basis["w"], J32[didx]))
    assert abs(E32 / E_items - 1) < 1e-7
    Js, _ = cpc.coulomb_matrix(P, off_d, U_d, c_d, U_rho, c_rho, "split", tiles_per_cta=0)
    assert abs(float(np.dot(basis["w"], Js.cpu().numpy())) / E_items - 1) < 1e-7


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("fp32", 5e-7)])
def test_lattice32_n16384(cpc, precision, tol):
    name = "lattice32_n16384"
    cfg = workloads.CONFIGS[name]
    n, b, M, L, sub_n = cfg["n"], cfg["b"], cfg["M"], cfg["L"], cfg["sub"]
    h = 2 * b / n
    geo = workloads.lattice_geometry(n, L, sub_n)
    P = cpc.make_newton_kernel(n, b, M, "master")
    sub = dev(np.stack([geo["sub_idx"]] * 3), torch.int32)
    S, V = cpc.lattice_potential_sum(P, [geo["edges"]] * 3, sub, precision)
    _, _, Pm0 = oracle_master_kernel(n, b, M)
    S0 = olat.assembled_vectors(Pm0, geo["edges"], n)
    for l in range(3):
        assert col_rel_err(S[l].cpu().numpy(), S0) < 1e-13
    pts = workloads.check_points(sub_n, cfg["n_check"], seed=7)
    Vs = V[pts[:, 0], pts[:, 1], pts[:, 2]].double().cpu().numpy()
    idx = geo["sub_idx"][pts]
    V0 = olat.potential_on_points([S0] * 3, h, idx)
    assert np.max(np.abs(Vs / V0 - 1)) < tol
    # physical check: direct sum of 1/|x - x_k| over the 32^3 charges
    x = -b + (idx + 0.5) * h
    q = -b + geo["edges"] * h
    Q = np.array(np.meshgrid(q, q, q, indexing="ij")).reshape(3, -1).T
    ref = np.array([np.sum(1.0 / np.linalg.norm(Q - xi, axis=1)) for xi in x])
    assert np.max(np.abs(Vs / ref - 1)) < 5e-5


@pytest.mark.parametrize("name", ["lattice_energy24_n4096", "lattice_energy256_n16384"])
def test_lattice_interaction_energy_fullsize(cpc, name):
    # hydrogen lattices of the printed energy table (Sec. 5.3): 24^3 and 256^3
    # charges 2 bohr apart; the device sum against the oracle's traced tensor
    # sum and against the direct sum of Eq. EnergyLatSum
    cfg = workloads.CONFIGS[name]
    n, b, M, L, cells = cfg["n"], cfg["b"], cfg["M"], cfg["L"], cfg["cells"]
    h = 2 * b / n
    edges = [workloads.lattice_energy_edges(n, L, cells)] * 3
    P = cpc.make_newton_kernel(n, b, M, "master")
    E = cpc.lattice_interaction_energy(P, edges).item()
    _, _, Pm0 = oracle_master_kernel(n, b, M)
    assert abs(E / olat.interaction_energy_tensor(Pm0, edges, n, h) - 1) < 1e-12
    assert abs(E / olat.interaction_energy_direct(edges, h) - 1) < 2e-8


def test_nuclear80_n4096_nuclear_matrix(cpc):
    # Sec. 3.3: all 3240 nuclear-attraction entries of the 80-function basis
    # (10 nuclei) in the float32 form, and a sample in float64, against the oracle
    from oracle import nuclear as onuc
    name = "nuclear80_n4096"
    cfg = workloads.CONFIGS[name]
    n, b, M = cfg["n"], cfg["b"], cfg["M"]
    basis = workloads.basis_for(name, 3)
    nb = cfg["n_basis"]
    nuc, Z = workloads.nuclei_for(basis, n, b, 5)
    P = cpc.make_newton_kernel(n, b, M, "master")
    _, _, Pm0 = oracle_master_kernel(n, b, M)
    rng = np.random.default_rng(4)
    all_items = ocoul.item_list(nb)
    sample = [all_items[int(i)] for i in rng.choice(len(all_items), 12, replace=False)] + [(0, 0), (nb - 1, nb - 1)]
    V0 = onuc.nuclear_items(n, b, basis, Pm0, sample, nuc, Z)
    _, _, U_s, c_s, off_s = _coulomb_inputs(cpc, n, b, basis, sample)
    V64, _ = cpc.nuclear_matrix(P, off_s, U_s, c_s, nuc, dev(Z), "fp64")
    assert np.max(np.abs(V64.cpu().numpy() - V0)) < TOL64 * np.max(np.abs(V0))
    _, _, U_all, c_all, off_all = _coulomb_inputs(cpc, n, b, basis, all_items)
    V32, _ = cpc.nuclear_matrix(P, off_all, U_all, c_all, nuc, dev(Z), "fp32")
    V32 = V32.cpu().numpy()
    idx = [all_items.index(it) for it in sample]
    assert np.max(np.abs(V32[idx] - V0)) < 1e-5 * np.max(np.abs(V0))
    assert np.all(np.isfinite(V32))
    # the trace (the nuclear energy of a density with unit weights) of the float32
    # form against the float64 form at the stated 1e-7 (all diagonal entries are negative)
    diag = [(mu, mu) for mu in range(nb)]
    _, _, U_d, c_d, off_d = _coulomb_inputs(cpc, n, b, basis, diag)
    V64d, _ = cpc.nuclear_matrix(P, off_d, U_d, c_d, nuc, dev(Z), "fp64")
    didx = [all_items.index(it) for it in diag]
    assert abs(V32[didx].sum() / V64d.cpu().numpy().sum() - 1) < 1e-7


def test_tei80_n4096_cholesky(cpc):
    # Sec. 3.2 at full size: 80 s primitives (3240 pairs) on the 4096 grid;
    # J(D) for a diagonal and a random symmetric D against the oracle's own
    # density fitting and Cholesky (each within its truncation), and the
    # diagonal-density J against the Coulomb-matrix path of the library
    from oracle import tei as otei
    name = "tei80_n4096"
    cfg = workloads.CONFIGS[name]
    n, b, M, nb = cfg["n"], cfg["b"], cfg["M"], cfg["n_prims"]
    h = 2 * b / n
    g = workloads.gaussian_mixture(nb, cfg["a_lo"], cfg["a_hi"], 11, centres=cfg["centres"],
                                   cluster_radius=cfg["cluster_radius"])
    P = cpc.make_newton_kernel(n, b, M)
    U = cpc.cp_sample_gaussians(n, b, dev(g["a"]), dev(g["X"]))
    pa0, pb0 = otei.pair_list(nb)
    pa, pb = dev(pa0, torch.int32), dev(pb0, torch.int32)
    L, ranks = cpc.tei_cholesky(P, U, pa, pb, cfg["tol_df"], 1e-8, 128, cfg["max_rank_b"])
    _, _, P0 = oracle_conv_kernel(n, b, M)
    U0 = ocp.sample_gaussians(n, b, g["a"], g["X"])
    L0, *_ = otei.tei_cholesky(U0, P0, h, pa0, pb0, cfg["tol_df"], 1e-8, 128, cfg["max_rank_b"])
    rng = np.random.default_rng(5)
    X = rng.standard_normal((nb, nb))
    w = rng.uniform(0.0, 2.0, nb)
    for D in (np.diag(w), X + X.T):
        J = cpc.tei_coulomb(L, ranks, pa, pb, dev(D)).cpu().numpy()
        J0 = otei.coulomb_from_cholesky(L0, D, pa0, pb0)
        assert np.max(np.abs(J - J0)) < 1e-6 * np.max(np.abs(J0))
        K = cpc.tei_exchange(L, ranks, pa, pb, dev(D)).cpu().numpy()
        K0 = otei.exchange_from_cholesky(L0, D, pa0, pb0)
        assert np.max(np.abs(K - K0)) < 1e-6 * np.max(np.abs(K0))
    # the same J for D = diag(w) from the Coulomb-matrix path (V_H factors of
    # rho = sum w g^2, no density fitting, no Cholesky)
    d1 = dev(np.ones(nb))
    idx = dev(np.arange(nb), torch.int32)
    U_rho, c_rho = cpc.cp_hadamard_pairs(U, idx, idx, d1, dev(w))
    U_it, c_it = cpc.cp_hadamard_pairs(U, pa, pb, d1)
    off = dev(np.arange(len(pa0) + 1), torch.int32)
    Jc, _ = cpc.coulomb_matrix(P, off, U_it, c_it, U_rho, c_rho, "fp64", tiles_per_cta=0)
    Jd = cpc.tei_coulomb(L, ranks, pa, pb, dev(np.diag(w))).cpu().numpy()
    Jc = Jc.cpu().numpy()
    # set by the density fitting at tol_df = 1e-14 (the oracle measures
    # 1.5e-7 of max |J|; 1.3e-6 at tol_df = 1e-12), not by the Cholesky
    # truncation (tol_b = 1e-8: at most 8e-7 of max |J| here)
    assert np.max(np.abs(Jd - Jc)) < 1e-6 * np.max(np.abs(Jc))
