"""Pins for the CP convolution, E_H and its adjoint (oracle/cp.py).

Each check compares against something the oracle does not compute itself:
brute-force dense 3D convolution, analytic Gaussian Coulomb integrals under
grid refinement, exact invariants, and finite differences."""
import math

import numpy as np
import pytest

import workloads
from oracle import closed_forms as cf
from oracle import cp, kernel_vectors as kv, sinc


def _kernel(n, b, M):
    t, a = sinc.conv_nodes(n, b, M)
    return kv.conv_kernel_vectors(n, b, t, a)


def _mixture(R, seed, a_lo=0.5, a_hi=2.0, half=1.5):
    return workloads.gaussian_mixture(R, a_lo, a_hi, seed, centre_half=half)


def test_cp_convolution_equals_dense_3d_convolution():
    n, b, M = 10, 3.0, 6
    P = _kernel(n, b, M)
    g = _mixture(3, 11, 0.3, 3.0, 1.0)
    U = cp.sample_gaussians(n, b, g["a"], g["X"])
    f = cp.full_tensor(U, g["c"])
    # dense kernel tensor over offsets -(n-1)..n-1 per axis, from the 1D vectors
    off = np.abs(np.arange(-(n - 1), n))
    Pd = np.einsum("qi,qj,qk->ijk", P[:, off], P[:, off], P[:, off])
    V = np.zeros((n, n, n))
    for i in range(n):
        for j in range(n):
            for k in range(n):
                # V[i,j,k] = sum_{i',j',k'} f[i',j',k'] P[(i-i'), (j-j'), (k-k')]
                V[i, j, k] = np.sum(f * Pd[i - np.arange(n) + n - 1][:, j - np.arange(n) + n - 1][:, :, k - np.arange(n) + n - 1])
    W = cp.convolve_factors(U, P)
    R_N = P.shape[0]
    Vcp = np.zeros((n, n, n))
    for k in range(3):
        for q in range(R_N):
            col = k * R_N + q
            Vcp += g["c"][k] * np.einsum("i,j,l->ijl", W[0, col], W[1, col], W[2, col])
    assert np.max(np.abs(Vcp - V)) < 1e-13 * np.max(np.abs(V))
    h = 2 * b / n
    E_dense = h ** 3 * np.sum(f * V)
    E = cp.hartree_energy(U, g["c"], P, h)
    assert abs(E / E_dense - 1) < 1e-13


def _energy(n, b, M, g):
    P = _kernel(n, b, M)
    U = cp.sample_gaussians(n, b, g["a"], g["X"])
    return cp.hartree_energy(U, g["c"], P, 2 * b / n)


def test_energy_converges_to_closed_form_at_second_order():
    # E_H -> 2 pi^{5/2}/(ab sqrt(a+b)) F0(...) summed over pairs, error O(h^2)
    b, M = 8.0, 40
    g = _mixture(4, 3)
    g["c"] = np.abs(g["c"]) + 0.2
    exact = cf.mixture_energy(g["a"], g["X"], g["c"])
    E = {n: _energy(n, b, M, g) for n in (64, 128, 256)}
    e1, e2, e3 = (E[n] - exact for n in (64, 128, 256))
    assert 3.0 < e1 / e2 < 5.0 and 3.0 < e2 / e3 < 5.0, (e1, e2, e3)
    rich = (4 * E[256] - E[128]) / 3
    assert abs(rich / exact - 1) < 2e-5, (rich / exact - 1, e3 / exact)


def test_single_gaussian_potential_at_cell_centres():
    # V_i = sum_j f_j P_{i-j} -> (pi/a)^{3/2} erf(sqrt(a) r)/r, O(h^2)
    b, M, a = 8.0, 40, 1.0
    errs = []
    for n in (64, 128, 256):
        h = 2 * b / n
        X = np.array([[0.0, 0.0, 0.0]])
        P = _kernel(n, b, M)
        U = cp.sample_gaussians(n, b, np.array([a]), X)
        W = cp.convolve_factors(U, P)
        x = cp.cell_centres(n, b)
        # evaluation point nearest to (1.5, -0.7, 2.2): cell centres move with n,
        # so compare each grid against the closed form at its own point
        idx = [int(np.argmin(np.abs(x - v))) for v in (1.5, -0.7, 2.2)]
        V = sum(W[0, q, idx[0]] * W[1, q, idx[1]] * W[2, q, idx[2]] for q in range(P.shape[0]))
        ref = cf.gaussian_potential(a, X[0], np.array([x[i] for i in idx]))
        errs.append(V / ref - 1)
    # the nearest cell centre moves slightly with n, so only require a clear
    # second-order-like decrease and a small final error
    assert abs(errs[2]) < 2e-6 and 3.0 < errs[1] / errs[2] < 8.0 and 3.0 < errs[0] / errs[1] < 8.0, errs


def test_symmetry_linearity_and_concatenation():
    n, b, M = 48, 6.0, 20
    h = 2 * b / n
    P = _kernel(n, b, M)
    R_N = P.shape[0]
    f = _mixture(3, 21)
    g = _mixture(4, 22)
    Uf = cp.sample_gaussians(n, b, f["a"], f["X"])
    Ug = cp.sample_gaussians(n, b, g["a"], g["X"])
    Wf = cp.convolve_factors(Uf, P)
    Wg = cp.convolve_factors(Ug, P)

    def cross(Ua, ca, Wb, cb):
        tot = 0.0
        for q in range(R_N):
            prod = np.ones((Ua.shape[1], Wb.shape[1] // R_N))
            for l in range(3):
                prod *= Ua[l] @ Wb[l, q::R_N].T
            tot += ca @ prod @ cb
        return h ** 3 * tot

    fg = cross(Uf, f["c"], Wg, g["c"])
    gf = cross(Ug, g["c"], Wf, f["c"])
    assert abs(fg - gf) < 1e-13 * abs(fg)
    # rank concatenation (Sec. 2.5, Eq. conc): E(f + g) = E(f) + E(g) + 2 <f, P g>
    Ucat = np.concatenate([Uf, Ug], axis=1)
    ccat = np.concatenate([f["c"], g["c"]])
    Ecat = cp.hartree_energy(Ucat, ccat, P, h)
    Ef = cp.hartree_energy(Uf, f["c"], P, h)
    Eg = cp.hartree_energy(Ug, g["c"], P, h)
    assert abs(Ecat - (Ef + Eg + 2 * fg)) < 1e-12 * (abs(Ef) + abs(Eg) + 2 * abs(fg))
    # quadratic in c
    assert abs(cp.hartree_energy(Uf, 2.5 * f["c"], P, h) / Ef - 6.25) < 1e-13
    assert Ef > 0 and Eg > 0 and Ecat > 0


def test_translation_by_whole_cells():
    n, b, M = 64, 8.0, 20
    h = 2 * b / n
    P = _kernel(n, b, M)
    g = _mixture(4, 31)
    E0 = cp.hartree_energy(cp.sample_gaussians(n, b, g["a"], g["X"]), g["c"], P, h)
    X1 = g["X"] + h * np.array([3, -2, 5])
    E1 = cp.hartree_energy(cp.sample_gaussians(n, b, g["a"], X1), g["c"], P, h)
    assert abs(E1 / E0 - 1) < 1e-12


def test_adjoint_against_finite_differences():
    n, b, M = 32, 5.0, 12
    h = 2 * b / n
    P = _kernel(n, b, M)
    g = _mixture(5, 41)
    U = cp.sample_gaussians(n, b, g["a"], g["X"])
    dU, dc = cp.hartree_energy_adjoint(U, g["c"], P, h)
    rng = np.random.default_rng(0)
    for _ in range(12):
        l, k, i = rng.integers(3), rng.integers(5), rng.integers(n)
        eps = 1e-5 * max(1.0, abs(U[l, k, i]))
        Up = U.copy(); Up[l, k, i] += eps
        Um = U.copy(); Um[l, k, i] -= eps
        fd = (cp.hartree_energy(Up, g["c"], P, h) - cp.hartree_energy(Um, g["c"], P, h)) / (2 * eps)
        assert abs(fd - dU[l, k, i]) < 1e-7 * np.max(np.abs(dU)), (fd, dU[l, k, i])
    for k in range(5):
        cp_ = g["c"].copy(); cp_[k] += 1e-5
        cm = g["c"].copy(); cm[k] -= 1e-5
        fd = (cp.hartree_energy(U, cp_, P, h) - cp.hartree_energy(U, cm, P, h)) / 2e-5
        assert abs(fd - dc[k]) < 1e-8 * np.max(np.abs(dc))
    # chain rule to exponents and centres, against FD through re-sampling
    da, dX = cp.gaussian_param_grad(n, b, g["a"], g["X"], U, dU)
    for k in range(5):
        for which in ("a", "X0", "X2"):
            gp = {key: v.copy() for key, v in g.items()}
            gm = {key: v.copy() for key, v in g.items()}
            if which == "a":
                gp["a"][k] += 1e-5; gm["a"][k] -= 1e-5; ref = da[k]
            else:
                l = int(which[1]); gp["X"][k, l] += 1e-5; gm["X"][k, l] -= 1e-5; ref = dX[k, l]
            Ep = cp.hartree_energy(cp.sample_gaussians(n, b, gp["a"], gp["X"]), g["c"], P, h)
            Em = cp.hartree_energy(cp.sample_gaussians(n, b, gm["a"], gm["X"]), g["c"], P, h)
            fd = (Ep - Em) / 2e-5
            assert abs(fd - ref) < 1e-6 * (abs(ref) + np.max(np.abs(da))), (which, k, fd, ref)


def test_parameter_gradients_approach_closed_form():
    # discrete gradients -> derivatives of the analytic mixture energy, O(h^2)
    b, M = 8.0, 40
    g = _mixture(3, 51)
    da_ex, dX_ex, dc_ex = cf.mixture_energy_grad(g["a"], g["X"], g["c"])
    res = {}
    for n in (64, 128):
        h = 2 * b / n
        P = _kernel(n, b, M)
        U = cp.sample_gaussians(n, b, g["a"], g["X"])
        dU, dc = cp.hartree_energy_adjoint(U, g["c"], P, h)
        da, dX = cp.gaussian_param_grad(n, b, g["a"], g["X"], U, dU)
        res[n] = (da, dX, dc)
    for i, ex in enumerate((da_ex, dX_ex, dc_ex)):
        rich = (4 * res[128][i] - res[64][i]) / 3
        scale = np.max(np.abs(ex))
        assert np.max(np.abs(rich - ex)) < 2e-4 * scale, (i, np.max(np.abs(rich - ex)) / scale)
        assert np.max(np.abs(res[128][i] - ex)) < 2e-2 * scale


def test_closed_form_gradient_self_check():
    # the analytic gradient used above agrees with finite differences of the analytic energy
    g = _mixture(3, 61)
    da, dX, dc = cf.mixture_energy_grad(g["a"], g["X"], g["c"])
    for k in range(3):
        ap = g["a"].copy(); ap[k] += 1e-6
        am = g["a"].copy(); am[k] -= 1e-6
        fd = (cf.mixture_energy(ap, g["X"], g["c"]) - cf.mixture_energy(am, g["X"], g["c"])) / 2e-6
        assert abs(fd - da[k]) < 1e-7 * max(1, abs(da[k]))
        Xp = g["X"].copy(); Xp[k, 1] += 1e-6
        Xm = g["X"].copy(); Xm[k, 1] -= 1e-6
        fd = (cf.mixture_energy(g["a"], Xp, g["c"]) - cf.mixture_energy(g["a"], Xm, g["c"])) / 2e-6
        assert abs(fd - dX[k, 1]) < 1e-7 * max(1, abs(dX[k, 1]))


def test_single_column_direct_convolution_matches_toeplitz():
    rng = np.random.default_rng(3)
    for n in (16, 100, 257):
        u = rng.standard_normal(n)
        p = rng.standard_normal(n)
        w = cp.conv1d_direct(u, p)
        # brute force from the definition w[i] = sum_j u[j] p[|i-j|]
        ref = np.array([sum(u[j] * p[abs(i - j)] for j in range(n)) for i in range(n)])
        assert np.max(np.abs(w - ref)) < 1e-12 * np.max(np.abs(ref))
        assert np.max(np.abs(cp.conv1d(u, p) - ref)) < 1e-12 * np.max(np.abs(ref))
