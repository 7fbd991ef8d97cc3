"""Exact integral of 1/|x| over an axis-aligned box (the potential of a uniform
rectangular prism, a textbook closed form), used to pin Galerkin entries."""
import math


def _F(x, y, z):
    r = math.sqrt(x * x + y * y + z * z)
    s = 0.0
    if x * y != 0.0:
        s += x * y * math.log(z + r)
    if y * z != 0.0:
        s += y * z * math.log(x + r)
    if z * x != 0.0:
        s += z * x * math.log(y + r)
    if x != 0.0:
        s -= 0.5 * x * x * math.atan(y * z / (x * r))
    if y != 0.0:
        s -= 0.5 * y * y * math.atan(z * x / (y * r))
    if z != 0.0:
        s -= 0.5 * z * z * math.atan(x * y / (z * r))
    return s


def box_nonneg(x0, x1, y0, y1, z0, z1):
    """int over [x0,x1]x[y0,y1]x[z0,z1] of 1/|x|, all bounds >= 0."""
    tot = 0.0
    for i, x in enumerate((x0, x1)):
        for j, y in enumerate((y0, y1)):
            for k, z in enumerate((z0, z1)):
                tot += (-1) ** (i + j + k + 1) * _F(x, y, z)
    return tot


def box(lo, hi):
    """int over the box prod [lo_l, hi_l] of 1/|x| for any signs (split at 0)."""
    segs = []
    for l in range(3):
        a, b = lo[l], hi[l]
        if a < 0.0 < b:
            segs.append([(0.0, -a), (0.0, b)])
        elif b <= 0.0:
            segs.append([(-b, -a)])
        else:
            segs.append([(a, b)])
    tot = 0.0
    for s0 in segs[0]:
        for s1 in segs[1]:
            for s2 in segs[2]:
                tot += box_nonneg(s0[0], s0[1], s1[0], s1[1], s2[0], s2[1])
    return tot


def cell(lo, hi, gl_points=16):
    """int of 1/|x| over a box: the closed form near the origin, where it is well
    conditioned, and tensor Gauss-Legendre far away (the closed form sums
    corner terms of size r^2 to a result of size h^3/r and cancels there)."""
    import numpy as np
    lo = np.asarray(lo, dtype=float)
    hi = np.asarray(hi, dtype=float)
    width = float(np.max(hi - lo))
    nearest = np.sqrt(np.sum(np.maximum(0.0, np.maximum(lo, -hi)) ** 2))
    if nearest < 3.0 * width:
        return box(lo, hi)
    xg, wg = np.polynomial.legendre.leggauss(gl_points)
    pts = [0.5 * (hi[l] - lo[l]) * xg + 0.5 * (hi[l] + lo[l]) for l in range(3)]
    ws = [0.5 * (hi[l] - lo[l]) * wg for l in range(3)]
    X, Y, Z = np.meshgrid(*pts, indexing="ij")
    Wt = ws[0][:, None, None] * ws[1][None, :, None] * ws[2][None, None, :]
    return float(np.sum(Wt / np.sqrt(X * X + Y * Y + Z * Z)))
