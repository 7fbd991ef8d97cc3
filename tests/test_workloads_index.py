"""The index bookkeeping of workloads.py (used by bench.py) lists the same
product functions, in the same order, as the oracle's Coulomb-matrix module."""
import numpy as np

import workloads
from oracle import coulomb as ocoul
from oracle import tei as otei


def test_item_and_density_pairs_match_the_oracle():
    basis = workloads.basis_for("basis80_n4096", 3)
    nb = len(basis["fn_first"]) - 1
    items, ia, ib, off = workloads.basis_item_pairs(basis)
    assert items == ocoul.item_list(nb)
    ja, jb, _, joff = ocoul.item_pairs(basis, items)
    assert np.array_equal(ia, ja) and np.array_equal(ib, jb) and np.array_equal(off, joff)
    pa, pb, wt = workloads.basis_density_pairs(basis)
    qa, qb, coef = ocoul.density_pairs(basis)
    assert np.array_equal(pa, qa) and np.array_equal(pb, qb)
    # the oracle's coefficient is the weight times the contraction coefficients
    assert np.allclose(wt * basis["prim_d"][pa] * basis["prim_d"][pb], coef, rtol=1e-15, atol=0)


def test_upper_pairs_match_the_oracle():
    for nb in (1, 2, 7, 80):
        a, b = workloads.upper_pairs(nb)
        c, d = otei.pair_list(nb)
        assert np.array_equal(a, c) and np.array_equal(b, d)
