"""The library's float64 host set-up (nodes, weights, cell integrals; no GPU)
against the independent oracle implementation of the same readings."""
import numpy as np
import pytest

from tests.gpu_util import oracle_conv_kernel, oracle_master_kernel


@pytest.fixture(scope="module")
def cpc():
    import paper_1504_06289_gb300 as m
    from paper_1504_06289_gb300 import build
    build.build()
    return m


@pytest.mark.parametrize("n,b,M,kind", [(128, 10.0, 20, "conv"), (8192, 20.0, 30, "conv"),
                                        (16, 2.0, 3, "conv"), (4096, 16.0, 25, "conv"),
                                        (4096, 20.0, 25, "conv"), (256, 8.0, 12, "master"),
                                        (16384, 64.0, 30, "master")])
def test_host_tables_match_oracle(cpc, n, b, M, kind):
    t, a, p, hs, u0 = cpc.make_newton_kernel_tables(n, b, M, kind)
    t0, a0, p0 = oracle_conv_kernel(n, b, M) if kind == "conv" else oracle_master_kernel(n, b, M)
    assert np.max(np.abs(t / t0 - 1)) < 1e-12
    assert np.max(np.abs(a / a0 - 1)) < 1e-12
    peak = np.max(np.abs(p0), axis=1, keepdims=True)
    assert np.max(np.abs(p - p0) / peak) < 1e-12
    assert np.allclose(np.log(t[1:] / t[:-1]), hs, rtol=1e-12)
    assert abs(np.log(t[len(t) // 2]) - u0) < 1e-12


def test_host_tables_reject_bad_sizes(cpc):
    from paper_1504_06289_gb300 import CpcError
    for args in [(100, 1.0, 5, "conv"), (16384, 1.0, 5, "conv"), (64, -1.0, 5, "conv"), (64, 1.0, 0, "conv"),
                 (64, 1.0, 65, "master"), (8, 1.0, 5, "master")]:
        with pytest.raises(CpcError):
            cpc.make_newton_kernel_tables(*args)
