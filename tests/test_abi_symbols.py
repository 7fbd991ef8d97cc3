"""The C-ABI library loads and exports every function include/cpc.h declares (CPU only)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
LIB = os.path.join(ROOT, "paper_1504_06289_gb300", "libcpc.so")


def declared():
    text = open(os.path.join(ROOT, "include", "cpc.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"^[A-Za-z_][\w\s\*]*?\b([a-z_][a-z0-9_]*)\s*\(", text, flags=re.M)))


@pytest.fixture(scope="module")
def lib():
    if not os.path.exists(LIB):
        from paper_1504_06289_gb300 import build
        build.build()
    return ctypes.CDLL(LIB)


def test_header_declares_the_main_entry_points():
    names = declared()
    for n in ("make_newton_kernel", "cp_convolve", "cp_hartree_energy", "coulomb_matrix",
              "lattice_potential_sum", "lattice_interaction_energy"):
        assert n in names


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_only_the_api_is_exported():
    import subprocess
    out = subprocess.run(["nm", "-D", "--defined-only", LIB], capture_output=True, text=True).stdout
    exported = sorted(l.split()[-1] for l in out.splitlines() if " T " in l)
    assert exported == declared()


def test_binding_prototypes_cover_the_header():
    from paper_1504_06289_gb300 import _abi
    assert sorted(_abi.PROTOTYPES) == declared()


def test_status_strings(lib):
    lib.cpc_status_string.restype = ctypes.c_char_p
    for code in (0, -1, -2, -3, -4, -5):
        assert lib.cpc_status_string(code)
    assert b"unknown" in lib.cpc_status_string(7)
