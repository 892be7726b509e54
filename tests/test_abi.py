"""The C-ABI library builds for sm_103a, loads, and exports every symbol that
include/randutv.h declares; host-side argument checks return their status
before any CUDA call (no GPU needed)."""
import ctypes
import os
import re

import pytest

import paper_2104_05782_gb300 as rutv
from paper_2104_05782_gb300 import build as rbuild

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    rbuild.build()
    return rutv.load()


def declared_functions():
    names = []
    for fn in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names += re.findall(r"\b(randutv_\w+)\s*\(", src)
    return sorted(set(names))


def test_header_declares_entry_points():
    names = declared_functions()
    for want in ("randutv_factor", "randutv_factor_ex", "randutv_workspace_size", "randutv_factor_host",
                 "randutv_status_string"):
        assert want in names


def test_library_exports_every_declared_symbol(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name
        assert isinstance(getattr(lib, name), ctypes._CFuncPtr)


def test_status_strings(lib):
    assert rutv.status_string(0) == "ok"
    assert "invalid" in rutv.status_string(rutv.RANDUTV_EINVAL)
    assert rutv.status_string(99) == "unknown status"


@pytest.mark.parametrize("m,n,lda,b,q", [
    (3, 5, 3, 2, 1),     # m < n
    (5, 3, 5, 0, 1),     # b < 1
    (5, 3, 5, 2, -1),    # q < 0
    (5, 3, 4, 2, 1),     # lda < m
    (-1, 0, 1, 2, 1),    # negative size
])
def test_invalid_arguments_rejected_on_host(lib, m, n, lda, b, q):
    fake = 256  # never dereferenced: validation fails first
    assert rutv.randutv_factor(m, n, fake, lda, b, q, 0, fake, fake, fake) == rutv.RANDUTV_EINVAL
    assert rutv.randutv_factor_ex(m, n, fake, lda, b, q, 0, fake, fake, fake) == rutv.RANDUTV_EINVAL


def test_null_t_rejected(lib):
    assert rutv.randutv_factor(4, 3, 256, 4, 2, 1, 0, None, None, None) == rutv.RANDUTV_EINVAL


def test_workspace_size_host_logic(lib):
    assert rutv.randutv_workspace_size(3, 5, 2) == 0          # m < n
    assert rutv.randutv_workspace_size(5, 3, 0) == 0          # b < 1
