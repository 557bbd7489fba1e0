"""The C-ABI library builds for sm_103a, loads, and exports every symbol that
include/cfft.h declares; argument checks that need no device behave."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    text = open(os.path.join(ROOT, "include", "cfft.h")).read()
    return sorted(set(re.findall(r"\b(cfft_[a-z0-9_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__
    __graft_entry__.build()
    from paper_1404_7357_gb300 import cfft
    return cfft


def test_header_and_binding_agree(lib):
    assert declared_symbols() == sorted(lib.EXPORTS)


def test_every_declared_symbol_is_exported(lib):
    handle = lib.lib()
    for name in declared_symbols():
        assert hasattr(handle, name), name


def test_null_context_arguments(lib):
    h = lib.lib()
    assert h.cfft_create(None, 0, None) == 1               # CFFT_ERR_ARG
    assert h.cfft_set_substrate(None, 2.2, 0.05, 6.28) == 1
    assert h.cfft_tabulate_reactions(None, 4, 10.0, 64, 0, 1) == 1
    assert h.cfft_last_error(None) == b"null context"
    h.cfft_destroy(None)                                   # ignored


def test_create_without_device_fails_cleanly(lib):
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a device is present")
    out = ctypes.c_void_p()
    assert lib.lib().cfft_create(ctypes.byref(out), 0, None) == 4  # CFFT_ERR_CUDA
    assert out.value is None
