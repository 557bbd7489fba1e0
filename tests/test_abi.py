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


def _header_struct(name):
    """Field (name, C type) list of `typedef struct { ... } name;` in include/cfft.h."""
    text = open(os.path.join(ROOT, "include", "cfft.h")).read()
    m = re.search(r"typedef struct \{([^}]*)\}\s*" + name + r"\s*;", text)
    assert m, name
    fields = []
    for decl in m.group(1).split(";"):
        decl = re.sub(r"/\*.*?\*/", "", decl, flags=re.S).strip()
        if not decl:
            continue
        ctype, names = decl.split(None, 1)
        fields += [(n.strip(), ctype) for n in names.split(",")]
    return fields


@pytest.mark.parametrize("cname,pyname", [("cfft_info", "Info"), ("cfft_batch_info", "BatchInfo"),
                                          ("cfft_batch_item", "BatchItem"), ("cfft_solve_info", "SolveInfo"),
                                          ("cfft_cartesian_info", "CartesianInfo")])
def test_struct_layouts_match_header(lib, cname, pyname):
    """The ctypes mirrors of the ABI structs list the header's fields in its order with the
    same C types (a field added on one side only would shift every later one)."""
    from paper_1404_7357_gb300 import cfft
    ctypes_of = {"int": ctypes.c_int, "double": ctypes.c_double}
    header = _header_struct(cname)
    binding = getattr(cfft, pyname)._fields_
    assert [n for n, _ in header] == [n for n, _ in binding]
    for (n, ct), (_, pt) in zip(header, binding):
        assert ctypes_of[ct] is pt, (cname, n)


def test_option_ids_match_header(lib):
    """Every option constant of the binding has the value of the header's enum."""
    from paper_1404_7357_gb300 import cfft
    text = open(os.path.join(ROOT, "include", "cfft.h")).read()
    enum = dict((k, int(v)) for k, v in re.findall(r"CFFT_OPT_([A-Z0-9_]+)\s*=\s*(\d+)", text))
    assert enum
    for name, value in enum.items():
        assert getattr(cfft, "OPT_" + name) == value, name


def _unbound_context(cfft, n_mbf):
    """A Context object with no C context behind it: enough to exercise the binding's
    own argument checks, which run before any library call."""
    import torch
    c = object.__new__(cfft.Context)
    c._torch = torch
    c._h = ctypes.c_void_p()
    c.device = 0
    c.n_mbf = n_mbf
    return c


def test_fill_binding_rejects_bad_layouts(lib):
    import numpy as np
    import torch
    c = _unbound_context(lib, 4)
    pos = np.zeros((3, 2))
    rot = np.zeros(3, dtype=np.int32)
    z = np.zeros((12, 13), dtype=np.complex64)
    assert c._check_layout(pos, rot, z, device=False) == 3
    assert c._check_layout(pos, None, np.zeros((12, 12), dtype=np.complex128), device=False) == 3
    bad = [
        (pos.astype(np.float32), rot, z),                   # positions not float64
        (np.zeros((3, 3)), rot, z),                          # not (A, 2)
        (pos, rot.astype(np.int64), z),                      # rotations not int32
        (pos, np.zeros(2, dtype=np.int32), z),               # one rotation per element
        (pos, rot, np.zeros((11, 12), dtype=np.complex64)),  # fewer than A*M rows
        (pos, rot, np.zeros((12, 11), dtype=np.complex64)),  # fewer than A*M columns
        (pos, rot, np.zeros((12, 12), dtype=np.float64)),    # not complex
    ]
    for p, r, m in bad:
        with pytest.raises(ValueError):
            c._check_layout(p, r, m, device=False)
    # the device entry points take CUDA tensors only
    with pytest.raises(ValueError):
        c._check_layout(torch.zeros((3, 2), dtype=torch.float64), None,
                        torch.zeros((12, 12), dtype=torch.complex64), device=True)


def test_static_backprojection_and_spectra_bindings_refuse_host_tensors(lib):
    import torch
    grid = torch.zeros((1, 1, 1, 101), dtype=torch.complex64)
    table = torch.zeros((1, 1, 1, 64), dtype=torch.complex64)
    with pytest.raises(ValueError):
        lib.backproject_static(grid, table, 1, 0, 10.0, 50, 0.1, 4, 8, 10.0, stream=0)
    c = _unbound_context(lib, 2)
    with pytest.raises(ValueError):
        c.mbf_spectra(torch.zeros((8, 2), dtype=torch.complex64))


def test_static_backprojection_argument_checks_need_no_device(lib):
    h = lib.lib()
    dummy = ctypes.c_void_p(16)   # never dereferenced: every case below is refused first

    def call(**kw):
        a = dict(device=0, grid=dummy, table=dummy, series_per_q=1, q_max=0, n_rho=64, rho_max=1.0,
                 grid_half=64, delta_s=0.1, sigma=4, taps=8, beta=10.0, margin=24.0)
        a.update(kw)
        return h.cfft_backproject_static(a["device"], None, a["grid"], a["table"], a["series_per_q"],
                                         a["q_max"], a["n_rho"], a["rho_max"], a["grid_half"],
                                         a["delta_s"], a["sigma"], a["taps"], a["beta"], a["margin"], 0)
    for kw in ({"taps": 5}, {"taps": 14}, {"sigma": 3}, {"grid": None}, {"n_rho": 1},
               {"rho_max": float("nan")}, {"q_max": 65}, {"device": -1}, {"delta_s": 0.0}):
        assert call(**kw) == 1, kw                              # CFFT_ERR_ARG


def test_header_is_plain_c(tmp_path):
    """include/cfft.h is a C header (C99, pedantic): plain pointers and sizes, no C++ or
    torch types, so that any C caller can use the library."""
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    src = tmp_path / "use_header.c"
    src.write_text('#include "cfft.h"\nint main(void) { cfft_ctx* c = 0; (void)c; return (int)CFFT_OK; }\n')
    r = subprocess.run([cc, "-std=c99", "-Wall", "-Wextra", "-pedantic", "-Werror", "-fsyntax-only",
                        "-I", os.path.join(ROOT, "include"), str(src)], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr


def test_readme_c_example_compiles(tmp_path):
    """The C example of README.md stays valid against include/cfft.h (syntax and types)."""
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    text = open(os.path.join(ROOT, "README.md")).read()
    m = re.search(r"```c\n(.*?)```", text, flags=re.S)
    assert m, "README.md has no C example"
    src = tmp_path / "readme_example.c"
    src.write_text(m.group(1))
    r = subprocess.run([cc, "-std=c99", "-Wall", "-Wextra", "-Werror", "-fsyntax-only",
                        "-I", os.path.join(ROOT, "include"), str(src)], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr


def test_fill_binding_before_an_element_leaves_the_state_error_to_the_library(lib):
    """Without an element the binding has no MBF count; it checks what it can and lets the
    library report the call order (CFFT_ERR_STATE) instead of failing on its own."""
    import numpy as np
    c = _unbound_context(lib, 1)
    del c.n_mbf
    assert c._check_layout(np.zeros((2, 2)), None, np.zeros((1, 1), dtype=np.complex64), device=False) == 2
