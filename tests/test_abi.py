"""The C-ABI library builds for sm_103a, loads without a GPU, and exports every
entry point that include/*.h declares (no compute calls here)."""
import ctypes
import glob
import os
import re

import pytest

from conftest import ROOT

HEADER = os.path.join(ROOT, "include", "nc_pcg.h")


def declared_symbols():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        for m in re.finditer(r"^NC_API\s+[\w\s\*]+?\b(\w+)\s*\(", text, re.M):
            names.add(m.group(1))
    return sorted(names)


@pytest.fixture(scope="module")
def libpath():
    from paper_2008_01440_gb300.build import build
    return build()


def test_header_declares_entry_points():
    names = declared_symbols()
    for required in ("pcg_setup", "pcg_solve", "pcg_apply_poly", "nc_matrix_csr", "nc_bounds_lanczos"):
        assert required in names


def test_library_exports_every_declared_symbol(libpath):
    lib = ctypes.CDLL(libpath)
    missing = [n for n in declared_symbols() if not hasattr(lib, n)]
    assert not missing, missing


def test_host_only_entry_points(libpath):
    lib = ctypes.CDLL(libpath)
    lib.nc_version.restype = ctypes.c_char_p
    assert b"sm_103a" in lib.nc_version()
    lib.nc_strerror.restype = ctypes.c_char_p
    assert lib.nc_strerror(0) == b"ok"
    # argument validation happens before any CUDA call
    h = ctypes.c_void_p()
    assert lib.nc_matrix_csr(ctypes.c_int64(-1), ctypes.c_int64(0), None, None, None, ctypes.byref(h)) == 1
    assert lib.nc_matrix_csr(ctypes.c_int64(0), ctypes.c_int64(0), None, None, None, ctypes.byref(h)) == 0
    assert lib.nc_matrix_destroy(h) == 0
    assert lib.pcg_setup(None, ctypes.c_double(1.0), ctypes.c_double(2.0), 3, ctypes.c_double(1.0), None, None,
                         ctypes.byref(h)) == 1


def test_binding_imports_and_matches_header(libpath):
    import paper_2008_01440_gb300 as nc
    from paper_2008_01440_gb300 import binding
    assert set(binding._SIGS) == set(declared_symbols())
    assert nc.nc_version().startswith("ncpcg")


def test_built_only_for_sm103a():
    from paper_2008_01440_gb300 import build
    assert build.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]


def _header_struct_fields(name):
    """Field names, in order, of `typedef struct { ... } name;` in the header."""
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    m = re.search(r"typedef struct \{([^{}]*)\}\s*" + name + r"\s*;", text)
    assert m, name
    names = []
    for decl in m.group(1).split(";"):
        parts = [p.strip() for p in decl.strip().split(",") if p.strip()]
        if parts:   # "double theta, delta, sigma": the type prefixes the first name only
            names.append(re.findall(r"(\w+)$", parts[0])[0])
            names.extend(parts[1:])
    return names


def test_binding_structs_match_header(libpath):
    """The ctypes mirrors of the option, info and result structs list the
    header's fields in the header's order (an ABI mismatch would shift every
    field after it)."""
    from paper_2008_01440_gb300 import binding
    for name in ("nc_options", "nc_solver_info", "nc_result"):
        cls = getattr(binding, name)
        assert [f for f, _ in cls._fields_] == _header_struct_fields(name), name
    o = binding.make_options(poly="newton", persistent=True, apply_dtype="f32")
    assert (o.poly_form, o.use_graph, o.apply_dtype) == (1, 2, 1)


def _header_constants():
    """NAME = value pairs of the header's enums and integer #defines."""
    text = re.sub(r"/\*.*?\*/", "", open(HEADER).read(), flags=re.S)
    out = {}
    for body in re.findall(r"typedef enum\s*\{([^{}]*)\}", text):
        for name, val in re.findall(r"\b(NC_\w+)\s*=\s*(-?\d+)", body):
            out[name] = int(val)
    for name, val in re.findall(r"^#define\s+(NC_\w+)\s+\(?(-?\d+)[uU]?\)?\s*$", text, re.M):
        out[name] = int(val)
    return out


def test_binding_constants_match_header():
    """Every enum value or integer constant of the header that the binding
    defines has the header's value (status codes, dtypes, layouts, forms)."""
    from paper_2008_01440_gb300 import binding
    consts = _header_constants()
    for required in ("NC_OK", "NC_F64", "NC_FORMAT_SELL", "NC_FORMAT_PSELL", "NC_POLY_NEWTON"):
        assert required in consts, required
    checked = [n for n in consts if hasattr(binding, n)]
    assert len(checked) >= 15
    mismatched = {n: (getattr(binding, n), consts[n]) for n in checked if getattr(binding, n) != consts[n]}
    assert not mismatched, mismatched
    assert binding._FORMATS["psell"] == consts["NC_FORMAT_PSELL"]


def test_setup_rejects_bad_options_before_any_device_call(libpath):
    """pcg_setup validates its options before it touches the device: an
    empty matrix handle (no CUDA) is enough to see every rejection."""
    from paper_2008_01440_gb300 import binding as b
    h = ctypes.c_void_p()
    assert b.lib.nc_matrix_csr(0, 0, None, None, None, ctypes.byref(h)) == b.NC_OK
    S = ctypes.c_void_p()

    try:
        o = b.make_options()
        o.spmv_format = b.NC_FORMAT_PSELL + 1
        assert b.lib.pcg_setup(h, 0.1, 2.0, 3, 1.0, ctypes.byref(o), None, ctypes.byref(S)) == b.NC_ERR_ARG
        o = b.make_options(spmv_format="psell")
        o.apply_dtype = 7
        assert b.lib.pcg_setup(h, 0.1, 2.0, 3, 1.0, ctypes.byref(o), None, ctypes.byref(S)) == b.NC_ERR_ARG
        o = b.make_options()
        o.rr_period = -1
        assert b.lib.pcg_setup(h, 0.1, 2.0, 3, 1.0, ctypes.byref(o), None, ctypes.byref(S)) == b.NC_ERR_ARG
        # the Newton form: k = 2^nlev - 1 only, float64 only
        o = b.make_options(poly="newton")
        assert b.lib.pcg_setup(h, 0.1, 2.0, 4, 1.0, ctypes.byref(o), None, ctypes.byref(S)) == b.NC_ERR_ARG
        o = b.make_options(poly="newton", apply_dtype="f32")
        assert b.lib.pcg_setup(h, 0.1, 2.0, 7, 1.0, ctypes.byref(o), None, ctypes.byref(S)) == b.NC_ERR_UNSUPPORTED
        # the interval and the scale
        o = b.make_options()
        for lo, hi, s in ((0.0, 2.0, 1.0), (2.0, 1.0, 1.0), (0.1, float("inf"), 1.0), (0.1, 2.0, 0.0)):
            assert b.lib.pcg_setup(h, lo, hi, 3, s, ctypes.byref(o), None, ctypes.byref(S)) == b.NC_ERR_ARG
        assert not S.value
    finally:
        assert b.lib.nc_matrix_destroy(h) == b.NC_OK


def test_host_side_matrix_entry_points(libpath):
    """Stencil handles, their Jacobi scaling and their Gershgorin bound are
    host-only: checked here against the assembled CSR's largest absolute row
    sum (brute force), with the argument checks the header documents."""
    import numpy as np
    import workloads as W
    from paper_2008_01440_gb300 import binding as b
    h, hs = ctypes.c_void_p(), ctypes.c_void_p()
    g = ctypes.c_double()
    for bad in ((0, 4, 4, 6.0), (4, 4, 4, float("nan")), (2048, 1024, 1024, 6.0)):
        assert b.lib.nc_matrix_stencil7(*bad[:3], bad[3], 1.0, 1.0, 1.0, ctypes.byref(h)) == b.NC_ERR_ARG
    for dims, c in (((5, 4, 3), (6.0, 1.0, 0.5, 0.25)), ((1, 1, 5), (2.0, 1.0, 1.0, 1.0)),
                    ((2, 7, 1), (3.0, 0.4, 0.9, 0.3))):
        assert b.lib.nc_matrix_stencil7(*dims, *c, ctypes.byref(h)) == b.NC_OK
        try:
            A = W.stencil7_to_csr(W.Stencil7(*dims, *c))
            rows = np.repeat(np.arange(A.n), np.diff(A.rowptr))
            ref = np.zeros(A.n)
            np.add.at(ref, rows, np.abs(A.val))
            assert b.lib.nc_gershgorin(h, None, ctypes.byref(g)) == b.NC_OK
            assert abs(g.value - ref.max()) <= 1e-14 * ref.max()
            # Jacobi scaling: constant diagonal c0, so the bound scales by 1/c0
            assert b.lib.nc_matrix_jacobi(h, None, ctypes.byref(hs)) == b.NC_OK
            assert b.lib.nc_gershgorin(hs, None, ctypes.byref(g)) == b.NC_OK
            assert abs(g.value - ref.max() / c[0]) <= 1e-14 * ref.max() / c[0]
            h2 = ctypes.c_void_p()
            assert b.lib.nc_matrix_jacobi(hs, None, ctypes.byref(h2)) == b.NC_ERR_ARG   # already scaled
            assert b.lib.nc_matrix_destroy(hs) == b.NC_OK
        finally:
            assert b.lib.nc_matrix_destroy(h) == b.NC_OK
    assert b.lib.nc_matrix_stencil7(4, 4, 4, -1.0, 1.0, 1.0, 1.0, ctypes.byref(h)) == b.NC_OK
    assert b.lib.nc_matrix_jacobi(h, None, ctypes.byref(hs)) == b.NC_ERR_ARG          # c0 <= 0
    assert b.lib.nc_matrix_destroy(h) == b.NC_OK
    assert b.lib.nc_matrix_destroy(None) == b.NC_ERR_ARG


def test_status_strings_and_option_defaults(libpath):
    from paper_2008_01440_gb300 import binding as b
    consts = _header_constants()
    codes = sorted({v for k, v in consts.items() if k == "NC_OK" or k.startswith("NC_ERR_")})
    lib = ctypes.CDLL(libpath)
    lib.nc_strerror.restype = ctypes.c_char_p
    texts = [lib.nc_strerror(c) for c in codes]
    assert len(set(texts)) == len(codes) and b"unknown status" not in texts
    assert lib.nc_strerror(max(codes) + 1) == b"unknown status"
    o = b.nc_options()
    b.lib.nc_options_default(ctypes.byref(o))
    assert (o.apply_dtype, o.rr_period, o.x0_is_zero, o.use_graph, o.spmv_format, o.poly_form) == \
        (b.NC_F64, 0, 0, 1, b.NC_FORMAT_AUTO, consts["NC_POLY_CHEBYSHEV"])


def test_batch_create_checks_arguments_first(libpath):
    from paper_2008_01440_gb300 import binding as b
    B = ctypes.c_void_p()
    for args in ((0, 100, 8, 0), (4, 0, 8, 0), (4, 100, 0, 0), (4, 100, 5000, 0), (4, 100, 8, 1 << 12)):
        assert b.lib.pcg_batch_create(*args, None, ctypes.byref(B)) == b.NC_ERR_ARG
        assert not B.value


def test_binding_refuses_tensor_on_another_device(libpath):
    """Every entry point launches on the current device; a tensor that lives on
    another one must be refused before any pointer reaches the library."""
    from paper_2008_01440_gb300 import binding
    binding._check_device(0, 0, "v")
    binding._check_device(3, 3, "v")
    with pytest.raises(ValueError, match="cuda:1 but the current device is cuda:0"):
        binding._check_device(1, 0, "v")
    import torch
    with pytest.raises(TypeError):
        binding._ptr(torch.zeros(4, dtype=torch.float64), torch.float64, 4, "v")   # host tensor
