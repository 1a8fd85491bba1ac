"""Host-side checks of the C ABI: the library loads without a GPU, exports
every function include/magnitude.h declares, and the binding's structs match
the header's layout.  No device work runs here."""
import ctypes
import os
import re

import pytest

import paper_2607_23354_gb300 as M

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    src = open(os.path.join(ROOT, "include", "magnitude.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(mag_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_2607_23354_gb300 import build
    build.build()
    return M.load_library()


def test_every_declared_symbol_is_exported(lib):
    names = _declared_functions()
    assert len(names) >= 14
    for name in names:
        assert hasattr(lib, name), name
    assert set(names) == set(M.SIGNATURES), set(names) ^ set(M.SIGNATURES)


def test_status_strings(lib):
    for code, name in [(0, "MAG_OK"), (1, "MAG_EINVAL"), (2, "MAG_EDUPLICATE"), (3, "MAG_ENOTPD"),
                       (4, "MAG_ENOCONV"), (5, "MAG_ENOBRACKET"), (6, "MAG_ENOMEM"), (7, "MAG_ECUDA"),
                       (8, "MAG_ETIMEOUT")]:
        assert M.status_string(code) == name
    assert M.status_string(99) == "MAG_UNKNOWN"


def test_options_defaults_and_struct_sizes(lib):
    o = M.mag_options()
    assert lib.mag_options_default(ctypes.byref(o)) == 0
    assert o.precision == M.PREC_AUTO and o.ir_tol == 1e-14 and o.allow_fallback == 1
    assert o.residual_mode == M.RESID_AUTO and o.ir_max_iters > 0
    # sizes follow the C layout (natural alignment on both x86-64 and aarch64)
    assert ctypes.sizeof(M.mag_options) == 112
    assert ctypes.sizeof(M.mag_batch_desc) == 32
    assert ctypes.sizeof(M.mag_info) == 6 * 4 + 6 * 8 + 2 * 4 + 6 * 8 + 8 + 2 * 4 + 2 * 8 + 4 * 8 + 2 * 8 + 8 + 2 * 4 + 4 * 8 + 2 * 4 + 8 + 8 * 4
    assert lib.mag_options_default(None) == M.MAG_EINVAL


def test_null_context_is_rejected(lib):
    assert lib.mag_ctx_destroy(None) == 0
    assert lib.mag_last_error(None) == b"no context"
    b = ctypes.c_double(0)
    assert lib.mag_workspace_bytes(None, 100, 3, ctypes.byref(b)) == M.MAG_EINVAL
    assert lib.mag_solve(None, None, 10, 2, 1.0, None, None, None) == M.MAG_EINVAL


def test_python_options_marshal(lib):
    o = M.Options(precision="fp64", residual_mode="stored", ir_tol=1e-13, ir_max_iters=7).to_c()
    assert o.precision == M.PREC_FP64 and o.residual_mode == M.RESID_STORED
    assert o.ir_tol == 1e-13 and o.ir_max_iters == 7
    # the sweep kind and the exact distances: defaults as the C defaults
    d = M.mag_options()
    assert lib.mag_options_default(ctypes.byref(d)) == 0
    o = M.Options().to_c()
    assert o.sweep_kind == d.sweep_kind == 0 and o.exact_distances == d.exact_distances == 1
    o = M.Options(sweeps="progress", exact_distances=False, fp16_gmres=1, gmres_matvec="fp64").to_c()
    assert o.sweep_kind == 2 and o.exact_distances == 0 and o.fp16_gmres == 1 and o.gmres_matvec == 1
    assert M.Options(sweeps="chain_fp32").to_c().sweep_kind == 1
    with pytest.raises(ValueError):
        M.Options(sweeps="fast").to_c()


def test_product_path_has_no_oracle_import():
    pkg = os.path.join(ROOT, "paper_2607_23354_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                txt = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in txt and "from oracle" not in txt, f
                assert "oracle.c" not in txt, f
