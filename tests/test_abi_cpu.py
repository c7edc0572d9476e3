"""Host-side checks of the C ABI that need no GPU: the library builds for
sm_103a, loads, and exports every entry point the header declares."""

import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2310_15235_gb300 import build_lib
    build_lib.build()
    import paper_2310_15235_gb300 as t2
    return t2


def test_header_declares_the_boundary(lib):
    syms = lib.exported_symbols()
    for name in ("trevr2_build", "trevr2_J", "trevr2_free", "trevr2_last_error", "trevr2_status",
                 "trevr2_tree_info_get", "trevr2_tree_export", "trevr2_alpha_table",
                 "trevr2_healpix_pix2vec", "trevr2_healpix_vec2pix"):
        assert name in syms


def test_library_exports_every_declared_symbol(lib):
    so = ctypes.CDLL(lib.library_path())
    missing = [s for s in lib.exported_symbols() if not hasattr(so, s)]
    assert not missing, missing
    out = subprocess.run(["nm", "-D", "--defined-only", lib.library_path()], capture_output=True,
                         text=True, check=True).stdout
    exported = {line.split()[-1] for line in out.splitlines() if " T " in line}
    assert set(lib.exported_symbols()) <= exported


def test_last_error_without_gpu_work(lib):
    so = lib.load_library()
    # argument validation happens on the host before any CUDA call
    rc = so.trevr2_build(None, None, None, None, None, -1, 1, None, 0.0, 12, None, None)
    assert rc == -1
    assert b"out is NULL" in so.trevr2_last_error()
    handle = ctypes.c_void_p()
    rc = so.trevr2_build(None, None, None, None, None, 10, 1, None, 0.0, 12, None,
                         ctypes.byref(handle))
    assert rc == -1 and b"NULL input" in so.trevr2_last_error()
    rc = so.trevr2_build(None, None, None, None, None, 0, 9, None, 0.0, 12, None,
                         ctypes.byref(handle))
    assert rc == -5
    assert so.trevr2_J(None, None, 0, 2, ctypes.c_float(0.75), None, 0, 0, None, None) == -1
    assert so.trevr2_free(None) == 0


def test_python_layer_fails_loudly_without_library(monkeypatch, tmp_path):
    import paper_2310_15235_gb300 as t2
    monkeypatch.setattr(t2, "_LIB_PATH", str(tmp_path / "missing.so"))
    monkeypatch.setattr(t2, "_lib", None)
    with pytest.raises(RuntimeError, match="no CPU fallback"):
        t2.load_library()


def test_flag_values_agree(lib):
    """The header's flag bits, the Python binding's constants and the
    oracle's flags are the same numbers."""
    import os
    import re

    import oracle
    hdr = open(os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                            "include", "trevr2.h")).read()
    defs = {m.group(1): int(m.group(2)) for m in
            re.finditer(r"#define TREVR2_([A-Z]+) (\d+)u", hdr)}
    for name in ("SOFT", "THICK", "ASYNC", "LINEAR", "BUCKET", "PP", "CSM"):
        assert getattr(lib, name) == defs[name], name
    for name in ("SOFT", "THICK", "LINEAR", "BUCKET", "PP", "CSM"):
        assert getattr(oracle, "FLAG_" + name) == defs[name], name
    bits = [defs[n] for n in ("SOFT", "THICK", "ASYNC", "LINEAR", "BUCKET", "PP", "CSM")]
    assert len(set(bits)) == len(bits) and all(b & (b - 1) == 0 for b in bits)


def test_testing_aids_match_header(lib):
    """The binding's testing-aid settings are the header's, and the library
    rejects an unknown setting on the host (no GPU work)."""
    with open(os.path.join(ROOT, "include", "trevr2.h")) as f:
        hdr = f.read()
    defs = {m.group(1): int(m.group(2)) for m in
            re.finditer(r"#define TREVR2_(DEBUG_[A-Z_]+) (\d+)", hdr)}
    assert defs == {"DEBUG_FAIL_ALLOC": lib.DEBUG_FAIL_ALLOC,
                    "DEBUG_SOURCE_STACK": lib.DEBUG_SOURCE_STACK}
    so = lib.load_library()
    assert so.trevr2_debug_set(99, 0) == -1
    assert b"unknown setting" in so.trevr2_last_error()
    assert so.trevr2_debug_set(lib.DEBUG_FAIL_ALLOC, -1) == 0
    assert so.trevr2_debug_pool_used(None) == -1
    assert so.trevr2_kernel_binary_version(None) == -1


def test_new_entry_points_validate_on_host(lib):
    so = lib.load_library()
    assert so.trevr2_set_tau_refine(None, ctypes.c_double(0.1), None) == -1
    assert b"tree is NULL" in so.trevr2_last_error()
    tgt = (ctypes.c_double * 3)(0.5, 0.5, 0.5)
    assert so.trevr2_J_directed(None, None, 0, 2, ctypes.c_float(0.75), None, 0, 16, tgt,
                                None, None) == -1
    assert so.trevr2_J_directed(None, None, 0, 2, ctypes.c_float(0.75), None, 0, 16, None,
                                None, None) == -1
    assert b"target is NULL" in so.trevr2_last_error()
