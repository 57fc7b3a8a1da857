"""Host-side checks of the C ABI (no GPU needed): libsj.so builds for sm_103a,
loads, and exports every entry point include/sj.h declares; the Python
binding declares exactly those signatures."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
INCLUDE = os.path.join(ROOT, "include")


def declared_functions():
    names = set()
    for f in sorted(os.listdir(INCLUDE)):
        if f.endswith(".h"):
            text = re.sub(r"/\*.*?\*/", "", open(os.path.join(INCLUDE, f)).read(), flags=re.S)
            names |= set(re.findall(r"\b(sj_[a-z0-9_]+)\s*\(", text))
    return sorted(names)


@pytest.fixture(scope="module")
def libsj():
    from paper_1403_0802_gb300 import build
    so = build.build()
    return C.CDLL(so)


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ("sj_pip_layer_create", "sj_p2p_layer_create", "sj_pip_join", "sj_p2p_join", "sj_layer_destroy",
                 "sj_bucket_points", "sj_last_error"):
        assert must in names


def test_library_exports_every_declared_symbol(libsj):
    missing = [n for n in declared_functions() if not hasattr(libsj, n)]
    assert not missing, missing


def test_binding_covers_the_header(libsj):
    from paper_1403_0802_gb300 import _lib
    assert sorted(_lib.SIGNATURES) == declared_functions()


def test_version_and_error_string_without_gpu(libsj):
    libsj.sj_version.restype = C.c_char_p
    libsj.sj_last_error.restype = C.c_char_p
    assert b"sm_103a" in libsj.sj_version()
    assert libsj.sj_last_error() == b""


def test_argument_errors_are_synchronous_and_need_no_gpu(libsj):
    """Argument checks run before any CUDA call: a bad grid is rejected."""
    from paper_1403_0802_gb300 import _lib
    lib = _lib.lib()
    bad = _lib.sj_grid(0.0, 0.0, -1.0, 1.0, 4, 4)       # x1 < x0
    h = C.c_void_p()
    st = lib.sj_p2p_layer_create(None, 0, None, 0, 1.0, C.byref(bad), None, C.byref(h))
    assert st == _lib.SJ_ERR_INVALID
    assert b"grid" in lib.sj_last_error()
    st = lib.sj_bucket_points(None, 0, C.byref(bad), None, None, None)
    assert st == _lib.SJ_ERR_INVALID


def test_struct_layouts_match_header():
    from paper_1403_0802_gb300 import _lib
    assert C.sizeof(_lib.sj_grid) == 40
    assert C.sizeof(_lib.sj_opts) == 24
    assert C.sizeof(_lib.sj_run_stats) == 80
    assert C.sizeof(_lib.sj_layer_info) == 48


def test_binding_imports_without_a_gpu():
    """The Python front end imports on a CPU-only host (the library is only
    loaded, never called)."""
    from paper_1403_0802_gb300 import api, synth  # noqa: F401
    assert api.FORMS == {"fp64": 0, "fp32x": 1}
    o = api._opts("fp32x", "persistent", 32, True)
    assert (o.form, o.launch, o.pts_per_item, o.flags) == (1, 1, 32, 1)


def test_request_struct_layout():
    from paper_1403_0802_gb300 import _lib
    assert C.sizeof(_lib.sj_request) == 40


def test_server_struct_layouts_and_argument_checks(libsj):
    """include/sj_serve.h: struct sizes, and argument errors reported without
    touching a GPU."""
    from paper_1403_0802_gb300 import _lib
    assert C.sizeof(_lib.sj_serve_request) == 48
    assert C.sizeof(_lib.sj_server_stats) == 48
    lib = _lib.lib()
    h = C.c_void_p()
    assert lib.sj_server_create(None, None, None, 0, 1 << 20, 1000, 8, C.byref(h)) == _lib.SJ_ERR_INVALID
    assert b"layer" in lib.sj_last_error()
    t = C.c_int64()
    assert lib.sj_server_submit(None, None, C.byref(t)) == _lib.SJ_ERR_INVALID
    assert lib.sj_server_destroy(None) == _lib.SJ_OK
