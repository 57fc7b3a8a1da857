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
    # element counts stop at 2^31 - 2^22 (32-bit grid-stride indices never overflow)
    big = _lib.sj_grid(0.0, 0.0, 1.0, 1.0, 1 << 20, 1 << 11)       # 2^31 cells
    assert lib.sj_bucket_points(None, 0, C.byref(big), None, None, None) == _lib.SJ_ERR_INVALID
    e = C.c_void_p()
    assert lib.sj_engine_create((1 << 31) - (1 << 22) + 1, 8, None, C.byref(e)) == _lib.SJ_ERR_INVALID
    for w in (-1.0, float("nan")):    # a per-call P2P window is checked before the layer is touched
        st = lib.sj_p2p_join_window(None, None, 0, w, None, None, None, None)
        assert st == _lib.SJ_ERR_INVALID
        assert b"window" in lib.sj_last_error()


def test_struct_layouts_match_header():
    from paper_1403_0802_gb300 import _lib
    assert C.sizeof(_lib.sj_grid) == 40
    assert C.sizeof(_lib.sj_opts) == 24
    assert C.sizeof(_lib.sj_run_stats) == 104
    assert C.sizeof(_lib.sj_layer_info) == 48


def test_binding_imports_without_a_gpu():
    """The Python front end imports on a CPU-only host (the library is only
    loaded, never called)."""
    from paper_1403_0802_gb300 import api, synth  # noqa: F401
    assert api.FORMS == {"fp64": 0, "fp32x": 1}
    o = api._opts("fp32x", "persistent", 32, True)
    assert (o.form, o.launch, o.pts_per_item, o.flags) == (1, 1, 32, 1)


C_STRUCTS = ("sj_grid", "sj_opts", "sj_layer_info", "sj_run_stats", "sj_peak_rates", "sj_request",
             "sj_serve_request", "sj_server_stats")


def test_struct_layouts_match_the_c_compiler(tmp_path):
    """Every struct the binding declares has the size and field offsets that
    the host C compiler gives the header's struct."""
    import shutil
    import subprocess
    from paper_1403_0802_gb300 import _lib
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "sj.h"', '#include "sj_serve.h"', '#include "sj_peaks.h"',
             "int main(void) {"]
    for name in C_STRUCTS:
        lines.append(f'printf("{name} %zu\\n", sizeof({name}));')
        for f, _ in getattr(_lib, name)._fields_:
            lines.append(f'printf("{name}.{f} %zu\\n", offsetof({name}, {f}));')
    lines += ["return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-std=c11", "-I", INCLUDE, str(src), "-o", str(exe)], check=True)
    got = dict(l.split() for l in subprocess.run([str(exe)], check=True, capture_output=True,
                                                  text=True).stdout.splitlines())
    for name in C_STRUCTS:
        T = getattr(_lib, name)
        assert int(got[name]) == C.sizeof(T), name
        for f, _ in T._fields_:
            assert int(got[f"{name}.{f}"]) == getattr(T, f).offset, (name, f)


def test_server_struct_layouts_and_argument_checks(libsj):
    """include/sj_serve.h: struct sizes, and argument errors reported without
    touching a GPU."""
    from paper_1403_0802_gb300 import _lib
    lib = _lib.lib()
    h = C.c_void_p()
    assert lib.sj_server_create(None, None, None, 0, 1 << 20, 1000, 8, C.byref(h)) == _lib.SJ_ERR_INVALID
    assert b"layer" in lib.sj_last_error()
    t = C.c_int64()
    assert lib.sj_server_submit(None, None, C.byref(t)) == _lib.SJ_ERR_INVALID
    assert lib.sj_server_destroy(None) == _lib.SJ_OK


def test_fault_injection_and_checked_build_without_gpu(libsj):
    """The fault hook is host-side state (armed, counted, disarmed without a
    GPU); server calls check their arguments first; the bounds-checked build
    says so, the normal build does not."""
    from paper_1403_0802_gb300 import _lib, build
    lib = _lib.lib()
    assert lib.sj_fault_inject(7, 0, 1) == _lib.SJ_ERR_INVALID
    assert lib.sj_fault_inject(_lib.SJ_FAULT_ALLOC, -1, 1) == _lib.SJ_ERR_INVALID
    assert lib.sj_fault_inject(_lib.SJ_FAULT_ALLOC, 2, 3) == _lib.SJ_OK
    assert lib.sj_fault_pending() == 3
    assert lib.sj_fault_inject(_lib.SJ_FAULT_NONE, 0, 0) == _lib.SJ_OK
    assert lib.sj_fault_pending() == 0
    assert lib.sj_server_cancel(None, 0) == _lib.SJ_ERR_INVALID
    assert lib.sj_server_wait_for(None, 0, 1.0, None) == _lib.SJ_ERR_INVALID
    assert lib.sj_bounds_checked() == 0
    checked = C.CDLL(build.build(checked=True))
    checked.sj_bounds_checked.restype = C.c_int32
    assert checked.sj_bounds_checked() == 1
