"""ctypes front end of the CPU oracle (sj_oracle.c).

TEST INFRASTRUCTURE ONLY: the test suite, the smoke check and the benchmark's
CPU-baseline leg are the only users.  The CUDA path never imports this module.

Every function takes and returns numpy arrays; the arithmetic lives in the C
file (FP64, -ffp-contract=off, no fast-math), which cites the paper section of
each step.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sj_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_SO = os.path.join(_OUT_DIR, "libsj_oracle.so")
_lock = threading.Lock()
_lib = None

OK, INVALID, OOM, GRID_COVER = 0, -1, -2, -3


class Grid(C.Structure):
    _fields_ = [("x0", C.c_double), ("y0", C.c_double), ("x1", C.c_double), ("y1", C.c_double),
                ("nx", C.c_int32), ("ny", C.c_int32)]


_SO_SAN = os.path.join(_OUT_DIR, "libsj_oracle_san.so")


def build(force: bool = False, sanitize: bool = False) -> str:
    """Compile the oracle with gcc (OpenMP when available).  sanitize=True:
    a separate build with AddressSanitizer and UndefinedBehaviorSanitizer
    (single-threaded; a process loading it needs the ASan runtime preloaded)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    so = _SO_SAN if sanitize else _SO
    if not force and os.path.exists(so) and os.path.getmtime(so) >= os.path.getmtime(_SRC):
        return so
    base = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared", "-std=c11",
            "-Wall", "-Wno-unknown-pragmas"]
    tmp = so + f".tmp{os.getpid()}"
    if sanitize:
        subprocess.run(base + ["-g", "-fno-omit-frame-pointer", "-fsanitize=address,undefined",
                               "-fno-sanitize-recover=undefined", _SRC, "-o", tmp, "-lm"], check=True)
        os.replace(tmp, so)
        return so
    try:
        subprocess.run(base + ["-fopenmp", _SRC, "-o", tmp, "-lm"], check=True, capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base + [_SRC, "-o", tmp, "-lm"], check=True)
    os.replace(tmp, so)
    return so


def use(path: str):
    """Load the oracle from `path` (e.g. the sanitized build) instead of the
    default build; only before the first call."""
    global _SO
    with _lock:
        if _lib is not None:
            raise RuntimeError("the oracle is already loaded")
        _SO = path


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = C.CDLL(_SO if os.path.basename(_SO) != "libsj_oracle.so" else build())
        d, i32, i64, p = C.c_double, C.c_int32, C.c_int64, C.c_void_p
        gp = C.POINTER(Grid)
        sig = {
            "or_set_threads": (None, [C.c_int]),
            "or_max_threads": (C.c_int, []),
            "or_set_exact": (None, [C.c_int]),
            "or_cross_sign": (C.c_int, [d, d, d, d, d, d]),
            "or_point_cell": (i64, [gp, d, d]),
            "or_point_cells": (None, [gp, p, i64, p]),
            "or_cell_counts": (C.c_int, [gp, p, i64, p]),
            "or_pip_mbb": (C.c_int, [gp, p, i64, p, i64, p, i32, p]),
            "or_p2p_mbb": (C.c_int, [gp, p, i64, p, i32, p]),
            "or_cand_csr": (C.c_int, [gp, p, i32, d, C.c_int, p, p]),
            "or_pip_polygon": (C.c_int, [d, d, p, p, p, i32]),
            "or_pip_brute": (C.c_int, [gp, p, i64, p, p, p, i32, p, p]),
            "or_pip_grid": (C.c_int, [gp, p, i64, p, p, p, p, p, p, p]),
            "or_seg_dist": (d, [d, d, d, d, d, d]),
            "or_line_dist": (d, [d, d, p, p, i32]),
            "or_p2p_brute": (C.c_int, [gp, p, i64, p, p, i32, d, p, p, p, p]),
            "or_p2p_grid": (C.c_int, [gp, p, i64, p, p, d, p, p, p, p, p, p]),
        }
        for name, (res, args) in sig.items():
            f = getattr(lib, name)
            f.restype = res
            f.argtypes = args
        _lib = lib
        return lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _i64(a):
    return np.ascontiguousarray(a, dtype=np.int64)


def _grid(g) -> Grid:
    if isinstance(g, Grid):
        return g
    return Grid(float(g["x0"]), float(g["y0"]), float(g["x1"]), float(g["y1"]), int(g["nx"]), int(g["ny"]))


class OracleError(RuntimeError):
    def __init__(self, code):
        super().__init__(f"oracle status {code}")
        self.code = code


def _check(rc):
    if rc != OK:
        raise OracleError(rc)


def set_threads(n: int | None = None) -> int:
    lib = _load()
    n = lib.or_max_threads() if n is None else int(n)
    lib.or_set_threads(n)
    return n


class exact_predicates:
    """Context manager: PIP crossing signs from the exact value of the
    determinant (Shewchuk's adaptive predicate) instead of its FP64 value."""

    def __enter__(self):
        _load().or_set_exact(1)
        return self

    def __exit__(self, *exc):
        _load().or_set_exact(0)


def cross_sign(hx, hy, lx, ly, px, py) -> int:
    """Sign (-1, 0, 1) the crossing rule takes for
    (hx - lx)(py - ly) - (hy - ly)(px - lx) in the current mode."""
    return int(_load().or_cross_sign(float(hx), float(hy), float(lx), float(ly), float(px), float(py)))


def point_cell(g, x: float, y: float) -> int:
    return int(_load().or_point_cell(C.byref(_grid(g)), float(x), float(y)))


def point_cells(g, pts) -> np.ndarray:
    pts = _f64(pts)
    out = np.empty(len(pts), np.int64)
    _load().or_point_cells(C.byref(_grid(g)), _ptr(pts), len(pts), _ptr(out))
    return out


def cell_counts(g, pts) -> np.ndarray:
    gg = _grid(g)
    pts = _f64(pts)
    out = np.empty(gg.nx * gg.ny + 1, np.int64)
    _check(_load().or_cell_counts(C.byref(gg), _ptr(pts), len(pts), _ptr(out)))
    return out


def pip_mbb(g, verts, ring_off, poly_ring_off) -> np.ndarray:
    verts, ring_off, poly_ring_off = _f64(verts), _i64(ring_off), _i64(poly_ring_off)
    P = len(poly_ring_off) - 1
    out = np.empty((P, 4), np.float64)
    _check(_load().or_pip_mbb(C.byref(_grid(g)), _ptr(verts), len(verts), _ptr(ring_off), len(ring_off) - 1,
                              _ptr(poly_ring_off), P, _ptr(out)))
    return out


def p2p_mbb(g, verts, line_off) -> np.ndarray:
    verts, line_off = _f64(verts), _i64(line_off)
    L = len(line_off) - 1
    out = np.empty((L, 4), np.float64)
    _check(_load().or_p2p_mbb(C.byref(_grid(g)), _ptr(verts), len(verts), _ptr(line_off), L, _ptr(out)))
    return out


def cand_csr(g, mbb, R: float = 0.0, expand: bool = False):
    """Per-cell candidate lists: (cand_start int64 [G+1], cand_ids int32 [M])."""
    gg = _grid(g)
    mbb = _f64(mbb)
    G = gg.nx * gg.ny
    start = np.empty(G + 1, np.int64)
    lib = _load()
    _check(lib.or_cand_csr(C.byref(gg), _ptr(mbb), len(mbb), float(R), int(expand), _ptr(start), None))
    ids = np.empty(int(start[-1]), np.int32)
    _check(lib.or_cand_csr(C.byref(gg), _ptr(mbb), len(mbb), float(R), int(expand), _ptr(start), _ptr(ids)))
    return start, ids


def pip_polygon(px, py, verts, ring_off, poly_ring_off, p: int) -> int:
    verts, ring_off, poly_ring_off = _f64(verts), _i64(ring_off), _i64(poly_ring_off)
    return int(_load().or_pip_polygon(float(px), float(py), _ptr(verts), _ptr(ring_off), _ptr(poly_ring_off),
                                      int(p)))


def pip_brute(g, pts, verts, ring_off, poly_ring_off, with_hits: bool = False):
    pts, verts, ring_off, poly_ring_off = _f64(pts), _f64(verts), _i64(ring_off), _i64(poly_ring_off)
    out = np.empty(len(pts), np.int32)
    nh = np.empty(len(pts), np.int32) if with_hits else None
    _check(_load().or_pip_brute(C.byref(_grid(g)), _ptr(pts), len(pts), _ptr(verts), _ptr(ring_off),
                                _ptr(poly_ring_off), len(poly_ring_off) - 1, _ptr(out), _ptr(nh)))
    return (out, nh) if with_hits else out


def pip_grid(g, pts, verts, ring_off, poly_ring_off, cand_start, cand_ids, with_hits: bool = False):
    pts, verts, ring_off, poly_ring_off = _f64(pts), _f64(verts), _i64(ring_off), _i64(poly_ring_off)
    cand_start = _i64(cand_start)
    cand_ids = np.ascontiguousarray(cand_ids, np.int32)
    out = np.empty(len(pts), np.int32)
    nh = np.empty(len(pts), np.int32) if with_hits else None
    _check(_load().or_pip_grid(C.byref(_grid(g)), _ptr(pts), len(pts), _ptr(verts), _ptr(ring_off),
                               _ptr(poly_ring_off), _ptr(cand_start), _ptr(cand_ids), _ptr(out), _ptr(nh)))
    return (out, nh) if with_hits else out


def seg_dist(px, py, ax, ay, bx, by) -> float:
    return float(_load().or_seg_dist(float(px), float(py), float(ax), float(ay), float(bx), float(by)))


def line_dist(px, py, verts, line_off, l: int) -> float:
    verts, line_off = _f64(verts), _i64(line_off)
    return float(_load().or_line_dist(float(px), float(py), _ptr(verts), _ptr(line_off), int(l)))


def p2p_brute(g, pts, verts, line_off, R: float):
    """Returns (id int32, d float64, d_best float64, d_second float64) per point."""
    pts, verts, line_off = _f64(pts), _f64(verts), _i64(line_off)
    n = len(pts)
    oid, od, d1, d2 = np.empty(n, np.int32), np.empty(n), np.empty(n), np.empty(n)
    _check(_load().or_p2p_brute(C.byref(_grid(g)), _ptr(pts), n, _ptr(verts), _ptr(line_off),
                                len(line_off) - 1, float(R), _ptr(oid), _ptr(od), _ptr(d1), _ptr(d2)))
    return oid, od, d1, d2


def p2p_grid(g, pts, verts, line_off, R: float, cand_start, cand_ids):
    """Returns (id int32, d float64, d_best float64, d_second float64) per point."""
    pts, verts, line_off = _f64(pts), _f64(verts), _i64(line_off)
    cand_start = _i64(cand_start)
    cand_ids = np.ascontiguousarray(cand_ids, np.int32)
    n = len(pts)
    oid, od, d1, d2 = np.empty(n, np.int32), np.empty(n), np.empty(n), np.empty(n)
    _check(_load().or_p2p_grid(C.byref(_grid(g)), _ptr(pts), n, _ptr(verts), _ptr(line_off), float(R),
                               _ptr(cand_start), _ptr(cand_ids), _ptr(oid), _ptr(od), _ptr(d1), _ptr(d2)))
    return oid, od, d1, d2


# ---------------------------------------------------------------- whole joins (filter + refine)

def pip_join(g, pts, verts, ring_off, poly_ring_off, with_hits: bool = False):
    mbb = pip_mbb(g, verts, ring_off, poly_ring_off)
    cs, ci = cand_csr(g, mbb)
    return pip_grid(g, pts, verts, ring_off, poly_ring_off, cs, ci, with_hits=with_hits)


def p2p_join(g, pts, verts, line_off, R: float):
    mbb = p2p_mbb(g, verts, line_off)
    cs, ci = cand_csr(g, mbb, R, expand=True)
    return p2p_grid(g, pts, verts, line_off, R, cs, ci)
