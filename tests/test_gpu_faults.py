"""Failure paths, injected on the host (sj_fault_inject): device allocations
that fail as out of memory at layer build, join, host-buffer join and engine
round; each call reports SJ_ERR_OOM, leaves its outputs untouched, and the
library keeps working (the next call is correct).  No GPU fault is caused:
the failing call is a fake of cudaMalloc's out-of-memory return.  Also the
bounds-checked build, run on small in-range cases against the oracle."""
import os
import subprocess
import sys

import numpy as np
import pytest

from paper_1403_0802_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1403_0802_gb300 import _lib, api, build
    build.build()
    yield api, _lib
    _lib.lib().sj_fault_inject(_lib.SJ_FAULT_NONE, 0, 0)


def arm(L, after, count=1):
    assert L.lib().sj_fault_inject(L.SJ_FAULT_ALLOC, after, count) == L.SJ_OK


def test_layer_build_out_of_memory(lib, oracle):
    api, L = lib
    w = synth.pip_stars(n_points=20_000, n_side=8)
    P = w.polygons
    ref = oracle.pip_join(w.grid, w.points, P.verts, P.ring_off, P.poly_ring_off)
    for after in (0, 3, 11, 25):                   # the allocation that fails: early, middle, late
        arm(L, after)
        with pytest.raises(L.SJError) as e:
            api.pip_layer(P.verts, P.ring_off, P.poly_ring_off, w.grid)
        assert e.value.status == L.SJ_ERR_OOM, after
        assert L.lib().sj_fault_pending() == 0
    with api.pip_layer(P.verts, P.ring_off, P.poly_ring_off, w.grid) as layer:
        np.testing.assert_array_equal(api.pip_join(layer, w.points, form="fp32x").cpu().numpy(), ref)
    wl = synth.p2p_walks(n_points=1000, n_lines=2000)
    for after in (0, 7, 20):
        arm(L, after)
        with pytest.raises(L.SJError) as e:
            api.p2p_layer(wl.polylines.verts, wl.polylines.line_off, wl.D, wl.grid)
        assert e.value.status == L.SJ_ERR_OOM


def test_join_out_of_memory_leaves_outputs(lib, oracle):
    api, L = lib
    w = synth.p2p_walks(n_points=50_000, n_lines=5_000)
    Lw = w.polylines
    rid, rd, _, _ = oracle.p2p_join(w.grid, w.points, Lw.verts, Lw.line_off, w.D)
    with api.p2p_layer(Lw.verts, Lw.line_off, w.D, w.grid) as layer:
        pts = torch.as_tensor(w.points, device="cuda")
        oid = torch.full((len(pts),), 7, dtype=torch.int32, device="cuda")
        od = torch.full((len(pts),), -3.0, dtype=torch.float64, device="cuda")
        for form in ("fp64", "fp32x"):
            arm(L, 0)
            with pytest.raises(L.SJError) as e:
                api.p2p_join(layer, pts, oid, od, form=form)
            assert e.value.status == L.SJ_ERR_OOM
            torch.cuda.synchronize()
            assert bool((oid == 7).all()) and bool((od == -3.0).all())
        arm(L, 0)                                  # host-buffer join: its device buffer
        hid = np.full(len(pts), 7, np.int32)
        with pytest.raises(L.SJError) as e:
            api.p2p_join_host(layer, w.points, hid, form="fp64")
        assert e.value.status == L.SJ_ERR_OOM and (hid == 7).all()
        gid, gd = api.p2p_join(layer, pts, oid, od, form="fp64")
        np.testing.assert_array_equal(gid.cpu().numpy(), rid)
        ok = rid >= 0
        assert np.all(np.abs(gd.cpu().numpy()[ok] - rd[ok]) <= 1e-12 * np.maximum(rd[ok], 1.0))


def test_engine_round_out_of_memory(lib):
    api, L = lib
    w = synth.pip_stars(n_points=30_000, n_side=8)
    P = w.polygons
    with api.pip_layer(P.verts, P.ring_off, P.poly_ring_off, w.grid) as layer:
        pts = torch.as_tensor(w.points, device="cuda")
        want = api.pip_join(layer, pts, form="fp32x")
        out = torch.full((len(pts),), 7, dtype=torch.int32, device="cuda")
        stream = torch.cuda.Stream()
        with api.Engine(max_points=100_000, max_requests=4, form="fp32x") as eng:
            arm(L, 0)                              # the layer's workspace, built on its first round
            with pytest.raises(L.SJError) as e:
                eng.round([(layer, pts, out, None)], stream)
            assert e.value.status == L.SJ_ERR_OOM
            stream.synchronize()
            assert bool((out == 7).all())
            eng.round([(layer, pts, out, None)], stream)
            stream.synchronize()
            assert torch.equal(out, want)


def test_bounds_checked_build_on_in_range_cases():
    """The bounds-checked build (-DSJ_CHECK_BOUNDS) in a process of its own:
    PIP and P2P joins in both forms, a host-buffer join, an engine round and
    the no-alloc join against the oracle, every guard silent."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    code = f"""
import sys
sys.path.insert(0, {ROOT!r}); sys.path.insert(0, {os.path.join(ROOT, 'tests')!r})
import numpy as np, torch
from paper_1403_0802_gb300 import _lib, build
_lib.use(build.build(checked=True))
from paper_1403_0802_gb300 import api, synth
from oracle import oracle as O
from parity import P2PRef
O.build()
assert _lib.lib().sj_bounds_checked() == 1
w = synth.pip_tiles(n_points=300_001, layer=2, grid_n=256)
P = w.polygons
ref = O.pip_join(w.grid, w.points, P.verts, P.ring_off, P.poly_ring_off)
with api.pip_layer(P.verts, P.ring_off, P.poly_ring_off, w.grid) as layer:
    for form in ("fp64", "fp32x"):
        for kw in ({{}}, {{"pts_per_item": 7, "edges_per_chunk": 4, "block": 2}}):
            np.testing.assert_array_equal(api.pip_join(layer, w.points, form=form, **kw).cpu().numpy(), ref)
    np.testing.assert_array_equal(api.pip_join_host(layer, w.points, form="fp32x"), ref)
    pts = torch.as_tensor(w.points, device="cuda")
    out = torch.empty(len(pts), dtype=torch.int32, device="cuda")
    with api.Engine(max_points=400_000, max_requests=4, form="fp32x") as eng:
        s = torch.cuda.Stream()
        eng.round([(layer, pts, out, None)], s)
        s.synchronize()
    np.testing.assert_array_equal(out.cpu().numpy(), ref)
w = synth.p2p_walks(n_points=200_003, n_lines=10_000)
L = w.polylines
r = P2PRef(O, w.grid, L.verts, L.line_off, w.D)
rr = r.join(w.points)
with api.p2p_layer(L.verts, L.line_off, w.D, w.grid) as layer:
    pts = torch.as_tensor(w.points, device="cuda")
    for form in ("fp64", "fp32x"):
        gid, gd = api.p2p_join(layer, pts, form=form)
        r.check(w.points, gid.cpu().numpy(), gd.cpu().numpy(), form, ref=rr)
        oid = torch.empty(len(pts), dtype=torch.int32, device="cuda")
        od = torch.empty(len(pts), dtype=torch.float64, device="cuda")
        api.p2p_join_noalloc(layer, pts, oid, od, form=form)
        torch.cuda.synchronize()
        r.check(w.points, oid.cpu().numpy(), od.cpu().numpy(), form, ref=rr)
print("checked ok")
"""
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=900)
    assert r.returncode == 0 and "checked ok" in r.stdout, r.stdout[-2000:] + r.stderr[-4000:]
