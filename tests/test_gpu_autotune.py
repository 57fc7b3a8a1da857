"""The autotuner times every (grid, points per item, block, edges per chunk,
form) setting of a small workload through the library and returns the table
with its fastest row; every launch setting gives the same results."""
import numpy as np
import pytest

from paper_1403_0802_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mods():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1403_0802_gb300 import api, autotune, build
    build.build()
    return api, autotune


def test_autotuner_table(mods):
    api, autotune = mods
    w = synth.p2p_walks(n_points=100_000, n_lines=5_000)
    res = autotune.autotune(w, grids=(256, 512), ppis=(32, 128), forms=("fp32x", "fp64"), blocks=(2, 8),
                            edges=(0, 16), steps=2)
    table = res["table"]
    assert len(table) == 32
    assert {(r["grid"], r["pts_per_item"], r["form"], r["block"], r["edges_per_chunk"]) for r in table} == {
        (g, p, f, b, e) for g in (256, 512) for p in (32, 128) for f in ("fp32x", "fp64") for b in (2, 8)
        for e in (0, 16)}
    assert all(r["ms"] > 0 and r["points_per_s"] > 0 for r in table)
    assert res["best"]["ms"] == min(r["ms"] for r in table)
    w = synth.pip_stars(n_points=50_000, n_side=8)
    res = autotune.autotune(w, grids=(128,), ppis=(64,), steps=2)
    assert len(res["table"]) == 1 and res["best"]["form"] == "fp32x"


@pytest.mark.parametrize("form", ["fp64", "fp32x"])
def test_launch_knobs_do_not_change_results(mods, oracle, form):
    """Warps per block 2 / 4 / 8 and edge budgets that cut heavy cells into
    small items (PIP heavy-tail tiling, 1 M points; P2P walks, 1 M points):
    PIP ids equal the oracle's for every setting; P2P results pass the parity
    bar and their ids agree between settings wherever the oracle's answer is
    unique (FP64: bit for bit)."""
    api, _ = mods
    from parity import P2PRef
    w = synth.pip_tiles(n_points=1_000_003, layer=2)
    P = w.polygons
    ref = oracle.pip_join(w.grid, w.points, P.verts, P.ring_off, P.poly_ring_off)
    with api.pip_layer(P.verts, P.ring_off, P.poly_ring_off, w.grid) as layer:
        pts = torch.as_tensor(w.points, device="cuda")
        for block, epc, ppi in ((2, 0, 64), (8, 0, 128), (4, 16, 64), (8, 200, 128), (2, 1, 7)):
            layer.reset_stats()
            got = api.pip_join(layer, pts, form=form, block=block, edges_per_chunk=epc, pts_per_item=ppi)
            np.testing.assert_array_equal(got.cpu().numpy(), ref)
            if epc:
                assert layer.stats()["items"] > 0
    w = synth.p2p_walks(n_points=1_000_003, n_lines=30_000)
    L = w.polylines
    pref = P2PRef(oracle, w.grid, L.verts, L.line_off, w.D)
    r = pref.join(w.points)
    u = pref.unique(w.points, ref=r)
    first = None
    with api.p2p_layer(L.verts, L.line_off, w.D, w.grid) as layer:
        pts = torch.as_tensor(w.points, device="cuda")
        for block, epc, ppi in ((2, 0, 128), (8, 0, 128), (4, 8, 128), (8, 40, 64)):
            gid, gd = api.p2p_join(layer, pts, form=form, block=block, edges_per_chunk=epc, pts_per_item=ppi)
            gid, gd = gid.cpu().numpy(), gd.cpu().numpy()
            pref.check(w.points, gid, gd, form, ref=r)
            if first is None:
                first = (gid, gd)
            elif form == "fp64":
                np.testing.assert_array_equal(gid, first[0])
                np.testing.assert_array_equal(gd, first[1])
            else:
                np.testing.assert_array_equal(gid[u], first[0][u])
        with pytest.raises(Exception) as e:
            api.p2p_join(layer, pts[:10], form=form, block=3)
        assert "block" in str(e.value)
        with pytest.raises(Exception) as e:
            api.p2p_join(layer, pts[:10], form=form, edges_per_chunk=-1)
        assert "edges_per_chunk" in str(e.value)
