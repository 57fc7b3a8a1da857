"""The autotuner times every (grid, points per item, form) setting of a small
workload through the library and returns the table with its fastest row."""
import pytest

from paper_1403_0802_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_autotuner_table():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1403_0802_gb300 import autotune, build
    build.build()
    w = synth.p2p_walks(n_points=100_000, n_lines=5_000)
    res = autotune.autotune(w, grids=(256, 512), ppis=(32, 128), forms=("fp32x", "fp64"), steps=2)
    table = res["table"]
    assert len(table) == 8
    assert {(r["grid"], r["pts_per_item"], r["form"]) for r in table} == {
        (g, p, f) for g in (256, 512) for p in (32, 128) for f in ("fp32x", "fp64")}
    assert all(r["ms"] > 0 and r["points_per_s"] > 0 for r in table)
    assert res["best"]["ms"] == min(r["ms"] for r in table)
    w = synth.pip_stars(n_points=50_000, n_side=8)
    res = autotune.autotune(w, grids=(128,), ppis=(64,), steps=2)
    assert len(res["table"]) == 1 and res["best"]["form"] == "fp32x"
