"""sj_p2p_join_noalloc: the P2P join for callers that cannot allocate device
memory (it takes its scratch from a fixed array inside libsj.so).  It must
give what sj_p2p_join gives, call after call, even though every call reuses
the scratch the previous call left behind.  This file sorts last so that a
run stopping at its first failure has already run every other test."""
import numpy as np
import pytest

from paper_1403_0802_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1403_0802_gb300 import api, build
    build.build()
    return api


@pytest.fixture(scope="module")
def walks():
    return synth.p2p_walks(n_points=300_001, n_lines=20_000)


def same_result(a_id, a_d, b_id, b_d):
    """The tolerance of the P2P parity tests: equal ids, distances within
    1e-12 * max(d, 1 m), +inf where there is no polyline within D."""
    a_id, a_d, b_id, b_d = (t.cpu().numpy() for t in (a_id, a_d, b_id, b_d))
    np.testing.assert_array_equal(a_id, b_id)
    hit = b_id >= 0
    assert np.all(np.isinf(a_d[~hit])) and np.all(np.isinf(b_d[~hit]))
    assert np.all(np.abs(a_d[hit] - b_d[hit]) <= 1e-12 * np.maximum(b_d[hit], 1.0))


@pytest.mark.parametrize("form", ["fp64", "fp32x"])
def test_noalloc_matches_allocating_join_twice_in_a_row(lib, walks, form):
    api = lib
    L = walks.polylines
    with api.p2p_layer(L.verts, L.line_off, walks.D, walks.grid) as layer:
        pts = torch.as_tensor(walks.points, device="cuda")
        batches = [pts, pts[170_000:].contiguous()]         # second call: another batch, leftover scratch
        for p in batches:
            # same work items as the no-alloc join (64 points per item): the
            # FP32X certification of a point depends on the other points of its item
            ref_id, ref_d = api.p2p_join(layer, p, form=form, pts_per_item=64)
            out_id = torch.full((p.shape[0],), 7, dtype=torch.int32, device="cuda")
            out_d = torch.full((p.shape[0],), -1.0, dtype=torch.float64, device="cuda")
            api.p2p_join_noalloc(layer, p, out_id, out_d, form=form)
            torch.cuda.synchronize()
            same_result(out_id, out_d, ref_id, ref_d)
            assert (ref_id >= 0).float().mean().item() > 0.3


def test_noalloc_rejects_sizes_beyond_its_scratch(lib, walks):
    from paper_1403_0802_gb300._lib import SJError, SJ_ERR_INVALID
    api = lib
    L = walks.polylines
    with api.p2p_layer(L.verts, L.line_off, walks.D, walks.grid) as layer:
        too_many = torch.zeros((524_289, 2), dtype=torch.float64, device="cuda")
        out_id = torch.empty(524_289, dtype=torch.int32, device="cuda")
        with pytest.raises(SJError) as e:
            api.p2p_join_noalloc(layer, too_many, out_id, None)
        assert e.value.status == SJ_ERR_INVALID and "524288" in str(e.value)
    big_grid = synth.grid(2048)                             # 4,194,304 cells > 1,048,576
    with api.p2p_layer(L.verts, L.line_off, walks.D, big_grid) as layer:
        p = torch.as_tensor(walks.points[:10], device="cuda")
        with pytest.raises(SJError) as e:
            api.p2p_join_noalloc(layer, p, torch.empty(10, dtype=torch.int32, device="cuda"), None)
        assert e.value.status == SJ_ERR_INVALID and "cells" in str(e.value)
    # SJ_FP32X needs grid coordinates below 1e30 (its cell-relative FP32
    # coordinates and rounding bounds assume them): refused as by sj_p2p_join
    huge = dict(x0=0.0, y0=0.0, x1=4e30, y1=4e30, nx=4, ny=4)
    hv = np.array([[1e30, 1e30]], np.float64)              # a one-vertex polyline: a point
    with api.p2p_layer(hv, np.array([0, 1], np.int64), 100.0, huge) as layer:
        p = torch.tensor([[1e30, 1e30]], dtype=torch.float64, device="cuda")
        oid = torch.empty(1, dtype=torch.int32, device="cuda")
        od = torch.empty(1, dtype=torch.float64, device="cuda")
        for join in (lambda: api.p2p_join_noalloc(layer, p, oid, od, form="fp32x"),
                     lambda: api.p2p_join(layer, p, oid, od, form="fp32x")):
            with pytest.raises(SJError) as e:
                join()
            assert e.value.status == SJ_ERR_INVALID and "1e30" in str(e.value)
        api.p2p_join_noalloc(layer, p, oid, od, form="fp64")
        torch.cuda.synchronize()
        assert int(oid[0]) == 0 and float(od[0]) == 0.0
