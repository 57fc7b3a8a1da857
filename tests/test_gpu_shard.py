"""MultiDeviceJoin on the devices of this machine (with one GPU, two
replicas on the same device joined from two host threads): results of a
request split across replicas equal the single join."""
import numpy as np
import pytest

from paper_1403_0802_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_multi_device_join_equals_single_join():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1403_0802_gb300 import api, build
    from paper_1403_0802_gb300.shard import MultiDeviceJoin
    build.build()
    devs = list(range(torch.cuda.device_count()))
    devs = devs if len(devs) > 1 else [0, 0]
    w = synth.p2p_walks(n_points=500_001, n_lines=20_000)
    L = w.polylines
    with api.p2p_layer(L.verts, L.line_off, w.D, w.grid) as layer:
        rid, rd = api.p2p_join(layer, w.points, form="fp64")
    with MultiDeviceJoin.p2p(L.verts, L.line_off, w.D, w.grid, devices=devs) as mj:
        ids, d = mj.join(w.points, form="fp64")
    np.testing.assert_array_equal(ids, rid.cpu().numpy())
    np.testing.assert_array_equal(d, rd.cpu().numpy())
    wp = synth.pip_stars(n_points=300_007)
    P = wp.polygons
    with api.pip_layer(P.verts, P.ring_off, P.poly_ring_off, wp.grid) as layer:
        ref = api.pip_join(layer, wp.points, form="fp32x").cpu().numpy()
    with MultiDeviceJoin.pip(P.verts, P.ring_off, P.poly_ring_off, wp.grid, devices=devs) as mj:
        np.testing.assert_array_equal(mj.join(wp.points, form="fp32x"), ref)
