"""The continuous-batching serving loop: requests that arrive while others are
on the GPU are admitted as memory frees up and joined in shared rounds, and
each request's result is the same in the mix as alone.  PIP ids are checked
bit for bit against the join alone; every P2P request is checked against the
oracle at its window (ids exact except oracle near-ties within 1e-9 relative
or distances within 1e-9 of the window; distances within the form's bound),
and its ids equal those of the join alone wherever the oracle's answer is
unique (FP64: ids and distances equal bit for bit)."""
import numpy as np
import pytest

from paper_1403_0802_gb300 import synth
from parity import P2PRef, PIPRef

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def server(oracle):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1403_0802_gb300 import api, build, serve
    build.build()
    wp = synth.pip_tiles(n_points=300_000, layer=1)
    wl = synth.p2p_walks_lognormal(n_points=300_000, n_lines=20_000)
    pip = api.pip_layer(wp.polygons.verts, wp.polygons.ring_off, wp.polygons.poly_ring_off, wp.grid)
    p2p = api.p2p_layer(wl.polylines.verts, wl.polylines.line_off, wl.D, wl.grid)
    pool_p = torch.from_numpy(wp.points).pin_memory()
    pool_l = torch.from_numpy(wl.points).pin_memory()
    srv = serve.Server(pip, p2p, form="fp32x", round_points=400_000, max_requests=256,
                       hbm_budget=40_000_000)
    srv.ref = P2PRef(oracle, wl.grid, wl.polylines.verts, wl.polylines.line_off, wl.D)
    srv.pref = PIPRef(oracle, wp.grid, wp.polygons.verts, wp.polygons.ring_off, wp.polygons.poly_ring_off)
    yield api, serve, srv, pool_p, pool_l
    srv.close()
    pip.close()
    p2p.close()


def check_p2p_request(api, srv, r, form):
    """A served P2P request against the oracle at its window, and against the
    same join alone (FP64: bit for bit; FP32X: equal ids wherever the oracle's
    answer is unique -- a point's FP32 certificate can depend on the other
    points of its work item, and an uncertified point is redone in FP64)."""
    pts = r.pts.numpy()
    a_id, a_d = r.out_id.numpy(), r.out_d.numpy()
    ref = srv.ref.join(pts, r.window)
    srv.ref.check(pts, a_id, a_d, form, window=r.window, ref=ref)
    rid, rd = api.p2p_join(srv.layers[r.kind], r.pts.cuda(), form=form, window=r.window)
    b_id, b_d = rid.cpu().numpy(), rd.cpu().numpy()
    if form == "fp64":
        np.testing.assert_array_equal(a_id, b_id)
        np.testing.assert_array_equal(a_d, b_d)
    else:
        u = srv.ref.unique(pts, r.window, ref=ref)
        np.testing.assert_array_equal(a_id[u], b_id[u])


@pytest.mark.parametrize("mode,form", [("batched", None), ("per_request", None), ("per_request", "fp64")])
def test_mix_equals_alone(server, mode, form):
    api, serve, srv, pool_p, pool_l = server
    # arrivals every ~5 us on average: requests arrive while others are on the GPU
    reqs = serve.make_stream(80, rate_per_s=200_000.0, pool_pip=pool_p, pool_p2p=pool_l, size_min=100,
                             size_max=60_000, seed=5)
    stats = srv.run(reqs, mode=mode, form=form)
    assert stats["requests"] == 80 and stats["p99_ms"] >= stats["p50_ms"] > 0
    if mode == "batched":
        assert stats["rounds"] < 80            # requests really shared rounds
    form = form or srv.form
    for r in reqs:
        layer = srv.layers[r.kind]
        pts = r.pts.cuda()
        if r.kind == serve.PIP:
            ref = api.pip_join(layer, pts, form=form).cpu()
            assert torch.equal(r.out_id, ref), r.rid
            np.testing.assert_array_equal(r.out_id.numpy(), srv.pref.join(r.pts.numpy()))
        else:
            check_p2p_request(api, srv, r, form)


@pytest.mark.parametrize("mode", ["batched", "per_request"])
def test_per_request_windows(server, mode):
    """P2P requests with their own windows (below the layer's D) share rounds
    with unwindowed ones; each equals sj_p2p_join_window at its window."""
    api, serve, srv, pool_p, pool_l = server
    reqs = serve.make_stream(60, rate_per_s=200_000.0, pool_pip=pool_p, pool_p2p=pool_l, size_min=100,
                             size_max=60_000, seed=9, pip_frac=0.3, p2p_windows=(0.0, 10.0, 40.0, 100.0))
    assert len({r.window for r in reqs if r.kind == serve.P2P}) > 2
    srv.run(reqs, mode=mode)
    for r in reqs:
        layer = srv.layers[r.kind]
        pts = r.pts.cuda()
        if r.kind == serve.PIP:
            assert torch.equal(r.out_id, api.pip_join(layer, pts, form=srv.form).cpu()), r.rid
            continue
        check_p2p_request(api, srv, r, srv.form)
        assert np.all(r.out_d.numpy()[r.out_id.numpy() >= 0] <= r.window)


def test_arrivals_are_not_admitted_early(server):
    """A request submitted with a future arrival time is not served before it
    (its latency is measured from that arrival)."""
    api, serve, srv, pool_p, pool_l = server
    import ctypes as C
    from paper_1403_0802_gb300 import _lib as L
    lib = L.lib()
    pts = pool_p[:1000].contiguous()
    out = torch.empty(1000, dtype=torch.int32, pin_memory=True)
    req = L.sj_serve_request(L.SJ_SERVE_PIP, 0, pts.data_ptr(), 1000, out.data_ptr(), None, 0.0)
    t_arr = lib.sj_server_now(srv.handle) + 0.05
    req.not_before = t_arr
    tk, lat = C.c_int64(), C.c_double()
    L.check(lib.sj_server_submit(srv.handle, C.byref(req), C.byref(tk)), "submit")
    L.check(lib.sj_server_wait(srv.handle, tk.value, C.byref(lat)), "wait")
    assert lib.sj_server_now(srv.handle) >= t_arr
    assert 0.0 < lat.value < 0.05
    ref = api.pip_join(srv.layers[serve.PIP], pts.cuda(), form=srv.form).cpu()
    assert torch.equal(out, ref)


def test_admission_waits_for_device_memory(server):
    """A budget that holds only a couple of requests at a time: requests queue
    until earlier ones release their arena blocks, every one completes, and the
    results equal the joins alone."""
    api, serve, srv, pool_p, pool_l = server
    tight = serve.Server(srv.layers[serve.PIP], srv.layers[serve.P2P], form=srv.form, round_points=400_000,
                         max_requests=64, hbm_budget=3_000_000)
    try:
        reqs = serve.make_stream(40, rate_per_s=0.0, pool_pip=pool_p, pool_p2p=pool_l, size_min=20_000,
                                 size_max=60_000, seed=9)
        stats = tight.run(reqs, mode="batched")
        assert stats["requests"] == 40
        assert tight.stats()["completed"] == 40
        for r in reqs:
            pts = r.pts.cuda()
            if r.kind == serve.PIP:
                ref = api.pip_join(srv.layers[serve.PIP], pts, form=srv.form).cpu()
                assert torch.equal(r.out_id, ref), r.rid
            else:
                check_p2p_request(api, srv, r, srv.form)
    finally:
        tight.close()


def test_admission_refusal_cancellation_and_deadline(server):
    """Injected admission refusal (the server keeps serving), a request
    cancelled before it is admitted (its wait reports SJ_ERR_CANCELLED and its
    outputs stay untouched), and a wait with a deadline that gives up
    (SJ_ERR_TIMEOUT) on a request still ahead, then completes it."""
    api, serve, srv, pool_p, pool_l = server
    import ctypes as C
    from paper_1403_0802_gb300 import _lib as L
    lib = L.lib()
    pts = pool_p[:2000].contiguous()
    outs = [torch.full((2000,), 7, dtype=torch.int32, pin_memory=True) for _ in range(4)]
    tk, lat = C.c_int64(), C.c_double()

    def req(k, delay):
        r = L.sj_serve_request(L.SJ_SERVE_PIP, 0, pts.data_ptr(), 2000, outs[k].data_ptr(), None, 0.0)
        r.not_before = lib.sj_server_now(srv.handle) + delay
        return r

    want = api.pip_join(srv.layers[serve.PIP], pts.cuda(), form=srv.form).cpu()
    assert lib.sj_fault_inject(L.SJ_FAULT_ADMIT, 1, 1) == L.SJ_OK
    r0 = req(0, 0.0)
    L.check(lib.sj_server_submit(srv.handle, C.byref(r0), C.byref(tk)), "submit")
    t0 = tk.value
    r1 = req(1, 0.0)
    assert lib.sj_server_submit(srv.handle, C.byref(r1), C.byref(tk)) == L.SJ_ERR_BUSY
    L.check(lib.sj_server_wait(srv.handle, t0, C.byref(lat)), "wait")
    assert torch.equal(outs[0], want) and bool((outs[1] == 7).all())
    # cancelled before admission (arrives in 0.5 s)
    r2 = req(2, 0.5)
    L.check(lib.sj_server_submit(srv.handle, C.byref(r2), C.byref(tk)), "submit")
    t2 = tk.value
    assert lib.sj_server_cancel(srv.handle, t2) == L.SJ_OK
    assert lib.sj_server_wait(srv.handle, t2, C.byref(lat)) == L.SJ_ERR_CANCELLED
    assert bool((outs[2] == 7).all())
    # a deadline that runs out, then the request completes
    r3 = req(3, 0.3)
    L.check(lib.sj_server_submit(srv.handle, C.byref(r3), C.byref(tk)), "submit")
    t3 = tk.value
    assert lib.sj_server_wait_for(srv.handle, t3, 0.01, C.byref(lat)) == L.SJ_ERR_TIMEOUT
    assert lib.sj_server_cancel(srv.handle, 10 ** 9) == L.SJ_ERR_INVALID
    L.check(lib.sj_server_wait_for(srv.handle, t3, 10.0, C.byref(lat)), "wait_for")
    assert torch.equal(outs[3], want)
    assert lib.sj_server_cancel(srv.handle, t3) == L.SJ_ERR_INVALID     # already waited for


def test_serving_on_the_full_layers(oracle):
    """The serving workload's layers (40,000 tiles; 150,000 lognormal walks,
    D = 100 m), requests of 100 k - 3 M points arriving while others run,
    batched rounds of up to 6 M points: every request checked against the
    oracle on a seeded 20,000-point sample of its points (PIP ids bit for bit;
    P2P with the parity bar)."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1403_0802_gb300 import api, build, serve
    build.build()
    wp = synth.pip_tiles(n_points=8_000_000, layer=1, grid_n=1024)
    wl = synth.p2p_walks_lognormal(n_points=8_000_000, n_lines=150_000, D=100.0, grid_n=512)
    P, L = wp.polygons, wl.polylines
    pref = PIPRef(oracle, wp.grid, P.verts, P.ring_off, P.poly_ring_off)
    lref = P2PRef(oracle, wl.grid, L.verts, L.line_off, wl.D)
    pool_p = torch.from_numpy(wp.points).pin_memory()
    pool_l = torch.from_numpy(wl.points).pin_memory()
    with api.pip_layer(P.verts, P.ring_off, P.poly_ring_off, wp.grid) as pip, \
            api.p2p_layer(L.verts, L.line_off, wl.D, wl.grid) as p2p:
        srv = serve.Server(pip, p2p, form="fp32x", round_points=6_000_000, max_requests=256)
        try:
            reqs = serve.make_stream(24, rate_per_s=40.0, pool_pip=pool_p, pool_p2p=pool_l, size_min=100_000,
                                     size_max=3_000_000, seed=11)
            stats = srv.run(reqs, mode="batched")
        finally:
            srv.close()
    assert stats["requests"] == 24
    rng = np.random.default_rng(12)
    for r in reqs:
        idx = np.sort(rng.choice(r.n, min(r.n, 20_000), replace=False))
        pts = np.ascontiguousarray(r.pts.numpy()[idx])
        if r.kind == serve.PIP:
            np.testing.assert_array_equal(r.out_id.numpy()[idx], pref.join(pts))
        else:
            lref.check(pts, r.out_id.numpy()[idx], r.out_d.numpy()[idx], "fp32x")
