"""Serving loop: continuous batching over streams with HBM-budget admission.

Each request's result is the same alone and in a concurrent mix; storm frames
equal the direct apply-flips + guard + render sequence; admission refusal,
cancellation and bounded waits are host-side outcomes (no device fault)."""
import numpy as np
import pytest

from paper_2606_21791_gb300 import synth as S

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def G():
    import torch
    import paper_2606_21791_gb300 as P
    P.build()
    from paper_2606_21791_gb300 import gs
    gs.load_library()
    torch.cuda.init()
    return gs


def _scenes(G):
    a = S.make_scene(5000, 0, S.FP32, 70)
    b = S.make_scene(20000, 3, S.FP16, 71, layout="clusters")
    ha = G.gs_load_scene(a.planes, a.n, 0, S.FP32)
    hb = G.gs_load_scene(b.planes, b.n, 3, S.FP16)
    return (a, ha), (b, hb)


def _requests(G, torch, ids, cams_b, flips_b):
    """A mixed list of render and campaign requests with their output buffers."""
    reqs = []
    for i, (sid, W, H, elev) in enumerate([(0, 256, 256, 0.0), (1, 320, 208, 20.0), (0, 200, 136, -15.0),
                                           (1, 256, 256, 35.0), (0, 256, 256, 60.0), (1, 160, 160, -40.0)]):
        cam = S.ring_cameras(1, W, H, elevation_deg=elev)[0]
        img = torch.full((H * W * 3,), -1.0, dtype=torch.float32, device="cuda")
        reqs.append(("render", G.make_request(G.GS_REQ_RENDER, ids[sid], cam, dev_rgb=img), img))
    for j in range(2):
        fl = flips_b[j * 48:(j + 1) * 48]
        d = G.to_device(fl)
        out = G.device_bytes(len(fl) * len(cams_b) * 24)
        reqs.append(("campaign", G.make_request(G.GS_REQ_CAMPAIGN, ids[1], dev_flips=d, nflips=len(fl),
                                                dev_results=out), (out, d)))
    return reqs


def _run(G, torch, server, reqs, together):
    tickets = []
    if together:
        order = np.random.default_rng(5).permutation(len(reqs))
        tickets = {int(i): G.gs_server_submit(server, reqs[i][1]) for i in order}
        for i in order:
            G.gs_server_wait(server, tickets[int(i)])
    else:
        for r in reqs:
            G.gs_server_wait(server, G.gs_server_submit(server, r[1]))
    torch.cuda.synchronize()
    res = []
    for kind, _, buf in reqs:
        if kind == "render":
            res.append(buf.cpu().numpy().copy())
        else:
            res.append(buf[0].cpu().numpy().copy())
    return res


def test_results_identical_alone_and_in_the_mix(G):
    import torch
    (a, ha), (b, hb) = _scenes(G)
    cams_b = S.ring_cameras(2, 192, 160)
    G.gs_set_views(hb, cams_b)
    flips_b = S.flips_stratified(96, b.n, b.nwords, S.FP16, 72)
    try:
        alone_srv = G.gs_server_create(40 << 30, 1)
        ids = [G.gs_server_add_scene(alone_srv, ha), G.gs_server_add_scene(alone_srv, hb)]
        reqs = _requests(G, torch, ids, cams_b, flips_b)
        alone = _run(G, torch, alone_srv, reqs, together=False)
        G.gs_server_destroy(alone_srv)

        mix_srv = G.gs_server_create(40 << 30, 4)
        ids = [G.gs_server_add_scene(mix_srv, ha), G.gs_server_add_scene(mix_srv, hb)]
        reqs = _requests(G, torch, ids, cams_b, flips_b)
        mixed = _run(G, torch, mix_srv, reqs, together=True)
        stats = G.gs_server_stats(mix_srv)
        G.gs_server_destroy(mix_srv)
        assert stats["completed"] == len(reqs)
        for x, y in zip(alone, mixed):
            assert np.array_equal(x.view(np.uint8), y.view(np.uint8))
        assert all((r >= 0).all() for r, (k, _, _) in zip(alone, reqs) if k == "render")
    finally:
        G.gs_free_scene(ha)
        G.gs_free_scene(hb)


def test_storm_frames_match_direct_calls(G):
    """An upset storm accumulates upsets in the resident model; each frame is
    flips, then the guard (Algorithm 1), then the render."""
    import torch
    sc = S.make_scene(30000, 3, S.FP32, 73, layout="clusters")
    h_srv = G.gs_load_scene(sc.planes, sc.n, 3, S.FP32)
    h_ref = G.gs_load_scene(sc.planes, sc.n, 3, S.FP32)
    cam = S.ring_cameras(1, 256, 192)[0]
    rng = np.random.default_rng(74)
    srv = G.gs_server_create(40 << 30, 3)
    try:
        sid = G.gs_server_add_scene(srv, h_srv)
        for frame in range(5):
            fl = S.flips_at(rng.integers(0, sc.n, size=200), 0, 0)
            fl["word"] = rng.integers(0, 59, size=200)
            fl["bit"] = rng.integers(0, 32, size=200)
            d = G.to_device(fl)
            img = torch.empty(256 * 192 * 3, dtype=torch.float32, device="cuda")
            cl = torch.zeros(1, dtype=torch.int64, device="cuda")
            t = G.gs_server_submit(srv, G.make_request(G.GS_REQ_STORM, sid, cam, guard_mode=0,
                                                       word_mask=S.GUARD_WORDS_DEFAULT, dev_flips=d, nflips=200,
                                                       dev_rgb=img, dev_clamps=cl))
            G.gs_server_wait(srv, t)
            # direct calls on the reference copy
            G.gs_apply_flips(h_ref, d, 200)
            cl_ref = torch.zeros(1, dtype=torch.int64, device="cuda")
            G.gs_guard(h_ref, 0, S.GUARD_WORDS_DEFAULT, cl_ref)
            ref = torch.empty_like(img)
            G.gs_render(h_ref, cam, ref)
            torch.cuda.synchronize()
            assert int(cl.item()) == int(cl_ref.item())
            assert torch.equal(img, ref)
            assert not torch.isnan(img).any()    # the guard removed every non-finite value
    finally:
        G.gs_server_destroy(srv)
        G.gs_free_scene(h_srv)
        G.gs_free_scene(h_ref)


def test_admission_refusal_cancel_and_timeout(G):
    import torch
    sc = S.make_scene(200000, 3, S.FP32, 75, layout="clusters")
    h = G.gs_load_scene(sc.planes, sc.n, 3, S.FP32)
    try:
        tiny = G.gs_server_create(1 << 20, 1)            # 1 MiB: the scene itself does not fit
        with pytest.raises(G.GsError) as e:
            G.gs_server_add_scene(tiny, h)
        assert e.value.status == G.GS_ERR_BUSY
        G.gs_server_destroy(tiny)

        resident = sc.n * sc.nwords * 4
        small = G.gs_server_create(resident + (4 << 20), 1)   # scene fits, a render's scratch does not
        sid = G.gs_server_add_scene(small, h)
        cam = S.ring_cameras(1, 640, 480)[0]
        img = torch.empty(640 * 480 * 3, dtype=torch.float32, device="cuda")
        with pytest.raises(G.GsError) as e:
            G.gs_server_submit(small, G.make_request(G.GS_REQ_RENDER, sid, cam, dev_rgb=img))
        assert e.value.status == G.GS_ERR_BUSY
        G.gs_server_destroy(small)

        srv = G.gs_server_create(40 << 30, 1)
        sid = G.gs_server_add_scene(srv, h)
        tickets = [G.gs_server_submit(srv, G.make_request(G.GS_REQ_RENDER, sid, cam, dev_rgb=img)) for _ in range(6)]
        # the last one is still queued behind five renders on the single slot: cancel it
        G.gs_server_cancel(srv, tickets[-1])
        with pytest.raises(G.GsError) as e:
            G.gs_server_wait(srv, tickets[-1])
        assert e.value.status == G.GS_ERR_STATE
        for t in tickets[:-1]:
            r = G.gs_server_wait(srv, t)
            assert r["status"] == 0 and r["t_done_ms"] >= r["t_start_ms"] >= r["t_submit_ms"]
        # bounded wait on a request that cannot have finished yet returns GS_ERR_TIMEOUT
        big = [G.gs_server_submit(srv, G.make_request(G.GS_REQ_RENDER, sid, cam, dev_rgb=img)) for _ in range(8)]
        with pytest.raises(G.GsError) as e:
            G.gs_server_wait(srv, big[-1], timeout_ms=0)
        assert e.value.status == G.GS_ERR_TIMEOUT
        for t in big:
            G.gs_server_wait(srv, t)
        G.gs_server_destroy(srv)
    finally:
        G.gs_free_scene(h)
