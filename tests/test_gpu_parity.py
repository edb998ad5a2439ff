"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Bit-exact: flipped words, guard outputs and clamp counts, field boxes, tile
lists from the same (depth, rect) input, footprint counts from the same images.
Floating point: pixels within 2e-3 absolute on >= 99.9% of pixels, PSNR within
0.05 dB."""
import math

import numpy as np
import pytest

import footprint_attribution as FA
import oracle as O
from paper_2606_21791_gb300 import synth as S

pytestmark = pytest.mark.gpu

PIX_TOL = 2e-3
PIX_FRAC = 0.999
PSNR_TOL = 0.05


@pytest.fixture(scope="module")
def G():
    import torch
    import paper_2606_21791_gb300 as P
    P.build()
    from paper_2606_21791_gb300 import gs
    gs.load_library()
    torch.cuda.init()
    return gs


def _torch():
    import torch
    return torch


def _load(G, scene):
    return G.gs_load_scene(scene.planes, scene.n, scene.sh_degree, scene.fmt)


def _read(G, h, scene):
    out = np.empty_like(scene.planes)
    G.gs_read_planes(h, out)
    return out


def _render_gpu(G, h, cams):
    torch = _torch()
    cams = np.atleast_1d(cams)
    tot = sum(int(c["width"]) * int(c["height"]) * 3 for c in cams)
    buf = torch.empty(tot, dtype=torch.float32, device="cuda")
    G.gs_render(h, cams, buf)
    torch.cuda.synchronize()
    out, off = [], 0
    for c in cams:
        H, W = int(c["height"]), int(c["width"])
        out.append(buf[off:off + H * W * 3].cpu().numpy().reshape(H, W, 3))
        off += H * W * 3
    return out


def _pix_agree(a, b):
    both_nan = np.isnan(a) & np.isnan(b)
    d = np.abs(a.astype(np.float64) - b.astype(np.float64))
    ok = (d <= PIX_TOL) | both_nan
    return ok.all(axis=-1).mean()


def _psnr(sse, npx):
    return O.psnr(float(sse), npx)


# ---------------------------------------------------------------------------
# (a) injection, (f) guard: bit exact
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("fmt", [S.FP32, S.FP16, S.BF16])
def test_apply_flips_bit_exact(G, fmt):
    torch = _torch()
    sc = S.make_scene(3001, 3, fmt, 50, layout="clusters")
    flips = S.flips_stratified(4000, sc.n, sc.nwords, fmt, 51)
    flips = np.concatenate([flips, flips[:17]])        # duplicates cancel
    h = _load(G, sc)
    try:
        d = G.to_device(flips)
        G.gs_apply_flips(h, d, len(flips))
        torch.cuda.synchronize()
        assert np.array_equal(_read(G, h, sc), O.apply_flips(sc.planes, fmt, flips))
        assert G.gs_scene_errors(h) == 0
        bad = S.flips_at(np.array([sc.n]), 0, 0)       # out-of-range site: skipped and flagged
        G.gs_apply_flips(h, G.to_device(bad), 1)
        torch.cuda.synchronize()
        assert G.gs_scene_errors(h) == 1
    finally:
        G.gs_free_scene(h)


@pytest.mark.parametrize("fmt", [S.FP32, S.FP16, S.BF16])
def test_field_box_bit_exact(G, fmt):
    sc = S.make_scene(20011, 3, fmt, 52, layout="clusters")
    v = sc.planes.copy()
    v[5, 7] = S.encode(np.array([np.nan], np.float32), fmt)[0]   # NaN words are ignored
    sc = S.Scene(v, fmt, 3)
    h = _load(G, sc)
    try:
        lo, hi = G.gs_field_box(h, sc.nwords)
        olo, ohi = O.field_box(sc.planes, fmt)
        assert np.array_equal(lo, olo) and np.array_equal(hi, ohi)
    finally:
        G.gs_free_scene(h)


@pytest.mark.parametrize("fmt", [S.FP32, S.FP16, S.BF16])
@pytest.mark.parametrize("mode", [0, 1])
@pytest.mark.parametrize("mask", [S.GUARD_WORDS_DEFAULT, S.GUARD_WORDS_SELECTIVE, (1 << 59) - 1])
def test_guard_bit_exact(G, fmt, mode, mask):
    torch = _torch()
    n = 40_003   # ragged against every vector width
    clean = S.make_scene(n, 3, fmt, 53, layout="clusters")
    nbox = 59 if mask == (1 << 59) - 1 else 14
    if mode == 0:
        lo, hi = O.field_box(clean.planes, fmt)
    else:
        lo, hi = S.prim_boxes(clean, nbox, 54)
    rng = np.random.default_rng(55)
    fl = S.flips_at(rng.integers(0, n, size=5000), 0, 0)
    fl["word"] = rng.integers(0, 59, size=5000)
    fl["bit"] = rng.integers(0, S.FORMAT_BITS[fmt], size=5000)
    bad_planes = O.apply_flips(clean.planes, fmt, fl)
    ref, nref = O.guard(bad_planes, fmt, mask, mode, lo, hi)
    # the GPU scene's FIELD box is computed from what it loads: load clean, then flip
    h = _load(G, clean)
    try:
        if mode == 1:
            G.gs_set_prim_box(h, lo, hi, nbox)
        G.gs_apply_flips(h, G.to_device(fl), len(fl))
        cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
        G.gs_guard(h, mode, mask, cnt)
        torch.cuda.synchronize()
        assert int(cnt.item()) == nref and nref > 0
        assert np.array_equal(_read(G, h, clean), ref)
        # guarding again finds nothing (Theorem 1(i) on the guarded model)
        cnt.zero_()
        G.gs_guard(h, mode, mask, cnt)
        torch.cuda.synchronize()
        assert int(cnt.item()) == 0
    finally:
        G.gs_free_scene(h)


@pytest.mark.parametrize("fmt", [S.FP32, S.FP16, S.BF16])
@pytest.mark.parametrize("mode", [0, 1])
def test_guard_bitmap(G, fmt, mode):
    """The guard's optional bitmap of clamped words is exactly the set of words
    the oracle's guard changes (a clamp always changes the word: the endpoint
    differs from an out-of-box or NaN value), with zero rows for the unguarded
    words and zero bits past n; its popcount is the clamp count, and the
    guarded model is the oracle's."""
    torch = _torch()
    n = 20_011   # not a multiple of 32
    clean = S.make_scene(n, 3, fmt, 63, layout="clusters")
    mask = S.GUARD_WORDS_DEFAULT
    if mode == 0:
        lo, hi = O.field_box(clean.planes, fmt)
    else:
        lo, hi = S.prim_boxes(clean, 14, 64)
    rng = np.random.default_rng(65)
    fl = S.flips_at(rng.integers(0, n, size=3000), 0, 0)
    fl["word"] = rng.integers(0, 59, size=3000)
    fl["bit"] = rng.integers(0, S.FORMAT_BITS[fmt], size=3000)
    bad = O.apply_flips(clean.planes, fmt, fl)
    ref, nref = O.guard(bad, fmt, mask, mode, lo, hi)
    words32 = -(-n // 32)
    changed = np.zeros((clean.nwords, words32 * 32), dtype=bool)
    changed[:, :n] = ref != bad
    expect = np.packbits(changed, axis=1, bitorder="little").view("<u4")
    h = _load(G, clean)
    try:
        if mode == 1:
            G.gs_set_prim_box(h, lo, hi, 14)
        G.gs_apply_flips(h, G.to_device(fl), len(fl))
        cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
        bm = torch.full((clean.nwords * words32,), -1, dtype=torch.int32, device="cuda")   # overwritten whole
        G.gs_guard_bitmap(h, mode, mask, bm, cnt)
        torch.cuda.synchronize()
        got = bm.cpu().numpy().view(np.uint32).reshape(clean.nwords, words32)
        assert nref > 0 and int(cnt.item()) == nref
        assert np.array_equal(got, expect)
        assert int(np.unpackbits(got.view(np.uint8)).sum()) == nref
        assert np.array_equal(_read(G, h, clean), ref)
    finally:
        G.gs_free_scene(h)


# ---------------------------------------------------------------------------
# (b) preprocess
# ---------------------------------------------------------------------------
def _gpu_records(G, h, cam, n):
    torch = _torch()
    buf = G.device_bytes(n * G.RECORD_DTYPE.itemsize)
    G.gs_preprocess(h, cam, buf)
    torch.cuda.synchronize()
    return G.from_device(buf, G.RECORD_DTYPE)[:n]


@pytest.mark.parametrize("fmt,degree,layout,n", [(S.FP32, 0, "cube", 5000), (S.FP32, 3, "clusters", 30000),
                                                 (S.FP16, 3, "clusters", 30000), (S.BF16, 3, "clusters", 30000)])
def test_preprocess_parity(G, fmt, degree, layout, n):
    sc = S.make_scene(n, degree, fmt, 56, layout=layout)
    cams = S.ring_cameras(2, 320, 208)
    h = _load(G, sc)
    try:
        for cam in cams:
            g = _gpu_records(G, h, cam, sc.n)
            o = O.preprocess(sc.planes, fmt, degree, cam)
            vis = o["visible"] == 1
            assert np.array_equal(g["visible"], o["visible"])
            for f in ("x0", "y0", "x1", "y1", "radius"):
                assert np.array_equal(g[f][vis], o[f][vis]), f
            # identical operation order, no contraction, exp rounded once from double:
            # every field of the record is bit-identical
            for f in ("depth", "mx", "my", "r", "g", "b", "ca", "cb", "cc", "opac"):
                assert np.array_equal(g[f][vis].view(np.uint32), o[f][vis].view(np.uint32)), f
    finally:
        G.gs_free_scene(h)


# ---------------------------------------------------------------------------
# (c) binning + radix sort: bit exact from the same per-primitive input
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("case", ["tiny", "clusters", "ties_and_giants", "grid_100x65", "grid_128x72"])
def test_bin_tiles_bit_exact(G, case):
    """Lists equal the oracle's bit for bit, from small grids to the benchmark's
    100 x 65 tiles and a 128 x 72 grid (two pair passes over 13 and 14 tile-id
    bits)."""
    torch = _torch()
    if case == "tiny":
        sc = S.make_scene(5000, 0, S.FP32, 57)
        cam = S.ring_cameras(1, 256, 256)[0]
        recs = O.preprocess(sc.planes, S.FP32, 0, cam)
    elif case in ("grid_100x65", "grid_128x72"):
        sc = S.make_scene(60000, 0, S.FP32, 59, layout="clusters")
        cam = S.ring_cameras(1, 1600, 1040)[0] if case == "grid_100x65" else S.ring_cameras(1, 2048, 1152)[0]
        recs = O.preprocess(sc.planes, S.FP32, 0, cam)
    else:
        sc = S.make_scene(60000, 0, S.FP32, 58, layout="clusters")
        cam = S.ring_cameras(1, 800, 600)[0]
        recs = O.preprocess(sc.planes, S.FP32, 0, cam)
        if case == "ties_and_giants":
            rng = np.random.default_rng(3)
            vis = np.nonzero(recs["visible"])[0]
            recs["depth"][vis[:5000]] = np.float32(12.5)     # many exact depth ties
            g = vis[5000:5010]                               # primitives covering most of the grid
            recs["x0"][g], recs["y0"][g] = 0, 0
            recs["x1"][g], recs["y1"][g] = 50, 38
            recs["depth"][g] = rng.uniform(5, 25, size=len(g)).astype(np.float32)
    W, H = int(cam["width"]), int(cam["height"])
    tx, ty = -(-W // 16), -(-H // 16)
    off_o, ids_o = O.bin_tiles(recs, W, H)
    rects = np.stack([recs["x0"], recs["y0"], recs["x1"], recs["y1"]], axis=1).astype(np.int32)
    rects[recs["visible"] == 0] = 0
    d_depth = torch.from_numpy(recs["depth"].copy()).cuda()
    d_rects = torch.from_numpy(rects.reshape(-1).copy()).cuda()
    d_off = torch.zeros(tx * ty + 1, dtype=torch.int32, device="cuda")
    cap = len(ids_o) + 10
    d_ids = torch.zeros(cap, dtype=torch.int32, device="cuda")
    total = G.gs_bin_tiles(d_depth, d_rects, sc.n, tx, ty, d_off, d_ids, cap)
    assert total == len(ids_o)
    assert np.array_equal(d_off.cpu().numpy().view(np.uint32), off_o)
    assert np.array_equal(d_ids.cpu().numpy().view(np.uint32)[:total], ids_o)
    # too-small capacity is reported, not overrun
    with pytest.raises(G.GsError) as e:
        G.gs_bin_tiles(d_depth, d_rects, sc.n, tx, ty, d_off, d_ids, max(total // 2, 1))
    assert e.value.status == G.GS_ERR_CAPACITY


def test_render_stage_times(G):
    """Stage timing of the full render: the counts it reports are the oracle's
    (pairs of the last view's tile lists; 4 depth-key passes and ceil(tile bits
    / 8) pair passes of the 8-bit radix sort), the times are positive, and the
    image is the same with timing on."""
    sc = S.make_scene(30000, 3, S.FP32, 62, layout="clusters")
    cams = S.ring_cameras(2, 480, 304)
    h = _load(G, sc)
    try:
        plain = _render_gpu(G, h, cams)
        with pytest.raises(G.GsError) as e:
            G.gs_read_render_ms(h)
        assert e.value.status == G.GS_ERR_STATE
        G.gs_time_kernels(h, True)
        with pytest.raises(G.GsError) as e:
            G.gs_read_render_ms(h)
        assert e.value.status == G.GS_ERR_STATE
        timed = _render_gpu(G, h, cams)
        ms, counts = G.gs_read_render_ms(h)
        for a, b in zip(plain, timed):
            assert np.array_equal(a.view(np.uint32), b.view(np.uint32))
        cam = cams[-1]
        W, H = int(cam["width"]), int(cam["height"])
        _, ids_o = O.bin_tiles(O.preprocess(sc.planes, S.FP32, 3, cam), W, H)
        ntiles = -(-W // 16) * -(-H // 16)
        assert counts == (sc.n, len(ids_o), 4, -(-int(math.ceil(math.log2(ntiles))) // 8))
        assert all(t > 0 for t in ms)
        G.gs_time_kernels(h, False)
        with pytest.raises(G.GsError):
            G.gs_read_render_ms(h)
    finally:
        G.gs_free_scene(h)


# ---------------------------------------------------------------------------
# (d) blend from the same records and lists; (e) compare from the same images
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("W,H", [(256, 256), (200, 136)])
def test_blend_lists_parity(G, W, H):
    torch = _torch()
    sc = S.make_scene(8000, 0, S.FP32, 59)
    v = sc.values().copy()
    v[3:6, :3] = 2.0          # a few exploded primitives
    v[10, 3] = np.nan         # non-finite opacity propagates
    planes = S.encode(v, S.FP32)
    cam = S.look_at_camera((1.0, 2.0, 14.0), width=W, height=H)
    recs = O.preprocess(planes, S.FP32, 0, cam)
    off, ids = O.bin_tiles(recs, W, H)
    ref = O.blend(recs, off, ids, W, H)
    d_recs = G.to_device(recs.astype(G.RECORD_DTYPE))
    d_off = torch.from_numpy(off.view(np.int32).copy()).cuda()
    d_ids = torch.from_numpy(ids.view(np.int32).copy()).cuda()
    img = torch.empty(H * W * 3, dtype=torch.float32, device="cuda")
    G.gs_blend_lists(d_recs, len(recs), d_off, d_ids, W, H, img)
    torch.cuda.synchronize()
    out = img.cpu().numpy().reshape(H, W, 3)
    assert _pix_agree(out, ref) >= PIX_FRAC
    assert np.array_equal(np.isnan(out), np.isnan(ref))


def test_compare_exact_counts(G):
    torch = _torch()
    rng = np.random.default_rng(7)
    K, H, W = 3, 67, 91
    a = rng.uniform(-0.2, 1.2, size=(K, H, W, 3)).astype(np.float32)
    b = a + rng.normal(0, 0.01, size=a.shape).astype(np.float32) * (rng.uniform(size=a.shape) < 0.3)
    a[0, 3, 4, 1] = np.nan
    a[1, 5, 6, 0] = np.inf
    b[2, 10, 10, 2] = a[2, 10, 10, 2] - np.float32(1 / 255)
    da = torch.from_numpy(a.reshape(-1).copy()).cuda()
    db = torch.from_numpy(b.reshape(-1).copy()).cuda()
    out = G.device_bytes(K * 24)
    G.gs_compare(da, db, H, W, K, out)
    torch.cuda.synchronize()
    r = G.from_device(out, G.RESULT_DTYPE)
    for k in range(K):
        o = O.compare(a[k], b[k])
        assert r[k]["footprint"] == o["footprint"] and r[k]["nonfinite"] == o["nonfinite"]
        assert r[k]["maxabs"] == o["maxabs"]
        assert abs(r[k]["sse"] - o["sse"]) <= 1e-6 * o["sse"] + 1e-9


# ---------------------------------------------------------------------------
# end to end
# ---------------------------------------------------------------------------
def test_render_tiny_matches_oracle(G):
    sc, cams, _ = S.tiny_workload()
    h = _load(G, sc)
    try:
        g = _render_gpu(G, h, cams)[0]
        o = O.render(sc.planes, S.FP32, 0, cams[0])
        assert _pix_agree(g, o) >= PIX_FRAC
        assert np.abs(g - o).max() < 1e-4
    finally:
        G.gs_free_scene(h)


@pytest.mark.parametrize("fmt", [S.FP32, S.FP16, S.BF16])
def test_render_degree3_clusters_matches_oracle(G, fmt):
    sc = S.make_scene(40000, 3, fmt, 60, layout="clusters")
    cams = S.ring_cameras(2, 400, 272)
    h = _load(G, sc)
    try:
        gi = _render_gpu(G, h, cams)
        for k in range(2):
            o = O.render(sc.planes, fmt, 3, cams[k])
            assert _pix_agree(gi[k], o) >= PIX_FRAC
    finally:
        G.gs_free_scene(h)


def _campaign_gpu(G, h, flips, K, fpv=1, guard=-1, mask=S.GUARD_WORDS_DEFAULT, full=False):
    torch = _torch()
    nvar = len(flips) // fpv
    out = G.device_bytes(nvar * K * 24)
    d = G.to_device(flips)
    fn = G.gs_inject_and_render_full if full else G.gs_inject_and_render
    fn(h, d, nvar, fpv, guard, mask, out)
    torch.cuda.synchronize()
    return G.from_device(out, G.RESULT_DTYPE).reshape(nvar, K)


def test_campaign_tiny_matches_oracle(G):
    sc, cams, flips = S.tiny_workload()
    h = _load(G, sc)
    try:
        G.gs_set_views(h, cams)
        g = _campaign_gpu(G, h, flips, 1)
        o, _, _ = O.campaign(sc.planes, S.FP32, 0, cams, flips, nthreads=O.max_threads())
        npx = 256 * 256 * 3
        gp = np.array([_psnr(x, npx) for x in g["sse"].ravel()])
        op = np.array([_psnr(x, npx) for x in o["sse"].ravel()])
        assert np.abs(gp - op).max() <= PSNR_TOL
        assert np.array_equal(g["nonfinite"] > 0, o["nonfinite"] > 0)
        att = FA.attribute(G, h, sc, cams, flips, g["footprint"], o["footprint"])
        print("footprint attribution, 5,000 Gaussians:", att)
        assert att["unexplained"] == 0, att
    finally:
        G.gs_free_scene(h)


@pytest.mark.parametrize("fmt", [S.FP32, S.FP16, S.BF16])
@pytest.mark.parametrize("guard", [-1, 0, 1, 2])
def test_dirty_tile_equals_full_rerender(G, fmt, guard):
    """Batched dirty-tile records are bit-identical to one-variant-at-a-time full
    re-renders of the same variants (guard off, FIELD, PRIM, ECC emulation)."""
    sc = S.make_scene(30000, 3, fmt, 61, layout="clusters")
    cams = S.ring_cameras(2, 320, 240)
    flips = S.flips_stratified(59 * S.FORMAT_BITS[fmt], sc.n, sc.nwords, fmt, 62)
    h = _load(G, sc)
    try:
        if guard == 1:
            lo, hi = S.prim_boxes(sc, 14, 63)
            G.gs_set_prim_box(h, lo, hi, 14)
        G.gs_set_views(h, cams)
        a = _campaign_gpu(G, h, flips, 2, guard=guard)
        b = _campaign_gpu(G, h, flips, 2, guard=guard, full=True)
        for f in ("sse", "maxabs", "footprint", "nonfinite", "clamps"):
            assert np.array_equal(a[f], b[f]), f
        assert (a["footprint"] > 0).any()
        # the scene is left unchanged by both
        assert np.array_equal(_read(G, h, sc), sc.planes)
    finally:
        G.gs_free_scene(h)


def test_campaign_batching_guard_matches_oracle(G):
    """fp16 storage, degree-3 clusters, PRIM guard on: GPU campaign vs oracle."""
    fmt = S.FP16
    sc = S.make_scene(20000, 3, fmt, 64, layout="clusters")
    cams = S.ring_cameras(1, 240, 240)
    flips = S.flips_stratified(59 * 16, sc.n, sc.nwords, fmt, 65)[::4]
    lo, hi = S.prim_boxes(sc, 14, 66)
    h = _load(G, sc)
    try:
        G.gs_set_prim_box(h, lo, hi, 14)
        G.gs_set_views(h, cams)
        g = _campaign_gpu(G, h, flips, 1, guard=1)
        o, cl, _ = O.campaign(sc.planes, fmt, 3, cams, flips, guard_mode=1, word_mask=S.GUARD_WORDS_DEFAULT,
                              box_lo=lo, box_hi=hi, nthreads=O.max_threads())
        assert np.array_equal(g["clamps"][:, 0], cl.astype(np.uint32))
        npx = 240 * 240 * 3
        gp = np.array([_psnr(x, npx) for x in g["sse"].ravel()])
        op = np.array([_psnr(x, npx) for x in o["sse"].ravel()])
        assert np.abs(gp - op).max() <= PSNR_TOL
        att = FA.attribute(G, h, sc, cams, flips, g["footprint"], o["footprint"], guard=1,
                           mask=S.GUARD_WORDS_DEFAULT, box_lo=lo, box_hi=hi)
        print("footprint attribution, 20,000 Gaussians fp16 PRIM guard:", att)
        assert att["unexplained"] == 0, att
    finally:
        G.gs_free_scene(h)


def test_multi_flip_variants_match_oracle(G):
    sc, cams, _ = S.tiny_workload()
    flips = S.flips_multi(40 * 25, sc.n, sc.nwords, S.FP32, 67)
    h = _load(G, sc)
    try:
        G.gs_set_views(h, cams)
        g = _campaign_gpu(G, h, flips, 1, fpv=25)
        o, _, _ = O.campaign(sc.planes, S.FP32, 0, cams, flips, flips_per_variant=25, nthreads=O.max_threads())
        npx = 256 * 256 * 3
        gp = np.array([_psnr(x, npx) for x in g["sse"].ravel()])
        op = np.array([_psnr(x, npx) for x in o["sse"].ravel()])
        assert np.abs(gp - op).max() <= PSNR_TOL
        assert np.array_equal(g["nonfinite"] > 0, o["nonfinite"] > 0)
    finally:
        G.gs_free_scene(h)


def test_graphs_on_and_off_identical(G):
    sc, cams, flips = S.tiny_workload()
    h = _load(G, sc)
    try:
        G.gs_set_views(h, cams)
        a = _campaign_gpu(G, h, flips, 1)
        G.gs_set_graphs(h, False)
        b = _campaign_gpu(G, h, flips, 1)
        assert np.array_equal(a.view(np.uint8), b.view(np.uint8))
    finally:
        G.gs_free_scene(h)


def test_clean_scene_with_nonfinite_pixels(G):
    """A clean scene whose render already holds NaN pixels (NaN colour words
    propagate through the blend): every variant's non-finite count includes the
    clean image's NaN pixels that the variant leaves in place.  Dirty-tile records
    equal full re-renders bit for bit and match the oracle's counts."""
    sc, cams, flips = S.tiny_workload()
    planes = sc.planes.copy()
    rng = np.random.default_rng(S.SEED_BASE + 68)
    bad = rng.choice(sc.n, 40, replace=False)
    planes[11, bad] = np.uint32(0x7FC00000)   # DC red coefficient := NaN
    sc = S.Scene(planes=planes, fmt=sc.fmt, sh_degree=sc.sh_degree)
    h = _load(G, sc)
    try:
        G.gs_set_views(h, cams)
        clean_or = O.render(sc.planes, S.FP32, 0, cams[0])
        n_clean_bad = int((~np.isfinite(clean_or)).any(axis=2).sum())
        assert n_clean_bad > 0
        a = _campaign_gpu(G, h, flips, 1)
        b = _campaign_gpu(G, h, flips, 1, full=True)
        for f in ("sse", "maxabs", "footprint", "nonfinite", "clamps"):
            assert np.array_equal(a[f], b[f]), f
        o, _, _ = O.campaign(sc.planes, S.FP32, 0, cams, flips, nthreads=O.max_threads())
        assert (a["nonfinite"] > 0).all()
        dn = np.abs(a["nonfinite"].astype(np.int64) - o["nonfinite"].astype(np.int64))
        assert (dn <= 2).all(), dn.max()
        npx = 256 * 256 * 3
        gp = np.array([_psnr(x, npx) for x in a["sse"].ravel()])
        op = np.array([_psnr(x, npx) for x in o["sse"].ravel()])
        assert np.abs(gp - op).max() <= PSNR_TOL
    finally:
        G.gs_free_scene(h)


@pytest.mark.parametrize("fmt", [S.FP32, S.FP16, S.BF16])
def test_ecc_campaign_matches_oracle(G, fmt):
    """ECC sign+exponent emulation (Table 4): corrected upsets give the clean
    record exactly; the others match the oracle's campaign."""
    sc = S.make_scene(20000, 3, fmt, 71, layout="clusters")
    cams = S.ring_cameras(1, 240, 240)
    nbits = S.FORMAT_BITS[fmt]
    flips = S.flips_stratified(59 * nbits, sc.n, sc.nwords, fmt, 72)
    mask = (1 << 59) - 1
    h = _load(G, sc)
    try:
        G.gs_set_views(h, cams)
        g = _campaign_gpu(G, h, flips, 1, guard=2, mask=mask)
        o, _, _ = O.campaign(sc.planes, fmt, 3, cams, flips, guard_mode=2, word_mask=mask, nthreads=O.max_threads())
        corr = O.ecc_corrects(fmt, mask, flips)
        assert corr.any() and (~corr).any()
        for f in ("sse", "maxabs", "footprint", "nonfinite", "clamps"):
            assert (g[corr][f] == 0).all(), f
        npx = 240 * 240 * 3
        gp = np.array([_psnr(x, npx) for x in g["sse"].ravel()])
        op = np.array([_psnr(x, npx) for x in o["sse"].ravel()])
        assert np.abs(gp - op).max() <= PSNR_TOL
        assert np.array_equal(g["nonfinite"] > 0, o["nonfinite"] > 0)
        assert (o[corr]["footprint"] == 0).all()
        att = FA.attribute(G, h, sc, cams, flips[~corr], g[~corr]["footprint"], o[~corr]["footprint"])
        print(f"footprint attribution, ECC fmt {fmt}:", att)
        assert att["unexplained"] == 0, att
    finally:
        G.gs_free_scene(h)


@pytest.mark.parametrize("guard", [-1, 0, 2])
def test_contamination_regions_match_oracle(G, guard):
    """Sort-first contamination masks (Sec. 5): predicted cells bit for bit (they
    come from the bit-exact tile rects), actual cells equal on >= 99% of the
    (variant, view) pairs, records equal to the plain campaign call."""
    torch = _torch()
    sc = S.make_scene(30000, 3, S.FP32, 74, layout="clusters")
    cams = S.ring_cameras(2, 320, 240)
    flips = S.flips_stratified(59 * 32, sc.n, sc.nwords, S.FP32, 75)[::2]
    mask = S.GUARD_WORDS_DEFAULT
    h = _load(G, sc)
    try:
        G.gs_set_views(h, cams)
        out = G.device_bytes(len(flips) * 2 * 24)
        reg = torch.zeros(len(flips) * 2 * 2, dtype=torch.int64, device="cuda")
        G.gs_inject_and_render_regions(h, G.to_device(flips), len(flips), guard, mask, out, reg)
        torch.cuda.synchronize()
        g = G.from_device(out, G.RESULT_DTYPE).reshape(len(flips), 2)
        r = reg.cpu().numpy().view(np.uint64).reshape(len(flips), 2, 2)
        ref = _campaign_gpu(G, h, flips, 2, guard=guard, mask=mask)
        for f in ("sse", "maxabs", "footprint", "nonfinite", "clamps"):
            assert np.array_equal(g[f], ref[f]), f
        kw = {}
        if guard == 0:
            lo, hi = G.gs_field_box(h, 59)
            kw = dict(box_lo=lo, box_hi=hi)
        _, _, _, act, pred = O.campaign(sc.planes, S.FP32, 3, cams, flips, guard_mode=guard, word_mask=mask,
                                        nthreads=O.max_threads(), regions=True, **kw)
        assert np.array_equal(r[:, :, 1], pred)
        assert (r[:, :, 0] == act).mean() >= 0.99
        assert ((r[:, :, 0] & ~r[:, :, 1]) == 0).all()
    finally:
        G.gs_free_scene(h)


def test_ssim_image_pairs_match_oracle(G):
    torch = _torch()
    rng = np.random.default_rng(S.SEED_BASE + 78)
    H, W = 67, 91                     # ragged: partial tiles on both edges
    a = rng.random((2, H, W, 3), dtype=np.float32)
    b = a.copy()
    b[0] += rng.normal(0, 0.05, b[0].shape).astype(np.float32)
    b[1, 10:30, 20:50] = 0.0
    b[1, 5, 5, 0] = np.nan
    da, db = torch.from_numpy(a).cuda(), torch.from_numpy(b).cuda()
    out = torch.zeros(2, dtype=torch.float64, device="cuda")
    G.gs_ssim(db, da, H, W, 2, out)
    torch.cuda.synchronize()
    g = out.cpu().numpy()
    o = np.array([O.ssim(b[k], a[k]) for k in range(2)])
    assert np.abs(g - o).max() < 5e-5, (g, o)
    G.gs_ssim(da, da, H, W, 2, out)
    torch.cuda.synchronize()
    assert (out.cpu().numpy() == 1.0).all()


def test_dirty_tile_ssim_equals_full_frame_ssim(G):
    """The campaign's SSIM, from re-blended pixels only, equals gs_ssim of the
    full re-rendered frame bit for bit, and the oracle's SSIM within 5e-5."""
    torch = _torch()
    sc = S.make_scene(30000, 3, S.FP32, 79, layout="clusters")
    cams = S.ring_cameras(2, 320, 240)
    flips = S.flips_stratified(59 * 32, sc.n, sc.nwords, S.FP32, 80)[::4]
    B, K, H, W = len(flips), 2, 240, 320
    h = _load(G, sc)
    try:
        G.gs_set_views(h, cams)
        d = G.to_device(flips)
        out = G.device_bytes(B * K * 24)
        ss = torch.zeros(B * K, dtype=torch.float64, device="cuda")
        G.gs_inject_and_render_ex(h, d, B, -1, S.GUARD_WORDS_DEFAULT, out, None, ss)
        torch.cuda.synchronize()
        g = G.from_device(out, G.RESULT_DTYPE).reshape(B, K)
        ssim = ss.cpu().numpy().reshape(B, K)
        ref = _campaign_gpu(G, h, flips, K)
        for f in ("sse", "maxabs", "footprint", "nonfinite"):
            assert np.array_equal(g[f], ref[f]), f
        changed = np.nonzero(g["sse"].sum(axis=1) > 0)[0]
        assert len(changed) > 4
        sample = np.concatenate([changed[:: max(1, len(changed) // 12)], np.nonzero(g["sse"].sum(axis=1) == 0)[0][:2]])
        clean = torch.empty(K * H * W * 3, dtype=torch.float32, device="cuda")
        for k in range(K):
            G.gs_clean_image(h, k, clean[k * H * W * 3:(k + 1) * H * W * 3])
        img = torch.empty_like(clean)
        one = torch.zeros(K, dtype=torch.float64, device="cuda")
        for i in sample:
            fi = G.to_device(flips[i:i + 1])
            G.gs_apply_flips(h, fi, 1)
            G.gs_render(h, cams, img)
            G.gs_apply_flips(h, fi, 1)   # XOR back
            G.gs_ssim(img, clean, H, W, K, one)
            torch.cuda.synchronize()
            assert np.array_equal(one.cpu().numpy(), ssim[i]), (i, one.cpu().numpy(), ssim[i])
        assert np.array_equal(_read(G, h, sc), sc.planes)
        _, _, _, o = O.campaign(sc.planes, S.FP32, 3, cams, flips[sample], nthreads=O.max_threads(), ssim=True)
        assert np.abs(o - ssim[sample]).max() < 5e-5
    finally:
        G.gs_free_scene(h)


def test_campaign_edge_cases(G):
    """Empty batch; ragged views (not multiples of the tile) and an odd view count;
    a batch split over launches (2049 variants with the 2048 cap); invalid upsets
    (site, word or bit out of range) give the clean record; an ECC word index
    beyond 64 is not a protected word."""
    torch = _torch()
    sc = S.make_scene(8000, 3, S.FP32, 81, layout="clusters")
    cams = S.ring_cameras(3, 250, 130)
    h = _load(G, sc)
    try:
        G.gs_set_views(h, cams)
        K = 3
        out = G.device_bytes(24)
        G.gs_inject_and_render(h, G.to_device(S.flips_at(np.array([0], np.uint32), 0, 0)), 0, 1, -1,
                               S.GUARD_WORDS_DEFAULT, out)   # B = 0: nothing to do
        torch.cuda.synchronize()
        flips = S.flips_stratified(2049, sc.n, sc.nwords, S.FP32, 82)
        G.gs_set_batch(h, 2048)
        a = _campaign_gpu(G, h, flips, K)
        G.gs_set_batch(h, 64)
        b = _campaign_gpu(G, h, flips, K)
        for f in ("sse", "maxabs", "footprint", "nonfinite", "clamps"):
            assert np.array_equal(a[f], b[f]), f
        sample = np.arange(0, 2049, 97)
        o, _, _ = O.campaign(sc.planes, S.FP32, 3, cams, flips[sample], nthreads=O.max_threads())
        npx = 250 * 130 * 3
        dp = np.abs(np.array([_psnr(x, npx) for x in a[sample]["sse"].ravel()]) -
                    np.array([_psnr(x, npx) for x in o["sse"].ravel()]))
        assert dp.max() <= PSNR_TOL
        full = _campaign_gpu(G, h, flips[sample], K, full=True)
        for f in ("sse", "maxabs", "footprint", "nonfinite"):
            assert np.array_equal(full[f], a[sample][f]), f
        bad = np.concatenate([S.flips_at(np.array([sc.n], np.uint32), 3, 31), S.flips_at(np.array([5], np.uint32), 59, 0),
                              S.flips_at(np.array([5], np.uint32), 3, 32)])
        r = _campaign_gpu(G, h, bad, K)
        for f in ("sse", "maxabs", "footprint", "nonfinite", "clamps"):
            assert (r[f] == 0).all(), f
        # The plain loop saves, applies and restores the sites: an invalid site is
        # skipped by all three (the scene stays clean, the error flag is raised),
        # one variant at a time and as part of a multi-upset variant.
        G.gs_scene_errors(h)   # clear
        before = _read(G, h, sc)
        for guard in (-1, 0):   # guard off, FIELD guard
            r = _campaign_gpu(G, h, bad, K, guard=guard, full=True)
            for f in ("sse", "maxabs", "footprint", "nonfinite", "clamps"):
                assert (r[f] == 0).all(), (guard, f)
        assert G.gs_scene_errors(h) & 1
        mixed = np.concatenate([bad, S.flips_at(np.array([7], np.uint32), 10, 30)])   # 3 invalid + 1 valid
        r = _campaign_gpu(G, h, mixed, K, fpv=4, full=True)
        one = _campaign_gpu(G, h, mixed[3:], K, full=True)
        for f in ("sse", "maxabs", "footprint", "nonfinite"):
            assert np.array_equal(r[f], one[f]), f
        assert G.gs_scene_errors(h) & 1
        assert np.array_equal(_read(G, h, sc).view(np.uint32), before.view(np.uint32))
        far = S.flips_at(np.array([5], np.uint32), 70, 0)   # word 70 >= 64: invalid, not protected
        r = _campaign_gpu(G, h, far, K, guard=2, mask=(1 << 59) - 1)
        assert (r["sse"] == 0).all()
    finally:
        G.gs_free_scene(h)


# ---------------------------------------------------------------------------
# render tile shapes (gs_set_tile, gs_autotune_tile)
# ---------------------------------------------------------------------------
TILE_SHAPES = [(8, 8), (32, 8), (16, 8)]


@pytest.mark.parametrize("tile", TILE_SHAPES)
def test_tile_shape_matches_oracle(G, tile):
    """At each tile shape: the records' tile rects are the oracle's bit for bit,
    the render agrees with the oracle's render at that shape, and a FIELD-guarded
    campaign over two ragged views agrees in PSNR with every footprint decision
    equal or attributed to a threshold."""
    sc = S.make_scene(30000, 3, S.FP32, 93, layout="clusters")
    cams = S.ring_cameras(2, 200, 120)   # ragged against every tile edge
    flips = S.flips_stratified(59 * 32, sc.n, sc.nwords, S.FP32, 94)[::8]
    h = _load(G, sc)
    try:
        G.gs_set_tile(h, *tile)
        assert G.gs_get_tile(h) == tile
        g = _gpu_records(G, h, cams[0], sc.n)
        o = O.preprocess(sc.planes, S.FP32, 3, cams[0], tile)
        vis = o["visible"] == 1
        assert np.array_equal(g["visible"], o["visible"])
        for f in ("x0", "y0", "x1", "y1", "radius"):
            assert np.array_equal(g[f][vis], o[f][vis]), f
        imgs = _render_gpu(G, h, cams)
        for k in range(2):
            assert _pix_agree(imgs[k], O.render(sc.planes, S.FP32, 3, cams[k], tile)) >= PIX_FRAC
        G.gs_set_views(h, cams)
        gr = _campaign_gpu(G, h, flips, 2, guard=0)
        lo, hi = O.field_box(sc.planes, S.FP32)
        orc, cl, _ = O.campaign(sc.planes, S.FP32, 3, cams, flips, guard_mode=0, word_mask=S.GUARD_WORDS_DEFAULT,
                                box_lo=lo, box_hi=hi, tile=tile, nthreads=O.max_threads())
        assert np.array_equal(gr["clamps"][:, 0], cl.astype(np.uint32))
        npx = 200 * 120 * 3
        gp = np.array([_psnr(x, npx) for x in gr["sse"].ravel()])
        op = np.array([_psnr(x, npx) for x in orc["sse"].ravel()])
        assert np.abs(gp - op).max() <= PSNR_TOL
        assert np.array_equal(gr["nonfinite"] > 0, orc["nonfinite"] > 0)
        att = FA.attribute(G, h, sc, cams, flips, gr["footprint"], orc["footprint"], guard=0,
                           mask=S.GUARD_WORDS_DEFAULT, tile=tile)
        print(f"footprint attribution, tiles {tile}:", att)
        assert att["unexplained"] == 0, att
    finally:
        G.gs_free_scene(h)


@pytest.mark.parametrize("tile", TILE_SHAPES)
@pytest.mark.parametrize("guard", [-1, 1])
def test_dirty_tile_equals_full_rerender_at_tile_shapes(G, tile, guard):
    """The dirty-tile engine on other tile shapes: records bit-identical to full
    re-renders of the same variants (guard off and PRIM boxes), the scene left
    unchanged."""
    sc = S.make_scene(30000, 3, S.FP32, 95, layout="clusters")
    cams = S.ring_cameras(2, 328, 244)
    flips = S.flips_stratified(59 * 32, sc.n, sc.nwords, S.FP32, 96)
    h = _load(G, sc)
    try:
        if guard == 1:
            lo, hi = S.prim_boxes(sc, 14, 97)
            G.gs_set_prim_box(h, lo, hi, 14)
        G.gs_set_views(h, cams)
        G.gs_set_tile(h, *tile)   # rebuilds the views for the new tiles
        a = _campaign_gpu(G, h, flips, 2, guard=guard)
        b = _campaign_gpu(G, h, flips, 2, guard=guard, full=True)
        for f in ("sse", "maxabs", "footprint", "nonfinite", "clamps"):
            assert np.array_equal(a[f], b[f]), f
        assert (a["footprint"] > 0).any()
        assert np.array_equal(_read(G, h, sc), sc.planes)
    finally:
        G.gs_free_scene(h)


def test_autotune_tile_and_batch(G):
    """gs_autotune_tile leaves the scene on one of the candidate shapes with its
    batch; records at that shape equal a direct call; the dirty-tile SSIM is
    refused on other shapes than 16 x 16 and works again after switching back."""
    torch = _torch()
    sc = S.make_scene(20000, 3, S.FP32, 98, layout="clusters")
    cams = S.ring_cameras(2, 240, 160)
    flips = S.flips_stratified(59 * 32, sc.n, sc.nwords, S.FP32, 99)
    h = _load(G, sc)
    try:
        G.gs_set_views(h, cams)
        d = G.to_device(flips)
        (tw, th), b, us = G.gs_autotune_tile(h, d, len(flips), -1, S.GUARD_WORDS_DEFAULT)
        assert (tw, th) in [(16, 16), (8, 8), (32, 8)] and b in (8, 16, 32, 64, 128, 256, 512, 1024, 2048)
        assert G.gs_get_tile(h) == (tw, th) and us > 0
        a = _campaign_gpu(G, h, flips, 2)
        full = _campaign_gpu(G, h, flips, 2, full=True)
        for f in ("sse", "maxabs", "footprint", "nonfinite"):
            assert np.array_equal(a[f], full[f]), f
        G.gs_set_tile(h, 8, 8)
        out = G.device_bytes(len(flips) * 2 * 24)
        ss = torch.zeros(len(flips) * 2, dtype=torch.float64, device="cuda")
        with pytest.raises(G.GsError) as e:
            G.gs_inject_and_render_ex(h, d, len(flips), -1, S.GUARD_WORDS_DEFAULT, out, None, ss)
        assert e.value.status == G.GS_ERR_STATE
        G.gs_set_tile(h, 16, 16)
        G.gs_inject_and_render_ex(h, d, len(flips), -1, S.GUARD_WORDS_DEFAULT, out, None, ss)
        torch.cuda.synchronize()
        # the same as a scene that never left 16 x 16 tiles, bit for bit
        h2 = _load(G, sc)
        try:
            G.gs_set_views(h2, cams)
            out2 = G.device_bytes(len(flips) * 2 * 24)
            ss2 = torch.zeros_like(ss)
            G.gs_inject_and_render_ex(h2, d, len(flips), -1, S.GUARD_WORDS_DEFAULT, out2, None, ss2)
            torch.cuda.synchronize()
            assert np.array_equal(ss.cpu().numpy(), ss2.cpu().numpy())
            assert np.array_equal(G.from_device(out, G.RESULT_DTYPE), G.from_device(out2, G.RESULT_DTYPE))
        finally:
            G.gs_free_scene(h2)
    finally:
        G.gs_free_scene(h)


def test_host_buffer_entry_point_equals_device_one(G):
    """gs_inject_and_render_host (host upsets in, host records out, the copies
    inside the call) gives the records of gs_inject_and_render, for single-flip
    variants (dirty-tile engine) and multi-flip variants (full re-renders),
    from pageable numpy buffers."""
    sc = S.make_scene(20000, 3, S.FP32, 101, layout="clusters")
    cams = S.ring_cameras(2, 200, 152)
    flips = S.flips_stratified(59 * 32, sc.n, sc.nwords, S.FP32, 102)[:600]
    h = _load(G, sc)
    try:
        G.gs_set_views(h, cams)
        for fpv in (1, 3):
            nvar = len(flips) // fpv
            dev = _campaign_gpu(G, h, flips[:nvar * fpv], 2, fpv=fpv)
            host = np.zeros(nvar * 2, dtype=G.RESULT_DTYPE)
            G.gs_inject_and_render_host(h, np.ascontiguousarray(flips[:nvar * fpv]), nvar, fpv, -1,
                                        S.GUARD_WORDS_DEFAULT, host)
            host = host.reshape(nvar, 2)
            for f in ("sse", "maxabs", "footprint", "nonfinite", "clamps"):
                assert np.array_equal(host[f], dev[f]), (fpv, f)
        G.gs_inject_and_render_host(h, None, 0, 1, -1, S.GUARD_WORDS_DEFAULT, None)   # B = 0: nothing to do
    finally:
        G.gs_free_scene(h)
