"""Parity at the benchmark's full sizes, in the launch configuration bench.py
times, on sampled outputs the oracle computes one by one.

* 2,000,000 Gaussians, 4 views 1600x1040, batch 2048 (the largest batch the
  benchmark's autotuner picks from): the clean frame of view 0 against the
  oracle's render; a sample of the step's variants against the oracle campaign
  in view 0; the sampled variants' records against full re-renders (bit for bit).
* 134,826 Gaussians, 800x800, fp32/fp16/bf16 storage, stratified upsets (one
  format with per-primitive guard boxes): GPU campaign vs oracle campaign.
* 66,000,000 Gaussians (guard stress): after 2,000 upsets and the FIELD guard,
  the words of every flipped primitive equal the oracle's guard of the same
  words with the same box, the box equals torch's min/max of the planes, and
  the clamp count equals the oracle's."""
import numpy as np
import pytest

import footprint_attribution as FA
import oracle as O
from paper_2606_21791_gb300 import synth as S

pytestmark = pytest.mark.gpu

PIX_TOL = 2e-3
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


def _records(G, h, flips, K, full=False, guard=-1, mask=S.GUARD_WORDS_DEFAULT):
    import torch
    out = G.device_bytes(len(flips) * K * 24)
    fn = G.gs_inject_and_render_full if full else G.gs_inject_and_render
    fn(h, G.to_device(flips), len(flips), 1, guard, mask, out)
    torch.cuda.synchronize()
    return G.from_device(out, G.RESULT_DTYPE).reshape(len(flips), K)


def _psnr(x, npx):
    return np.array([O.psnr(float(v), npx) for v in np.ravel(x)])


def test_scale_workload_step_matches_oracle(G):
    import torch
    sc, cams, flips = S.scale_workload()
    h = G.gs_load_scene(sc.planes, sc.n, 3, S.FP32)
    try:
        G.gs_set_views(h, cams)
        G.gs_set_batch(h, 2048)
        # clean frame of view 0
        W, H = int(cams[0]["width"]), int(cams[0]["height"])
        clean_gpu = torch.empty(W * H * 3, dtype=torch.float32, device="cuda")
        G.gs_clean_image(h, 0, clean_gpu)
        clean_gpu = clean_gpu.cpu().numpy().reshape(H, W, 3)
        clean_or = O.render(sc.planes, S.FP32, 3, cams[0])
        ok = (np.abs(clean_gpu.astype(np.float64) - clean_or) <= PIX_TOL).all(axis=2).mean()
        assert ok >= 0.999, ok
        # one step: 2048 variants x 4 views in one launch
        step = flips[:2048]
        g = _records(G, h, step, 4)
        # sample: 16 variants, view 0, against the oracle
        sample = np.arange(0, 2048, 128)
        o, _, _ = O.campaign(sc.planes, S.FP32, 3, cams[0:1], step[sample], clean_imgs=[clean_or],
                             nthreads=O.max_threads())
        npx = W * H * 3
        dp = np.abs(_psnr(g[sample, 0]["sse"], npx) - _psnr(o[:, 0]["sse"], npx))
        assert dp.max() <= PSNR_TOL, dp.max()
        assert np.array_equal(g[sample, 0]["nonfinite"] > 0, o[:, 0]["nonfinite"] > 0)
        att = FA.attribute(G, h, sc, cams, step[sample], g[sample, 0]["footprint"], o[:, 0]["footprint"],
                           views=[0], nthreads=O.max_threads())
        print("footprint attribution, 2M Gaussians view 0:", att)
        assert att["unexplained"] == 0, att
        # the sampled variants re-rendered in full give the same records bit for bit
        f = _records(G, h, step[sample], 4, full=True)
        for fld in ("sse", "maxabs", "footprint", "nonfinite"):
            assert np.array_equal(f[fld], g[sample][fld]), fld
    finally:
        G.gs_free_scene(h)


def test_scale_workload_at_32x8_tiles_matches_oracle(G):
    """The benchmark workload on 32x8 tiles (a shape the tile autotuner may
    pick): one batch of 2048 variants x 4 views; 8 sampled variants in view 1
    against the oracle rendering with the same tiles (PSNR, non-finite flags,
    footprints exact or attributed), and the sampled records equal full
    re-renders bit for bit."""
    sc, cams, flips = S.scale_workload()
    h = G.gs_load_scene(sc.planes, sc.n, 3, S.FP32)
    try:
        G.gs_set_views(h, cams)
        G.gs_set_tile(h, 32, 8)
        G.gs_set_batch(h, 2048)
        step = flips[4096:6144]
        g = _records(G, h, step, 4)
        sample = np.arange(7, 2048, 256)
        o, _, _ = O.campaign(sc.planes, S.FP32, 3, cams[1:2], step[sample], tile=(32, 8), nthreads=O.max_threads())
        W, H = int(cams[1]["width"]), int(cams[1]["height"])
        npx = W * H * 3
        dp = np.abs(_psnr(g[sample, 1]["sse"], npx) - _psnr(o[:, 0]["sse"], npx))
        assert dp.max() <= PSNR_TOL, dp.max()
        assert np.array_equal(g[sample, 1]["nonfinite"] > 0, o[:, 0]["nonfinite"] > 0)
        att = FA.attribute(G, h, sc, cams, step[sample], g[sample, 1]["footprint"], o[:, 0]["footprint"],
                           views=[1], nthreads=O.max_threads(), tile=(32, 8))
        print("footprint attribution, 2M Gaussians view 1, 32x8 tiles:", att)
        assert att["unexplained"] == 0, att
        f = _records(G, h, step[sample], 4, full=True)
        for fld in ("sse", "maxabs", "footprint", "nonfinite"):
            assert np.array_equal(f[fld], g[sample][fld]), fld
    finally:
        G.gs_free_scene(h)


@pytest.mark.parametrize("fmt,guard", [(S.FP32, -1), (S.FP16, 1), (S.BF16, -1)])
def test_batching_workload_matches_oracle(G, fmt, guard):
    sc, cams, flips = S.batching_workload(fmt, count=50_000)
    nbits = S.FORMAT_BITS[fmt]
    # one upset per (word, bit) cell, taken from the stratified list
    sample = flips[::len(flips) // (59 * nbits)][: 59 * nbits]
    h = G.gs_load_scene(sc.planes, sc.n, 3, fmt)
    try:
        kw = {}
        if guard == 1:
            lo, hi = S.prim_boxes(sc, 14, S.SEED_BASE + 60)
            G.gs_set_prim_box(h, lo, hi, 14)
            kw = dict(guard_mode=1, word_mask=S.GUARD_WORDS_DEFAULT, box_lo=lo, box_hi=hi)
        G.gs_set_views(h, cams)
        G.gs_set_batch(h, 32)
        g = _records(G, h, sample, 1, guard=guard)
        o, cl, _ = O.campaign(sc.planes, fmt, 3, cams, sample, nthreads=O.max_threads(), **kw)
        npx = 800 * 800 * 3
        dp = np.abs(_psnr(g["sse"], npx) - _psnr(o["sse"], npx))
        assert dp.max() <= PSNR_TOL, dp.max()
        assert np.array_equal(g["nonfinite"] > 0, o["nonfinite"] > 0)
        att = FA.attribute(G, h, sc, cams, sample, g["footprint"], o["footprint"], guard=guard,
                           mask=S.GUARD_WORDS_DEFAULT, box_lo=kw.get("box_lo"), box_hi=kw.get("box_hi"),
                           nthreads=O.max_threads())
        print(f"footprint attribution, 134,826 Gaussians fmt {fmt} guard {guard}:", att)
        assert att["unexplained"] == 0, att
        if guard == 1:
            assert np.array_equal(g["clamps"][:, 0], cl.astype(np.uint32))
    finally:
        G.gs_free_scene(h)


def test_guard_stress_66m_matches_oracle_on_flipped_primitives(G):
    import torch
    n = 66_000_000
    planes = S.make_scene_torch(n, 3, S.FP32, S.SEED_BASE + 4)
    h = G.gs_load_scene(planes, n, 3, S.FP32)
    try:
        # FIELD box against torch's min/max of the guarded planes
        lo, hi = G.gs_field_box(h, 59)
        v = planes[:14].view(torch.float32)
        mn = v.amin(dim=1).cpu().numpy()
        mx = v.amax(dim=1).cpu().numpy()
        assert np.array_equal(lo[:14].view(np.float32), mn) and np.array_equal(hi[:14].view(np.float32), mx)
        del v
        fl = S.flips_multi(2000, n, 14, S.FP32, S.SEED_BASE + 61)   # sites over the 14 guarded words
        prims = np.unique(fl["prim"])
        idx = torch.from_numpy(prims.astype(np.int64)).cuda()
        before = planes[:, idx].cpu().numpy().view(np.uint32)       # [59, m] clean words of those primitives
        del planes
        torch.cuda.empty_cache()
        G.gs_apply_flips(h, G.to_device(fl), len(fl))
        cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
        G.gs_guard(h, 0, S.GUARD_WORDS_DEFAULT, cnt)
        torch.cuda.synchronize()
        dev_planes = torch.empty((59, n), dtype=torch.int32, device="cuda")
        G.gs_read_planes(h, dev_planes)
        after = dev_planes[:, idx].cpu().numpy().view(np.uint32)
        del dev_planes
        # oracle: the same flips on the gathered words, then the guard with the GPU's box
        remap = {p: i for i, p in enumerate(prims.tolist())}
        lf = fl.copy()
        lf["prim"] = [remap[int(p)] for p in fl["prim"]]
        bad = O.apply_flips(before, S.FP32, lf)
        ref, nref = O.guard(bad, S.FP32, S.GUARD_WORDS_DEFAULT, 0, lo, hi)
        assert np.array_equal(after, ref)
        assert int(cnt.item()) == nref and nref > 0
    finally:
        G.gs_free_scene(h)
        torch.cuda.empty_cache()
