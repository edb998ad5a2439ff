"""Attribution of end-to-end footprint differences between the CUDA path and the
oracle (Definition 1: pixels whose largest channel change exceeds 1/255).

The two renderers share every preprocess bit (tested bit for bit) and differ only
in the exponential inside alpha.  A pixel's footprint decision can therefore
differ only where one of the thresholds met on the way is within rounding of
being crossed:

* ``delta``: the oracle's |change| at the pixel is within 1e-5 of 1/255;
* ``alpha``: some entry walked at the pixel (clean or corrupted render) has an
  alpha within 1e-5 (relative) of the 1/255 skip cut-off;
* ``stop``: some entry's T' is within 1e-5 (relative) of the 1e-4 stop.

``attribute`` re-renders each (variant, view) whose footprint counts differ, on
both sides, finds the pixels whose decisions differ and sorts them into those
classes.  Every differing pixel must fall into one; the tests print the counts.
"""
from __future__ import annotations

import concurrent.futures as cf

import numpy as np

import oracle as O

MARGIN = 1e-5
THR = np.float32(1.0 / 255.0)


def _clamp01(x):
    x = np.asarray(x, dtype=np.float32)
    return np.where(x > 0, np.minimum(x, np.float32(1)), np.float32(0)).astype(np.float32)


def change(img, clean):
    """Per pixel: the largest channel |change| of clamped images, in fp32 (the
    arithmetic of the compare on both sides)."""
    return np.abs(_clamp01(img) - _clamp01(clean)).max(axis=-1)


def gpu_variant_images(G, h, scene, cams, flips, guard=-1, mask=0):
    """Full GPU re-render of one variant in every view: apply its flips in the
    scene, guard (FIELD or PRIM), render, then write the clean planes back."""
    import torch
    cams = np.atleast_1d(cams)
    G.gs_apply_flips(h, G.to_device(flips), len(flips))
    if guard in (0, 1):
        clamps = G.device_bytes(8)
        G.gs_guard(h, guard, mask, clamps)
    tot = sum(int(c["width"]) * int(c["height"]) * 3 for c in cams)
    buf = torch.empty(tot, dtype=torch.float32, device="cuda")
    G.gs_render(h, cams, buf)
    torch.cuda.synchronize()
    G.gs_write_planes(h, scene.planes)
    out, off = [], 0
    host = buf.cpu().numpy()
    for c in cams:
        H, W = int(c["height"]), int(c["width"])
        out.append(host[off:off + H * W * 3].reshape(H, W, 3))
        off += H * W * 3
    return out


def gpu_clean_images(G, h, cams):
    import torch
    out = []
    for k, c in enumerate(np.atleast_1d(cams)):
        H, W = int(c["height"]), int(c["width"])
        buf = torch.empty(H * W * 3, dtype=torch.float32, device="cuda")
        G.gs_clean_image(h, k, buf)
        torch.cuda.synchronize()
        out.append(buf.cpu().numpy().reshape(H, W, 3))
    return out


def oracle_variant(scene, cam, flips, guard=-1, mask=0, box_lo=None, box_hi=None, tile=(16, 16)):
    p = O.apply_flips(scene.planes, scene.fmt, flips)
    if guard in (0, 1):
        if guard == 0 and box_lo is None:
            box_lo, box_hi = O.field_box(scene.planes, scene.fmt)
        p, _ = O.guard(p, scene.fmt, mask, guard, box_lo, box_hi)
    return O.render_margins(p, scene.fmt, scene.sh_degree, cam, tile)


def attribute(G, h, scene, cams, flips, g_fp, o_fp, fpv=1, guard=-1, mask=0, box_lo=None, box_hi=None,
              views=None, nthreads=8, tile=(16, 16)):
    """g_fp, o_fp: footprint counts [nvar, len(views)] from the engine and the
    oracle campaign; views: the camera indices they cover (default all); tile:
    the render tile shape of both sides.
    Returns {"variants": pairs compared, "mismatched_pairs": ..., "pixels": ...,
    "delta": ..., "alpha": ..., "stop": ..., "unexplained": ...}; asserts that
    each side's footprint count equals its own per-pixel decisions."""
    cams = np.atleast_1d(cams)
    views = list(range(len(cams))) if views is None else list(views)
    g_fp = np.asarray(g_fp).reshape(-1, len(views))
    o_fp = np.asarray(o_fp).reshape(-1, len(views))
    bad = sorted({int(v) for v, _ in zip(*np.nonzero(g_fp != o_fp))})
    res = dict(variants=int(g_fp.size), mismatched_pairs=int((g_fp != o_fp).sum()), pixels=0, delta=0, alpha=0,
               stop=0, unexplained=0)
    if not bad:
        return res
    sel = [cams[k] for k in views]
    clean_g = gpu_clean_images(G, h, cams)
    with cf.ThreadPoolExecutor(max_workers=nthreads) as ex:   # the oracle's C calls release the GIL
        clean_o = list(ex.map(lambda c: O.render_margins(scene.planes, scene.fmt, scene.sh_degree, c, tile), sel))
        jobs = {}
        for v in bad:
            fv = flips[v * fpv:(v + 1) * fpv]
            for j, k in enumerate(views):
                if g_fp[v, j] != o_fp[v, j]:
                    jobs[(v, j)] = ex.submit(oracle_variant, scene, cams[k], fv, guard, mask, box_lo, box_hi, tile)
        for v in bad:
            fv = flips[v * fpv:(v + 1) * fpv]
            imgs_g = gpu_variant_images(G, h, scene, cams, fv, guard, mask)
            for j, k in enumerate(views):
                if (v, j) not in jobs:
                    continue
                img_o, mg_o = jobs[(v, j)].result()
                c = classify(imgs_g[k], clean_g[k], img_o, mg_o, clean_o[j][0], clean_o[j][1])
                assert c["gpu_footprint"] == int(g_fp[v, j]), (v, k, c, int(g_fp[v, j]))
                assert c["oracle_footprint"] == int(o_fp[v, j]), (v, k, c, int(o_fp[v, j]))
                for key in ("pixels", "delta", "alpha", "stop", "unexplained"):
                    res[key] += c[key]
    return res


def classify(img_g, clean_g, img_o, margins_o, clean_o, clean_margins_o):
    """Per-pixel footprint decisions of one (variant, view) on both sides and the
    class of every pixel where they differ (see the module docstring)."""
    dg = change(img_g, clean_g)
    do = change(img_o, clean_o)
    fg, fo = dg > THR, do > THR
    diff = fg != fo
    near_d = np.abs(do.astype(np.float64) - float(THR)) <= MARGIN
    near_a = np.minimum(margins_o[..., 0], clean_margins_o[..., 0]) <= MARGIN
    near_s = np.minimum(margins_o[..., 1], clean_margins_o[..., 1]) <= MARGIN
    return {"gpu_footprint": int(fg.sum()), "oracle_footprint": int(fo.sum()), "pixels": int(diff.sum()),
            "delta": int((diff & near_d).sum()), "alpha": int((diff & ~near_d & near_a).sum()),
            "stop": int((diff & ~near_d & ~near_a & near_s).sum()),
            "unexplained": int((diff & ~near_d & ~near_a & ~near_s).sum())}
