"""CPU oracle of the SEU-injection / 3DGS-render / support-guard path (ctypes wrapper).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  The product path
(``paper_2606_21791_gb300``) never imports it and has no CPU fallback.

The arithmetic lives in ``gs_oracle.c`` (plain C, fp32 render math with every
operation rounded, double metric sums); this module only marshals numpy arrays.
It shares nothing with the CUDA path except the seeded input generators.
"""
from __future__ import annotations

import ctypes as C
import math
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gs_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

REC_DTYPE = np.dtype([
    ("mx", "<f4"), ("my", "<f4"), ("ca", "<f4"), ("cb", "<f4"), ("cc", "<f4"),
    ("r", "<f4"), ("g", "<f4"), ("b", "<f4"), ("opac", "<f4"), ("depth", "<f4"),
    ("x0", "<i4"), ("y0", "<i4"), ("x1", "<i4"), ("y1", "<i4"), ("radius", "<i4"), ("visible", "<i4"),
])
METRICS_DTYPE = np.dtype([("sse", "<f8"), ("maxabs", "<f4"), ("footprint", "<u4"),
                          ("nonfinite", "<u4"), ("pad", "<u4")])

PSNR_MSE_FLOOR = 1e-10   # PSNR capped at 100 dB for averaging


def build(force: bool = False) -> str:
    """Compile gs_oracle.c with gcc (no FP contraction, no fast-math, OpenMP)."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-std=c11", "-O2", "-fPIC", "-shared", "-ffp-contract=off", "-fno-fast-math",
           "-fopenmp", "-o", tmp, _SRC, "-lm"]
    subprocess.check_call(cmd)
    os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = C.CDLL(_LIB)
            vp, u64, i32, i64 = C.c_void_p, C.c_uint64, C.c_int, C.c_int64
            L.or_apply_flips.argtypes = [vp, i32, u64, i32, vp, i64]
            L.or_field_box.argtypes = [vp, i32, u64, i32, vp, vp]
            L.or_guard.argtypes = [vp, i32, u64, i32, u64, i32, vp, vp, i32, vp]
            L.or_preprocess.argtypes = [vp, i32, u64, i32, vp, i32, i32, vp]
            L.or_bin.argtypes = [vp, u64, i32, i32, vp, vp, u64]
            L.or_bin.restype = i64
            L.or_blend.argtypes = [vp, vp, vp, i32, i32, i32, i32, vp]
            L.or_blend_brute.argtypes = [vp, u64, i32, i32, i32, i32, vp]
            L.or_compare.argtypes = [vp, vp, i32, i32, vp]
            L.or_render.argtypes = [vp, i32, u64, i32, vp, i32, i32, vp]
            L.or_render_margins.argtypes = [vp, i32, u64, i32, vp, i32, i32, vp, vp]
            L.or_campaign.argtypes = [vp, i32, u64, i32, i32, vp, i32, i32, i32, vp, vp, i64, i32, i32,
                                      u64, vp, vp, i32, vp, vp, i32, vp, vp, vp]
            L.or_ssim.argtypes = [vp, vp, i32, i32]
            L.or_ssim.restype = C.c_double
            L.or_region_actual.argtypes = [vp, vp, i32, i32]
            L.or_region_actual.restype = u64
            L.or_region_rect.argtypes = [vp, i32, i32, i32, i32]
            L.or_region_rect.restype = u64
            L.or_sh_basis.argtypes = [C.c_float, C.c_float, C.c_float, i32, vp]
            L.or_exp_f32.argtypes = [vp, vp, i64]
            L.or_ecc_first_bit.argtypes = [i32]
            L.or_ecc_corrects.argtypes = [i32, u64, vp]
            L.or_max_threads.restype = i32
            _lib = L
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p) if a is not None else None


def _c(a, dtype=None):
    return np.ascontiguousarray(a, dtype=dtype) if a is not None else None


def max_threads() -> int:
    return int(lib().or_max_threads())


def apply_flips(planes: np.ndarray, fmt: int, flips: np.ndarray) -> np.ndarray:
    """Return a copy of ``planes`` with every flip XOR-ed in, in list order."""
    out = np.array(planes, copy=True, order="C")
    f = _c(flips)
    rc = lib().or_apply_flips(_p(out), fmt, out.shape[1], out.shape[0], _p(f), len(f))
    if rc != 0:
        raise ValueError("flip site out of range")
    return out


def field_box(planes: np.ndarray, fmt: int):
    """Algorithm 1 precompute: per-word (lo, hi) storage words (uint32 arrays)."""
    p = _c(planes)
    lo = np.zeros(p.shape[0], dtype=np.uint32)
    hi = np.zeros(p.shape[0], dtype=np.uint32)
    lib().or_field_box(_p(p), fmt, p.shape[1], p.shape[0], _p(lo), _p(hi))
    return lo, hi


def guard(planes: np.ndarray, fmt: int, word_mask: int, mode: int, box_lo, box_hi):
    """Algorithm 1 per-frame clamp on a copy; returns (guarded planes, clamp count).
    mode 0 = FIELD (box_lo/hi: uint32[nwords] storage words), 1 = PRIM (planes)."""
    out = np.array(planes, copy=True, order="C")
    lo, hi = _c(box_lo), _c(box_hi)
    nbox = out.shape[0] if mode == 0 else lo.shape[0]
    cnt = np.zeros(1, dtype=np.uint64)
    rc = lib().or_guard(_p(out), fmt, out.shape[1], out.shape[0], word_mask, mode, _p(lo), _p(hi), nbox, _p(cnt))
    if rc != 0:
        raise ValueError("guarded word outside the per-primitive box planes")
    return out, int(cnt[0])


def _cam(cam):
    from paper_2606_21791_gb300.synth import CAMERA_DTYPE  # dtype only (layout of the camera record)
    return np.ascontiguousarray(np.asarray(cam, dtype=CAMERA_DTYPE).reshape(-1))


def preprocess(planes, fmt: int, sh_degree: int, cam, tile=(16, 16)) -> np.ndarray:
    p = _c(planes)
    c = _cam(cam)
    out = np.zeros(p.shape[1], dtype=REC_DTYPE)
    lib().or_preprocess(_p(p), fmt, p.shape[1], sh_degree, _p(c), tile[0], tile[1], _p(out))
    return out


def bin_tiles(recs: np.ndarray, width: int, height: int, tile=(16, 16)):
    """Per-tile lists: (offsets[ntiles+1], ids[total]) sorted front to back."""
    tx = (width + tile[0] - 1) // tile[0]
    ty = (height + tile[1] - 1) // tile[1]
    r = _c(recs)
    vis = r["visible"] != 0
    total = int(((r["x1"] - r["x0"]).astype(np.int64) * (r["y1"] - r["y0"]))[vis].sum())
    offsets = np.zeros(tx * ty + 1, dtype=np.uint32)
    ids = np.zeros(max(total, 1), dtype=np.uint32)
    got = lib().or_bin(_p(r), len(r), tx, ty, _p(offsets), _p(ids), total)
    assert got == total
    return offsets, ids[:total]


def blend(recs, offsets, ids, width: int, height: int, tile=(16, 16)) -> np.ndarray:
    img = np.zeros((height, width, 3), dtype=np.float32)
    r, o, i = _c(recs), _c(offsets), _c(ids)
    if len(i) == 0:
        i = np.zeros(1, dtype=np.uint32)
    lib().or_blend(_p(r), _p(o), _p(i), width, height, tile[0], tile[1], _p(img))
    return img


def blend_brute(recs, width: int, height: int, tile=(16, 16)) -> np.ndarray:
    img = np.zeros((height, width, 3), dtype=np.float32)
    r = _c(recs)
    lib().or_blend_brute(_p(r), len(r), width, height, tile[0], tile[1], _p(img))
    return img


def render(planes, fmt: int, sh_degree: int, cam, tile=(16, 16)) -> np.ndarray:
    c = _cam(cam)
    p = _c(planes)
    img = np.zeros((int(c[0]["height"]), int(c[0]["width"]), 3), dtype=np.float32)
    rc = lib().or_render(_p(p), fmt, p.shape[1], sh_degree, _p(c), tile[0], tile[1], _p(img))
    assert rc == 0
    return img


def render_margins(planes, fmt: int, sh_degree: int, cam, tile=(16, 16)):
    """The render of ``render`` and, per pixel, how close its blend decisions came
    to their thresholds: margins[..., 0] = min |alpha - 1/255| / (1/255) over the
    entries walked, margins[..., 1] = min |T' - 1e-4| / 1e-4 (inf where no entry
    was tested).  Used to attribute footprint differences between two renderers
    whose exponentials round differently."""
    c = _cam(cam)
    p = _c(planes)
    H, W = int(c[0]["height"]), int(c[0]["width"])
    img = np.zeros((H, W, 3), dtype=np.float32)
    mg = np.zeros((H, W, 2), dtype=np.float32)
    rc = lib().or_render_margins(_p(p), fmt, p.shape[1], sh_degree, _p(c), tile[0], tile[1], _p(img), _p(mg))
    assert rc == 0
    return img, mg


def compare(a: np.ndarray, b: np.ndarray) -> np.ndarray:
    a = _c(a, np.float32)
    b = _c(b, np.float32)
    H, W = a.shape[0], a.shape[1]
    out = np.zeros(1, dtype=METRICS_DTYPE)
    lib().or_compare(_p(a), _p(b), H, W, _p(out))
    return out[0]


def campaign(planes, fmt: int, sh_degree: int, cams, flips, flips_per_variant: int = 1,
             guard_mode: int = -1, word_mask: int = (1 << 14) - 1, box_lo=None, box_hi=None,
             clean_imgs=None, tile=(16, 16), nthreads: int = 1, regions: bool = False, ssim: bool = False):
    """Per variant: copy, flip, (guard), render each view, compare with clean.
    guard_mode: -1 off, 0 FIELD box, 1 PRIM boxes, 2 ECC emulation (upsets on
    the sign/exponent bits of the words in word_mask are corrected).
    Returns (metrics[nvar, K], clamps[nvar], clean_imgs); with regions=True also
    the contamination masks (actual[nvar, K], predicted[nvar, K]) over the 8x8
    screen cells; with ssim=True the SSIM of every (variant, view) is appended
    last (ssim[nvar, K])."""
    p = _c(planes)
    c = _cam(cams)
    K = len(c)
    if clean_imgs is None:
        clean_imgs = [render(p, fmt, sh_degree, c[k], tile) for k in range(K)]
    flat = np.ascontiguousarray(np.concatenate([np.asarray(x, np.float32).reshape(-1) for x in clean_imgs]))
    f = _c(flips)
    nvar = len(f) // flips_per_variant
    out = np.zeros(nvar * K, dtype=METRICS_DTYPE)
    clamps = np.zeros(nvar, dtype=np.uint64)
    ra = np.zeros(nvar * K, dtype=np.uint64) if regions else None
    rp = np.zeros(nvar * K, dtype=np.uint64) if regions else None
    ss = np.zeros(nvar * K, dtype=np.float64) if ssim else None
    lo, hi = _c(box_lo), _c(box_hi)
    nbox = 0 if lo is None else (p.shape[0] if guard_mode == 0 else lo.shape[0])
    rc = lib().or_campaign(_p(p), fmt, p.shape[1], p.shape[0], sh_degree, _p(c), K, tile[0], tile[1], _p(flat),
                           _p(f), nvar, flips_per_variant, guard_mode, word_mask, _p(lo), _p(hi), nbox,
                           _p(out), _p(clamps), nthreads, _p(ra), _p(rp), _p(ss))
    if rc != 0:
        raise ValueError("campaign failed (flip site or box out of range)")
    res = (out.reshape(nvar, K), clamps, clean_imgs)
    if regions:
        res += (ra.reshape(nvar, K), rp.reshape(nvar, K))
    if ssim:
        res += (ss.reshape(nvar, K),)
    return res


def ssim(a: np.ndarray, b: np.ndarray) -> float:
    """SSIM of image a against image b (H x W x 3 float32)."""
    a = _c(a, np.float32)
    b = _c(b, np.float32)
    return float(lib().or_ssim(_p(a), _p(b), a.shape[0], a.shape[1]))


def region_actual(a: np.ndarray, b: np.ndarray) -> int:
    """8x8-cell mask of the footprint pixels of image a against image b."""
    a = _c(a, np.float32)
    b = _c(b, np.float32)
    H, W = a.shape[0], a.shape[1]
    return int(lib().or_region_actual(_p(a), _p(b), H, W))


def region_rect(rec, width: int, height: int, tile=(16, 16)) -> int:
    """8x8-cell mask of the pixels a preprocessed record's tile rect covers."""
    r = np.ascontiguousarray(np.asarray(rec, dtype=REC_DTYPE).reshape(1))
    return int(lib().or_region_rect(_p(r), width, height, tile[0], tile[1]))


def ecc_first_bit(fmt: int) -> int:
    """First bit the sign+exponent code protects (fp32 23, fp16 10, bf16 7)."""
    return int(lib().or_ecc_first_bit(fmt))


def ecc_corrects(fmt: int, word_mask: int, flips: np.ndarray) -> np.ndarray:
    """Per flip: corrected by the sign+exponent code over the words in word_mask."""
    f = _c(flips)
    return np.array([bool(lib().or_ecc_corrects(fmt, word_mask, f[i:i + 1].ctypes.data)) for i in range(len(f))])


def exp_f32(x: np.ndarray) -> np.ndarray:
    """The activations' fp32 exponential (Cody-Waite reduction + degree-7 Taylor)."""
    x = _c(x, np.float32)
    y = np.empty_like(x)
    lib().or_exp_f32(_p(x), _p(y), x.size)
    return y


def sh_basis(x: float, y: float, z: float, degree: int = 3) -> np.ndarray:
    Y = np.zeros(16, dtype=np.float32)
    lib().or_sh_basis(x, y, z, degree, _p(Y))
    return Y[: (degree + 1) ** 2]


def psnr(sse: float, npix_channels: int, cap: bool = True) -> float:
    """PSNR = 10 log10(1 / MSE) over H*W*3 channels of [0,1] images; with ``cap``
    the MSE is floored at 1e-10 (100 dB), otherwise MSE = 0 gives +inf."""
    mse = sse / npix_channels
    if cap:
        mse = max(mse, PSNR_MSE_FLOOR)
    elif mse == 0.0:
        return math.inf
    return 10.0 * math.log10(1.0 / mse)
