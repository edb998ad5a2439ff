"""Seeded synthetic inputs: 3DGS scenes, pinhole cameras, upset lists, guard boxes.

This module is the one place that both the CUDA path's tests/benchmark and the
CPU oracle's tests draw their inputs from.  It holds random draws and input
shaping only -- none of the method's arithmetic (no injection, no guard, no
projection, no blending, no metric).

Parameter layout (Sec. 3 "Parameter layout"): a primitive stores, in
optimisation space, mean (3), logarithmic scale (3), quaternion (4, w first),
opacity logit (1), SH DC colour (3) and the higher-order SH coefficients
((l+1)^2 - 1) x 3, coefficient-major.  At SH degree 3 that is 59 words per
primitive, at degree 0 it is 14.  Scenes are held as structure-of-arrays planes
``planes[word, prim]`` in the storage format (fp32 / fp16 / bf16 bits).

Value distributions follow the workloads the study runs on (trained synthetic
scenes of 6.7k to 2M primitives, replicated up to 66M): means uniform in a cube
or in Gaussian clusters, log-scales N(-4.5, 1), quaternions normalised from
N(0,1)^4, opacity logits N(0, 2), DC colour N(0, 0.5), higher-order SH N(0, 0.05)
(second arguments are standard deviations).
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

FP32, FP16, BF16 = 0, 1, 2
FORMAT_NAMES = {FP32: "fp32", FP16: "fp16", BF16: "bf16"}
FORMAT_BITS = {FP32: 32, FP16: 16, BF16: 16}
FORMAT_DTYPE = {FP32: np.uint32, FP16: np.uint16, BF16: np.uint16}

# word map: 0-2 mean, 3-5 log-scale, 6-9 quaternion (w,x,y,z), 10 opacity logit,
# 11-13 SH DC, 14.. higher-order SH (coefficient-major, 3 channels each)
FIELDS = {
    "mean": (0, 3),
    "log_scale": (3, 6),
    "rotation": (6, 10),
    "opacity": (10, 11),
    "sh_dc": (11, 14),
    "sh_rest": (14, 59),
}
GUARD_WORDS_DEFAULT = (1 << 14) - 1          # the 14 non-SH-rest words
GUARD_WORDS_SELECTIVE = (0b111 << 3) | (1 << 10)  # log-scale + opacity only

FLIP_DTYPE = np.dtype([("prim", "<u4"), ("word", "<u2"), ("bit", "u1"), ("pad", "u1")])

CAMERA_DTYPE = np.dtype([
    ("R", "<f4", (9,)), ("t", "<f4", (3,)),
    ("fx", "<f4"), ("fy", "<f4"), ("cx", "<f4"), ("cy", "<f4"),
    ("width", "<i4"), ("height", "<i4"), ("znear", "<f4"), ("zfar", "<f4"),
])


def words_for_degree(sh_degree: int) -> int:
    return 14 + ((sh_degree + 1) ** 2 - 1) * 3


# ----------------------------------------------------------------------------
# storage-format encoding of generated fp32 values (round to nearest even)
# ----------------------------------------------------------------------------
def f32_to_bf16_bits(x: np.ndarray) -> np.ndarray:
    u = np.ascontiguousarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    nan = np.isnan(np.asarray(x, dtype=np.float32))
    lsb = (u >> 16) & 1
    r = ((u + 0x7FFF + lsb) >> 16).astype(np.uint16)
    r[nan] = ((u[nan] >> 16) | 0x40).astype(np.uint16)
    return r


def bf16_bits_to_f32(b: np.ndarray) -> np.ndarray:
    return (np.asarray(b, dtype=np.uint32) << 16).view(np.float32)


def encode(values_f32: np.ndarray, fmt: int) -> np.ndarray:
    v = np.ascontiguousarray(values_f32, dtype=np.float32)
    if fmt == FP32:
        return v.view(np.uint32).copy()
    if fmt == FP16:
        return v.astype(np.float16).view(np.uint16).copy()
    if fmt == BF16:
        return f32_to_bf16_bits(v)
    raise ValueError(fmt)


def decode(bits: np.ndarray, fmt: int) -> np.ndarray:
    """Exact up-conversion of storage words to float32 (used by tests)."""
    if fmt == FP32:
        return np.asarray(bits, dtype=np.uint32).view(np.float32)
    if fmt == FP16:
        return np.asarray(bits, dtype=np.uint16).view(np.float16).astype(np.float32)
    if fmt == BF16:
        return bf16_bits_to_f32(bits)
    raise ValueError(fmt)


def _step_bits(bits: np.ndarray, fmt: int, up: bool) -> np.ndarray:
    """Next representable storage value toward +inf (up) or -inf (sign-magnitude order)."""
    width = FORMAT_BITS[fmt]
    sign = np.int64(1) << (width - 1)
    b = bits.astype(np.int64)
    key = np.where(b & sign, -(b & (sign - 1)), b & (sign - 1))
    key = key + (1 if up else -1)
    out = np.where(key >= 0, key, sign | (-key))
    return out.astype(FORMAT_DTYPE[fmt])


def _round_directed(x64: np.ndarray, fmt: int, down: bool) -> np.ndarray:
    """Round float64 values into the storage format toward -inf (down) or +inf."""
    shape = x64.shape
    x = x64.reshape(-1)
    enc = encode(x.astype(np.float32), fmt)
    for _ in range(4):
        val = decode(enc, fmt).astype(np.float64)
        bad = (val > x) if down else (val < x)
        if not np.any(bad):
            break
        enc[bad] = _step_bits(enc[bad], fmt, up=not down)
    return enc.reshape(shape)


# ----------------------------------------------------------------------------
# scenes
# ----------------------------------------------------------------------------
@dataclass
class Scene:
    planes: np.ndarray        # [nwords, n] storage bits (uint32 or uint16)
    fmt: int
    sh_degree: int

    @property
    def n(self) -> int:
        return int(self.planes.shape[1])

    @property
    def nwords(self) -> int:
        return int(self.planes.shape[0])

    def values(self) -> np.ndarray:
        return decode(self.planes, self.fmt)


def scene_values(n: int, sh_degree: int, seed: int, layout: str = "cube",
                 clusters: int = 4, cube: float = 5.0, centre_box: float = 3.0) -> np.ndarray:
    """Float32 parameter planes [nwords, n] drawn from the workload recipe.

    layout "cube": means uniform in [-cube, cube]^3.
    layout "clusters": ``clusters`` centres uniform in [-centre_box, centre_box]^3,
    primitive i belongs to cluster (i * clusters) // n, mean = centre + N(0, 1).
    """
    rng = np.random.default_rng(seed)
    nw = words_for_degree(sh_degree)
    v = np.empty((nw, n), dtype=np.float32)
    if layout == "cube":
        v[0:3] = rng.uniform(-cube, cube, size=(3, n))
    elif layout == "clusters":
        centres = rng.uniform(-centre_box, centre_box, size=(clusters, 3))
        cid = (np.arange(n, dtype=np.int64) * clusters) // max(n, 1)
        v[0:3] = (centres[cid] + rng.standard_normal((n, 3))).T
    else:
        raise ValueError(layout)
    v[3:6] = rng.normal(-4.5, 1.0, size=(3, n))
    q = rng.standard_normal((4, n))
    q /= np.linalg.norm(q, axis=0, keepdims=True)
    v[6:10] = q
    v[10] = rng.normal(0.0, 2.0, size=n)
    v[11:14] = rng.normal(0.0, 0.5, size=(3, n))
    if nw > 14:
        v[14:] = rng.normal(0.0, 0.05, size=(nw - 14, n))
    return v


def make_scene(n: int, sh_degree: int, fmt: int, seed: int, layout: str = "cube", **kw) -> Scene:
    vals = scene_values(n, sh_degree, seed, layout, **kw)
    return Scene(planes=encode(vals, fmt), fmt=fmt, sh_degree=sh_degree)


def make_scene_torch(n: int, sh_degree: int, fmt: int, seed: int, device="cuda", clusters: int = 4):
    """Clustered scene generated with torch's seeded generator on ``device``.

    Used for the multi-million-primitive workloads, where drawing on the host
    would dominate the run.  Same recipe as ``scene_values(layout="clusters")``
    (different random stream).  Returns a [nwords, n] tensor of storage bits
    (int32 for fp32 storage, int16 for fp16/bf16)."""
    import torch
    g = torch.Generator(device=device)
    g.manual_seed(seed)
    nw = words_for_degree(sh_degree)
    v = torch.empty((nw, n), dtype=torch.float32, device=device)
    centres = (torch.rand((clusters, 3), generator=g, device=device) * 2 - 1) * 3.0
    cid = (torch.arange(n, device=device, dtype=torch.int64) * clusters) // max(n, 1)
    v[0:3] = (centres[cid] + torch.randn((n, 3), generator=g, device=device)).T
    v[3:6] = torch.randn((3, n), generator=g, device=device) * 1.0 - 4.5
    q = torch.randn((4, n), generator=g, device=device)
    v[6:10] = q / q.norm(dim=0, keepdim=True)
    v[10] = torch.randn(n, generator=g, device=device) * 2.0
    v[11:14] = torch.randn((3, n), generator=g, device=device) * 0.5
    if nw > 14:
        v[14:] = torch.randn((nw - 14, n), generator=g, device=device) * 0.05
    if fmt == FP32:
        return v.view(torch.int32)
    if fmt == FP16:
        return v.to(torch.float16).view(torch.int16)
    return v.to(torch.bfloat16).view(torch.int16)


# ----------------------------------------------------------------------------
# cameras (world -> camera rotation R, translation t; x right, y down, z forward)
# ----------------------------------------------------------------------------
def look_at_camera(eye, target=(0.0, 0.0, 0.0), up=(0.0, 1.0, 0.0), width=256, height=256,
                   fov_x_deg=60.0, znear=0.01, zfar=1e10) -> np.ndarray:
    eye = np.asarray(eye, dtype=np.float64)
    f = np.asarray(target, dtype=np.float64) - eye
    f /= np.linalg.norm(f)
    r = np.cross(f, np.asarray(up, dtype=np.float64))
    r /= np.linalg.norm(r)
    d = np.cross(f, r)
    R = np.stack([r, d, f])
    t = -R @ eye
    focal = (width / 2.0) / math.tan(math.radians(fov_x_deg) / 2.0)
    cam = np.zeros((), dtype=CAMERA_DTYPE)
    cam["R"] = R.reshape(-1)
    cam["t"] = t
    cam["fx"] = focal
    cam["fy"] = focal
    cam["cx"] = width / 2.0
    cam["cy"] = height / 2.0
    cam["width"] = width
    cam["height"] = height
    cam["znear"] = znear
    cam["zfar"] = zfar
    return cam


def ring_cameras(k: int, width: int, height: int, distance: float = 15.0, elevation_deg: float = 0.0,
                 fov_x_deg: float = 60.0) -> np.ndarray:
    """``k`` views on a ring around the origin, evenly spaced in azimuth."""
    cams = np.zeros(k, dtype=CAMERA_DTYPE)
    el = math.radians(elevation_deg)
    for i in range(k):
        az = 2.0 * math.pi * i / k
        eye = (distance * math.cos(el) * math.sin(az), distance * math.sin(el),
               distance * math.cos(el) * math.cos(az))
        cams[i] = look_at_camera(eye, width=width, height=height, fov_x_deg=fov_x_deg)
    return cams


# ----------------------------------------------------------------------------
# upset lists
# ----------------------------------------------------------------------------
_FIVE_FIELDS = ("mean", "log_scale", "rotation", "opacity", "sh_dc")


def flips_uniform_fields(count: int, n: int, fmt: int, seed: int) -> np.ndarray:
    """Field uniform over the five non-SH-rest fields, then component, primitive, bit."""
    rng = np.random.default_rng(seed)
    out = np.zeros(count, dtype=FLIP_DTYPE)
    nbits = FORMAT_BITS[fmt]
    for i in range(count):
        f = _FIVE_FIELDS[rng.integers(0, len(_FIVE_FIELDS))]
        a, b = FIELDS[f]
        out[i]["word"] = a + rng.integers(0, b - a)
        out[i]["prim"] = rng.integers(0, n)
        out[i]["bit"] = rng.integers(0, nbits)
    return out


def flips_stratified(count: int, n: int, nwords: int, fmt: int, seed: int) -> np.ndarray:
    """Exhaustive campaign stratified over every (word, bit) cell.

    Each of the nwords * nbits cells receives floor(count / cells) upsets, the
    remainder going to cells in (word, bit) index order; the primitive of each
    upset is uniform.  The list is returned in cell order."""
    rng = np.random.default_rng(seed)
    nbits = FORMAT_BITS[fmt]
    cells = nwords * nbits
    per, rem = divmod(count, cells)
    reps = np.full(cells, per, dtype=np.int64)
    reps[:rem] += 1
    cell = np.repeat(np.arange(cells, dtype=np.int64), reps)
    out = np.zeros(count, dtype=FLIP_DTYPE)
    out["word"] = cell // nbits
    out["bit"] = cell % nbits
    out["prim"] = rng.integers(0, n, size=count)
    return out


def flips_top_bits(count: int, n: int, nwords: int, seed: int, frac_top: float = 0.7) -> np.ndarray:
    """fp32 list: ``frac_top`` of the upsets on bits 24-31 of log-scale (3-5) and
    opacity (10); the rest uniform over every word and bit.  Shuffled."""
    rng = np.random.default_rng(seed)
    out = np.zeros(count, dtype=FLIP_DTYPE)
    ntop = int(round(count * frac_top))
    top_words = np.array([3, 4, 5, 10], dtype=np.int64)
    out["word"][:ntop] = top_words[rng.integers(0, 4, size=ntop)]
    out["bit"][:ntop] = rng.integers(24, 32, size=ntop)
    out["word"][ntop:] = rng.integers(0, nwords, size=count - ntop)
    out["bit"][ntop:] = rng.integers(0, 32, size=count - ntop)
    out["prim"] = rng.integers(0, n, size=count)
    return out[rng.permutation(count)]


def flips_multi(k: int, n: int, nwords: int, fmt: int, seed: int) -> np.ndarray:
    """k distinct sites drawn without replacement over the whole stored bit budget."""
    rng = np.random.default_rng(seed)
    nbits = FORMAT_BITS[fmt]
    total = n * nwords * nbits
    sites = rng.choice(total, size=k, replace=False) if total < 2**62 else None
    out = np.zeros(k, dtype=FLIP_DTYPE)
    out["bit"] = sites % nbits
    sites //= nbits
    out["word"] = sites % nwords
    out["prim"] = sites // nwords
    return out


def flips_at(prim, word, bit) -> np.ndarray:
    prim = np.atleast_1d(prim)
    out = np.zeros(prim.shape[0], dtype=FLIP_DTYPE)
    out["prim"] = prim
    out["word"] = word
    out["bit"] = bit
    return out


# ----------------------------------------------------------------------------
# per-primitive guard boxes  [v - u1 * w, v + u2 * w],  w = 0.2 * |field range|
# ----------------------------------------------------------------------------
def prim_boxes(scene: Scene, nbox_words: int, seed: int, width_frac: float = 0.2):
    """Per-primitive, per-component boxes for words [0, nbox_words).

    u1, u2 ~ U(0,1) independently per (primitive, component); w is width_frac
    times the component's range over the clean scene.  Endpoints are rounded
    outward in the storage format (lo toward -inf, hi toward +inf) so that the
    clean value stays inside its box.  Returns (lo, hi) storage-bit planes."""
    rng = np.random.default_rng(seed)
    v = scene.values()[:nbox_words].astype(np.float64)
    rngw = width_frac * (v.max(axis=1, keepdims=True) - v.min(axis=1, keepdims=True))
    u1 = rng.uniform(0.0, 1.0, size=v.shape)
    u2 = rng.uniform(0.0, 1.0, size=v.shape)
    lo = _round_directed(v - u1 * rngw, scene.fmt, down=True)
    hi = _round_directed(v + u2 * rngw, scene.fmt, down=False)
    return lo, hi


# ----------------------------------------------------------------------------
# named workloads
# ----------------------------------------------------------------------------
SEED_BASE = 20261202


def tiny_workload():
    """5,000 primitives in a cube, SH degree 0, fp32, one 256x256 view at distance
    15 with 60 deg horizontal FOV, 200 upsets over the five non-SH-rest fields."""
    scene = make_scene(5000, 0, FP32, SEED_BASE + 0, layout="cube")
    cams = ring_cameras(1, 256, 256)
    flips = flips_uniform_fields(200, scene.n, FP32, SEED_BASE + 100)
    return scene, cams, flips


def scale_workload(n: int = 2_000_000, count: int = 20_000, width: int = 1600, height: int = 1040, views: int = 4):
    """2,000,000 primitives in 4 clusters, SH degree 3, fp32, four 1600x1040 views
    on a ring (90 deg apart, elevation 0), 20,000 upsets with 70% on bits 24-31 of
    log-scale and opacity."""
    scene = make_scene(n, 3, FP32, SEED_BASE + 2, layout="clusters")
    cams = ring_cameras(views, width, height)
    flips = flips_top_bits(count, scene.n, scene.nwords, SEED_BASE + 102)
    return scene, cams, flips


def prim_boxes_torch(planes, fmt: int, nbox_words: int, seed: int, width_frac: float = 0.2):
    """Device version of ``prim_boxes`` for fp32 storage (multi-million-primitive
    workloads): returns (lo, hi) int32 tensors [nbox_words, n] of storage bits."""
    import torch
    assert fmt == FP32
    v = planes[:nbox_words].view(torch.float32)
    g = torch.Generator(device=v.device)
    g.manual_seed(seed)
    lo = torch.empty_like(v)
    hi = torch.empty_like(v)
    for w in range(nbox_words):
        x = v[w].double()
        wdt = width_frac * (x.max() - x.min())
        l64 = x - torch.rand(x.shape, generator=g, device=v.device, dtype=torch.float64) * wdt
        h64 = x + torch.rand(x.shape, generator=g, device=v.device, dtype=torch.float64) * wdt
        l32 = l64.float()
        h32 = h64.float()
        l32 = torch.where(l32.double() > l64, torch.nextafter(l32, torch.full_like(l32, -float("inf"))), l32)
        h32 = torch.where(h32.double() < h64, torch.nextafter(h32, torch.full_like(h32, float("inf"))), h32)
        lo[w] = l32
        hi[w] = h32
    return lo.view(torch.int32).contiguous(), hi.view(torch.int32).contiguous()


def batching_workload(fmt: int, n: int = 134_826, count: int = 50_000):
    """134,826 primitives in 4 clusters, SH degree 3, one 800x800 view, campaign
    stratified over all 59 words and every bit of the format."""
    scene = make_scene(n, 3, fmt, SEED_BASE + 1, layout="clusters")
    cams = ring_cameras(1, 800, 800)
    flips = flips_stratified(count, scene.n, scene.nwords, fmt, SEED_BASE + 101 + fmt)
    return scene, cams, flips
