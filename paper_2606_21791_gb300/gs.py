"""Thin ctypes binding of libgs (include/gs.h).  Argument marshalling only: every
step of the hot path runs in the CUDA kernels of libgs.so.  PyTorch provides
device memory (tensors) and streams; there is no CPU fallback -- if libgs.so is
missing or no CUDA device is present the calls raise.

Functions keep the C names.  Device buffers are passed as torch CUDA tensors
(or raw integer pointers), host buffers as numpy arrays.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

from . import synth

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libgs.so")

GS_OK, GS_ERR_ARG, GS_ERR_OOM, GS_ERR_CUDA, GS_ERR_TIMEOUT, GS_ERR_BUSY, GS_ERR_STATE, GS_ERR_CAPACITY = range(8)
GS_GUARD_OFF, GS_GUARD_FIELD, GS_GUARD_PRIM, GS_GUARD_ECC = -1, 0, 1, 2
STATUS_NAMES = {0: "GS_OK", 1: "GS_ERR_ARG", 2: "GS_ERR_OOM", 3: "GS_ERR_CUDA", 4: "GS_ERR_TIMEOUT",
                5: "GS_ERR_BUSY", 6: "GS_ERR_STATE", 7: "GS_ERR_CAPACITY"}

FLIP_DTYPE = synth.FLIP_DTYPE
CAMERA_DTYPE = synth.CAMERA_DTYPE
RESULT_DTYPE = np.dtype([("sse", "<f8"), ("maxabs", "<f4"), ("footprint", "<u4"), ("nonfinite", "<u4"),
                         ("clamps", "<u4")])
RECORD_DTYPE = np.dtype([
    ("mx", "<f4"), ("my", "<f4"), ("ca", "<f4"), ("cb", "<f4"), ("cc", "<f4"),
    ("r", "<f4"), ("g", "<f4"), ("b", "<f4"), ("opac", "<f4"), ("depth", "<f4"),
    ("x0", "<i4"), ("y0", "<i4"), ("x1", "<i4"), ("y1", "<i4"), ("radius", "<i4"), ("visible", "<i4"),
])
assert RESULT_DTYPE.itemsize == 24 and RECORD_DTYPE.itemsize == 64 and FLIP_DTYPE.itemsize == 8
assert CAMERA_DTYPE.itemsize == 80

# every symbol include/gs.h declares, with (restype, argtypes)
_vp, _u64, _i32, _i64 = C.c_void_p, C.c_uint64, C.c_int, C.c_int64
SIGNATURES = {
    "gs_last_error": (C.c_char_p, []),
    "gs_version": (C.c_char_p, []),
    "gs_load_scene": (_i32, [_vp, _i32, _u64, _i32, _i32, C.POINTER(_vp)]),
    "gs_free_scene": (_i32, [_vp]),
    "gs_scene_info": (_i32, [_vp, _vp, _vp, _vp, _vp]),
    "gs_scene_planes": (_i32, [_vp, C.POINTER(_vp)]),
    "gs_read_planes": (_i32, [_vp, _vp, _i32, _vp]),
    "gs_write_planes": (_i32, [_vp, _vp, _i32, _vp]),
    "gs_scene_errors": (_i32, [_vp, _vp]),
    "gs_apply_flips": (_i32, [_vp, _vp, _i64, _vp]),
    "gs_field_box": (_i32, [_vp, _vp, _vp]),
    "gs_set_prim_box": (_i32, [_vp, _vp, _vp, _i32, _i32]),
    "gs_guard": (_i32, [_vp, _i32, _u64, _vp, _vp]),
    "gs_guard_bitmap": (_i32, [_vp, _i32, _u64, _vp, _vp, _vp]),
    "gs_render": (_i32, [_vp, _vp, _i32, _vp, _vp]),
    "gs_compare": (_i32, [_vp, _vp, _i32, _i32, _i32, _vp, _vp]),
    "gs_compare_noalloc": (_i32, [_vp, _vp, _i32, _i32, _i32, _vp, _vp]),
    "gs_set_views": (_i32, [_vp, _vp, _i32, _vp]),
    "gs_clean_image": (_i32, [_vp, _i32, _vp, _vp]),
    "gs_inject_and_render": (_i32, [_vp, _vp, _i32, _i32, _i32, _u64, _vp, _vp]),
    "gs_inject_and_render_full": (_i32, [_vp, _vp, _i32, _i32, _i32, _u64, _vp, _vp]),
    "gs_inject_and_render_host": (_i32, [_vp, _vp, _i32, _i32, _i32, _u64, _vp, _vp]),
    "gs_inject_and_render_regions": (_i32, [_vp, _vp, _i32, _i32, _u64, _vp, _vp, _vp]),
    "gs_inject_and_render_ex": (_i32, [_vp, _vp, _i32, _i32, _u64, _vp, _vp, _vp, _vp]),
    "gs_ssim": (_i32, [_vp, _vp, _i32, _i32, _i32, _vp, _vp]),
    "gs_set_graphs": (_i32, [_vp, _i32]),
    "gs_set_batch": (_i32, [_vp, _i32]),
    "gs_count_work": (_i32, [_vp, _i32]),
    "gs_time_kernels": (_i32, [_vp, _i32]),
    "gs_read_kernel_ms": (_i32, [_vp, _vp]),
    "gs_read_render_ms": (_i32, [_vp, _vp, _vp]),
    "gs_read_work": (_i32, [_vp, _vp]),
    "gs_autotune": (_i32, [_vp, _vp, _i32, _i32, _u64, _vp, _vp, _vp]),
    "gs_set_tile": (_i32, [_vp, _i32, _i32, _vp]),
    "gs_get_tile": (_i32, [_vp, _vp, _vp]),
    "gs_autotune_tile": (_i32, [_vp, _vp, _i32, _i32, _u64, _vp, _vp, _vp, _vp, _vp]),
    "gs_preprocess": (_i32, [_vp, _vp, _vp, _vp]),
    "gs_bin_tiles": (_i32, [_vp, _vp, _u64, _i32, _i32, _vp, _vp, _u64, _vp, _vp]),
    "gs_blend_lists": (_i32, [_vp, _u64, _vp, _vp, _i32, _i32, _vp, _vp]),
    "gs_server_create": (_i32, [_u64, _i32, C.POINTER(_vp)]),
    "gs_server_add_scene": (_i32, [_vp, _vp, _vp]),
    "gs_server_submit": (_i32, [_vp, _vp, C.c_double, _vp]),
    "gs_server_wait": (_i32, [_vp, _u64, _i32, _vp]),
    "gs_server_cancel": (_i32, [_vp, _u64]),
    "gs_server_stats": (_i32, [_vp, _vp]),
    "gs_server_now": (_i32, [_vp, _vp]),
    "gs_server_destroy": (_i32, [_vp]),
}

GS_REQ_RENDER, GS_REQ_CAMPAIGN, GS_REQ_STORM = 0, 1, 2
REQUEST_DTYPE = np.dtype([("kind", "<i4"), ("scene", "<i4"), ("cam", CAMERA_DTYPE), ("guard_mode", "<i4"),
                          ("nflips", "<i4"), ("word_mask", "<u8"), ("dev_flips", "<u8"), ("dev_rgb", "<u8"),
                          ("dev_results", "<u8"), ("dev_clamps", "<u8")])
RESPONSE_DTYPE = np.dtype([("ticket", "<u8"), ("status", "<i4"), ("slot", "<i4"), ("t_submit_ms", "<f8"),
                           ("t_start_ms", "<f8"), ("t_done_ms", "<f8")])
assert REQUEST_DTYPE.itemsize == 136 and RESPONSE_DTYPE.itemsize == 40

_lock = threading.Lock()
_lib = None


class GsError(RuntimeError):
    def __init__(self, status: int, where: str, msg: str):
        super().__init__(f"{where}: {STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


def load_library(path: str = LIB_PATH) -> C.CDLL:
    """Load libgs.so (built by buildlib.build()); raises if it is absent."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(path):
                raise RuntimeError(f"libgs.so not found at {path}: run __graft_entry__.build() (no CPU fallback)")
            L = C.CDLL(path)
            for name, (res, args) in SIGNATURES.items():
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
            _lib = L
    return _lib


def _check(st: int, where: str):
    if st != GS_OK:
        msg = load_library().gs_last_error()
        raise GsError(st, where, msg.decode() if msg else "")


def _ptr(x):
    """Raw pointer of a torch tensor / numpy array / int / None."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if isinstance(x, np.ndarray):
        assert x.flags["C_CONTIGUOUS"]
        return x.ctypes.data
    if hasattr(x, "data_ptr"):
        assert x.is_contiguous()
        return x.data_ptr()
    raise TypeError(type(x))


def _stream(stream):
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def _cams(cams) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(cams, dtype=CAMERA_DTYPE).reshape(-1))


# ----------------------------------------------------------------------------
# C entry points
# ----------------------------------------------------------------------------
def gs_version() -> str:
    return load_library().gs_version().decode()


def gs_load_scene(planes, n: int, sh_degree: int, fmt: int):
    """planes: numpy [nwords, n] storage bits (host) or torch CUDA tensor (device)."""
    on_dev = not isinstance(planes, np.ndarray)
    if not on_dev:
        planes = np.ascontiguousarray(planes)
    h = C.c_void_p()
    _check(load_library().gs_load_scene(_ptr(planes), int(on_dev), n, sh_degree, fmt, C.byref(h)), "gs_load_scene")
    return h.value


def gs_free_scene(scene):
    _check(load_library().gs_free_scene(scene), "gs_free_scene")


def gs_scene_info(scene):
    n, d, f, w = C.c_uint64(), C.c_int(), C.c_int(), C.c_int()
    _check(load_library().gs_scene_info(scene, C.byref(n), C.byref(d), C.byref(f), C.byref(w)), "gs_scene_info")
    return n.value, d.value, f.value, w.value


def gs_scene_planes(scene) -> int:
    p = C.c_void_p()
    _check(load_library().gs_scene_planes(scene, C.byref(p)), "gs_scene_planes")
    return p.value


def gs_read_planes(scene, dst, stream=None):
    on_dev = not isinstance(dst, np.ndarray)
    _check(load_library().gs_read_planes(scene, _ptr(dst), int(on_dev), _stream(stream)), "gs_read_planes")
    return dst


def gs_write_planes(scene, src, stream=None):
    on_dev = not isinstance(src, np.ndarray)
    if not on_dev:
        src = np.ascontiguousarray(src)
    _check(load_library().gs_write_planes(scene, _ptr(src), int(on_dev), _stream(stream)), "gs_write_planes")


def gs_scene_errors(scene) -> int:
    f = np.zeros(1, dtype=np.uint32)
    _check(load_library().gs_scene_errors(scene, _ptr(f)), "gs_scene_errors")
    return int(f[0])


def gs_apply_flips(scene, dev_flips, count: int, stream=None):
    _check(load_library().gs_apply_flips(scene, _ptr(dev_flips), count, _stream(stream)), "gs_apply_flips")


def gs_field_box(scene, nwords: int):
    lo = np.zeros(nwords, dtype=np.uint32)
    hi = np.zeros(nwords, dtype=np.uint32)
    _check(load_library().gs_field_box(scene, _ptr(lo), _ptr(hi)), "gs_field_box")
    return lo, hi


def gs_set_prim_box(scene, lo, hi, nbox_words: int):
    on_dev = not isinstance(lo, np.ndarray)
    if not on_dev:
        lo, hi = np.ascontiguousarray(lo), np.ascontiguousarray(hi)
    _check(load_library().gs_set_prim_box(scene, _ptr(lo), _ptr(hi), int(on_dev), nbox_words), "gs_set_prim_box")


def gs_guard(scene, mode: int, word_mask: int, dev_clamps=None, stream=None):
    _check(load_library().gs_guard(scene, mode, word_mask, _ptr(dev_clamps), _stream(stream)), "gs_guard")


def gs_guard_bitmap(scene, mode: int, word_mask: int, dev_bitmap, dev_clamps=None, stream=None):
    """gs_guard plus the bitmap of clamped words (device uint32[nwords * ceil(n / 32)])."""
    _check(load_library().gs_guard_bitmap(scene, mode, word_mask, _ptr(dev_clamps), _ptr(dev_bitmap),
                                          _stream(stream)), "gs_guard_bitmap")


def gs_render(scene, cams, dev_rgb, stream=None):
    c = _cams(cams)
    _check(load_library().gs_render(scene, _ptr(c), len(c), _ptr(dev_rgb), _stream(stream)), "gs_render")


def gs_compare(dev_a, dev_b, H: int, W: int, K: int, dev_out, stream=None):
    _check(load_library().gs_compare(_ptr(dev_a), _ptr(dev_b), H, W, K, _ptr(dev_out), _stream(stream)), "gs_compare")


def gs_compare_noalloc(dev_a, dev_b, H: int, W: int, K: int, dev_out, stream=None):
    """gs_compare without any device allocation (fixed 64-pair scratch in the library)."""
    _check(load_library().gs_compare_noalloc(_ptr(dev_a), _ptr(dev_b), H, W, K, _ptr(dev_out), _stream(stream)),
           "gs_compare_noalloc")


def gs_set_views(scene, cams, stream=None):
    c = _cams(cams)
    _check(load_library().gs_set_views(scene, _ptr(c), len(c), _stream(stream)), "gs_set_views")


def gs_clean_image(scene, k: int, dev_rgb, stream=None):
    _check(load_library().gs_clean_image(scene, k, _ptr(dev_rgb), _stream(stream)), "gs_clean_image")


def gs_inject_and_render(scene, dev_flips, B: int, flips_per_variant: int, guard_mode: int, word_mask: int,
                         dev_out, stream=None):
    _check(load_library().gs_inject_and_render(scene, _ptr(dev_flips), B, flips_per_variant, guard_mode, word_mask,
                                               _ptr(dev_out), _stream(stream)), "gs_inject_and_render")


def gs_inject_and_render_regions(scene, dev_flips, B: int, guard_mode: int, word_mask: int, dev_out,
                                 dev_regions, stream=None):
    """dev_regions: device buffer of B*K*2 uint64 ([actual, predicted] cell masks)."""
    _check(load_library().gs_inject_and_render_regions(scene, _ptr(dev_flips), B, guard_mode, word_mask,
                                                       _ptr(dev_out), _ptr(dev_regions), _stream(stream)),
           "gs_inject_and_render_regions")


def gs_inject_and_render_ex(scene, dev_flips, B: int, guard_mode: int, word_mask: int, dev_out, dev_regions=None,
                            dev_ssim=None, stream=None):
    """Single-flip campaign with optional region masks (B*K*2 uint64) and SSIM (B*K float64)."""
    _check(load_library().gs_inject_and_render_ex(scene, _ptr(dev_flips), B, guard_mode, word_mask, _ptr(dev_out),
                                                  _ptr(dev_regions), _ptr(dev_ssim), _stream(stream)),
           "gs_inject_and_render_ex")


def gs_ssim(dev_test, dev_clean, H: int, W: int, K: int, dev_out, stream=None):
    """SSIM of K image pairs into dev_out (K float64, device)."""
    _check(load_library().gs_ssim(_ptr(dev_test), _ptr(dev_clean), H, W, K, _ptr(dev_out), _stream(stream)), "gs_ssim")


def gs_inject_and_render_host(scene, host_flips, B: int, flips_per_variant: int, guard_mode: int, word_mask: int,
                              host_out, stream=None):
    """Host buffers in and out (numpy arrays or pinned torch CPU tensors);
    returns after the records are in host_out."""
    _check(load_library().gs_inject_and_render_host(scene, _ptr(host_flips), B, flips_per_variant, guard_mode,
                                                    word_mask, _ptr(host_out), _stream(stream)),
           "gs_inject_and_render_host")


def gs_inject_and_render_full(scene, dev_flips, B: int, flips_per_variant: int, guard_mode: int, word_mask: int,
                              dev_out, stream=None):
    _check(load_library().gs_inject_and_render_full(scene, _ptr(dev_flips), B, flips_per_variant, guard_mode,
                                                    word_mask, _ptr(dev_out), _stream(stream)),
           "gs_inject_and_render_full")


def gs_set_graphs(scene, enable: bool):
    _check(load_library().gs_set_graphs(scene, int(bool(enable))), "gs_set_graphs")


def gs_count_work(scene, enable: bool):
    _check(load_library().gs_count_work(scene, int(bool(enable))), "gs_count_work")


def gs_read_work(scene):
    c = np.zeros(16, dtype=np.uint64)
    _check(load_library().gs_read_work(scene, _ptr(c)), "gs_read_work")
    return {"evaluations": int(c[0]), "tiles": int(c[1]), "entries": int(c[2]), "tiles_unchanged": int(c[3]),
            "dropped_stop_key": int(c[4]), "dropped_tile_reach": int(c[5]), "dropped_no_reach": int(c[6]),
            "dropped_pixel_stop": int(c[7]), "warp_steps": int(c[8]), "warp_steps_blending": int(c[9]),
            "blocks_blended": int(c[10]), "cycles_setup": int(c[11]), "cycles_walk": int(c[12]),
            "cycles_compare": int(c[13]), "active_pixels": int(c[14]), "active_pixel_steps": int(c[15])}


def gs_time_kernels(scene, enable: bool):
    _check(load_library().gs_time_kernels(scene, int(bool(enable))), "gs_time_kernels")


def gs_read_kernel_ms(scene):
    """(plan kernel ms, blend + compare kernel ms) of the last dirty-tile batch."""
    ms = (C.c_float * 2)()
    _check(load_library().gs_read_kernel_ms(scene, ms), "gs_read_kernel_ms")
    return float(ms[0]), float(ms[1])


def gs_read_render_ms(scene):
    """Stage times of the last view of the last gs_render (kernel timing on):
    ((preprocess ms, binning + sort ms, blend ms),
     (primitives, tile pairs, depth-key radix passes, pair radix passes))."""
    ms = (C.c_float * 3)()
    counts = (C.c_uint64 * 4)()
    _check(load_library().gs_read_render_ms(scene, ms, counts), "gs_read_render_ms")
    return tuple(float(x) for x in ms), tuple(int(x) for x in counts)


def gs_set_batch(scene, batch: int):
    _check(load_library().gs_set_batch(scene, batch), "gs_set_batch")


def gs_autotune(scene, dev_flips, count: int, guard_mode: int, word_mask: int, stream=None):
    b = C.c_int()
    us = C.c_float()
    _check(load_library().gs_autotune(scene, _ptr(dev_flips), count, guard_mode, word_mask, C.byref(b), C.byref(us),
                                      _stream(stream)), "gs_autotune")
    return b.value, us.value


def gs_set_tile(scene, tile_w: int, tile_h: int, stream=None):
    _check(load_library().gs_set_tile(scene, tile_w, tile_h, _stream(stream)), "gs_set_tile")


def gs_get_tile(scene):
    w, h = C.c_int(), C.c_int()
    _check(load_library().gs_get_tile(scene, C.byref(w), C.byref(h)), "gs_get_tile")
    return w.value, h.value


def gs_autotune_tile(scene, dev_flips, count: int, guard_mode: int, word_mask: int, stream=None):
    """Returns ((tile_w, tile_h), batch, us per variant) the scene now uses."""
    tw, th, b = C.c_int(), C.c_int(), C.c_int()
    us = C.c_float()
    _check(load_library().gs_autotune_tile(scene, _ptr(dev_flips), count, guard_mode, word_mask, C.byref(tw),
                                           C.byref(th), C.byref(b), C.byref(us), _stream(stream)), "gs_autotune_tile")
    return (tw.value, th.value), b.value, us.value


def gs_preprocess(scene, cam, dev_out, stream=None):
    c = _cams(cam)
    _check(load_library().gs_preprocess(scene, _ptr(c), _ptr(dev_out), _stream(stream)), "gs_preprocess")


def gs_bin_tiles(dev_depth, dev_rects, n: int, tiles_x: int, tiles_y: int, dev_offsets, dev_ids, ids_cap: int,
                 stream=None) -> int:
    total = np.zeros(1, dtype=np.uint64)
    _check(load_library().gs_bin_tiles(_ptr(dev_depth), _ptr(dev_rects), n, tiles_x, tiles_y, _ptr(dev_offsets),
                                       _ptr(dev_ids), ids_cap, _ptr(total), _stream(stream)), "gs_bin_tiles")
    return int(total[0])


def gs_blend_lists(dev_recs, n: int, dev_offsets, dev_ids, W: int, H: int, dev_rgb, stream=None):
    _check(load_library().gs_blend_lists(_ptr(dev_recs), n, _ptr(dev_offsets), _ptr(dev_ids), W, H, _ptr(dev_rgb),
                                         _stream(stream)), "gs_blend_lists")


def gs_server_create(hbm_budget_bytes: int, slots: int):
    h = C.c_void_p()
    _check(load_library().gs_server_create(hbm_budget_bytes, slots, C.byref(h)), "gs_server_create")
    return h.value


def gs_server_add_scene(server, scene) -> int:
    sid = np.zeros(1, dtype=np.int32)
    _check(load_library().gs_server_add_scene(server, scene, _ptr(sid)), "gs_server_add_scene")
    return int(sid[0])


def make_request(kind: int, scene: int, cam=None, guard_mode: int = -1, word_mask: int = 0, dev_flips=None,
                 nflips: int = 0, dev_rgb=None, dev_results=None, dev_clamps=None) -> np.ndarray:
    r = np.zeros(1, dtype=REQUEST_DTYPE)
    r["kind"], r["scene"], r["guard_mode"], r["nflips"], r["word_mask"] = kind, scene, guard_mode, nflips, word_mask
    if cam is not None:
        r["cam"] = np.asarray(cam, dtype=CAMERA_DTYPE)
    for f, v in (("dev_flips", dev_flips), ("dev_rgb", dev_rgb), ("dev_results", dev_results),
                 ("dev_clamps", dev_clamps)):
        r[f] = _ptr(v) or 0
    return r


def gs_server_submit(server, request: np.ndarray, arrival_ms: float = -1.0) -> int:
    t = np.zeros(1, dtype=np.uint64)
    _check(load_library().gs_server_submit(server, _ptr(request), arrival_ms, _ptr(t)), "gs_server_submit")
    return int(t[0])


def gs_server_wait(server, ticket: int, timeout_ms: int = -1):
    r = np.zeros(1, dtype=RESPONSE_DTYPE)
    _check(load_library().gs_server_wait(server, ticket, timeout_ms, _ptr(r)), "gs_server_wait")
    return r[0]


def gs_server_cancel(server, ticket: int):
    _check(load_library().gs_server_cancel(server, ticket), "gs_server_cancel")


def gs_server_stats(server) -> dict:
    st = np.zeros(6, dtype=np.uint64)
    _check(load_library().gs_server_stats(server, _ptr(st)), "gs_server_stats")
    return dict(zip(("budget", "resident", "scratch", "queued", "completed", "mem_delayed"), (int(x) for x in st)))


def gs_server_now(server) -> float:
    t = np.zeros(1, dtype=np.float64)
    _check(load_library().gs_server_now(server, _ptr(t)), "gs_server_now")
    return float(t[0])


def gs_server_destroy(server):
    _check(load_library().gs_server_destroy(server), "gs_server_destroy")


# ----------------------------------------------------------------------------
# small helpers for torch buffers of C structs
# ----------------------------------------------------------------------------
def device_bytes(nbytes: int, device="cuda"):
    import torch
    return torch.empty(max(int(nbytes), 1), dtype=torch.uint8, device=device)


def to_device(arr: np.ndarray, device="cuda"):
    import torch
    a = np.ascontiguousarray(arr)
    t = torch.from_numpy(a.view(np.uint8).reshape(-1).copy())
    return t.to(device)


def from_device(t, dtype) -> np.ndarray:
    return t.cpu().numpy().view(dtype)
