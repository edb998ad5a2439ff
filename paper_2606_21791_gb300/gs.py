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
GS_GUARD_OFF, GS_GUARD_FIELD, GS_GUARD_PRIM = -1, 0, 1
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
    "gs_scene_errors": (_i32, [_vp, _vp]),
    "gs_apply_flips": (_i32, [_vp, _vp, _i64, _vp]),
    "gs_field_box": (_i32, [_vp, _vp, _vp]),
    "gs_set_prim_box": (_i32, [_vp, _vp, _vp, _i32, _i32]),
    "gs_guard": (_i32, [_vp, _i32, _u64, _vp, _vp]),
    "gs_render": (_i32, [_vp, _vp, _i32, _vp, _vp]),
    "gs_compare": (_i32, [_vp, _vp, _i32, _i32, _i32, _vp, _vp]),
    "gs_set_views": (_i32, [_vp, _vp, _i32, _vp]),
    "gs_clean_image": (_i32, [_vp, _i32, _vp, _vp]),
    "gs_inject_and_render": (_i32, [_vp, _vp, _i32, _i32, _i32, _u64, _vp, _vp]),
    "gs_inject_and_render_full": (_i32, [_vp, _vp, _i32, _i32, _i32, _u64, _vp, _vp]),
    "gs_set_graphs": (_i32, [_vp, _i32]),
    "gs_preprocess": (_i32, [_vp, _vp, _vp, _vp]),
    "gs_bin_tiles": (_i32, [_vp, _vp, _u64, _i32, _i32, _vp, _vp, _u64, _vp, _vp]),
    "gs_blend_lists": (_i32, [_vp, _u64, _vp, _vp, _i32, _i32, _vp, _vp]),
}

_lock = threading.Lock()
_lib = None


class GsError(RuntimeError):
    def __init__(self, status: int, where: str, msg: str):
        super().__init__(f"{where}: {STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


def load_library(path: str = LIB_PATH) -> C.CDLL:
    """Load libgs.so (built by build.py); raises if it is absent."""
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


def gs_render(scene, cams, dev_rgb, stream=None):
    c = _cams(cams)
    _check(load_library().gs_render(scene, _ptr(c), len(c), _ptr(dev_rgb), _stream(stream)), "gs_render")


def gs_compare(dev_a, dev_b, H: int, W: int, K: int, dev_out, stream=None):
    _check(load_library().gs_compare(_ptr(dev_a), _ptr(dev_b), H, W, K, _ptr(dev_out), _stream(stream)), "gs_compare")


def gs_set_views(scene, cams, stream=None):
    c = _cams(cams)
    _check(load_library().gs_set_views(scene, _ptr(c), len(c), _stream(stream)), "gs_set_views")


def gs_clean_image(scene, k: int, dev_rgb, stream=None):
    _check(load_library().gs_clean_image(scene, k, _ptr(dev_rgb), _stream(stream)), "gs_clean_image")


def gs_inject_and_render(scene, dev_flips, B: int, flips_per_variant: int, guard_mode: int, word_mask: int,
                         dev_out, stream=None):
    _check(load_library().gs_inject_and_render(scene, _ptr(dev_flips), B, flips_per_variant, guard_mode, word_mask,
                                               _ptr(dev_out), _stream(stream)), "gs_inject_and_render")


def gs_inject_and_render_full(scene, dev_flips, B: int, flips_per_variant: int, guard_mode: int, word_mask: int,
                              dev_out, stream=None):
    _check(load_library().gs_inject_and_render_full(scene, _ptr(dev_flips), B, flips_per_variant, guard_mode,
                                                    word_mask, _ptr(dev_out), _stream(stream)),
           "gs_inject_and_render_full")


def gs_set_graphs(scene, enable: bool):
    _check(load_library().gs_set_graphs(scene, int(bool(enable))), "gs_set_graphs")


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
