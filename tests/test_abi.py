"""The C-ABI library loads and exports every symbol include/gs.h declares
(no compute calls: runs without a GPU)."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "gs.h")).read()
    return sorted(set(re.findall(r"GS_API\s+[\w\s\*]+?\b(gs_\w+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    import paper_2606_21791_gb300 as P
    P.build()
    from paper_2606_21791_gb300 import gs
    return gs.load_library()


def test_header_declares_the_boundary():
    names = _declared()
    for required in ("gs_load_scene", "gs_inject_and_render", "gs_guard", "gs_compare", "gs_render",
                     "gs_apply_flips", "gs_set_views"):
        assert required in names


def test_every_declared_symbol_is_exported_and_bound(lib):
    from paper_2606_21791_gb300 import gs
    for name in _declared():
        assert hasattr(lib, name), name
        assert name in gs.SIGNATURES, name
    assert set(gs.SIGNATURES) <= set(_declared())


def test_library_reports_version_and_errors_without_gpu(lib):
    from paper_2606_21791_gb300 import gs
    assert "sm_103a" in gs.gs_version()
    with pytest.raises(gs.GsError) as e:
        gs.gs_load_scene(None, 10, 7, 0)   # invalid SH degree: rejected before touching the device
    assert e.value.status == gs.GS_ERR_ARG


def test_struct_layouts_match_header():
    from paper_2606_21791_gb300 import gs
    src = open(os.path.join(ROOT, "include", "gs.h")).read()
    assert "uint32_t prim;\n    uint16_t word;\n    uint8_t bit;" in src
    assert gs.FLIP_DTYPE.itemsize == 8 and gs.RESULT_DTYPE.itemsize == 24
    assert gs.RECORD_DTYPE.itemsize == 64 and gs.CAMERA_DTYPE.itemsize == 80


def test_product_path_does_not_import_the_oracle():
    pkg = os.path.join(ROOT, "paper_2606_21791_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".h", ".cpp")):
                text = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in text and "from oracle" not in text, f
                assert "gs_oracle" not in text, f


def test_invalid_arguments_are_refused_before_the_device(lib):
    """Every call checks its arguments before it touches the device: a NULL
    scene or server, a NULL required buffer or an out-of-range size returns
    GS_ERR_ARG with a message, and never aborts (runs without a GPU)."""
    from paper_2606_21791_gb300 import gs
    calls = {
        "gs_scene_info": (None, None, None, None, None),
        "gs_apply_flips": (None, None, 1, None),
        "gs_field_box": (None, None, None),
        "gs_set_prim_box": (None, None, None, 0, 0),
        "gs_guard": (None, 0, 1, None, None),
        "gs_guard_bitmap": (None, 0, 1, None, None, None),
        "gs_render": (None, None, 1, None, None),
        "gs_compare": (None, None, 1, 1, 1, None, None),
        "gs_compare_noalloc": (None, None, 1, 1, 1, None, None),
        "gs_ssim": (None, None, 1, 1, 1, None, None),
        "gs_set_views": (None, None, 1, None),
        "gs_inject_and_render": (None, None, 1, 1, -1, 1, None, None),
        "gs_inject_and_render_full": (None, None, 1, 1, -1, 1, None, None),
        "gs_inject_and_render_host": (None, None, 1, 1, -1, 1, None, None),
        "gs_inject_and_render_regions": (None, None, 1, -1, 1, None, None, None),
        "gs_inject_and_render_ex": (None, None, 1, -1, 1, None, None, None, None),
        "gs_set_graphs": (None, 1),
        "gs_count_work": (None, 1),
        "gs_read_work": (None, None),
        "gs_time_kernels": (None, 1),
        "gs_read_kernel_ms": (None, None),
        "gs_read_render_ms": (None, None, None),
        "gs_set_batch": (None, 0),
        "gs_autotune": (None, None, 0, -1, 1, None, None, None),
        "gs_set_tile": (None, 16, 16, None),
        "gs_get_tile": (None, None, None),
        "gs_autotune_tile": (None, None, 0, -1, 1, None, None, None, None, None),
        "gs_preprocess": (None, None, None, None),
        "gs_bin_tiles": (None, None, 5, 1, 1, None, None, 1, None, None),
        "gs_blend_lists": (None, 0, None, None, 1, 1, None, None),
        "gs_server_create": (0, 0, None),
        "gs_server_submit": (None, None, 0.0, None),
        "gs_server_wait": (None, 0, 0, None),
        "gs_server_cancel": (None, 0),
        "gs_server_stats": (None, None),
        "gs_server_now": (None, None),
    }
    for name, args in calls.items():
        assert getattr(lib, name)(*args) == gs.GS_ERR_ARG, name
        assert lib.gs_last_error(), name
    assert lib.gs_server_destroy(None) == gs.GS_OK      # NULL is a no-op, like free


def test_binding_fails_loudly_without_the_library(tmp_path):
    """No CPU fallback: without libgs.so the binding raises (in a fresh process,
    since a loaded library is cached)."""
    import subprocess
    import sys
    code = ("from paper_2606_21791_gb300 import gs\n"
            f"gs.load_library({str(tmp_path / 'libgs.so')!r})\n")
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, cwd=ROOT, timeout=300)
    assert r.returncode != 0
    assert "no CPU fallback" in r.stderr
