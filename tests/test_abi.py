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
