"""The classifier behind the end-to-end footprint parity tests, on constructed
images (no GPU): a footprint decision that differs between the two renderers is
attributed to the 1/255 change threshold, the 1/255 alpha cut-off or the 1e-4
stop only when the oracle's own numbers put it within 1e-5 of that threshold."""
import numpy as np

import footprint_attribution as FA


def _case():
    H, W = 2, 4
    clean = np.full((H, W, 3), 0.5, np.float32)
    inf = np.full((H, W, 2), np.inf, np.float32)
    return clean, inf


def test_identical_renders_have_no_differences():
    clean, inf = _case()
    img = clean.copy()
    img[0, 0] += np.float32(0.1)
    c = FA.classify(img, clean, img, inf, clean, inf)
    assert c["gpu_footprint"] == c["oracle_footprint"] == 1 and c["pixels"] == 0


def test_each_threshold_class_and_the_unexplained_rest():
    clean, inf = _case()
    thr = float(np.float32(1 / 255))
    img_o = clean.copy()
    img_g = clean.copy()
    # (0,0): oracle change a hair above 1/255, GPU a hair below -> "delta"
    img_o[0, 0, 1] = np.float32(0.5 + thr + 2e-6)
    img_g[0, 0, 1] = np.float32(0.5 + thr - 2e-6)
    # (0,1): GPU changed by 0.004, oracle not at all, an alpha at the cut-off -> "alpha"
    img_g[0, 1, 0] = np.float32(0.504)
    # (0,2): the same, a T' at the stop -> "stop"
    img_g[0, 2, 2] = np.float32(0.504)
    # (0,3): the same with no threshold nearby -> "unexplained"
    img_g[0, 3, 0] = np.float32(0.51)
    mg = np.full_like(inf, 0.5)
    mg[0, 1, 0] = 3e-6
    mc = inf.copy()
    mc[0, 2, 1] = 8e-6
    c = FA.classify(img_g, clean, img_o, mg, clean, mc)
    assert c["pixels"] == 4
    assert (c["delta"], c["alpha"], c["stop"], c["unexplained"]) == (1, 1, 1, 1)
    assert c["oracle_footprint"] == 1 and c["gpu_footprint"] == 3


def test_change_clamps_and_counts_nan_as_zero():
    a = np.array([[[np.nan, 2.0, -1.0]]], np.float32)
    b = np.array([[[0.0, 1.0, 0.0]]], np.float32)
    assert FA.change(a, b)[0, 0] == 0.0
