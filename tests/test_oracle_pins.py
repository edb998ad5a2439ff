"""Pins of the CPU oracle against facts fixed outside it: closed forms, the
paper's printed constants, invariants of the method, library routines and brute
force.  A dropped term, a wrong sign or a transposed operand in the oracle
should fail at least one of these."""
import json
import math
import os

import numpy as np
import pytest
import scipy.special as sp

import oracle as O
from paper_2606_21791_gb300 import synth as S

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_constants.json")))
C0 = 0.5 / math.sqrt(math.pi)


def _planes_from_values(v, fmt=S.FP32):
    return S.encode(np.asarray(v, dtype=np.float32), fmt)


def _one_primitive(mean=(0, 0, 0), log_scale=(-2.0, -2.0, -2.0), quat=(1, 0, 0, 0), logit=0.0,
                   dc=(0.3, -0.2, 0.1), rest=None, sh_degree=0):
    nw = S.words_for_degree(sh_degree)
    v = np.zeros((nw, 1), dtype=np.float64)
    v[0:3, 0] = mean
    v[3:6, 0] = log_scale
    v[6:10, 0] = quat
    v[10, 0] = logit
    v[11:14, 0] = dc
    if rest is not None:
        v[14:, 0] = np.asarray(rest).reshape(-1)
    return v


def _sigmoid(x):
    return 1.0 / (1.0 + math.exp(-x))


def _expected_gaussian_image(cov2, mx, my, opac, rgb, W, H, tile, rect):
    """float64 image of one Gaussian with 2x2 covariance cov2 over white, restricted
    to the tile rect; returns (image, mask of pixels away from the 1/255 boundary)."""
    inv = np.linalg.inv(cov2)
    ys, xs = np.mgrid[0:H, 0:W]
    dx = xs + 0.5 - mx
    dy = ys + 0.5 - my
    q = inv[0, 0] * dx * dx + 2 * inv[0, 1] * dx * dy + inv[1, 1] * dy * dy
    alpha = opac * np.exp(-0.5 * q)
    tx, ty = xs // tile[0], ys // tile[1]
    inrect = (tx >= rect[0]) & (tx < rect[2]) & (ty >= rect[1]) & (ty < rect[3])
    use = inrect & (alpha >= 1 / 255)
    a = np.minimum(alpha, 0.99)
    img = np.ones((H, W, 3))
    for ch in range(3):
        img[..., ch] = np.where(use, rgb[ch] * a + (1 - a), 1.0)
    safe = np.abs(alpha - 1 / 255) > 1e-5
    return img, safe


def _rect(mx, my, r, W, H, tile):
    tx, ty = -(-W // tile[0]), -(-H // tile[1])
    x0 = min(max(math.floor((mx - r) / tile[0]), 0), tx)
    x1 = min(max(math.floor((mx + r) / tile[0]) + 1, 0), tx)
    y0 = min(max(math.floor((my - r) / tile[1]), 0), ty)
    y1 = min(max(math.floor((my + r) / tile[1]) + 1, 0), ty)
    return (x0, y0, x1, y1)


# ---------------------------------------------------------------------------
# closed forms of the forward render
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("log_s,logit,dc,W,H,tile", [
    (-2.0, 0.0, (0.3, -0.2, 0.1), 64, 64, (16, 16)),
    (-1.2, 3.0, (-0.5, 0.9, 0.0), 72, 56, (16, 16)),
    (-3.5, -1.0, (1.0, 0.2, -2.0), 80, 48, (8, 8)),
    (-0.8, 6.0, (0.0, 0.0, 0.0), 96, 64, (32, 8)),
])
def test_isotropic_gaussian_closed_form(log_s, logit, dc, W, H, tile):
    """One isotropic primitive on the optical axis: sigma_px^2 = (f s / d)^2 + 0.3,
    alpha = min(0.99, sigmoid(o) exp(-r^2 / (2 sigma_px^2))), pixel = rgb a + (1 - a)."""
    d = 15.0
    cam = S.look_at_camera((0, 0, d), width=W, height=H)
    v = _one_primitive(log_scale=(log_s,) * 3, logit=logit, dc=dc)
    img = O.render(_planes_from_values(v), S.FP32, 0, cam, tile)
    f = float(cam["fx"])
    s = math.exp(log_s)
    var = (f * s / d) ** 2 + 0.3
    r = math.ceil(3 * math.sqrt(var + math.sqrt(0.1)))
    rgb = [max(0.0, C0 * c + 0.5) for c in dc]
    mx, my = W / 2, H / 2
    exp_img, safe = _expected_gaussian_image(np.diag([var, var]), mx, my, _sigmoid(logit), rgb, W, H, tile,
                                             _rect(mx, my, r, W, H, tile))
    err = np.abs(img - exp_img).max(axis=2)
    assert err[safe].max() < 2e-6
    rec = O.preprocess(_planes_from_values(v), S.FP32, 0, cam, tile)[0]
    assert rec["radius"] == r
    assert abs(rec["ca"] - 1 / var) < 1e-6 / var and rec["cb"] == 0.0


@pytest.mark.parametrize("phi", [0.3, 1.1, -0.7])
def test_rotated_anisotropic_closed_form(phi):
    """Quaternion (cos(phi/2), 0, 0, sin(phi/2)) rotates the scale axes about the
    view axis; with the camera on +z looking at the origin (image y down) the 2D
    covariance is (f/d)^2 [[Sxx, -Sxy], [-Sxy, Syy]] + 0.3 I."""
    W = H = 96
    d = 12.0
    cam = S.look_at_camera((0, 0, d), width=W, height=H)
    sx, sy, sz = math.exp(-1.3), math.exp(-2.3), math.exp(-2.0)
    q = (math.cos(phi / 2), 0.0, 0.0, math.sin(phi / 2))
    v = _one_primitive(log_scale=(math.log(sx), math.log(sy), math.log(sz)), quat=q, logit=1.5, dc=(0.4, 0.1, -0.3))
    img = O.render(_planes_from_values(v), S.FP32, 0, cam)
    c, s = math.cos(phi), math.sin(phi)
    Sxx = sx * sx * c * c + sy * sy * s * s
    Syy = sx * sx * s * s + sy * sy * c * c
    Sxy = (sx * sx - sy * sy) * s * c
    k = (float(cam["fx"]) / d) ** 2
    cov2 = np.array([[k * Sxx + 0.3, -k * Sxy], [-k * Sxy, k * Syy + 0.3]])
    mid = 0.5 * (cov2[0, 0] + cov2[1, 1])
    det = np.linalg.det(cov2)
    r = math.ceil(3 * math.sqrt(mid + math.sqrt(max(0.1, mid * mid - det))))
    rgb = [max(0.0, C0 * ch + 0.5) for ch in (0.4, 0.1, -0.3)]
    exp_img, safe = _expected_gaussian_image(cov2, W / 2, H / 2, _sigmoid(1.5), rgb, W, H, (16, 16),
                                             _rect(W / 2, H / 2, r, W, H, (16, 16)))
    err = np.abs(img - exp_img).max(axis=2)
    assert err[safe].max() < 5e-6


def _real_sh_scipy(l, m, x, y, z):
    """Real SH from scipy's complex harmonics (which carry the Condon-Shortley
    phase): Y_l0, sqrt2 Re Y_l^m (m > 0), sqrt2 Im Y_l^|m| (m < 0)."""
    th = math.acos(max(-1.0, min(1.0, z)))
    ph = math.atan2(y, x)
    if m == 0:
        return float(sp.sph_harm_y(l, 0, th, ph).real)
    if m > 0:
        return float(math.sqrt(2) * sp.sph_harm_y(l, m, th, ph).real)
    return float(math.sqrt(2) * sp.sph_harm_y(l, -m, th, ph).imag)


def test_sh_basis_matches_scipy():
    rng = np.random.default_rng(5)
    for _ in range(20):
        v = rng.standard_normal(3)
        v /= np.linalg.norm(v)
        Y = O.sh_basis(*[float(t) for t in v.astype(np.float32)], 3)
        ref = [_real_sh_scipy(l, m, *v) for l in range(4) for m in range(-l, l + 1)]
        np.testing.assert_allclose(Y, ref, atol=2e-6)


def test_sh_basis_orthonormal_by_quadrature():
    """Gauss-Legendre in cos(theta) x uniform phi integrates products of degree <= 6 exactly."""
    nt, nph = 12, 24
    xs, ws = np.polynomial.legendre.leggauss(nt)
    G = np.zeros((16, 16))
    for ct, wt in zip(xs, ws):
        st = math.sqrt(1 - ct * ct)
        for j in range(nph):
            ph = 2 * math.pi * j / nph
            Y = O.sh_basis(float(st * math.cos(ph)), float(st * math.sin(ph)), float(ct), 3).astype(np.float64)
            G += np.outer(Y, Y) * wt * (2 * math.pi / nph)
    np.testing.assert_allclose(G, np.eye(16), atol=1e-5)


def test_sh_colour_layout_in_render():
    """Degree-3 colour of an opaque primitive seen from a generic direction:
    pixel = 0.99 (sum_lm c_lm Y_lm(dir) + 0.5) + 0.01 with dir = normalize(mean - eye)
    and the higher-order coefficients stored coefficient-major (15 x 3)."""
    W = H = 64
    eye = np.array([4.0, -3.0, 11.0])
    cam = S.look_at_camera(eye, width=W, height=H)
    rng = np.random.default_rng(9)
    rest = rng.normal(0, 0.08, size=(15, 3))
    dc = (0.6, 0.2, 0.4)
    v = _one_primitive(log_scale=(1.0, 1.0, 1.0), logit=12.0, dc=dc, rest=rest, sh_degree=3)
    img = O.render(_planes_from_values(v), S.FP32, 3, cam)
    dirv = -eye / np.linalg.norm(eye)
    Y = [_real_sh_scipy(l, m, *dirv) for l in range(4) for m in range(-l, l + 1)]
    coef = np.vstack([np.asarray(dc)[None, :], rest])
    rgb = np.maximum(coef.T @ np.asarray(Y) + 0.5, 0.0)
    rec = O.preprocess(_planes_from_values(v), S.FP32, 3, cam)[0]
    np.testing.assert_allclose([rec["r"], rec["g"], rec["b"]], rgb, atol=3e-6)
    # the pixel under the projected mean: alpha is capped at 0.99
    px, py = int(rec["mx"]), int(rec["my"])
    np.testing.assert_allclose(img[py, px], 0.99 * rgb + 0.01, atol=1e-5)


# ---------------------------------------------------------------------------
# injection: XOR semantics and Lemma 1
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("fmt", [S.FP32, S.FP16, S.BF16])
def test_flip_twice_is_identity_and_one_bit(fmt):
    rng = np.random.default_rng(3)
    nbits = S.FORMAT_BITS[fmt]
    planes = rng.integers(0, 2 ** nbits, size=(14, 257), dtype=np.uint64).astype(S.FORMAT_DTYPE[fmt])
    # plant NaN payloads and infinities
    nan = 0x7FC00123 if fmt == S.FP32 else 0x7E01
    planes[0, :5] = nan
    planes[1, :3] = 0x7F800000 if fmt == S.FP32 else (0x7C00 if fmt == S.FP16 else 0x7F80)
    flips = S.flips_at(rng.integers(0, 257, size=300), 0, 0)
    flips["word"] = rng.integers(0, 14, size=300)
    flips["bit"] = rng.integers(0, nbits, size=300)
    once = O.apply_flips(planes, fmt, flips[:1])
    x = (once ^ planes).astype(np.uint64)
    assert sum(bin(int(t)).count("1") for t in x.ravel()) == 1
    f0 = flips[0]
    assert int(x[f0["word"], f0["prim"]]) == 1 << int(f0["bit"])
    twice = O.apply_flips(O.apply_flips(planes, fmt, flips), fmt, flips[::-1])
    assert np.array_equal(twice, planes)
    with pytest.raises(ValueError):
        O.apply_flips(planes, fmt, S.flips_at(0, 0, nbits))


@pytest.mark.parametrize("fmtname,fmt", [("fp32", S.FP32), ("fp16", S.FP16), ("bf16", S.BF16)])
def test_lemma1_value_perturbation(fmtname, fmt):
    """Lemma 1: mantissa bit b changes a normal value by exactly 2^(e+b-p); the sign
    bit negates; exponent bit j scales by 2^(+-2^j) or leaves the normal range."""
    lay = GOLD["ieee_layout"][fmtname]
    p, sbit, ebits = lay["mantissa_p"], lay["sign_bit"], lay["exp_bits"]
    assert sbit == p + ebits
    rng = np.random.default_rng(11)
    vals = rng.normal(0, 3, size=64).astype(np.float32)
    planes = S.encode(vals[None, :], fmt)
    base = S.decode(planes, fmt)[0].astype(np.float64)
    n = len(vals)
    for b in range(p):
        out = S.decode(O.apply_flips(planes, fmt, S.flips_at(np.arange(n), 0, b)), fmt)[0].astype(np.float64)
        e = np.floor(np.log2(np.abs(base)))
        np.testing.assert_array_equal(np.abs(out - base), np.exp2(e + b - p))
    out = S.decode(O.apply_flips(planes, fmt, S.flips_at(np.arange(n), 0, sbit)), fmt)[0].astype(np.float64)
    np.testing.assert_array_equal(out, -base)
    bias = 2 ** (ebits - 1) - 1
    for j in range(ebits):
        with np.errstate(invalid="ignore"):   # exponent flips make Inf and NaN on purpose
            out = S.decode(O.apply_flips(planes, fmt, S.flips_at(np.arange(n), 0, p + j)), fmt)[0].astype(np.float64)
        e = np.floor(np.log2(np.abs(base))).astype(np.int64)
        E = e + bias
        Enew = E ^ (1 << j)
        for k in range(n):
            if 1 <= Enew[k] <= 2 * bias:      # still a normal number: exact power-of-two scaling
                assert out[k] == base[k] * 2.0 ** (int(Enew[k]) - int(E[k]))
            elif Enew[k] == 2 * bias + 1:     # all-ones exponent: Inf or NaN
                assert not np.isfinite(out[k])
            else:                              # zero exponent: subnormal or zero, |value| < 2^(1-bias)
                assert abs(out[k]) < 2.0 ** (1 - bias)


def _scale_from_conic(rec, f, d):
    var = 1.0 / float(rec["ca"])
    return math.sqrt(var - 0.3) * d / f


def test_prop1_sign_flip_scale_ratio_golden():
    """Prop. 1: the sign flip of a log-scale near -3 multiplies the scale by e^6."""
    g = GOLD["prop1_sign_flip"]
    d = 15.0
    cam = S.look_at_camera((0, 0, d), width=512, height=512)
    v = _one_primitive(log_scale=(g["theta"],) * 3)
    planes = _planes_from_values(v)
    f = float(cam["fx"])
    s0 = _scale_from_conic(O.preprocess(planes, S.FP32, 0, cam)[0], f, d)
    flipped = O.apply_flips(planes, S.FP32, S.flips_at(np.zeros(3, np.int64), [3, 4, 5], 31))
    s1 = _scale_from_conic(O.preprocess(flipped, S.FP32, 0, cam)[0], f, d)
    assert abs(s1 / s0 - g["scale_ratio"]) / g["scale_ratio"] < 2e-4
    assert 0.5 * g["scale_ratio_printed_order"] < s1 / s0 < 2 * g["scale_ratio_printed_order"]


# ---------------------------------------------------------------------------
# support guard (Algorithm 1, Theorems 1 and 2)
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("fmt", [S.FP32, S.FP16, S.BF16])
def test_field_box_is_min_max(fmt):
    sc = S.make_scene(3000, 3, fmt, 7, layout="clusters")
    lo, hi = O.field_box(sc.planes, fmt)
    vals = sc.values()
    np.testing.assert_array_equal(S.decode(lo.astype(S.FORMAT_DTYPE[fmt]), fmt), vals.min(axis=1))
    np.testing.assert_array_equal(S.decode(hi.astype(S.FORMAT_DTYPE[fmt]), fmt), vals.max(axis=1))


@pytest.mark.parametrize("fmt", [S.FP32, S.FP16, S.BF16])
@pytest.mark.parametrize("mode", [0, 1])
def test_guard_identity_on_clean_model(fmt, mode):
    """Theorem 1(i): the guard leaves a clean model unchanged (zero clamps)."""
    sc = S.make_scene(2000, 3, fmt, 8, layout="clusters")
    if mode == 0:
        lo, hi = O.field_box(sc.planes, fmt)
        mask = (1 << 59) - 1
    else:
        lo, hi = S.prim_boxes(sc, 14, 21)
        mask = S.GUARD_WORDS_DEFAULT
    out, n = O.guard(sc.planes, fmt, mask, mode, lo, hi)
    assert n == 0 and np.array_equal(out, sc.planes)


def _corrupt(planes, fmt, rng, count):
    nbits = S.FORMAT_BITS[fmt]
    fl = S.flips_at(rng.integers(0, planes.shape[1], size=count), 0, 0)
    fl["word"] = rng.integers(0, 14, size=count)
    fl["bit"] = rng.integers(nbits - 9, nbits, size=count)  # sign and exponent bits mostly
    return O.apply_flips(planes, fmt, fl)


@pytest.mark.parametrize("fmt", [S.FP32, S.FP16, S.BF16])
@pytest.mark.parametrize("mode", [0, 1])
def test_guard_clamps_into_box(fmt, mode):
    """Theorem 1(ii): after the guard every guarded component is inside its box;
    in-box values are untouched, out-of-box values move to the nearer endpoint,
    NaN moves to the low endpoint, and the count equals the number moved."""
    rng = np.random.default_rng(4)
    sc = S.make_scene(1500, 0, fmt, 9)
    if mode == 0:
        lo, hi = O.field_box(sc.planes, fmt)
        lov = S.decode(lo.astype(S.FORMAT_DTYPE[fmt]), fmt)[:, None]
        hiv = S.decode(hi.astype(S.FORMAT_DTYPE[fmt]), fmt)[:, None]
    else:
        lo, hi = S.prim_boxes(sc, 14, 22)
        lov, hiv = S.decode(lo, fmt), S.decode(hi, fmt)
    bad = _corrupt(sc.planes, fmt, rng, 900)
    bad[2, :4] = S.encode(np.array([np.nan, np.inf, -np.inf, np.nan], np.float32), fmt)
    mask = (1 << 14) - 1
    out, n = O.guard(bad, fmt, mask, mode, lo, hi)
    x = S.decode(bad, fmt)
    y = S.decode(out, fmt)
    inside = (x >= lov) & (x <= hiv)
    assert n == int((~inside).sum()) and n > 0
    assert np.array_equal(out[inside], bad[inside])
    assert np.all((y >= lov) & (y <= hiv))
    lo_b = np.broadcast_to(lov, x.shape)
    hi_b = np.broadcast_to(hiv, x.shape)
    np.testing.assert_array_equal(y[x > hiv], hi_b[x > hiv])
    np.testing.assert_array_equal(y[x < lov], lo_b[x < lov])
    np.testing.assert_array_equal(y[np.isnan(x)], lo_b[np.isnan(x)])


def test_guard_word_mask_and_prim_box_range():
    sc = S.make_scene(500, 3, S.FP32, 10, layout="clusters")
    lo, hi = O.field_box(sc.planes, S.FP32)
    bad = O.apply_flips(sc.planes, S.FP32, S.flips_at(np.array([1, 2]), [20, 4], 30))
    out, n = O.guard(bad, S.FP32, S.GUARD_WORDS_DEFAULT, 0, lo, hi)
    assert n == 1 and out[20, 1] == bad[20, 1] and out[4, 2] != bad[4, 2]
    plo, phi = S.prim_boxes(sc, 14, 1)
    with pytest.raises(ValueError):
        O.guard(bad, S.FP32, 1 << 20, 1, plo, phi)


def _pin_scene(n, seed, sh_degree=0, fmt=S.FP32):
    rng = np.random.default_rng(seed)
    v = S.scene_values(n, sh_degree, seed, layout="cube", cube=2.0)
    v[3:6] = rng.normal(-3.0, 0.5, size=(3, n))
    v[10] = rng.normal(1.0, 1.0, size=n)
    return S.Scene(planes=S.encode(v, fmt), fmt=fmt, sh_degree=sh_degree)


def test_thm2_guarded_extent_bounded_by_largest_trained_scale():
    """Theorem 2: under the guard a flipped primitive's log-scales lie in the box,
    so its tile footprint is no larger than the same primitive with every
    log-scale at the box maximum."""
    sc = _pin_scene(300, 12)
    cam = S.look_at_camera((0, 0, 8), width=128, height=128)
    lo, hi = O.field_box(sc.planes, S.FP32)
    hmax = S.decode(hi.astype(np.uint32), S.FP32)[3:6]
    rng = np.random.default_rng(2)
    for prim in rng.integers(0, sc.n, size=15):
        for word in (3, 4, 5):
            for bit in (31, 30, 29):
                bad = O.apply_flips(sc.planes, S.FP32, S.flips_at(prim, word, bit))
                g, _ = O.guard(bad, S.FP32, S.GUARD_WORDS_DEFAULT, 0, lo, hi)
                gv = S.decode(g, S.FP32)
                assert np.all(gv[3:6] <= hmax[:, None])
                big = g.copy()
                big[3:6, prim] = S.encode(hmax, S.FP32)
                r_g = O.preprocess(g, S.FP32, 0, cam)[prim]
                r_big = O.preprocess(big, S.FP32, 0, cam)[prim]
                if r_g["visible"]:
                    assert r_g["radius"] <= r_big["radius"]
                    area = (r_g["x1"] - r_g["x0"]) * (r_g["y1"] - r_g["y0"])
                    assert area <= (r_big["x1"] - r_big["x0"]) * (r_big["y1"] - r_big["y0"])


# ---------------------------------------------------------------------------
# comparison (Definitions 1 and 2, PSNR)
# ---------------------------------------------------------------------------
def test_compare_textbook_psnr_and_footprint():
    rng = np.random.default_rng(1)
    H, W = 37, 53
    a = rng.uniform(0.1, 0.9, size=(H, W, 3)).astype(np.float32)
    b = a.copy()
    thr = GOLD["definition1_footprint_threshold"]["threshold"]
    # known perturbations: 40 pixels by 0.05 in channel 1, 7 pixels by exactly 1/255 (not counted)
    idx = rng.choice(H * W, size=47, replace=False)
    big, edge = idx[:40], idx[40:]
    b.reshape(-1, 3)[big, 1] += np.float32(0.05)
    b.reshape(-1, 3)[edge, 0] = a.reshape(-1, 3)[edge, 0] - np.float32(1.0 / 255.0)
    m = O.compare(a, b)
    d = (a.astype(np.float64) - b.astype(np.float64))
    mse_ref = float(np.mean(d * d))
    assert abs(m["sse"] / (H * W * 3) - mse_ref) < 1e-12
    assert abs(O.psnr(m["sse"], H * W * 3) - 10 * math.log10(1 / mse_ref)) < 1e-6
    diff_edge = np.abs(a.reshape(-1, 3)[edge, 0] - b.reshape(-1, 3)[edge, 0])
    expected_foot = 40 + int((diff_edge > np.float32(thr)).sum())
    assert m["footprint"] == expected_foot
    assert m["nonfinite"] == 0
    # clamping to [0, 1]: out-of-range values compare after clamping, NaN counts as 0
    c = a.copy()
    c[0, 0] = [2.0, -1.0, np.nan]
    m2 = O.compare(c, a)
    assert m2["nonfinite"] == 1
    dd = np.array([1.0 - a[0, 0, 0], 0.0 - a[0, 0, 1], 0.0 - a[0, 0, 2]], dtype=np.float64)
    assert abs(m2["sse"] - float((dd ** 2).sum())) < 1e-6
    assert O.psnr(0.0, 10) == 100.0 and O.psnr(0.0, 10, cap=False) == math.inf
    assert GOLD["definition2_catastrophe_percent"]["percent"] == 1.0


# ---------------------------------------------------------------------------
# binning / blending: brute force and ordering
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("seed,tile", [(0, (16, 16)), (1, (8, 8)), (2, (16, 8)), (3, (32, 8))])
def test_brute_force_equals_tiled(seed, tile):
    sc = _pin_scene(200, 100 + seed)
    v = sc.values().copy()
    # a few exploded and non-finite primitives
    v[3:6, 0] = 2.5
    v[10, 1] = np.nan
    v[0, 2] = np.inf
    v[11, 3] = np.nan
    planes = S.encode(v, S.FP32)
    cam = S.look_at_camera((0.5, -0.3, 8), width=64, height=56)
    recs = O.preprocess(planes, S.FP32, 0, cam, tile)
    off, ids = O.bin_tiles(recs, 64, 56, tile)
    tiled = O.blend(recs, off, ids, 64, 56, tile)
    brute = O.blend_brute(recs, 64, 56, tile)
    assert np.array_equal(tiled.view(np.uint32), brute.view(np.uint32))
    assert np.array_equal(tiled.view(np.uint32), O.render(planes, S.FP32, 0, cam, tile).view(np.uint32))
    assert recs["visible"][2] == 0  # non-finite mean culls
    assert np.isnan(tiled).any()    # non-finite opacity / colour propagates


def test_equal_depth_ties_break_by_index():
    W = H = 32
    cam = S.look_at_camera((0, 0, 10), width=W, height=H)
    v = np.zeros((14, 3))
    v[3:6] = -1.5
    v[6] = 1.0
    v[10] = [0.0, 2.0, 1.0]
    v[11:14] = [[0.5, -0.5, 0.0]] * 3
    v[11:14, 0] = [1, 0, 0]
    v[11:14, 1] = [0, 1, 0]
    v[11:14, 2] = [0, 0, 1]
    planes = _planes_from_values(v)
    recs = O.preprocess(planes, S.FP32, 0, cam)
    assert len(set(recs["depth"].tolist())) == 1
    off, ids = O.bin_tiles(recs, W, H)
    for t in range(len(off) - 1):
        lst = ids[off[t]:off[t + 1]]
        assert list(lst) == sorted(lst)
    # reversing the depth order by moving primitive 0 back changes the order
    v[2, 0] = -0.5
    recs = O.preprocess(_planes_from_values(v), S.FP32, 0, cam)
    off, ids = O.bin_tiles(recs, W, H)
    assert list(ids[off[0]:off[1]])[-1] == 0


# ---------------------------------------------------------------------------
# campaign-level properties
# ---------------------------------------------------------------------------
def test_zero_flip_render_equals_clean():
    sc, cams, flips = S.tiny_workload()
    pairs = np.repeat(flips[:12], 2)      # each variant flips the same site twice
    m, cl, clean = O.campaign(sc.planes, S.FP32, 0, cams, pairs, flips_per_variant=2)
    assert np.all(m["sse"] == 0) and np.all(m["footprint"] == 0) and np.all(m["maxabs"] == 0)


def test_campaign_is_flip_guard_render_compare():
    sc = _pin_scene(400, 31)
    cams = S.ring_cameras(2, 64, 48, distance=8.0)
    flips = S.flips_uniform_fields(6, sc.n, S.FP32, 77)
    lo, hi = O.field_box(sc.planes, S.FP32)
    m, cl, clean = O.campaign(sc.planes, S.FP32, 0, cams, flips, guard_mode=0, word_mask=S.GUARD_WORDS_DEFAULT,
                              box_lo=lo, box_hi=hi, nthreads=2)
    for vi in range(len(flips)):
        bad = O.apply_flips(sc.planes, S.FP32, flips[vi:vi + 1])
        g, n = O.guard(bad, S.FP32, S.GUARD_WORDS_DEFAULT, 0, lo, hi)
        assert n == cl[vi]
        for k in range(2):
            ref = O.compare(O.render(g, S.FP32, 0, cams[k]), clean[k])
            assert ref["sse"] == m[vi, k]["sse"] and ref["footprint"] == m[vi, k]["footprint"]


def _severity(sc, cam, word, bits, prims, metric="maxabs"):
    flips = np.concatenate([S.flips_at(prims, word, b) for b in bits])
    m, _, _ = O.campaign(sc.planes, sc.fmt, sc.sh_degree, [cam], flips, nthreads=O.max_threads())
    return m[:, 0][metric].reshape(len(bits), len(prims))


@pytest.mark.parametrize("word", [3, 10])
def test_prop1_mantissa_slope_one_bit(word):
    """Prop. 1 with Lemma 1: for log-scale (phi = exp) and opacity (phi = sigmoid)
    mantissa bits, the peak pixel error doubles per bit before saturation
    (log2 slope near 1; the study measured 0.94)."""
    sc = _pin_scene(300, 40)
    cam = S.look_at_camera((0, 0, 8), width=96, height=96)
    recs = O.preprocess(sc.planes, S.FP32, 0, cam)
    rng = np.random.default_rng(6)
    prims = rng.choice(np.nonzero(recs["visible"])[0], size=40, replace=False)
    bits = list(range(8, 17))
    sev = _severity(sc, cam, word, bits, prims)
    med = np.median(sev, axis=1)
    assert np.all(med > 0)
    slope = np.polyfit(bits, np.log2(med), 1)[0]
    assert 0.8 <= slope <= 1.2, slope


def test_log_scale_sign_bit_is_most_severe():
    """Sec. 5.1: the log-scale sign bit has the largest mean footprint of any
    (field, bit) cell; mantissa bits are far milder."""
    sc = _pin_scene(300, 41)
    cam = S.look_at_camera((0, 0, 8), width=96, height=96)
    rng = np.random.default_rng(8)
    prims = rng.integers(0, sc.n, size=12)
    cells = []
    for word in range(14):
        for bit in (31, 30, 29, 28, 27, 22, 18):
            cells.append((word, bit))
    flips = np.concatenate([S.flips_at(prims, w, b) for (w, b) in cells])
    m, _, _ = O.campaign(sc.planes, S.FP32, 0, [cam], flips, nthreads=O.max_threads())
    foot = m[:, 0]["footprint"].reshape(len(cells), len(prims)).astype(np.float64)
    nonfin = m[:, 0]["nonfinite"].reshape(len(cells), len(prims))
    # non-finite renders are catastrophic by Definition 2 but carry no footprint ordering
    mean_foot = np.where(nonfin > 0, 0.0, foot).mean(axis=1)
    best = cells[int(np.argmax(mean_foot))]
    assert best[0] in (3, 4, 5) and best[1] == 31, best
    sign_mean = np.mean([mean_foot[cells.index((w, 31))] for w in (3, 4, 5)])
    mant_mean = np.mean([mean_foot[cells.index((w, 18))] for w in (3, 4, 5)])
    assert sign_mean > 20 * max(mant_mean, 1e-9)


def test_generic_view_covariance_from_projected_axes():
    """A primitive at the look-at target projects to the image centre, where the
    perspective Jacobian is (f/d) times the first two camera axes.  Its 2D
    covariance is then the sum over its three scaled principal axes (rotation from
    scipy's quaternion routine) of the outer products of their projections."""
    from scipy.spatial.transform import Rotation
    W, H = 96, 80
    eye = np.array([5.0, -4.0, 9.0])
    d = float(np.linalg.norm(eye))
    cam = S.look_at_camera(eye, width=W, height=H)
    Rcam = np.asarray(cam["R"], dtype=np.float64).reshape(3, 3)
    rng = np.random.default_rng(17)
    for _ in range(5):
        q = rng.standard_normal(4)
        q /= np.linalg.norm(q)
        ls = rng.uniform(-2.5, -1.0, size=3)
        v = _one_primitive(log_scale=tuple(ls), quat=tuple(q), logit=2.0)
        rec = O.preprocess(_planes_from_values(v), S.FP32, 0, cam)[0]
        rot = Rotation.from_quat([q[1], q[2], q[3], q[0]]).as_matrix()   # scipy is scalar-last
        k = float(cam["fx"]) / d
        cov = np.zeros((2, 2))
        for ax in range(3):
            a_img = k * (Rcam @ (rot[:, ax] * math.exp(ls[ax])))[:2]
            cov += np.outer(a_img, a_img)
        cov += 0.3 * np.eye(2)
        conic = np.array([[rec["ca"], rec["cb"]], [rec["cb"], rec["cc"]]], dtype=np.float64)
        np.testing.assert_allclose(np.linalg.inv(conic), cov, rtol=2e-5, atol=1e-6)
        assert abs(rec["mx"] - W / 2) < 1e-4 and abs(rec["my"] - H / 2) < 1e-4


def test_transmittance_cutoff_stops_pixel():
    """Front-to-back compositing stops a pixel before the primitive that would take
    its transmittance below 1e-4: with four opaque primitives stacked on the
    optical axis (alpha ~ 0.95 each), the fourth is excluded at the centre pixel."""
    W = H = 32
    d = 15.0
    cam = S.look_at_camera((0, 0, d), width=W, height=H)
    zs = [0.0, -1.0, -2.0, -3.0]
    cols = [(0.8, -0.6, 0.1), (-0.7, 0.9, 0.3), (0.2, 0.2, -0.9), (-0.9, -0.9, -0.9)]
    v = np.zeros((14, 4))
    v[6] = 1.0
    v[3:6] = 0.5
    v[10] = 3.9
    for i in range(4):
        v[2, i] = zs[i]
        v[11:14, i] = cols[i]
    img = O.render(_planes_from_values(v), S.FP32, 0, cam)
    f = float(cam["fx"])
    T, C = 1.0, np.zeros(3)
    stopped_at = None
    for i in range(4):
        var = (f * math.exp(0.5) / (d - zs[i])) ** 2 + 0.3
        a = min(0.99, _sigmoid(3.9) * math.exp(-0.5 * 0.5 / var))
        Tn = T * (1 - a)
        assert abs(Tn - 1e-4) > 1e-6
        if Tn < 1e-4:
            stopped_at = i
            break
        C += np.maximum(C0 * np.asarray(cols[i]) + 0.5, 0) * a * T
        T = Tn
    assert stopped_at == 3
    np.testing.assert_allclose(img[H // 2, W // 2], C + T, atol=2e-6)


def test_decision_margins_closed_form():
    """The blend's decision margins, per pixel, from the closed form of one
    isotropic primitive on the optical axis: alpha margin = |alpha - 1/255| /
    (1/255) and, where alpha passes the cut-off, T' margin = |1 - alpha - 1e-4| /
    1e-4; inf where no entry was tested (outside the tile rect or power > 0 never
    happens on the centre).  The image equals the plain render."""
    W = H = 64
    d = 15.0
    tile = (16, 16)
    log_s, logit = -1.6, 1.0
    cam = S.look_at_camera((0, 0, d), width=W, height=H)
    v = _one_primitive(log_scale=(log_s,) * 3, logit=logit)
    planes = _planes_from_values(v)
    img, mg = O.render_margins(planes, S.FP32, 0, cam, tile)
    assert np.array_equal(img, O.render(planes, S.FP32, 0, cam, tile))
    f = float(cam["fx"])
    var = (f * math.exp(log_s) / d) ** 2 + 0.3
    r = math.ceil(3 * math.sqrt(var + math.sqrt(0.1)))
    rect = _rect(W / 2, H / 2, r, W, H, tile)
    ys, xs = np.mgrid[0:H, 0:W]
    q = ((xs + 0.5 - W / 2) ** 2 + (ys + 0.5 - H / 2) ** 2) / var
    alpha = _sigmoid(logit) * np.exp(-0.5 * q)
    tx, ty = xs // tile[0], ys // tile[1]
    inrect = (tx >= rect[0]) & (tx < rect[2]) & (ty >= rect[1]) & (ty < rect[3])
    thr = float(np.float32(1 / 255))
    exp_a = np.abs(alpha - thr) / thr
    assert np.isinf(mg[..., 0][~inrect]).all() and np.isinf(mg[..., 1][~inrect]).all()
    np.testing.assert_allclose(mg[..., 0][inrect], exp_a[inrect], rtol=2e-5, atol=1e-6)
    passed = inrect & (alpha >= thr) & (np.abs(alpha - thr) > 1e-6)
    tthr = float(np.float32(1e-4))
    exp_t = np.abs(1 - np.minimum(alpha, 0.99) - tthr) / tthr
    np.testing.assert_allclose(mg[..., 1][passed], exp_t[passed], rtol=2e-5)
    assert np.isinf(mg[..., 1][inrect & (alpha < thr * (1 - 1e-6))]).all()


def test_decision_margins_near_the_transmittance_stop():
    """Two opaque primitives stacked on the axis: at the centre pixel the second
    one's T' = (1 - a1)(1 - a2) is the closest decision to the 1e-4 stop."""
    W = H = 32
    d = 15.0
    cam = S.look_at_camera((0, 0, d), width=W, height=H)
    v = np.zeros((14, 2))
    v[6] = 1.0
    v[3:6] = 0.5
    v[10] = 4.5
    v[2] = (0.0, -1.0)
    img, mg = O.render_margins(_planes_from_values(v), S.FP32, 0, cam)
    f = float(cam["fx"])
    T = 1.0
    best = math.inf
    for z in (0.0, -1.0):
        var = (f * math.exp(0.5) / (d - z)) ** 2 + 0.3
        a = min(0.99, _sigmoid(4.5) * math.exp(-0.5 * 0.5 / var))
        T = T * (1 - a)
        best = min(best, abs(T - 1e-4) / 1e-4)
    assert abs(mg[H // 2, W // 2, 1] - best) <= 1e-3 * best


def test_footprint_threshold_is_strict():
    """Definition 1 counts changes of MORE than one 8-bit level: a change of exactly
    1/255 (in fp32) is not in the footprint."""
    thr = np.float32(GOLD["definition1_footprint_threshold"]["threshold"])
    a = np.zeros((2, 2, 3), dtype=np.float32)
    b = np.zeros((2, 2, 3), dtype=np.float32)
    a[0, 0, 0] = thr
    a[0, 1, 2] = np.nextafter(thr, np.float32(1))
    m = O.compare(a, b)
    assert m["footprint"] == 1 and m["maxabs"] == np.nextafter(thr, np.float32(1))


def test_off_centre_covariance_uses_projection_jacobian():
    """Off the optical axis the 2D covariance is J Sigma_cam J^T + 0.3 I with J the
    Jacobian of the pinhole map (x, y, z) -> (f x / z + c_x, f y / z + c_y); here J
    is taken by central finite differences and Sigma_cam from the projected axes."""
    from scipy.spatial.transform import Rotation
    W, H = 128, 96
    eye = np.array([3.0, 2.0, 10.0])
    cam = S.look_at_camera(eye, width=W, height=H)
    Rc = np.asarray(cam["R"], dtype=np.float64).reshape(3, 3)
    tc = np.asarray(cam["t"], dtype=np.float64)
    f = float(cam["fx"])
    cx, cy = float(cam["cx"]), float(cam["cy"])

    def pix(pc):
        return np.array([f * pc[0] / pc[2] + cx, f * pc[1] / pc[2] + cy])

    rng = np.random.default_rng(23)
    for _ in range(6):
        mean = rng.uniform(-2.0, 2.0, size=3)
        q = rng.standard_normal(4)
        q /= np.linalg.norm(q)
        ls = rng.uniform(-2.5, -1.0, size=3)
        v = _one_primitive(mean=tuple(mean), log_scale=tuple(ls), quat=tuple(q), logit=2.0)
        rec = O.preprocess(_planes_from_values(v), S.FP32, 0, cam)[0]
        pc = Rc @ np.asarray(v[0:3, 0], dtype=np.float32).astype(np.float64) + tc
        h = 1e-5
        J = np.stack([(pix(pc + h * e) - pix(pc - h * e)) / (2 * h) for e in np.eye(3)], axis=1)
        rot = Rotation.from_quat([q[1], q[2], q[3], q[0]]).as_matrix()
        cov = 0.3 * np.eye(2)
        for ax in range(3):
            a_img = J @ (Rc @ (rot[:, ax] * math.exp(ls[ax])))
            cov += np.outer(a_img, a_img)
        conic = np.array([[rec["ca"], rec["cb"]], [rec["cb"], rec["cc"]]], dtype=np.float64)
        np.testing.assert_allclose(np.linalg.inv(conic), cov, rtol=1e-4, atol=1e-5)
        np.testing.assert_allclose([rec["mx"], rec["my"]], pix(pc), atol=2e-4)
        assert abs(rec["depth"] - pc[2]) < 1e-5


# ---------------------------------------------------------------------------
# the activations' fp32 exponential (Cody-Waite reduction + degree-7 Taylor)
# ---------------------------------------------------------------------------
def _exp_ulp_error(x):
    """ulp error of the oracle's exp against the double exponential; where the
    double result rounds past the largest float the oracle must give +inf (or
    the largest float: one ulp)."""
    y = O.exp_f32(x).astype(np.float64)
    ref = np.exp(x.astype(np.float64))
    with np.errstate(over="ignore"):   # the overflow region is what this selects
        over = ~np.isfinite(ref.astype(np.float32))
    assert ((y[over] == np.inf) | (y[over] == np.finfo(np.float32).max)).all()
    y, ref = y[~over], ref[~over]
    # spacing of fp32 at the reference value (the smallest subnormal step below 2^-126)
    sp = np.spacing(np.abs(ref).astype(np.float32)).astype(np.float64)
    sp = np.maximum(sp, 2.0 ** -149)
    return np.abs(y - ref) / sp


def test_exp_f32_within_one_ulp_sweep():
    # every 97th fp32 value in [-104, 89] (positive and negative halves)
    pos = np.arange(0, int(np.float32(89.0).view(np.uint32)), 97, dtype=np.uint32).view(np.float32)
    neg = np.arange(0x80000000, int(np.float32(-104.0).view(np.uint32)), 97, dtype=np.uint32).view(np.float32)
    x = np.concatenate([pos, neg])
    err = _exp_ulp_error(x)
    assert err.max() <= 1.0, (err.max(), x[err.argmax()])


@pytest.mark.parametrize("lo", [0.25, 0.5, 1.0, 2.0, 32.0, 64.0])
def test_exp_f32_within_one_ulp_exhaustive_binades(lo):
    # every fp32 value of [lo, 2 lo) and of (-2 lo, -lo]
    a = int(np.float32(lo).view(np.uint32))
    b = int(np.float32(2 * lo).view(np.uint32))
    x = np.arange(a, b, dtype=np.uint32).view(np.float32)
    x = np.concatenate([x, -x])
    x = x[x <= 89.0]
    err = _exp_ulp_error(x)
    assert err.max() <= 1.0, (err.max(), x[err.argmax()])


def test_exp_f32_special_values():
    x = np.array([np.nan, np.inf, -np.inf, 0.0, -0.0, 88.72283, 88.7229, 89.5, -87.3, -100.0, -103.2, -103.9,
                  -104.1, 1e-30, -1e-30], dtype=np.float32)
    y = O.exp_f32(x)
    assert np.isnan(y[0])
    assert y[1] == np.inf and y[2] == 0.0
    assert y[3] == 1.0 and y[4] == 1.0
    assert np.isfinite(y[5]) and y[6] == np.inf and y[7] == np.inf
    assert 0 < y[8] < 2.0 ** -125   # near the normal/subnormal boundary
    assert 0 < y[9] < 2.0 ** -126 and 0 < y[10] < 2.0 ** -126   # subnormal results
    assert y[11] == np.float32(2.0 ** -149)   # 7.5e-46 rounds up to the smallest subnormal
    assert y[12] == 0.0
    assert y[13] == 1.0 and y[14] == 1.0
    err = _exp_ulp_error(x[[5, 8, 9, 10, 11]])
    assert err.max() <= 1.0


# ---------------------------------------------------------------------------
# ECC sign+exponent emulation (Sec. 5 "Alternative defenses", Table 4)
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("fmtname,fmt", [("fp32", S.FP32), ("fp16", S.FP16), ("bf16", S.BF16)])
def test_ecc_protects_exactly_the_sign_and_exponent_bits(fmtname, fmt):
    lay = GOLD["ieee_layout"][fmtname]
    assert O.ecc_first_bit(fmt) == lay["mantissa_p"]
    assert lay["mantissa_p"] + lay["exp_bits"] + 1 == lay["bits"]
    fl = np.zeros(lay["bits"] * 3, dtype=S.FLIP_DTYPE)
    fl["bit"] = np.tile(np.arange(lay["bits"]), 3)
    fl["word"] = np.repeat([3, 10, 20], lay["bits"])
    got = O.ecc_corrects(fmt, (1 << 14) - 1, fl)   # words 0-13 protected, word 20 not
    want = (fl["bit"] >= lay["mantissa_p"]) & (fl["word"] < 14)
    assert np.array_equal(got, want)


def test_ecc_campaign_is_plain_campaign_on_mantissa_flips_and_clean_elsewhere():
    sc, cams, _ = S.tiny_workload()
    fl = S.flips_stratified(14 * 32, sc.n, sc.nwords, S.FP32, S.SEED_BASE + 69)
    mask = (1 << 14) - 1
    e, _, clean = O.campaign(sc.planes, S.FP32, 0, cams, fl, guard_mode=2, word_mask=mask, nthreads=O.max_threads())
    p, _, _ = O.campaign(sc.planes, S.FP32, 0, cams, fl, clean_imgs=clean, nthreads=O.max_threads())
    corr = fl["bit"] >= 23
    assert corr.any() and (~corr).any()
    for f in ("sse", "maxabs", "footprint", "nonfinite"):
        assert np.array_equal(e[~corr][f], p[~corr][f]), f
        assert (e[corr][f] == 0).all(), f


def test_ecc_removes_catastrophes_table4():
    """Table 4: the sign+exponent code drives the catastrophe rate to zero, while
    the unprotected model has catastrophic upsets on the same grid."""
    sc, cams, _ = S.tiny_workload()
    fl = S.flips_stratified(14 * 32 * 4, sc.n, sc.nwords, S.FP32, S.SEED_BASE + 70)
    npx = 256 * 256
    thr = GOLD["definition2_catastrophe_percent"]["percent"] / 100.0
    e, _, clean = O.campaign(sc.planes, S.FP32, 0, cams, fl, guard_mode=2, word_mask=(1 << 14) - 1,
                             nthreads=O.max_threads())
    p, _, _ = O.campaign(sc.planes, S.FP32, 0, cams, fl, clean_imgs=clean, nthreads=O.max_threads())
    cat = lambda r: (r["nonfinite"] > 0) | (r["footprint"] / npx > thr)
    assert cat(p).sum() > 0
    assert cat(e).sum() == 0


# ---------------------------------------------------------------------------
# contamination of a sort-first partition (Sec. 5, cross-node contamination)
# ---------------------------------------------------------------------------
from paper_2606_21791_gb300 import contamination as CT


def test_region_cells_of_known_pixels():
    W, H = 800, 1040          # cells of 100 x 130 pixels
    base = np.full((H, W, 3), 0.5, np.float32)
    cases = [((99, 0), 0), ((100, 0), 1), ((0, 129), 0), ((0, 130), 8), ((799, 1039), 63), ((450, 600), 4 * 8 + 4)]
    for (x, y), cell in cases:
        img = base.copy()
        img[y, x, 1] = 0.9
        assert O.region_actual(img, base) == 1 << cell, (x, y)
    # strict 1/255 threshold (Definition 1) and a NaN pixel (clamped to 0 against 0.5)
    img = base.copy()
    img[0, 0, 0] = np.float32(0.5) + np.float32(1.0 / 255.0)
    assert O.region_actual(img, base) == (1 << 0 if abs(float(img[0, 0, 0]) - 0.5) > np.float32(1 / 255) else 0)
    img = base.copy()
    img[1039, 0, 2] = np.nan
    assert O.region_actual(img, base) == 1 << 56


def test_region_rect_cells():
    rec = np.zeros(1, dtype=O.REC_DTYPE)
    rec["visible"] = 1
    rec["x0"], rec["x1"], rec["y0"], rec["y1"] = 6, 8, 7, 10   # pixels 96..127 x 112..159 of 800 x 1040
    assert O.region_rect(rec, 800, 1040) == (1 << 0) | (1 << 1) | (1 << 8) | (1 << 9)
    rec["visible"] = 0
    assert O.region_rect(rec, 800, 1040) == 0


@pytest.mark.parametrize("nodes", [4, 8, 16, 32, 64])
def test_partition_regions_equal_direct_pixel_regions(nodes):
    rng = np.random.default_rng(S.SEED_BASE + 73)
    W, H = 320, 240
    rx, ry = CT.PARTITIONS[nodes]
    for _ in range(20):
        b = rng.random((H, W, 3), dtype=np.float32)
        a = b.copy()
        k = rng.integers(1, 6)
        ys, xs = rng.integers(0, H, k), rng.integers(0, W, k)
        a[ys, xs, 0] = np.where(b[ys, xs, 0] > 0.5, 0.0, 1.0)
        direct = 0
        for y, x in zip(ys, xs):
            direct |= 1 << int((y * ry // H) * rx + (x * rx // W))
        got = int(CT.region_masks(np.array([O.region_actual(a, b)], np.uint64), nodes)[0])
        assert got == direct


def test_campaign_actual_contamination_within_prediction():
    """A pixel outside both tile rects of the flipped primitive keeps its tile
    list, so it cannot change: actual cells are a subset of predicted cells.
    Corrected (ECC) upsets predict no contamination."""
    sc, cams, flips = S.tiny_workload()
    m, _, clean, act, pred = O.campaign(sc.planes, S.FP32, 0, cams, flips, nthreads=O.max_threads(), regions=True)
    assert ((act & ~pred) == 0).all()
    assert ((act != 0) == (m["footprint"] > 0)).all()
    assert (pred != 0).sum() > (act != 0).sum() > 0
    s = CT.summary(act.ravel(), pred.ravel())
    assert all(v["actual_outside_predicted"] == 0 for v in s.values())
    e, _, _, act_e, pred_e = O.campaign(sc.planes, S.FP32, 0, cams, flips, guard_mode=2, word_mask=(1 << 14) - 1,
                                        clean_imgs=clean, nthreads=O.max_threads(), regions=True)
    corr = O.ecc_corrects(S.FP32, (1 << 14) - 1, flips)
    assert corr.any() and (pred_e[corr] == 0).all() and (act_e[corr] == 0).all()


# ---------------------------------------------------------------------------
# campaign analytics (Table 2 Wilson intervals, Sec. 5 scaling-law fit)
# ---------------------------------------------------------------------------
from paper_2606_21791_gb300 import analytics as AN


@pytest.mark.parametrize("k,n", [(0, 10), (1, 10), (5, 10), (10, 10), (7, 2512), (2782, 100000), (1, 1)])
def test_wilson_interval_matches_scipy(k, n):
    st = pytest.importorskip("scipy.stats")
    ci = st.binomtest(k, n).proportion_ci(confidence_level=0.95, method="wilson")
    lo, hi = AN.wilson(k, n)
    assert abs(lo - ci.low) < 1e-12 and abs(hi - ci.high) < 1e-12


def test_wilson_closed_forms():
    n, z = 400, AN.Z95
    lo, hi = AN.wilson(0, n)
    assert lo == 0.0 and abs(hi - z * z / (n + z * z)) < 1e-15
    lo, hi = AN.wilson(n // 2, n)
    assert abs((lo + hi) / 2 - 0.5) < 1e-15


def test_loglog_fit_recovers_power_law():
    N = np.array([5e3, 2e4, 8e4, 3e5])
    a, c, r2 = AN.loglog_fit(N, 7.5 * N ** -0.83)
    assert abs(a + 0.83) < 1e-12 and abs(c - math.log(7.5)) < 1e-10 and abs(r2 - 1.0) < 1e-12


def test_severity_table_pooling_and_definition2():
    # 3 variants per field word group, 2 views, 1000-pixel frames
    words = np.array([0, 3, 3, 6, 10, 11, 20, 20])
    fl = S.flips_at(np.zeros(len(words), np.uint32), words, 0)
    rec = np.zeros((len(words), 2), dtype=[("footprint", "<u4"), ("nonfinite", "<u4")])
    rec["footprint"][1] = (30, 10)      # log-scale: 2.0% averaged -> catastrophic
    rec["footprint"][2] = (10, 10)      # log-scale: 1.0%, not above 1% -> not catastrophic
    rec["nonfinite"][5] = (0, 1)        # DC: non-finite in one view -> catastrophic
    t = AN.severity_table(fl, rec, 1000)
    assert t["log-scale"]["n"] == 2 and t["log-scale"]["catastrophe_pct"] == 50.0
    assert t["log-scale"]["max"] == 2.0 and t["log-scale"]["mean"] == 1.5
    assert t["color (DC)"]["catastrophe_pct"] == 100.0 and t["color (SH)"]["n"] == 2
    assert t["mean"]["catastrophe_pct"] == 0.0


# ---------------------------------------------------------------------------
# SSIM (Sec. 3 "Metrics and severity"; Wang et al. 2004)
# ---------------------------------------------------------------------------
def test_ssim_identical_and_constant_images():
    rng = np.random.default_rng(S.SEED_BASE + 76)
    a = rng.random((30, 41, 3), dtype=np.float32)
    assert O.ssim(a, a) == 1.0
    c1, c2 = 0.25, 0.75
    x = np.full((20, 20, 3), c1, np.float32)
    y = np.full((20, 20, 3), c2, np.float32)
    C1 = 0.01 ** 2
    want = (2 * c1 * c2 + C1) / (c1 * c1 + c2 * c2 + C1)   # variances and covariance vanish
    assert abs(O.ssim(x, y) - want) < 1e-12


def test_ssim_equals_separable_gaussian_filter_form():
    nd = pytest.importorskip("scipy.ndimage")
    rng = np.random.default_rng(S.SEED_BASE + 77)
    a = rng.random((37, 52, 3), dtype=np.float32)
    b = np.clip(a + rng.normal(0, 0.05, a.shape).astype(np.float32), -0.2, 1.2).astype(np.float32)
    b[3, 7, 1] = np.nan
    ca, cb = np.clip(np.nan_to_num(a.astype(np.float64), nan=0.0), 0, 1), np.clip(np.nan_to_num(b.astype(np.float64), nan=0.0), 0, 1)
    f = lambda z: nd.gaussian_filter(z, sigma=1.5, truncate=5 / 1.5, mode="constant")
    vals = []
    for c in range(3):
        u, v = ca[..., c], cb[..., c]
        mx, my = f(u), f(v)
        vx, vy, cxy = f(u * u) - mx * mx, f(v * v) - my * my, f(u * v) - mx * my
        C1, C2 = 0.01 ** 2, 0.03 ** 2
        m = ((2 * mx * my + C1) * (2 * cxy + C2)) / ((mx * mx + my * my + C1) * (vx + vy + C2))
        vals.append(m[5:-5, 5:-5])
    want = float(np.mean(vals))
    assert abs(O.ssim(b, a) - want) < 1e-12
    assert abs(O.ssim(a, b) - O.ssim(b, a)) < 1e-12
