/*
 * gs_oracle.c -- plain, slow CPU oracle of the single-event-upset (SEU) hot path
 * of "Single-Event Upsets in 3D Gaussian Splatting Rendering" (arXiv 2606.21791):
 * bit-flip injection, the support guard, the 3DGS forward render, and the
 * per-pixel comparison against the clean frame.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the CPU-baseline
 * leg of the benchmark may load this library.  It shares no code, header, table
 * or constant with the CUDA path and must never be used as a fallback for it.
 *
 * Precision: the study renders in fp32 (storage may be fp16/bf16, math is fp32,
 * Sec. 3 "Single-bit upset model"), so every render decision here is taken in
 * fp32 with IEEE-754 rounding of each operation (built with -ffp-contract=off,
 * no fast-math); the activations' exponential is the fp32 rounding of the
 * double exponential.  Metric sums accumulate in double.
 *
 * Conventions that the paper leaves to its external renderer (the 3DGS forward
 * pass it cites in Sec. 2 "Gaussian splatting") are fixed here as follows:
 *   - quaternion word order (w, x, y, z); zero or non-finite norm culls;
 *   - pixel (i, j) has centre (i + 0.5, j + 0.5); principal point (cx, cy);
 *   - 2D covariance gets +0.3 on its diagonal (anti-aliasing low-pass), no
 *     opacity compensation; tx/z, ty/z clamped to +-1.3 * half-FOV tangent;
 *   - radius = ceil(3 sqrt(lambda_max)), lambda_max = mid + sqrt(max(0.1, mid^2 - det));
 *   - tile rect = tiles meeting the square [px - r, px + r] x [py - r, py + r];
 *   - colour = SH(dir = normalize(mean - camera centre)) + 0.5, clamped at 0 from below;
 *   - blending: skip power > 0, skip alpha < 1/255, cap alpha at 0.99, stop a
 *     pixel before the primitive that would take T below 1e-4; over white;
 *   - the exponent power = -(ca dx^2 + cc dy^2)/2 - cb dx dy is evaluated in
 *     fp32 as s = fma(cc dy, dy, ca dx dx), power = fma(-cb dx, dy, -s/2) (the
 *     paper fixes the quadratic form, not its rounding order);
 *   - non-finite geometry culls; non-finite appearance propagates (no fminf/fmaxf).
 * Parity on every function in this file is pinned by tests against closed forms,
 * invariants, brute force and library routines (see tests/test_oracle_pins.py).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_FP32 0
#define OR_FP16 1
#define OR_BF16 2

typedef struct {
    uint32_t prim;
    uint16_t word;
    uint8_t bit;
    uint8_t pad;
} or_flip;

typedef struct {
    float R[9];
    float t[3];
    float fx, fy, cx, cy;
    int32_t width, height;
    float znear, zfar;
} or_camera;

/* one preprocessed primitive for one view */
typedef struct {
    float mx, my;            /* projected mean, pixel coordinates */
    float ca, cb, cc;        /* conic = inverse 2D covariance [[ca, cb], [cb, cc]] */
    float r, g, b;           /* view-dependent colour */
    float opac;              /* sigmoid(opacity logit) */
    float depth;             /* camera-space z */
    int32_t x0, y0, x1, y1;  /* tile rect, half open */
    int32_t radius;
    int32_t visible;         /* 1 if binned into at least one tile */
} or_rec;

typedef struct {
    double sse;              /* sum over H*W*3 of squared clamped differences */
    float maxabs;            /* max |difference| of clamped values */
    uint32_t footprint;      /* pixels with max_c |difference| > 1/255 */
    uint32_t nonfinite;      /* pixels of the first image with a non-finite channel */
    uint32_t pad;
} or_metrics;

/* ------------------------------------------------------------------------- */
/* storage formats (Sec. 3 "Single-bit upset model")                          */
/* ------------------------------------------------------------------------- */
int or_word_bytes(int fmt) { return fmt == OR_FP32 ? 4 : 2; }

static float bits_to_float(uint32_t u) {
    float f;
    memcpy(&f, &u, 4);
    return f;
}

/* exact conversion of an IEEE binary16 word to binary32 */
static float half_to_float(uint16_t h) {
    uint32_t sign = (uint32_t)(h >> 15) << 31;
    uint32_t e = (h >> 10) & 0x1fu;
    uint32_t m = h & 0x3ffu;
    uint32_t u;
    if (e == 0x1fu) {
        u = sign | 0x7f800000u | (m << 13);
    } else if (e != 0) {
        u = sign | ((e - 15u + 127u) << 23) | (m << 13);
    } else if (m == 0) {
        u = sign;
    } else {
        /* subnormal: value = m * 2^-24; normalise */
        int shift = 0;
        while ((m & 0x400u) == 0) {
            m <<= 1;
            shift++;
        }
        m &= 0x3ffu;
        u = sign | ((uint32_t)(127 - 15 - shift + 1) << 23) | (m << 13);
    }
    return bits_to_float(u);
}

/* stored word (prim i of plane w) up-converted exactly to float */
float or_load(const void* planes, int fmt, uint64_t n, int w, uint64_t i) {
    if (fmt == OR_FP32) {
        const uint32_t* p = (const uint32_t*)planes;
        return bits_to_float(p[(uint64_t)w * n + i]);
    }
    const uint16_t* p = (const uint16_t*)planes;
    uint16_t h = p[(uint64_t)w * n + i];
    if (fmt == OR_FP16) return half_to_float(h);
    return bits_to_float((uint32_t)h << 16);
}

static uint32_t load_bits(const void* planes, int fmt, uint64_t idx) {
    if (fmt == OR_FP32) return ((const uint32_t*)planes)[idx];
    return ((const uint16_t*)planes)[idx];
}

static void store_bits(void* planes, int fmt, uint64_t idx, uint32_t v) {
    if (fmt == OR_FP32)
        ((uint32_t*)planes)[idx] = v;
    else
        ((uint16_t*)planes)[idx] = (uint16_t)v;
}

static float bits_value(uint32_t bits, int fmt) {
    if (fmt == OR_FP32) return bits_to_float(bits);
    if (fmt == OR_FP16) return half_to_float((uint16_t)bits);
    return bits_to_float(bits << 16);
}

/* ------------------------------------------------------------------------- */
/* (a) injection: reinterpret the stored word as an unsigned integer of its   */
/* width and flip one bit (Sec. 3 "Single-bit upset model"). Flips apply in   */
/* list order; returns -1 on an out-of-range site.                            */
/* ------------------------------------------------------------------------- */
int or_apply_flips(void* planes, int fmt, uint64_t n, int nwords, const or_flip* flips, int64_t count) {
    int nbits = 8 * or_word_bytes(fmt);
    for (int64_t k = 0; k < count; k++) {
        const or_flip* f = &flips[k];
        if (f->prim >= n || f->word >= nwords || f->bit >= nbits) return -1;
        uint64_t idx = (uint64_t)f->word * n + f->prim;
        uint32_t v = load_bits(planes, fmt, idx);
        v ^= (1u << f->bit);
        store_bits(planes, fmt, idx, v);
    }
    return 0;
}

/* ------------------------------------------------------------------------- */
/* (f) support guard, Algorithm 1.                                            */
/* ------------------------------------------------------------------------- */
/* total order on values used for min/max: -0.0 sorts below +0.0, NaN ignored */
static int value_less(float a, float b) {
    if (a < b) return 1;
    if (a == b && signbit(a) && !signbit(b)) return 1;
    return 0;
}

/* Algorithm 1, precompute: per (field, component) word, the min and max stored
 * value over all primitives; written back as storage words. */
int or_field_box(const void* planes, int fmt, uint64_t n, int nwords, uint32_t* lo_bits, uint32_t* hi_bits) {
    for (int w = 0; w < nwords; w++) {
        int have = 0;
        uint32_t lo = 0, hi = 0;
        float lov = 0.f, hiv = 0.f;
        for (uint64_t i = 0; i < n; i++) {
            uint32_t b = load_bits(planes, fmt, (uint64_t)w * n + i);
            float v = bits_value(b, fmt);
            if (isnan(v)) continue;
            if (!have) {
                lo = hi = b;
                lov = hiv = v;
                have = 1;
                continue;
            }
            if (value_less(v, lov)) {
                lo = b;
                lov = v;
            }
            if (value_less(hiv, v)) {
                hi = b;
                hiv = v;
            }
        }
        lo_bits[w] = lo;
        hi_bits[w] = hi;
    }
    return 0;
}

/* Algorithm 1, per frame: for every guarded word (bit w of word_mask) of every
 * primitive, a value that is non-finite or outside [lo, hi] is replaced by the
 * nearer endpoint (NaN goes to lo) and counted.  mode 0 (FIELD): box_lo/box_hi
 * hold one storage word per word index; mode 1 (PRIM): they are planes
 * [nbox_words][n] of per-primitive endpoints.  Returns the clamp count. */
int or_guard(void* planes, int fmt, uint64_t n, int nwords, uint64_t word_mask, int mode,
             const void* box_lo, const void* box_hi, int nbox_words, uint64_t* clamps_out) {
    uint64_t clamps = 0;
    for (int w = 0; w < nwords; w++) {
        if (!((word_mask >> w) & 1u)) continue;
        if (mode == 1 && w >= nbox_words) return -1;
        for (uint64_t i = 0; i < n; i++) {
            uint64_t idx = (uint64_t)w * n + i;
            float x = bits_value(load_bits(planes, fmt, idx), fmt);
            uint32_t lob, hib;
            if (mode == 0) {
                lob = ((const uint32_t*)box_lo)[w];
                hib = ((const uint32_t*)box_hi)[w];
            } else {
                lob = load_bits(box_lo, fmt, idx);
                hib = load_bits(box_hi, fmt, idx);
            }
            float lo = bits_value(lob, fmt), hi = bits_value(hib, fmt);
            if (x >= lo && x <= hi) continue;
            store_bits(planes, fmt, idx, (x > hi) ? hib : lob);
            clamps++;
        }
    }
    *clamps_out = clamps;
    return 0;
}

/* ------------------------------------------------------------------------- */
/* (b) preprocess: activations of Sec. 3 "Parameter layout" (exp of the       */
/* log-scale, normalised quaternion, logistic opacity) and the EWA projection */
/* of the 3DGS forward pass.                                                   */
/* ------------------------------------------------------------------------- */

/* real spherical-harmonic basis up to degree 3 at unit direction (x, y, z),
 * ordered by degree l and, within a degree, m = -l..l, with the signs of the
 * Condon-Shortley phase.  Constants from their closed forms. */
static void sh_basis(float x, float y, float z, int degree, float* Y) {
    const double pi = 3.14159265358979323846;
    float c0 = (float)(0.5 * sqrt(1.0 / pi));
    float c1 = (float)sqrt(3.0 / (4.0 * pi));
    Y[0] = c0;
    if (degree < 1) return;
    Y[1] = -c1 * y;
    Y[2] = c1 * z;
    Y[3] = -c1 * x;
    if (degree < 2) return;
    float c2a = (float)(0.5 * sqrt(15.0 / pi));
    float c2b = (float)(0.25 * sqrt(5.0 / pi));
    float c2c = (float)(0.25 * sqrt(15.0 / pi));
    float xx = x * x, yy = y * y, zz = z * z;
    float xy = x * y, yz = y * z, xz = x * z;
    Y[4] = c2a * xy;
    Y[5] = -c2a * yz;
    Y[6] = c2b * (2.0f * zz - xx - yy);
    Y[7] = -c2a * xz;
    Y[8] = c2c * (xx - yy);
    if (degree < 3) return;
    float c3a = (float)(0.25 * sqrt(35.0 / (2.0 * pi)));
    float c3b = (float)(0.5 * sqrt(105.0 / pi));
    float c3c = (float)(0.25 * sqrt(21.0 / (2.0 * pi)));
    float c3d = (float)(0.25 * sqrt(7.0 / pi));
    float c3e = (float)(0.25 * sqrt(105.0 / pi));
    Y[9] = -c3a * y * (3.0f * xx - yy);
    Y[10] = c3b * xy * z;
    Y[11] = -c3c * y * (4.0f * zz - xx - yy);
    Y[12] = c3d * z * (2.0f * zz - 3.0f * xx - 3.0f * yy);
    Y[13] = -c3c * x * (4.0f * zz - xx - yy);
    Y[14] = c3e * z * (xx - yy);
    Y[15] = -c3a * x * (xx - 3.0f * yy);
}

/* exposed for the basis pin test */
void or_sh_basis(float x, float y, float z, int degree, float* Y) { sh_basis(x, y, z, degree, Y); }

static int finite3(float a, float b, float c) { return isfinite(a) && isfinite(b) && isfinite(c); }

/* The exponential of the activations (exp of the log-scale, the logistic of the
 * opacity).  The paper fixes fp32 rendering but no exp; a plain expf differs
 * between math libraries by an ulp on many inputs, and for needle-like
 * primitives the 2x2 determinant a c - b^2 cancels so strongly that one ulp in a
 * scale decides whether the primitive is culled.  So the exponential is defined
 * here as one fixed fp32 evaluation: Cody and Waite's argument reduction,
 * exp(x) = 2^k exp(r) with k the nearest integer to x / ln 2 and
 * r = x - k ln 2 (ln 2 split into a head with 12 trailing zero bits, so k times
 * the head is exact, and a tail), then the Taylor polynomial of exp(r) to
 * degree 7 in Horner form with correctly rounded fused multiply-adds.  |r| is
 * at most about 0.347, so the truncation error is below 0.1 ulp and the result
 * is within about 1 ulp of exp(x) (pinned against the double exponential).  Any
 * fp32 evaluation of the same steps gives the same bits. */
static float pow2i(int e) { /* 2^e, -126 <= e <= 127 */
    const uint32_t b = (uint32_t)(e + 127) << 23;
    float f;
    memcpy(&f, &b, sizeof f);
    return f;
}

static float exp_f32(float x) {
    if (isnan(x)) return x;
    if (x > 89.0f) return INFINITY;
    if (x < -104.0f) return 0.0f; /* below half the smallest subnormal */
    const float k = rintf(x * 1.44269502f); /* 1 / ln 2 */
    float r = fmaf(-k, 0.693115234375f, x); /* head of ln 2 */
    r = fmaf(-k, 3.19461833e-05f, r);       /* tail of ln 2 */
    float p = 1.98412701e-04f;              /* 1/7! */
    p = fmaf(p, r, 1.38888892e-03f);        /* 1/6! */
    p = fmaf(p, r, 8.33333377e-03f);        /* 1/5! */
    p = fmaf(p, r, 4.16666679e-02f);        /* 1/4! */
    p = fmaf(p, r, 1.66666672e-01f);        /* 1/3! */
    p = fmaf(p, r, 0.5f);
    p = fmaf(p, r, 1.0f);
    p = fmaf(p, r, 1.0f);
    const int ki = (int)k; /* -150 ... 128 */
    if (ki > 127) return (p * pow2i(127)) * pow2i(ki - 127);
    if (ki < -126) return (p * pow2i(ki + 100)) * pow2i(-100); /* one rounding into the subnormals */
    return p * pow2i(ki);
}

/* exposed for the pin test */
void or_exp_f32(const float* x, float* y, int64_t n) {
    for (int64_t i = 0; i < n; i++) y[i] = exp_f32(x[i]);
}

void or_preprocess_one(const void* planes, int fmt, uint64_t n, int sh_degree, uint64_t i, const or_camera* cam,
                       int tile_w, int tile_h, or_rec* out) {
    memset(out, 0, sizeof(*out));
    const float* R = cam->R;
    const float* t = cam->t;
    float mu[3];
    for (int k = 0; k < 3; k++) mu[k] = or_load(planes, fmt, n, k, i);

    /* camera-space position p = R mu + t */
    float p[3];
    for (int r = 0; r < 3; r++) p[r] = R[3 * r + 0] * mu[0] + R[3 * r + 1] * mu[1] + R[3 * r + 2] * mu[2] + t[r];
    if (!finite3(p[0], p[1], p[2])) return;
    if (!(p[2] > cam->znear) || !(p[2] < cam->zfar)) return;

    /* scale s = exp(log-scale) */
    float s[3];
    for (int k = 0; k < 3; k++) s[k] = exp_f32(or_load(planes, fmt, n, 3 + k, i));

    /* rotation from the normalised quaternion (w, x, y, z) */
    float qw = or_load(planes, fmt, n, 6, i), qx = or_load(planes, fmt, n, 7, i);
    float qy = or_load(planes, fmt, n, 8, i), qz = or_load(planes, fmt, n, 9, i);
    float qn2 = qw * qw + qx * qx + qy * qy + qz * qz;
    if (!(qn2 > 0.0f) || !isfinite(qn2)) return;
    float qn = sqrtf(qn2);
    qw = qw / qn;
    qx = qx / qn;
    qy = qy / qn;
    qz = qz / qn;
    float Rq[9];
    Rq[0] = 1.0f - 2.0f * (qy * qy + qz * qz);
    Rq[1] = 2.0f * (qx * qy - qw * qz);
    Rq[2] = 2.0f * (qx * qz + qw * qy);
    Rq[3] = 2.0f * (qx * qy + qw * qz);
    Rq[4] = 1.0f - 2.0f * (qx * qx + qz * qz);
    Rq[5] = 2.0f * (qy * qz - qw * qx);
    Rq[6] = 2.0f * (qx * qz - qw * qy);
    Rq[7] = 2.0f * (qy * qz + qw * qx);
    Rq[8] = 1.0f - 2.0f * (qx * qx + qy * qy);

    /* world covariance Sigma = (Rq S)(Rq S)^T */
    float M[9];
    for (int r = 0; r < 3; r++)
        for (int c = 0; c < 3; c++) M[3 * r + c] = Rq[3 * r + c] * s[c];
    float Sg[9];
    for (int r = 0; r < 3; r++)
        for (int c = 0; c < 3; c++) Sg[3 * r + c] = M[3 * r + 0] * M[3 * c + 0] + M[3 * r + 1] * M[3 * c + 1] + M[3 * r + 2] * M[3 * c + 2];

    /* camera covariance V = R Sigma R^T */
    float RS[9], V[9];
    for (int r = 0; r < 3; r++)
        for (int c = 0; c < 3; c++) RS[3 * r + c] = R[3 * r + 0] * Sg[0 * 3 + c] + R[3 * r + 1] * Sg[1 * 3 + c] + R[3 * r + 2] * Sg[2 * 3 + c];
    for (int r = 0; r < 3; r++)
        for (int c = 0; c < 3; c++) V[3 * r + c] = RS[3 * r + 0] * R[3 * c + 0] + RS[3 * r + 1] * R[3 * c + 1] + RS[3 * r + 2] * R[3 * c + 2];

    /* EWA: Jacobian of the perspective projection at the (clamped) mean */
    float z = p[2];
    float limx = 1.3f * (0.5f * (float)cam->width / cam->fx);
    float limy = 1.3f * (0.5f * (float)cam->height / cam->fy);
    float ux = p[0] / z, uy = p[1] / z;
    if (ux < -limx) ux = -limx;
    if (ux > limx) ux = limx;
    if (uy < -limy) uy = -limy;
    if (uy > limy) uy = limy;
    float tx = ux * z, ty = uy * z;
    float J00 = cam->fx / z, J02 = -(cam->fx * tx) / (z * z);
    float J11 = cam->fy / z, J12 = -(cam->fy * ty) / (z * z);
    /* cov2 = J V J^T with J = [[J00, 0, J02], [0, J11, J12]] */
    float JV0[3], JV1[3];
    for (int c = 0; c < 3; c++) {
        JV0[c] = J00 * V[0 * 3 + c] + J02 * V[2 * 3 + c];
        JV1[c] = J11 * V[1 * 3 + c] + J12 * V[2 * 3 + c];
    }
    float a = JV0[0] * J00 + JV0[2] * J02 + 0.3f;
    float b = JV0[1] * J11 + JV0[2] * J12;
    float c = JV1[1] * J11 + JV1[2] * J12 + 0.3f;

    float det = a * c - b * b;
    if (!(det > 0.0f) || !isfinite(det)) return;
    float ca = c / det, cb = -b / det, cc = a / det;
    if (!finite3(ca, cb, cc)) return;
    float mid = 0.5f * (a + c);
    float disc = mid * mid - det;
    if (disc < 0.1f) disc = 0.1f;
    float lmax = mid + sqrtf(disc);
    float rad = ceilf(3.0f * sqrtf(lmax));
    if (!(rad > 0.0f) || !isfinite(rad)) return;

    float mx = cam->fx * (p[0] / z) + cam->cx;
    float my = cam->fy * (p[1] / z) + cam->cy;
    if (!isfinite(mx) || !isfinite(my)) return;

    int tiles_x = (cam->width + tile_w - 1) / tile_w;
    int tiles_y = (cam->height + tile_h - 1) / tile_h;
    float fx0 = floorf((mx - rad) / (float)tile_w), fx1 = floorf((mx + rad) / (float)tile_w) + 1.0f;
    float fy0 = floorf((my - rad) / (float)tile_h), fy1 = floorf((my + rad) / (float)tile_h) + 1.0f;
    if (fx0 < 0.0f) fx0 = 0.0f;
    if (fy0 < 0.0f) fy0 = 0.0f;
    if (fx1 > (float)tiles_x) fx1 = (float)tiles_x;
    if (fy1 > (float)tiles_y) fy1 = (float)tiles_y;
    if (fx0 > (float)tiles_x) fx0 = (float)tiles_x;
    if (fy0 > (float)tiles_y) fy0 = (float)tiles_y;
    if (fx1 < 0.0f) fx1 = 0.0f;
    if (fy1 < 0.0f) fy1 = 0.0f;
    int x0 = (int)fx0, x1 = (int)fx1, y0 = (int)fy0, y1 = (int)fy1;
    if (x1 <= x0 || y1 <= y0) return;

    /* colour: SH at the viewing direction, + 0.5, clamped below at 0 */
    float cpos[3];
    for (int k = 0; k < 3; k++) cpos[k] = -(R[0 * 3 + k] * t[0] + R[1 * 3 + k] * t[1] + R[2 * 3 + k] * t[2]);
    float d0 = mu[0] - cpos[0], d1 = mu[1] - cpos[1], d2 = mu[2] - cpos[2];
    float dn = sqrtf(d0 * d0 + d1 * d1 + d2 * d2);
    d0 = d0 / dn;
    d1 = d1 / dn;
    d2 = d2 / dn;
    float Y[16];
    sh_basis(d0, d1, d2, sh_degree, Y);
    int ncoef = (sh_degree + 1) * (sh_degree + 1);
    float rgb[3];
    for (int ch = 0; ch < 3; ch++) {
        float acc = Y[0] * or_load(planes, fmt, n, 11 + ch, i);
        for (int j = 1; j < ncoef; j++) acc = acc + Y[j] * or_load(planes, fmt, n, 14 + 3 * (j - 1) + ch, i);
        acc = acc + 0.5f;
        rgb[ch] = (acc < 0.0f) ? 0.0f : acc;
    }

    /* opacity = logistic(logit) */
    float o = or_load(planes, fmt, n, 10, i);
    float opac = 1.0f / (1.0f + exp_f32(-o));

    out->mx = mx;
    out->my = my;
    out->ca = ca;
    out->cb = cb;
    out->cc = cc;
    out->r = rgb[0];
    out->g = rgb[1];
    out->b = rgb[2];
    out->opac = opac;
    out->depth = z;
    out->x0 = x0;
    out->y0 = y0;
    out->x1 = x1;
    out->y1 = y1;
    out->radius = (int32_t)rad;
    out->visible = 1;
}

int or_preprocess(const void* planes, int fmt, uint64_t n, int sh_degree, const or_camera* cam, int tile_w,
                  int tile_h, or_rec* out) {
    for (uint64_t i = 0; i < n; i++) or_preprocess_one(planes, fmt, n, sh_degree, i, cam, tile_w, tile_h, &out[i]);
    return 0;
}

/* ------------------------------------------------------------------------- */
/* (c) binning: per tile, the primitives whose rect covers it, front to back  */
/* by depth with ties broken by primitive index.                               */
/* ------------------------------------------------------------------------- */
typedef struct {
    float depth;
    uint32_t id;
} depth_id;

static int cmp_depth_id(const void* pa, const void* pb) {
    const depth_id* a = (const depth_id*)pa;
    const depth_id* b = (const depth_id*)pb;
    if (a->depth < b->depth) return -1;
    if (a->depth > b->depth) return 1;
    if (a->id < b->id) return -1;
    if (a->id > b->id) return 1;
    return 0;
}

/* offsets: ntiles+1 entries; ids: capacity cap.  Returns the pair count, or -1
 * if cap is too small (offsets are then still valid). */
int64_t or_bin(const or_rec* recs, uint64_t n, int tiles_x, int tiles_y, uint32_t* offsets, uint32_t* ids,
               uint64_t cap) {
    int64_t ntiles = (int64_t)tiles_x * tiles_y;
    memset(offsets, 0, sizeof(uint32_t) * (size_t)(ntiles + 1));
    for (uint64_t i = 0; i < n; i++) {
        if (!recs[i].visible) continue;
        for (int ty = recs[i].y0; ty < recs[i].y1; ty++)
            for (int tx = recs[i].x0; tx < recs[i].x1; tx++) offsets[(int64_t)ty * tiles_x + tx + 1]++;
    }
    for (int64_t t = 0; t < ntiles; t++) offsets[t + 1] += offsets[t];
    uint64_t total = offsets[ntiles];
    if (total > cap) return -1;
    uint32_t* fill = (uint32_t*)calloc((size_t)ntiles, sizeof(uint32_t));
    for (uint64_t i = 0; i < n; i++) {
        if (!recs[i].visible) continue;
        for (int ty = recs[i].y0; ty < recs[i].y1; ty++)
            for (int tx = recs[i].x0; tx < recs[i].x1; tx++) {
                int64_t tile = (int64_t)ty * tiles_x + tx;
                ids[offsets[tile] + fill[tile]++] = (uint32_t)i;
            }
    }
    free(fill);
    depth_id* tmp = NULL;
    size_t tmpcap = 0;
    for (int64_t t = 0; t < ntiles; t++) {
        uint32_t a = offsets[t], b = offsets[t + 1];
        size_t len = b - a;
        if (len < 2) continue;
        if (len > tmpcap) {
            free(tmp);
            tmpcap = len;
            tmp = (depth_id*)malloc(sizeof(depth_id) * tmpcap);
        }
        for (size_t k = 0; k < len; k++) {
            tmp[k].id = ids[a + k];
            tmp[k].depth = recs[ids[a + k]].depth;
        }
        qsort(tmp, len, sizeof(depth_id), cmp_depth_id);
        for (size_t k = 0; k < len; k++) ids[a + k] = tmp[k].id;
    }
    free(tmp);
    return (int64_t)total;
}

/* ------------------------------------------------------------------------- */
/* (d) front-to-back alpha blending over white (Sec. 3 "Metrics and severity" */
/* composites over white; the cutoffs are 1/255 on alpha and 1e-4 on T).       */
/* ------------------------------------------------------------------------- */
/* margin (may be NULL): how close the pixel's discrete decisions came to their
 * thresholds, as relative distances over the entries walked up to the stop:
 * margin[0] = min |alpha - 1/255| / (1/255) over entries with power <= 0 (the
 * skip test), margin[1] = min |T' - 1e-4| / 1e-4 over entries that pass it (the
 * stop test).  A renderer whose exponential rounds differently can take another
 * decision only where one of these is small.  Diagnostic only: the pixel's
 * value does not depend on it. */
static void blend_pixel(const or_rec* recs, const uint32_t* list, size_t len, float pxc, float pyc, float* out3,
                        float* margin) {
    const double a_thr = (double)(1.0f / 255.0f), t_thr = (double)1e-4f;
    double ma = INFINITY, mt = INFINITY;
    float T = 1.0f;
    float C[3] = {0.0f, 0.0f, 0.0f};
    for (size_t k = 0; k < len; k++) {
        const or_rec* g = &recs[list[k]];
        float dx = g->mx - pxc;
        float dy = g->my - pyc;
        /* the exponent -(ca dx^2 + cc dy^2) / 2 - cb dx dy in fp32 as two fused
         * multiply-adds, the other products rounded on their own:
         * s = fma(cc dy, dy, ca dx dx), power = fma(-cb dx, dy, -s / 2) */
        float t1 = (g->ca * dx) * dx;
        float s = fmaf(g->cc * dy, dy, t1);
        float power = fmaf(-g->cb * dx, dy, -0.5f * s);
        if (power > 0.0f) continue;
        float alpha = g->opac * expf(power);
        if (margin) {
            double m = fabs((double)alpha - a_thr) / a_thr;
            if (m < ma) ma = m;
        }
        if (alpha < 1.0f / 255.0f) continue;
        if (alpha > 0.99f) alpha = 0.99f;
        float Tn = T * (1.0f - alpha);
        if (margin) {
            double m = fabs((double)Tn - t_thr) / t_thr;
            if (m < mt) mt = m;
        }
        if (Tn < 1e-4f) break;
        C[0] = C[0] + g->r * alpha * T;
        C[1] = C[1] + g->g * alpha * T;
        C[2] = C[2] + g->b * alpha * T;
        T = Tn;
    }
    out3[0] = C[0] + T * 1.0f;
    out3[1] = C[1] + T * 1.0f;
    out3[2] = C[2] + T * 1.0f;
    if (margin) {
        margin[0] = (float)ma;
        margin[1] = (float)mt;
    }
}

/* tiled blend of the per-tile sorted lists; img is H*W*3, row-major; margins
 * (H*W*2, may be NULL) as in blend_pixel */
static void blend_tiles(const or_rec* recs, const uint32_t* offsets, const uint32_t* ids, int W, int H, int tile_w,
                        int tile_h, float* img, float* margins) {
    int tiles_x = (W + tile_w - 1) / tile_w;
    for (int y = 0; y < H; y++)
        for (int x = 0; x < W; x++) {
            int64_t tile = (int64_t)(y / tile_h) * tiles_x + (x / tile_w);
            uint32_t a = offsets[tile], b = offsets[tile + 1];
            int64_t p = (int64_t)y * W + x;
            blend_pixel(recs, ids + a, b - a, (float)x + 0.5f, (float)y + 0.5f, &img[p * 3],
                        margins ? &margins[p * 2] : NULL);
        }
}

int or_blend(const or_rec* recs, const uint32_t* offsets, const uint32_t* ids, int W, int H, int tile_w,
             int tile_h, float* img) {
    blend_tiles(recs, offsets, ids, W, H, tile_w, tile_h, img, NULL);
    return 0;
}

/* brute force: for each pixel scan every primitive, keep those whose tile rect
 * contains the pixel's tile, order them by (depth, index), and blend.  No
 * binning pass. */
int or_blend_brute(const or_rec* recs, uint64_t n, int W, int H, int tile_w, int tile_h, float* img) {
    depth_id* cand = (depth_id*)malloc(sizeof(depth_id) * (n ? n : 1));
    uint32_t* list = (uint32_t*)malloc(sizeof(uint32_t) * (n ? n : 1));
    for (int y = 0; y < H; y++)
        for (int x = 0; x < W; x++) {
            int tx = x / tile_w, ty = y / tile_h;
            size_t m = 0;
            for (uint64_t i = 0; i < n; i++) {
                const or_rec* g = &recs[i];
                if (!g->visible) continue;
                if (tx < g->x0 || tx >= g->x1 || ty < g->y0 || ty >= g->y1) continue;
                cand[m].depth = g->depth;
                cand[m].id = (uint32_t)i;
                m++;
            }
            qsort(cand, m, sizeof(depth_id), cmp_depth_id);
            for (size_t k = 0; k < m; k++) list[k] = cand[k].id;
            blend_pixel(recs, list, m, (float)x + 0.5f, (float)y + 0.5f, &img[((int64_t)y * W + x) * 3], NULL);
        }
    free(cand);
    free(list);
    return 0;
}

/* ------------------------------------------------------------------------- */
/* (e) comparison against the clean frame: Definition 1 (footprint: pixels    */
/* changed by more than one 8-bit level), PSNR's squared error, peak error,   */
/* non-finite flag (Sec. 3 "Metrics and severity").  Differences are taken on */
/* images clamped to [0, 1] (NaN counts as 0); the non-finite count looks at  */
/* the raw first image.                                                       */
/* ------------------------------------------------------------------------- */
static float clamp01(float v) {
    if (v > 0.0f) return (v < 1.0f) ? v : 1.0f;
    return 0.0f;
}

int or_compare(const float* a, const float* b, int H, int W, or_metrics* out) {
    double sse = 0.0;
    float maxabs = 0.0f;
    uint32_t foot = 0, nonfin = 0;
    for (int64_t p = 0; p < (int64_t)H * W; p++) {
        float m = 0.0f;
        int bad = 0;
        for (int ch = 0; ch < 3; ch++) {
            float va = a[p * 3 + ch], vb = b[p * 3 + ch];
            if (!isfinite(va)) bad = 1;
            float d = clamp01(va) - clamp01(vb);
            float ad = fabsf(d);
            sse += (double)d * (double)d;
            if (ad > m) m = ad;
        }
        if (m > maxabs) maxabs = m;
        if (m > 1.0f / 255.0f) foot++;
        nonfin += (uint32_t)bad;
    }
    out->sse = sse;
    out->maxabs = maxabs;
    out->footprint = foot;
    out->nonfinite = nonfin;
    out->pad = 0;
    return 0;
}

/* ------------------------------------------------------------------------- */
/* whole forward render of one view                                           */
/* ------------------------------------------------------------------------- */
/* margins: H*W*2 decision margins of every pixel (as in blend_pixel), or NULL */
int or_render_margins(const void* planes, int fmt, uint64_t n, int sh_degree, const or_camera* cam, int tile_w,
                      int tile_h, float* img, float* margins) {
    int W = cam->width, H = cam->height;
    int tiles_x = (W + tile_w - 1) / tile_w, tiles_y = (H + tile_h - 1) / tile_h;
    int64_t ntiles = (int64_t)tiles_x * tiles_y;
    or_rec* recs = (or_rec*)malloc(sizeof(or_rec) * (n ? n : 1));
    or_preprocess(planes, fmt, n, sh_degree, cam, tile_w, tile_h, recs);
    uint64_t total = 0;
    for (uint64_t i = 0; i < n; i++)
        if (recs[i].visible) total += (uint64_t)(recs[i].x1 - recs[i].x0) * (uint64_t)(recs[i].y1 - recs[i].y0);
    uint32_t* offsets = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)(ntiles + 1));
    uint32_t* ids = (uint32_t*)malloc(sizeof(uint32_t) * (total ? total : 1));
    int64_t got = or_bin(recs, n, tiles_x, tiles_y, offsets, ids, total);
    int rc = (got < 0) ? -1 : 0;
    if (rc == 0) blend_tiles(recs, offsets, ids, W, H, tile_w, tile_h, img, margins);
    free(ids);
    free(offsets);
    free(recs);
    return rc;
}

int or_render(const void* planes, int fmt, uint64_t n, int sh_degree, const or_camera* cam, int tile_w, int tile_h,
              float* img) {
    return or_render_margins(planes, fmt, n, sh_degree, cam, tile_w, tile_h, img, NULL);
}

/* ------------------------------------------------------------------------- */
/* injection campaign (Sec. 3 "Parallel injection engine"): for each variant, */
/* corrupt a copy of the clean parameters with its flips, optionally guard it */
/* (Algorithm 1), render every view and compare with the clean render of the  */
/* same precision.  out: nvar*K metrics, clamps_out: nvar (may be NULL).       */
/* Variants run in parallel over nthreads OpenMP threads (each owns a copy).  */
/* ------------------------------------------------------------------------- */
/* ------------------------------------------------------------------------- */
/* ECC emulation (Sec. 5 "Alternative defenses", Table 4, "ECC sign+exp"): a  */
/* code that protects the sign and exponent bits of the stored words corrects */
/* any single upset there, so such an upset leaves the model unchanged;       */
/* mantissa upsets are not covered.  Protected bits: fp32 23-31, fp16 10-15,  */
/* bf16 7-15, of the words in word_mask.                                       */
/* ------------------------------------------------------------------------- */
int or_ecc_first_bit(int fmt) { return fmt == OR_FP32 ? 23 : (fmt == OR_FP16 ? 10 : 7); }

int or_ecc_corrects(int fmt, uint64_t word_mask, const or_flip* f) {
    return f->word < 64 && ((word_mask >> f->word) & 1ull) && (int)f->bit >= or_ecc_first_bit(fmt);
}

/* ------------------------------------------------------------------------- */
/* SSIM (Sec. 3 "Metrics and severity", Wang et al. 2004): per channel, local */
/* Gaussian-weighted means, variances and covariance over an 11x11 window     */
/* (sigma 1.5, weights normalised to sum 1), SSIM = (2 mx my + C1)(2 sxy + C2) */
/* / ((mx^2 + my^2 + C1)(sx^2 + sy^2 + C2)), C1 = 0.01^2, C2 = 0.03^2 (data    */
/* range 1), on images clamped to [0, 1] (NaN as 0, like the other metrics);   */
/* the mean over the windows that lie inside the frame and over the channels. */
/* Direct 2-D window sums in double.                                           */
/* ------------------------------------------------------------------------- */
double or_ssim(const float* a, const float* b, int H, int W) {
    const int R = 5;
    double w1[11], ws = 0.0;
    for (int i = -R; i <= R; i++) ws += (w1[i + R] = exp(-(double)(i * i) / (2.0 * 1.5 * 1.5)));
    for (int i = 0; i < 11; i++) w1[i] /= ws;
    const double C1 = 0.01 * 0.01, C2 = 0.03 * 0.03;
    if (H <= 2 * R || W <= 2 * R) return 1.0;
    double total = 0.0;
    for (int y = R; y < H - R; y++)
        for (int x = R; x < W - R; x++)
            for (int c = 0; c < 3; c++) {
                double mx = 0, my = 0, sxx = 0, syy = 0, sxy = 0;
                for (int dy = -R; dy <= R; dy++)
                    for (int dx = -R; dx <= R; dx++) {
                        const int64_t q = ((int64_t)(y + dy) * W + (x + dx)) * 3 + c;
                        const double w = w1[dy + R] * w1[dx + R];
                        const double u = clamp01(a[q]), v = clamp01(b[q]);
                        mx += w * u;
                        my += w * v;
                        sxx += w * u * u;
                        syy += w * v * v;
                        sxy += w * u * v;
                    }
                const double vx = sxx - mx * mx, vy = syy - my * my, cxy = sxy - mx * my;
                total += ((2 * mx * my + C1) * (2 * cxy + C2)) / ((mx * mx + my * my + C1) * (vx + vy + C2));
            }
    return total / (3.0 * (double)(H - 2 * R) * (double)(W - 2 * R));
}

/* ------------------------------------------------------------------------- */
/* Contamination of a sort-first partition (Sec. 5 "Cross-node contamination */
/* in distributed rendering"): each node renders the primitives whose        */
/* footprint overlaps its screen region, so an upset contaminates the regions */
/* its primitive reaches.  Regions are unions of the cells of an 8x8 screen   */
/* grid, cell of pixel (x, y) = (8x / W, 8y / H), bit 8 cy + cx; the 4-, 8-,  */
/* 16-, 32- and 64-node partitions (2x2, 4x2, 4x4, 8x4, 8x8) are unions of    */
/* cells.  Actual: cells holding a footprint pixel (Definition 1).            */
/* Predicted: cells met by the tile rect of the changed primitive before or   */
/* after the upset (the node that drew it and the one that draws it now).     */
/* ------------------------------------------------------------------------- */
static uint32_t or_load_bits(const void* planes, int fmt, uint64_t n, int w, uint64_t i) {
    if (fmt == OR_FP32) return ((const uint32_t*)planes)[(uint64_t)w * n + i];
    return ((const uint16_t*)planes)[(uint64_t)w * n + i];
}

static uint64_t cell_bit(int x, int y, int W, int H) {
    const int cx = (int)(((int64_t)x * 8) / W), cy = (int)(((int64_t)y * 8) / H);
    return 1ull << (cy * 8 + cx);
}

uint64_t or_region_actual(const float* a, const float* b, int H, int W) {
    uint64_t m = 0;
    for (int y = 0; y < H; y++)
        for (int x = 0; x < W; x++) {
            const int64_t p = ((int64_t)y * W + x) * 3;
            float mx = 0.0f;
            for (int ch = 0; ch < 3; ch++) {
                const float d = fabsf(clamp01(a[p + ch]) - clamp01(b[p + ch]));
                if (d > mx) mx = d;
            }
            if (mx > 1.0f / 255.0f) m |= cell_bit(x, y, W, H);
        }
    return m;
}

uint64_t or_region_rect(const or_rec* r, int W, int H, int tile_w, int tile_h) {
    if (!r->visible || r->x1 <= r->x0 || r->y1 <= r->y0) return 0;
    const int px0 = r->x0 * tile_w, py0 = r->y0 * tile_h;
    const int px1 = (r->x1 * tile_w < W ? r->x1 * tile_w : W) - 1; /* inclusive */
    const int py1 = (r->y1 * tile_h < H ? r->y1 * tile_h : H) - 1;
    uint64_t m = 0;
    for (int y = py0; y <= py1; y++)
        for (int x = px0; x <= px1; x++) m |= cell_bit(x, y, W, H);
    return m;
}

int or_campaign(const void* clean, int fmt, uint64_t n, int nwords, int sh_degree, const or_camera* cams, int K,
                int tile_w, int tile_h, const float* clean_imgs, const or_flip* flips, int64_t nvar,
                int flips_per_variant, int guard_mode, uint64_t word_mask, const void* box_lo, const void* box_hi,
                int nbox_words, or_metrics* out, uint64_t* clamps_out, int nthreads, uint64_t* reg_actual,
                uint64_t* reg_pred, double* ssim_out) {
    size_t bytes = (size_t)n * (size_t)nwords * (size_t)or_word_bytes(fmt);
    int64_t px = 0;
    for (int k = 0; k < K; k++) px += (int64_t)cams[k].width * cams[k].height * 3;
    int err = 0;
#ifdef _OPENMP
    if (nthreads < 1) nthreads = 1;
#pragma omp parallel num_threads(nthreads)
#endif
    {
        void* work = malloc(bytes ? bytes : 1);
        float* img = (float*)malloc(sizeof(float) * (size_t)(px ? px : 1));
#ifdef _OPENMP
#pragma omp for schedule(dynamic, 1)
#endif
        for (int64_t v = 0; v < nvar; v++) {
            memcpy(work, clean, bytes);
            const or_flip* fv = flips + v * flips_per_variant;
            if (guard_mode == 2) { /* ECC: corrected upsets are not applied */
                for (int f = 0; f < flips_per_variant; f++)
                    if (!or_ecc_corrects(fmt, word_mask, &fv[f]) && or_apply_flips(work, fmt, n, nwords, &fv[f], 1) != 0)
                        err = 1;
            } else if (or_apply_flips(work, fmt, n, nwords, fv, flips_per_variant) != 0) {
                err = 1;
                continue;
            }
            uint64_t cl = 0;
            if (guard_mode == 0 || guard_mode == 1) {
                if (or_guard(work, fmt, n, nwords, word_mask, guard_mode, box_lo, box_hi, nbox_words, &cl) != 0) err = 1;
            }
            if (clamps_out) clamps_out[v] = cl;
            int64_t off = 0;
            for (int k = 0; k < K; k++) {
                int64_t sz = (int64_t)cams[k].width * cams[k].height * 3;
                if (or_render(work, fmt, n, sh_degree, &cams[k], tile_w, tile_h, img + off) != 0) err = 1;
                or_compare(img + off, clean_imgs + off, cams[k].height, cams[k].width, &out[v * K + k]);
                if (reg_actual)
                    reg_actual[v * K + k] = or_region_actual(img + off, clean_imgs + off, cams[k].height, cams[k].width);
                if (ssim_out) ssim_out[v * K + k] = or_ssim(img + off, clean_imgs + off, cams[k].height, cams[k].width);
                if (reg_pred) {
                    uint64_t m = 0;
                    for (int f = 0; f < flips_per_variant; f++) {
                        const uint64_t p = fv[f].prim;
                        if (p >= n) continue;
                        int changed = 0;
                        for (int w = 0; w < nwords; w++)
                            if (or_load_bits(work, fmt, n, w, p) != or_load_bits(clean, fmt, n, w, p)) changed = 1;
                        if (!changed) continue;
                        or_rec rc, rv;
                        or_preprocess_one(clean, fmt, n, sh_degree, p, &cams[k], tile_w, tile_h, &rc);
                        or_preprocess_one(work, fmt, n, sh_degree, p, &cams[k], tile_w, tile_h, &rv);
                        m |= or_region_rect(&rc, cams[k].width, cams[k].height, tile_w, tile_h);
                        m |= or_region_rect(&rv, cams[k].width, cams[k].height, tile_w, tile_h);
                    }
                    reg_pred[v * K + k] = m;
                }
                off += sz;
            }
        }
        free(img);
        free(work);
    }
    return err ? -1 : 0;
}

int or_max_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
