// (b) preprocess: the activations of Sec. 3 "Parameter layout" (exp of the
// log-scale, normalised quaternion, logistic opacity, SH colour up to degree 3)
// and the EWA projection of the 3DGS forward pass, one thread per primitive.
//
// This translation unit is compiled with -fmad=false: every product and sum is
// rounded on its own, in a fixed order, so the geometry that decides binning
// (depth, projected mean, radius, tile rect) is reproducible bit for bit between
// the full preprocess, the dirty-tile injector below, and any fp32 evaluation
// with the same operation order.
//
// Conventions fixed here (the paper defers its renderer to an external library):
// quaternion (w, x, y, z); 2D covariance + 0.3 on the diagonal; tx/z, ty/z
// clamped to +-1.3 half-FOV tangents; radius = ceil(3 sqrt(lambda_max)) with
// lambda_max = mid + sqrt(max(0.1, mid^2 - det)); tile rect = tiles meeting
// [mx - r, mx + r] x [my - r, my + r]; colour = SH(normalize(mean - camera
// centre)) + 0.5 clamped at 0 from below; non-finite geometry culls, non-finite
// appearance propagates.
#include "gs_internal.h"

namespace gs {

namespace {

// real SH basis constants (closed forms)
constexpr float kC0 = 0.28209479177387814f;   // 1/(2 sqrt(pi))
constexpr float kC1 = 0.48860251190291992f;   // sqrt(3/(4 pi))
constexpr float kC2a = 1.0925484305920792f;   // sqrt(15/pi)/2
constexpr float kC2b = 0.31539156525252005f;  // sqrt(5/pi)/4
constexpr float kC2c = 0.54627421529603959f;  // sqrt(15/pi)/4
constexpr float kC3a = 0.59004358992664352f;  // sqrt(35/(2 pi))/4
constexpr float kC3b = 2.8906114426405538f;   // sqrt(105/pi)/2
constexpr float kC3c = 0.45704579946446572f;  // sqrt(21/(2 pi))/4
constexpr float kC3d = 0.37317633259011546f;  // sqrt(7/pi)/4
constexpr float kC3e = 1.4453057213202769f;   // sqrt(105/pi)/4

template <int FMT>
__device__ __forceinline__ float decode(uint32_t b) {
    if (FMT == GS_FP32) return __uint_as_float(b);
    if (FMT == GS_FP16) return __half2float(__ushort_as_half((unsigned short)b));
    return __uint_as_float(b << 16);
}

template <int FMT>
__device__ __forceinline__ uint32_t load_bits(const void* planes, uint64_t n, int w, uint64_t i) {
    if (FMT == GS_FP32) return __ldg((const uint32_t*)planes + (uint64_t)w * n + i);
    return __ldg((const unsigned short*)planes + (uint64_t)w * n + i);
}

__device__ __forceinline__ bool finite3(float a, float b, float c) {
    return isfinite(a) && isfinite(b) && isfinite(c);
}

// Exponential of the activations, one fixed fp32 evaluation: Cody and Waite's
// argument reduction, exp(x) = 2^k exp(r) with k the nearest integer to x / ln 2
// and r = x - k ln 2 (ln 2 as a head with 12 trailing zero bits, so k times the
// head is exact, plus a tail), then the degree-7 Taylor polynomial of exp(r) in
// Horner form with correctly rounded fused multiply-adds (|r| <= ~0.347: within
// about 1 ulp of exp).  Every fp32 evaluation of these steps gives the same
// bits, so cull decisions agree with any other such evaluation: for needle-like
// primitives the determinant a c - b^2 cancels so strongly that one ulp in a
// scale decides whether the primitive is culled.  No FP64 (slow on this part).
__device__ __forceinline__ float pow2i(int e) { return __int_as_float((e + 127) << 23); }   // -126 <= e <= 127

__device__ __forceinline__ float exp_f32(float x) {
    if (isnan(x)) return x;
    if (x > 89.0f) return INFINITY;
    if (x < -104.0f) return 0.0f;   // below half the smallest subnormal
    const float k = rintf(__fmul_rn(x, 1.44269502f));   // 1 / ln 2
    float r = __fmaf_rn(-k, 0.693115234375f, x);         // head of ln 2
    r = __fmaf_rn(-k, 3.19461833e-05f, r);               // tail of ln 2
    float p = 1.98412701e-04f;                           // 1/7!
    p = __fmaf_rn(p, r, 1.38888892e-03f);                // 1/6!
    p = __fmaf_rn(p, r, 8.33333377e-03f);                // 1/5!
    p = __fmaf_rn(p, r, 4.16666679e-02f);                // 1/4!
    p = __fmaf_rn(p, r, 1.66666672e-01f);                // 1/3!
    p = __fmaf_rn(p, r, 0.5f);
    p = __fmaf_rn(p, r, 1.0f);
    p = __fmaf_rn(p, r, 1.0f);
    const int ki = (int)k;   // -150 ... 128
    if (ki > 127) return __fmul_rn(__fmul_rn(p, pow2i(127)), pow2i(ki - 127));
    if (ki < -126) return __fmul_rn(__fmul_rn(p, pow2i(ki + 100)), pow2i(-100));   // one rounding into the subnormals
    return __fmul_rn(p, pow2i(ki));
}

// Conservative half extents of a box that contains every pixel centre where the
// blend can compute alpha >= 1/255 for this primitive.  The blend evaluates
// power = -(ca dx^2 + cc dy^2)/2 - cb dx dy in fp32 with every operation
// rounded, so its result is within g * M of the exact quadratic form of the
// fp32 conic, M = (|ca| dx^2 + |cc| dy^2)/2 + |cb| |dx dy|, g = 1e-6 (several
// ulps).  alpha >= 1/255 needs power >= -L, L = ln(255 opac) (+ a margin for
// the exponential), so candidate pixels satisfy d^T Q'' d <= 2 L with
// Q'' = [[ca - g (|ca| + |cb|), cb], [cb, cc - g (|cc| + |cb|)]].  If Q'' is
// positive definite its ellipse's bounding box is returned; otherwise the
// candidates are unbounded (near-degenerate conics) and the box is infinite.
// NaN opacity gives NaN extents, which never cull.
__device__ __forceinline__ void cull_extent(float ca, float cb, float cc, float opac, float* ex, float* ey) {
    float lim = logf(255.0f * opac);
    if (lim < -1e-3f) {   // alpha <= opac < 1/255 everywhere
        *ex = -INFINITY;
        *ey = -INFINITY;
        return;
    }
    if (isnan(lim)) {
        *ex = NAN;
        *ey = NAN;
        return;
    }
    // Q'' in fp32: the margin is doubled (2g) so that the fp32 rounding of these
    // few operations (~1e-7 relative) stays inside it, and the determinant is
    // lowered by a bound on its own rounding error, so the box can only grow.
    const float acb = fabsf(cb);
    const float qxx = ca - 2e-6f * (fabsf(ca) + acb);
    const float qyy = cc - 2e-6f * (fabsf(cc) + acb);
    const float pxy = qxx * qyy, pcb = cb * cb;
    const float det = (pxy - pcb) - 4.8e-7f * (fabsf(pxy) + pcb);
    // huge terms: the blend's own power can overflow (and be NaN, which it
    // blends), so such a record is never culled
    if (!(qxx > 0.0f) || !(det > 0.0f) || !(pxy < 1e37f) || !(fmaxf(fmaxf(fabsf(ca), fabsf(cc)), acb) < 1e30f)) {
        *ex = INFINITY;
        *ey = INFINITY;
        return;
    }
    const float q = 2.0f * (fmaxf(lim, 0.0f) + 1e-3f);
    *ex = sqrtf(q * qyy / det) * (1.0f + 1e-5f) + 0.01f;
    *ey = sqrtf(q * qxx / det) * (1.0f + 1e-5f) + 0.01f;
}

// Preprocess one primitive.  `src(w)` returns the float value of word w.
// Returns false when the primitive is culled (not binned).
template <typename Src>
__device__ __forceinline__ bool preprocess_core(Src src, int sh_degree, const DevCamera& cam, BlendRec& rec,
                                                uint2& rect, float& radius) {
    const float* R = cam.R;
    const float* t = cam.t;
    float mu0 = src(0), mu1 = src(1), mu2 = src(2);
    float p0 = R[0] * mu0 + R[1] * mu1 + R[2] * mu2 + t[0];
    float p1 = R[3] * mu0 + R[4] * mu1 + R[5] * mu2 + t[1];
    float z = R[6] * mu0 + R[7] * mu1 + R[8] * mu2 + t[2];
    if (!finite3(p0, p1, z)) return false;
    if (!(z > cam.znear) || !(z < cam.zfar)) return false;

    float s0 = exp_f32(src(3)), s1 = exp_f32(src(4)), s2 = exp_f32(src(5));

    float qw = src(6), qx = src(7), qy = src(8), qz = src(9);
    float qn2 = qw * qw + qx * qx + qy * qy + qz * qz;
    if (!(qn2 > 0.0f) || !isfinite(qn2)) return false;
    float qn = sqrtf(qn2);
    qw = qw / qn;
    qx = qx / qn;
    qy = qy / qn;
    qz = qz / qn;
    float r00 = 1.0f - 2.0f * (qy * qy + qz * qz);
    float r01 = 2.0f * (qx * qy - qw * qz);
    float r02 = 2.0f * (qx * qz + qw * qy);
    float r10 = 2.0f * (qx * qy + qw * qz);
    float r11 = 1.0f - 2.0f * (qx * qx + qz * qz);
    float r12 = 2.0f * (qy * qz - qw * qx);
    float r20 = 2.0f * (qx * qz - qw * qy);
    float r21 = 2.0f * (qy * qz + qw * qx);
    float r22 = 1.0f - 2.0f * (qx * qx + qy * qy);

    // M = Rq diag(s); Sigma = M M^T (symmetric: compute all 9 in a fixed order)
    float m00 = r00 * s0, m01 = r01 * s1, m02 = r02 * s2;
    float m10 = r10 * s0, m11 = r11 * s1, m12 = r12 * s2;
    float m20 = r20 * s0, m21 = r21 * s1, m22 = r22 * s2;
    float S[9];
    S[0] = m00 * m00 + m01 * m01 + m02 * m02;
    S[1] = m00 * m10 + m01 * m11 + m02 * m12;
    S[2] = m00 * m20 + m01 * m21 + m02 * m22;
    S[3] = m10 * m00 + m11 * m01 + m12 * m02;
    S[4] = m10 * m10 + m11 * m11 + m12 * m12;
    S[5] = m10 * m20 + m11 * m21 + m12 * m22;
    S[6] = m20 * m00 + m21 * m01 + m22 * m02;
    S[7] = m20 * m10 + m21 * m11 + m22 * m12;
    S[8] = m20 * m20 + m21 * m21 + m22 * m22;

    // camera covariance V = R Sigma R^T
    float RS[9], V[9];
#pragma unroll
    for (int r = 0; r < 3; r++)
#pragma unroll
        for (int c = 0; c < 3; c++) RS[3 * r + c] = R[3 * r + 0] * S[c] + R[3 * r + 1] * S[3 + c] + R[3 * r + 2] * S[6 + c];
#pragma unroll
    for (int r = 0; r < 3; r++)
#pragma unroll
        for (int c = 0; c < 3; c++)
            V[3 * r + c] = RS[3 * r + 0] * R[3 * c + 0] + RS[3 * r + 1] * R[3 * c + 1] + RS[3 * r + 2] * R[3 * c + 2];

    // perspective Jacobian at the mean, with the view-frustum clamp
    float limx = 1.3f * (0.5f * (float)cam.W / cam.fx);
    float limy = 1.3f * (0.5f * (float)cam.H / cam.fy);
    float ux = p0 / z, uy = p1 / z;
    if (ux < -limx) ux = -limx;
    if (ux > limx) ux = limx;
    if (uy < -limy) uy = -limy;
    if (uy > limy) uy = limy;
    float tx = ux * z, ty = uy * z;
    float j00 = cam.fx / z, j02 = -(cam.fx * tx) / (z * z);
    float j11 = cam.fy / z, j12 = -(cam.fy * ty) / (z * z);
    float jv00 = j00 * V[0] + j02 * V[6];
    float jv01 = j00 * V[1] + j02 * V[7];
    float jv02 = j00 * V[2] + j02 * V[8];
    float jv11 = j11 * V[4] + j12 * V[7];
    float jv12 = j11 * V[5] + j12 * V[8];
    float a = jv00 * j00 + jv02 * j02 + 0.3f;
    float b = jv01 * j11 + jv02 * j12;
    float c = jv11 * j11 + jv12 * j12 + 0.3f;

    float det = a * c - b * b;
    if (!(det > 0.0f) || !isfinite(det)) return false;
    float ca = c / det, cb = -b / det, cc = a / det;
    if (!finite3(ca, cb, cc)) return false;
    float mid = 0.5f * (a + c);
    float disc = mid * mid - det;
    if (disc < 0.1f) disc = 0.1f;
    float lmax = mid + sqrtf(disc);
    float rad = ceilf(3.0f * sqrtf(lmax));
    if (!(rad > 0.0f) || !isfinite(rad)) return false;
    radius = rad;

    float mx = cam.fx * (p0 / z) + cam.cx;
    float my = cam.fy * (p1 / z) + cam.cy;
    if (!isfinite(mx) || !isfinite(my)) return false;

    const float tw = (float)cam.tile_w, th = (float)cam.tile_h;
    const float ftx = (float)cam.tiles_x, fty = (float)cam.tiles_y;
    float fx0 = floorf((mx - rad) / tw), fx1 = floorf((mx + rad) / tw) + 1.0f;
    float fy0 = floorf((my - rad) / th), fy1 = floorf((my + rad) / th) + 1.0f;
    fx0 = fminf(fmaxf(fx0, 0.0f), ftx);   // operands finite here
    fy0 = fminf(fmaxf(fy0, 0.0f), fty);
    fx1 = fminf(fmaxf(fx1, 0.0f), ftx);
    fy1 = fminf(fmaxf(fy1, 0.0f), fty);
    int x0 = (int)fx0, x1 = (int)fx1, y0 = (int)fy0, y1 = (int)fy1;
    if (x1 <= x0 || y1 <= y0) return false;

    // colour: SH at the viewing direction
    float cp0 = -(R[0] * t[0] + R[3] * t[1] + R[6] * t[2]);
    float cp1 = -(R[1] * t[0] + R[4] * t[1] + R[7] * t[2]);
    float cp2 = -(R[2] * t[0] + R[5] * t[1] + R[8] * t[2]);
    float d0 = mu0 - cp0, d1 = mu1 - cp1, d2 = mu2 - cp2;
    float dn = sqrtf(d0 * d0 + d1 * d1 + d2 * d2);
    float x = d0 / dn, y = d1 / dn, zz_ = d2 / dn;
    float Y[16];
    Y[0] = kC0;
    int ncoef = 1;
    if (sh_degree >= 1) {
        Y[1] = -kC1 * y;
        Y[2] = kC1 * zz_;
        Y[3] = -kC1 * x;
        ncoef = 4;
    }
    if (sh_degree >= 2) {
        float xx = x * x, yy = y * y, zz = zz_ * zz_;
        float xy = x * y, yz = y * zz_, xz = x * zz_;
        Y[4] = kC2a * xy;
        Y[5] = -kC2a * yz;
        Y[6] = kC2b * (2.0f * zz - xx - yy);
        Y[7] = -kC2a * xz;
        Y[8] = kC2c * (xx - yy);
        ncoef = 9;
        if (sh_degree >= 3) {
            Y[9] = -kC3a * y * (3.0f * xx - yy);
            Y[10] = kC3b * xy * zz_;
            Y[11] = -kC3c * y * (4.0f * zz - xx - yy);
            Y[12] = kC3d * zz_ * (2.0f * zz - 3.0f * xx - 3.0f * yy);
            Y[13] = -kC3c * x * (4.0f * zz - xx - yy);
            Y[14] = kC3e * zz_ * (xx - yy);
            Y[15] = -kC3a * x * (xx - 3.0f * yy);
            ncoef = 16;
        }
    }
    float rgb[3];
#pragma unroll
    for (int ch = 0; ch < 3; ch++) {
        float acc = Y[0] * src(11 + ch);
        for (int j = 1; j < ncoef; j++) acc = acc + Y[j] * src(14 + 3 * (j - 1) + ch);
        acc = acc + 0.5f;
        rgb[ch] = (acc < 0.0f) ? 0.0f : acc;
    }
    float o = src(10);
    float opac = 1.0f / (1.0f + exp_f32(-o));

    rec.mx = mx;
    rec.my = my;
    rec.ca = ca;
    rec.cb = cb;
    rec.cc = cc;
    rec.opac = opac;
    cull_extent(ca, cb, cc, opac, &rec.ex, &rec.ey);
    rec.r = rgb[0];
    rec.g = rgb[1];
    rec.b = rgb[2];
    rec.depth = z;
    rect = make_uint2((uint32_t)x0 | ((uint32_t)y0 << 16), (uint32_t)x1 | ((uint32_t)y1 << 16));
    return true;
}

// The outputs of one preprocessed primitive: blend record, packed tile rect,
// depth-sort key and value (invisible: key 0xffffffff), and the debug record.
__device__ __forceinline__ void write_prep(uint64_t i, bool vis, BlendRec rec, uint2 rect, float rad, BlendRec* recs,
                                           uint2* rects, uint32_t* keys, uint32_t* vals, gs_record* dbg) {
    if (!vis) {
        rec = BlendRec{0, 0, 0, 0, 0, 0, -INFINITY, -INFINITY, 0, 0, 0, 0};
        rect = make_uint2(0, 0);
    }
    if (recs) recs[i] = rec;
    if (rects) rects[i] = rect;
    if (keys) {
        keys[i] = vis ? __float_as_uint(rec.depth) : 0xffffffffu;
        vals[i] = (uint32_t)i;
    }
    if (dbg) {
        gs_record g;
        memset(&g, 0, sizeof(g));
        if (vis) {
            g.mx = rec.mx;
            g.my = rec.my;
            g.ca = rec.ca;
            g.cb = rec.cb;
            g.cc = rec.cc;
            g.r = rec.r;
            g.g = rec.g;
            g.b = rec.b;
            g.opac = rec.opac;
            g.depth = rec.depth;
            g.x0 = rect.x & 0xffff;
            g.y0 = rect.x >> 16;
            g.x1 = rect.y & 0xffff;
            g.y1 = rect.y >> 16;
            g.radius = (int32_t)rad;
            g.visible = 1;
        }
        dbg[i] = g;
    }
}

constexpr int kPrepThreads = 128;

// A primitive's words, staged in shared memory (this thread's column only).
template <int FMT>
struct StagedSrc {
    const uint32_t (*sw)[kPrepThreads];
    int t;
    __device__ float operator()(int w) const { return decode<FMT>(sw[w][t]); }
};

// full preprocess: records, packed rects, depth-sort keys (invisible: 0xffffffff).
// One thread per primitive.  Each thread first copies its primitive's stored
// words into shared memory, eight loads in flight at a time (a warp reads 32
// consecutive words of one plane per load), then computes from there: the
// planes stream at full width instead of one dependent load per use.
template <int FMT>
__global__ __launch_bounds__(kPrepThreads) void k_preprocess(const void* planes, uint64_t n, int nwords,
                                                             int sh_degree, DevCamera cam, BlendRec* recs,
                                                             uint2* rects, uint32_t* keys, uint32_t* vals,
                                                             gs_record* dbg) {
    __shared__ uint32_t sw[kMaxWords][kPrepThreads];
    const int t = threadIdx.x;
    uint64_t i = (uint64_t)blockIdx.x * kPrepThreads + t;
    if (i >= n) return;
#pragma unroll 8
    for (int w = 0; w < nwords; w++) sw[w][t] = load_bits<FMT>(planes, n, w, i);
    BlendRec rec;
    uint2 rect = make_uint2(0, 0);
    float rad = 0.0f;
    const bool vis = preprocess_core(StagedSrc<FMT>{sw, t}, sh_degree, cam, rec, rect, rad);
    write_prep(i, vis, rec, rect, rad, recs, rects, keys, vals, dbg);
}

// ---------------------------------------------------------------------------
// Full preprocess with the parameter planes staged by bulk copies (TMA)
// ---------------------------------------------------------------------------
// Persistent blocks of 128 threads walk tiles of 128 consecutive primitives.
// For each tile one thread issues one bulk copy per parameter plane
// (cp.async.bulk: the tile's 128 words of that plane) into one of two
// shared-memory stages, completing on the stage's mbarrier, one tile ahead of
// the tile being computed: a block keeps a whole tile's words (30 KB in fp32)
// in flight while it computes the previous tile, where the per-thread kernel
// above keeps eight loads.  A bulk copy needs 16-byte aligned addresses and a
// size that is a multiple of 16 bytes; plane w of tile t starts at word
// w n + 128 t, so this kernel runs when n is a multiple of 4 (fp32) or 8
// (fp16/bf16) and the per-thread kernel otherwise.  Every wait is bounded: a
// block whose wait gives up sets bit 1 of the scene's device error word, waits
// (bounded again) for its copies in flight and returns.
constexpr int kTmaStages = 2;
constexpr unsigned kWaitLimit = 1u << 20;   // mbarrier polls before a wait gives up

__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, unsigned parity) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return done != 0u;
}

__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, unsigned parity) {
    for (unsigned it = 0; it < kWaitLimit; it++)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}

// a primitive's words in a stage: plane w at w * 128 words, this thread's column t
template <int FMT>
struct StageSrc {
    const unsigned char* st;
    int t;
    __device__ float operator()(int w) const {
        if (FMT == GS_FP32) return decode<FMT>(reinterpret_cast<const uint32_t*>(st)[w * kPrepThreads + t]);
        return decode<FMT>(reinterpret_cast<const unsigned short*>(st)[w * kPrepThreads + t]);
    }
};

template <int FMT>
__global__ __launch_bounds__(kPrepThreads) void k_preprocess_tma(const void* planes, uint64_t n, int nwords,
                                                                 int sh_degree, DevCamera cam, BlendRec* recs,
                                                                 uint2* rects, uint32_t* keys, uint32_t* vals,
                                                                 gs_record* dbg, unsigned int* err) {
    extern __shared__ __align__(128) unsigned char stage_mem[];
    __shared__ __align__(8) uint64_t bar[kTmaStages];
    constexpr unsigned esz = FMT == GS_FP32 ? 4u : 2u;
    const int t = threadIdx.x;
    const size_t stage_bytes = (size_t)nwords * kPrepThreads * esz;
    const uint64_t ntile = (n + kPrepThreads - 1) / kPrepThreads;
    if (t == 0) {
        for (int s = 0; s < kTmaStages; s++)
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(&bar[s])) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    // thread 0: the tile's planes into stage s, completing on bar[s]
    auto issue = [&](uint64_t tile, int s) {
        const uint64_t p0 = tile * kPrepThreads;
        const unsigned bytes = (unsigned)min((uint64_t)kPrepThreads, n - p0) * esz;
        unsigned char* dst = stage_mem + (size_t)s * stage_bytes;
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(&bar[s])),
                     "r"(bytes * (unsigned)nwords)
                     : "memory");
        for (int w = 0; w < nwords; w++) {
            const unsigned char* src = static_cast<const unsigned char*>(planes) + ((uint64_t)w * n + p0) * esz;
            asm volatile(
                "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                    smem_addr(dst + (size_t)w * kPrepThreads * esz)),
                "l"(src), "r"(bytes), "r"(smem_addr(&bar[s]))
                : "memory");
        }
    };
    uint64_t tile = blockIdx.x;
    if (t == 0 && tile < ntile) issue(tile, 0);
    // tile k of this block uses stage k & 1 for the (k >> 1)-th time: mbarrier phase parity (k >> 1) & 1
    for (int k = 0; tile < ntile; tile += gridDim.x, k++) {
        const int s = k & 1;
        const unsigned parity = (unsigned)(k >> 1) & 1u;
        const uint64_t next = tile + gridDim.x;
        // stage s ^ 1 was released by the barrier that ended the previous tile
        if (t == 0 && next < ntile) issue(next, s ^ 1);
        const bool ok = mbar_wait_bounded(&bar[s], parity);
        if (__syncthreads_or(!ok)) {
            if (t == 0) atomicOr(err, 2u);
            mbar_wait_bounded(&bar[s], parity);   // the block's copies in flight land first
            if (next < ntile) mbar_wait_bounded(&bar[s ^ 1], (unsigned)((k + 1) >> 1) & 1u);
            return;
        }
        const uint64_t i = tile * kPrepThreads + (uint64_t)t;
        if (i < n) {
            BlendRec rec;
            uint2 rect = make_uint2(0, 0);
            float rad = 0.0f;
            const bool vis = preprocess_core(StageSrc<FMT>{stage_mem + (size_t)s * stage_bytes, t}, sh_degree, cam,
                                             rec, rect, rad);
            write_prep(i, vis, rec, rect, rad, recs, rects, keys, vals, dbg);
        }
        __syncthreads();   // every thread is done with stage s before it is refilled
    }
}

// ---------------------------------------------------------------------------
// Dirty-tile injector: one warp per variant.  The lanes gather the flipped
// primitive's words, XOR the upset in the storage format and optionally guard
// them (Algorithm 1 applied to the only primitive that can leave its box); then
// lane k preprocesses the corrupted primitive for view k and describes the
// dirty tiles: the union of its clean and corrupted tile rects, each cut to the
// tiles its record's alpha >= 1/255 box reaches.  A record changes no pixel of
// a tile outside its box, so there it may stay in (clean record) or out of
// (corrupted record) the tile's merged list without changing a bit.  The
// per-view comparison accumulators are zeroed here (guard clamps reported on
// view 0).
// ---------------------------------------------------------------------------
struct SharedSrc {
    const float* v;
    __device__ float operator()(int w) const { return v[w]; }
};

constexpr int kPrepWarps = 8;

// The tiles of a binned rect (packed x0 | y0 << 16, x1 | y1 << 16) that hold a
// pixel centre of the record's alpha >= 1/255 box, packed the same way ((0, 0):
// none).  An entry changes no pixel outside that box, so a tile outside it is
// not dirty for this record.  A NaN or infinite box keeps the whole rect; the
// pixel bounds take one pixel of slack on each side against rounding.
__device__ __forceinline__ uint2 alpha_tiles(uint2 rect, const BlendRec& r, int tw, int th) {
    const float ex = r.ex, ey = r.ey;
    if (!(ex < INFINITY) || !(ey < INFINITY) || !isfinite(r.mx) || !isfinite(r.my)) return rect;   // no bound
    if (ex < 0.0f || ey < 0.0f) return make_uint2(0u, 0u);    // -inf: alpha < 1/255 everywhere
    const float x0 = rect.x & 0xffff, y0 = rect.x >> 16, x1 = rect.y & 0xffff, y1 = rect.y >> 16;
    // tiles [floor((mx - ex - 1) / tw), floor((mx + ex) / tw)] (clamped in float before converting)
    const float fx0 = fminf(fmaxf(floorf((r.mx - ex - 1.0f) / (float)tw), x0), x1);
    const float fx1 = fminf(fmaxf(floorf((r.mx + ex) / (float)tw) + 1.0f, x0), x1);
    const float fy0 = fminf(fmaxf(floorf((r.my - ey - 1.0f) / (float)th), y0), y1);
    const float fy1 = fminf(fmaxf(floorf((r.my + ey) / (float)th) + 1.0f, y0), y1);
    if (!(fx1 > fx0) || !(fy1 > fy0)) return make_uint2(0u, 0u);
    return make_uint2((uint32_t)fx0 | ((uint32_t)fy0 << 16), (uint32_t)fx1 | ((uint32_t)fy1 << 16));
}

template <int FMT>
__global__ __launch_bounds__(kPrepWarps * 32) void k_inject_prep(
    const void* planes, uint64_t n, int nwords, int sh_degree, const DevCamera* cams, int K, const gs_flip* flips,
    int B, int guard_mode, uint64_t mask, const uint32_t* box, const void* pblo, const void* pbhi, int nbox,
    const uint2* const* clean_rects, const BlendRec* const* clean_recs, DirtyDesc* desc, uint32_t* n_items,
    CmpAcc* acc) {
    __shared__ float sv[kPrepWarps][kMaxWords];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int b = blockIdx.x * kPrepWarps + wib;
    if (b >= B) return;   // whole warps only; no block-wide barrier below
    const gs_flip f = flips[b];
    const int nbits = FMT == GS_FP32 ? 32 : 16;
    // an upset the sign+exponent code corrects leaves the variant clean (zero record)
    const bool corrected =
        guard_mode == GS_GUARD_ECC && f.word < 64 && ((mask >> f.word) & 1ull) && f.bit >= ecc_first_bit(FMT);
    const bool ok = f.prim < n && f.word < nwords && f.bit < nbits && !corrected;
    const uint32_t p = ok ? f.prim : 0u;
    unsigned int clamps = 0;
    bool changed = false;   // does any stored word of the primitive end up different
    for (int w = lane; w < nwords; w += 32) {
        const uint32_t orig = load_bits<FMT>(planes, n, w, p);
        uint32_t bits = orig;
        if (ok && w == f.word) bits ^= (1u << f.bit);
        float x = decode<FMT>(bits);
        if ((guard_mode == GS_GUARD_FIELD || guard_mode == GS_GUARD_PRIM) && ((mask >> w) & 1ull)) {
            uint32_t lb, hb;
            if (guard_mode == GS_GUARD_FIELD) {
                lb = box[w];
                hb = box[kMaxWords + w];
            } else {
                lb = w < nbox ? load_bits<FMT>(pblo, n, w, p) : 0u;
                hb = w < nbox ? load_bits<FMT>(pbhi, n, w, p) : 0u;
            }
            const float lo = decode<FMT>(lb), hi = decode<FMT>(hb);
            if (!(x >= lo && x <= hi)) {
                clamps++;
                x = (x > hi) ? hi : lo;
            }
        }
        sv[wib][w] = x;
        changed |= __float_as_uint(x) != __float_as_uint(decode<FMT>(orig));
    }
    clamps = __reduce_add_sync(0xffffffffu, clamps);
    changed = ok && __any_sync(0xffffffffu, changed);
    __syncwarp();
    if (lane >= K) return;
    const int k = lane, bk = b * K + k;
    DirtyDesc d;
    d.prim = p;
    uint2 rect = make_uint2(0, 0);
    float rad = 0.0f;
    const bool nvb = ok && preprocess_core(SharedSrc{sv[wib]}, sh_degree, cams[k], d.rec, rect, rad);
    const uint2 orect_b = ok ? clean_rects[k][p] : make_uint2(0, 0);   // binned rects (contamination cells)
    const uint2 rect_b = nvb ? rect : make_uint2(0, 0);
    // dirty tiles: the binned rects cut to the records' alpha boxes
    if (nvb) rect = alpha_tiles(rect, d.rec, cams[k].tile_w, cams[k].tile_h);
    const uint2 orect = orect_b.y != 0u ? alpha_tiles(orect_b, clean_recs[k][p], cams[k].tile_w, cams[k].tile_h)
                                        : orect_b;
    const bool nv = nvb && (rect.x & 0xffff) < (rect.y & 0xffff) && (rect.x >> 16) < (rect.y >> 16);
    const uint32_t ox0 = orect.x & 0xffff, oy0 = orect.x >> 16, ox1 = orect.y & 0xffff, oy1 = orect.y >> 16;
    const bool ov = ox1 > ox0 && oy1 > oy0;
    uint32_t nx0 = rect.x & 0xffff, ny0 = rect.x >> 16, nx1 = rect.y & 0xffff, ny1 = rect.y >> 16;
    if (!nv) nx0 = ny0 = nx1 = ny1 = 0;
    const uint32_t an = nv ? (nx1 - nx0) * (ny1 - ny0) : 0u;
    const uint32_t ao = ov ? (ox1 - ox0) * (oy1 - oy0) : 0u;
    uint32_t ix = 0, iy = 0;
    if (nv && ov) {
        const int lx = max((int)nx0, (int)ox0), hx = min((int)nx1, (int)ox1);
        const int ly = max((int)ny0, (int)oy0), hy = min((int)ny1, (int)oy1);
        ix = hx > lx ? (uint32_t)(hx - lx) : 0u;
        iy = hy > ly ? (uint32_t)(hy - ly) : 0u;
    }
    const uint32_t items = an + ao - ix * iy;
    d.new_vis = nv;
    d.old_vis = ov;
    d.old_depth = ov ? clean_recs[k][p].depth : 0.0f;
    d.pad[0] = d.pad[1] = d.pad[2] = 0u;
    d.n_items = items;
    d.nx0 = (uint16_t)nx0;
    d.ny0 = (uint16_t)ny0;
    d.nx1 = (uint16_t)nx1;
    d.ny1 = (uint16_t)ny1;
    d.ox0 = (uint16_t)ox0;
    d.oy0 = (uint16_t)oy0;
    d.ox1 = (uint16_t)ox1;
    d.oy1 = (uint16_t)oy1;
    if (!nv) d.rec = BlendRec{0, 0, 0, 0, 0, 0, -INFINITY, -INFINITY, 0, 0, 0, 0};
    desc[bk] = d;
    n_items[bk] = items;
    CmpAcc z;
    z.sse_fx = 0ull;
    z.maxabs_bits = 0u;
    z.footprint = 0u;
    z.nonfinite = 0u;
    z.clamps = (k == 0) ? clamps : 0u;   // clamps reported once per variant, on view 0
    z.clean_nonfinite_replaced = 0u;
    z.pad = 0u;
    z.reg_actual = 0ull;
    z.ssim_fx = 0ull;
    // contamination prediction: the cells the primitive's tile rects meet, before
    // and after the upset, when its stored words changed
    const int tw = cams[k].tile_w, th = cams[k].tile_h;
    z.reg_pred = changed ? rect_cells(orect_b, cams[k].W, cams[k].H, tw, th) |
                               rect_cells(rect_b, cams[k].W, cams[k].H, tw, th)
                         : 0ull;
    acc[bk] = z;
}

// Exclusive scan of the dirty-tile counts of the B*K <= kMaxPairs (variant,
// view) pairs (single block of 1024 threads, kPairsPerThread consecutive pairs
// each); resets the work-queue counters.
constexpr int kPairsPerThread = kMaxPairs / 1024;
__global__ __launch_bounds__(1024) void k_items_scan(const uint32_t* n_items, int total, uint32_t* item_off,
                                                     unsigned int* queue) {
    __shared__ uint32_t wsum[32];
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    uint32_t a[kPairsPerThread];
    uint32_t items = 0;
#pragma unroll
    for (int j = 0; j < kPairsPerThread; j++) {
        const int p = tid * kPairsPerThread + j;
        a[j] = p < total ? n_items[p] : 0u;
        items += a[j];
    }
    uint32_t x = items;
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) wsum[wid] = x;
    __syncthreads();
    if (wid == 0) {
        uint32_t s = wsum[lane];
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t y = __shfl_up_sync(0xffffffffu, s, o);
            if (lane >= o) s += y;
        }
        wsum[lane] = s;
    }
    __syncthreads();
    uint32_t run = x - items + (wid > 0 ? wsum[wid - 1] : 0u);   // exclusive offset of this thread's first pair
#pragma unroll
    for (int j = 0; j < kPairsPerThread; j++) {
        const int p = tid * kPairsPerThread + j;
        if (p < total) item_off[p] = run;
        run += a[j];
        if (p == total - 1) item_off[total] = run;
    }
    if (tid == 0) {
        queue[0] = 0u;
        queue[1] = 0u;
        queue[2] = 0u;
        queue[3] = 0u;
        queue[4] = 0u;
        queue[6] += 1u;   // batch generation (tags of the dirty-tile SSIM maps)
    }
}

}  // namespace

DevCamera make_dev_camera(const gs_camera& c, int tile_w, int tile_h) {
    DevCamera d;
    memcpy(d.R, c.R, sizeof(d.R));
    memcpy(d.t, c.t, sizeof(d.t));
    d.fx = c.fx;
    d.fy = c.fy;
    d.cx = c.cx;
    d.cy = c.cy;
    d.W = c.width;
    d.H = c.height;
    d.znear = c.znear;
    d.zfar = c.zfar;
    d.tile_w = tile_w;
    d.tile_h = tile_h;
    d.tiles_x = (c.width + tile_w - 1) / tile_w;
    d.tiles_y = (c.height + tile_h - 1) / tile_h;
    return d;
}

template <int FMT>
gs_status launch_preprocess_fmt(const gs_scene* s, const DevCamera& cam, BlendRec* recs, uint2* rects,
                                uint32_t* keys, uint32_t* vals, gs_record* dbg, cudaStream_t st) {
    constexpr uint64_t esz = FMT == GS_FP32 ? 4 : 2;
    if ((s->n * esz) % 16 == 0) {   // every plane of every tile starts on a 16-byte boundary
        const int smem = (int)(kTmaStages * (uint64_t)s->nwords * kPrepThreads * esz);
        GS_CUDA(cudaFuncSetAttribute(k_preprocess_tma<FMT>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
        int per_sm = 0;
        GS_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_preprocess_tma<FMT>, kPrepThreads, smem));
        const uint64_t ntile = div_up(s->n, kPrepThreads);
        const unsigned blocks = (unsigned)std::min<uint64_t>(ntile, (uint64_t)std::max(per_sm, 1) * num_sms());
        k_preprocess_tma<FMT><<<blocks, kPrepThreads, smem, st>>>(s->planes, s->n, s->nwords, s->sh_degree, cam,
                                                                   recs, rects, keys, vals, dbg, s->dev_err);
    } else {
        k_preprocess<FMT><<<(unsigned)div_up(s->n, kPrepThreads), kPrepThreads, 0, st>>>(
            s->planes, s->n, s->nwords, s->sh_degree, cam, recs, rects, keys, vals, dbg);
    }
    GS_CUDA(cudaGetLastError());
    return GS_OK;
}

gs_status launch_preprocess(const gs_scene* s, const DevCamera& cam, BlendRec* recs, uint2* rects, uint32_t* keys,
                            uint32_t* vals, gs_record* dbg, cudaStream_t st) {
    if (s->n == 0) return GS_OK;
    if (s->fmt == GS_FP32) return launch_preprocess_fmt<GS_FP32>(s, cam, recs, rects, keys, vals, dbg, st);
    if (s->fmt == GS_FP16) return launch_preprocess_fmt<GS_FP16>(s, cam, recs, rects, keys, vals, dbg, st);
    return launch_preprocess_fmt<GS_BF16>(s, cam, recs, rects, keys, vals, dbg, st);
}

gs_status launch_inject_prep(const gs_scene* s, const DevCamera* dev_cams, int K, const gs_flip* flips, int B,
                             int guard_mode, uint64_t mask, const uint2* const* dev_clean_rects,
                             const BlendRec* const* dev_clean_recs, DirtyDesc* desc, uint32_t* item_off, CmpAcc* acc,
                             unsigned int* queue, cudaStream_t st) {
    if (B * K > kMaxPairs || K > 32) return set_error(GS_ERR_ARG, "B * K must be <= 8192 and K <= 32");
    // the per-(variant, view) item counts go to the tail of item_off, past the B*K+1 offsets
    uint32_t* n_items = item_off + (B * K + 1);
    const int blocks = (B + kPrepWarps - 1) / kPrepWarps;
#define GS_PREP(F)                                                                                            \
    k_inject_prep<F><<<blocks, kPrepWarps * 32, 0, st>>>(s->planes, s->n, s->nwords, s->sh_degree, dev_cams, K, \
                                                         flips, B, guard_mode, mask, s->dev_box, s->pbox_lo,    \
                                                         s->pbox_hi, s->nbox_words, dev_clean_rects,            \
                                                         dev_clean_recs, desc, n_items, acc)
    if (s->fmt == GS_FP32)
        GS_PREP(GS_FP32);
    else if (s->fmt == GS_FP16)
        GS_PREP(GS_FP16);
    else
        GS_PREP(GS_BF16);
#undef GS_PREP
    k_items_scan<<<1, 1024, 0, st>>>(n_items, B * K, item_off, queue);
    GS_CUDA(cudaGetLastError());
    return GS_OK;
}

}  // namespace gs
