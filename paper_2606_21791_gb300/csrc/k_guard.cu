// (a) single-bit upset injection and (f) the support guard (Algorithm 1).
//
// Injection (Sec. 3 "Single-bit upset model"): the stored word is reinterpreted
// as an unsigned integer of its width and one bit is XOR-ed.  Sites are applied
// with 32-bit atomicXor on the word that contains them, so duplicate sites in
// one launch cancel exactly as sequential XORs do.
//
// Guard (Algorithm 1, per frame): a data-parallel clamp over the SoA planes of
// the guarded words.  HBM-bound: each plane is streamed with 16-byte vector
// loads (4 fp32 or 8 fp16/bf16 words), several vectors in flight per thread;
// a word is written back only where a clamp fires; clamp counts are reduced per
// block and added to one 64-bit counter.
#include "gs_internal.h"

namespace gs {

namespace {

constexpr int kGuardThreads = 256;
constexpr int kGuardUnroll = 4;

// ecc_mask: words whose sign and exponent bits an error-correcting code
// protects; an upset there is corrected (not applied).  0: no code.
__global__ void k_apply_flips(void* planes, int fmt, uint64_t n, int nwords, const gs_flip* flips, int64_t count,
                              unsigned int* err, uint64_t ecc_mask) {
    int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= count) return;
    gs_flip f = flips[j];
    int nbits = fmt == GS_FP32 ? 32 : 16;
    if (f.prim >= n || f.word >= nwords || f.bit >= nbits) {
        if (err) atomicOr(err, 1u);
        return;
    }
    if (((ecc_mask >> f.word) & 1ull) && f.bit >= ecc_first_bit(fmt)) return;   // corrected
    uint64_t idx = (uint64_t)f.word * n + f.prim;
    if (fmt == GS_FP32) {
        atomicXor((unsigned int*)planes + idx, 1u << f.bit);
    } else {
        uintptr_t addr = (uintptr_t)((uint16_t*)planes + idx);
        unsigned int* w32 = (unsigned int*)(addr & ~(uintptr_t)3);
        unsigned int shift = (addr & 2) ? 16u : 0u;
        atomicXor(w32, 1u << (f.bit + shift));
    }
}

// The plain loop saves each site's word before applying the flips and writes it
// back afterwards.  A site that k_apply_flips rejects (primitive, word or bit out
// of range) is neither read nor written here: its index may lie outside the
// planes.
__device__ __forceinline__ bool site_valid(const gs_flip& f, int fmt, uint64_t n, int nwords) {
    return f.prim < n && f.word < nwords && f.bit < (fmt == GS_FP32 ? 32 : 16);
}

__global__ void k_save_sites(const void* planes, int fmt, uint64_t n, int nwords, const gs_flip* flips, int count,
                             uint32_t* saved) {
    int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= count) return;
    gs_flip f = flips[j];
    if (!site_valid(f, fmt, n, nwords)) return;
    uint64_t idx = (uint64_t)f.word * n + f.prim;
    saved[j] = fmt == GS_FP32 ? ((const uint32_t*)planes)[idx] : ((const uint16_t*)planes)[idx];
}

__global__ void k_restore_sites(void* planes, int fmt, uint64_t n, int nwords, const gs_flip* flips, int count,
                                const uint32_t* saved) {
    int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= count) return;
    gs_flip f = flips[j];
    if (!site_valid(f, fmt, n, nwords)) return;
    uint64_t idx = (uint64_t)f.word * n + f.prim;
    if (fmt == GS_FP32)
        ((uint32_t*)planes)[idx] = saved[j];
    else
        ((uint16_t*)planes)[idx] = (uint16_t)saved[j];
}

// ---------------------------------------------------------------------------
// Algorithm 1 precompute: min / max of every word plane.  Values are ordered by
// an order-preserving integer key of their storage bits (-0 below +0); NaN words
// are skipped.  dev_box: key_min[nwords], key_max[nwords].
// ---------------------------------------------------------------------------
__device__ __forceinline__ bool is_nan_bits(uint32_t b, int fmt) {
    if (fmt == GS_FP32) return (b & 0x7f800000u) == 0x7f800000u && (b & 0x007fffffu);
    if (fmt == GS_FP16) return (b & 0x7c00u) == 0x7c00u && (b & 0x03ffu);
    return (b & 0x7f80u) == 0x7f80u && (b & 0x007fu);
}

__device__ __forceinline__ uint32_t order_key(uint32_t b, int fmt) {
    uint32_t sign = fmt == GS_FP32 ? 0x80000000u : 0x8000u;
    uint32_t all = fmt == GS_FP32 ? 0xffffffffu : 0xffffu;
    return (b & sign) ? (~b & all) : (b | sign);
}

__global__ void k_field_box(const void* planes, int fmt, uint64_t n, uint32_t* kmin, uint32_t* kmax) {
    int w = blockIdx.y;
    uint32_t lo = 0xffffffffu, hi = 0u;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
        uint32_t b = fmt == GS_FP32 ? ((const uint32_t*)planes)[(uint64_t)w * n + i]
                                    : ((const uint16_t*)planes)[(uint64_t)w * n + i];
        if (is_nan_bits(b, fmt)) continue;
        uint32_t k = order_key(b, fmt);
        lo = min(lo, k);
        hi = max(hi, k);
    }
    for (int o = 16; o > 0; o >>= 1) {
        lo = min(lo, __shfl_xor_sync(0xffffffffu, lo, o));
        hi = max(hi, __shfl_xor_sync(0xffffffffu, hi, o));
    }
    if ((threadIdx.x & 31) == 0) {
        atomicMin(&kmin[w], lo);
        atomicMax(&kmax[w], hi);
    }
}

__global__ void k_box_init(uint32_t* kmin, uint32_t* kmax, int nwords) {
    int w = threadIdx.x;
    if (w < nwords) {
        kmin[w] = 0xffffffffu;
        kmax[w] = 0u;
    }
}

// ---------------------------------------------------------------------------
// guard clamp
// ---------------------------------------------------------------------------
struct GuardParams {
    int nplanes;
    uint8_t word[kMaxWords];
    float lo[kMaxWords];      // FIELD box values
    float hi[kMaxWords];
    uint32_t lob[kMaxWords];  // FIELD box storage words
    uint32_t hib[kMaxWords];
};

// clamp one value; returns the word to store (== old if in box) and sets *hit
__device__ __forceinline__ uint32_t clamp_word(uint32_t bits, float x, float lo, float hi, uint32_t lob, uint32_t hib,
                                               unsigned int* hit) {
    if (x >= lo && x <= hi) return bits;
    *hit += 1u;
    return (x > hi) ? hib : lob;
}

template <int FMT, bool PRIM>
__global__ __launch_bounds__(kGuardThreads) void k_guard(void* __restrict__ planes, const void* __restrict__ plo,
                                                         const void* __restrict__ phi, uint64_t n, GuardParams gp,
                                                         unsigned long long* clamps) {
    using W = typename std::conditional<FMT == GS_FP32, uint32_t, uint16_t>::type;
    constexpr int kPer = 16 / sizeof(W);   // words per 16-byte vector
    const int p = blockIdx.y;
    const int w = gp.word[p];
    W* base = (W*)planes + (uint64_t)w * n;
    const W* lbase = PRIM ? (const W*)plo + (uint64_t)w * n : nullptr;
    const W* hbase = PRIM ? (const W*)phi + (uint64_t)w * n : nullptr;
    const float flo = gp.lo[p], fhi = gp.hi[p];
    const uint32_t flob = gp.lob[p], fhib = gp.hib[p];
    unsigned int hit = 0;

    auto value = [](uint32_t b) -> float {
        if (FMT == GS_FP32) return __uint_as_float(b);
        if (FMT == GS_FP16) return __half2float(__ushort_as_half((unsigned short)b));
        return __uint_as_float(b << 16);
    };
    auto one = [&](uint64_t i) {
        uint32_t b = base[i];
        float x = value(b);
        uint32_t lb = PRIM ? (uint32_t)lbase[i] : flob;
        uint32_t hb = PRIM ? (uint32_t)hbase[i] : fhib;
        float lo = PRIM ? value(lb) : flo;
        float hi = PRIM ? value(hb) : fhi;
        unsigned int before = hit;
        uint32_t nb = clamp_word(b, x, lo, hi, lb, hb, &hit);
        if (hit != before) base[i] = (W)nb;
    };

    // a plane is aligned to 16 B only when w * n * sizeof(W) is; peel the head
    uintptr_t addr = (uintptr_t)base;
    uint64_t head = ((16 - (addr & 15)) & 15) / sizeof(W);
    if (head > n) head = n;
    // the box planes are separate allocations with the same per-plane offsets,
    // so they share the parameter plane's 16-byte alignment
    uint64_t nvec = (n - head) / kPer;
    uint64_t tail0 = head + nvec * kPer;
    const uint64_t gtid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const uint64_t gstride = (uint64_t)gridDim.x * blockDim.x;
    if (gtid < head) one(gtid);
    if (gtid < n - tail0) one(tail0 + gtid);

    uint4* vb = (uint4*)(base + head);
    const uint4* vl = PRIM ? (const uint4*)(lbase + head) : nullptr;
    const uint4* vh = PRIM ? (const uint4*)(hbase + head) : nullptr;
    for (uint64_t v0 = gtid; v0 < nvec; v0 += gstride * kGuardUnroll) {
        uint4 d[kGuardUnroll], l[kGuardUnroll], h[kGuardUnroll];
#pragma unroll
        for (int u = 0; u < kGuardUnroll; u++) {
            uint64_t v = v0 + (uint64_t)u * gstride;
            if (v < nvec) {
                d[u] = __ldcs(vb + v);
                if (PRIM) {
                    l[u] = __ldcs(vl + v);
                    h[u] = __ldcs(vh + v);
                }
            }
        }
#pragma unroll
        for (int u = 0; u < kGuardUnroll; u++) {
            uint64_t v = v0 + (uint64_t)u * gstride;
            if (v >= nvec) continue;
            const W* dw = (const W*)&d[u];
            const W* lw = (const W*)&l[u];
            const W* hw = (const W*)&h[u];
            unsigned int before = hit;
            W out[kPer];
#pragma unroll
            for (int e = 0; e < kPer; e++) {
                uint32_t b = dw[e];
                float x = value(b);
                uint32_t lb = PRIM ? (uint32_t)lw[e] : flob;
                uint32_t hb = PRIM ? (uint32_t)hw[e] : fhib;
                float lo = PRIM ? value(lb) : flo;
                float hi = PRIM ? value(hb) : fhi;
                out[e] = (W)clamp_word(b, x, lo, hi, lb, hb, &hit);
            }
            if (hit != before) {
                W* dst = base + head + v * kPer;
#pragma unroll
                for (int e = 0; e < kPer; e++)
                    if (out[e] != dw[e]) dst[e] = out[e];   // an endpoint never equals an out-of-box word
            }
        }
    }
    // block reduction of the clamp count
    for (int o = 16; o > 0; o >>= 1) hit += __shfl_xor_sync(0xffffffffu, hit, o);
    __shared__ unsigned int wsum[kGuardThreads / 32];
    if ((threadIdx.x & 31) == 0) wsum[threadIdx.x >> 5] = hit;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned int s = 0;
        for (int i = 0; i < kGuardThreads / 32; i++) s += wsum[i];
        if (s && clamps) atomicAdd(clamps, (unsigned long long)s);
    }
}

// Clamped-word bitmap, an optional output of the guard: bit (i % 32) of
// bitmap[w * words32 + i / 32] is set when the guard clamps word w of primitive
// i -- the decision of k_guard (value outside [lo, hi], NaN included), taken
// on the words before the clamp, so this runs before k_guard.  One thread per
// (primitive, guarded plane); a warp covers 32 consecutive primitives, so lane
// 0 writes each bitmap word whole.  The loop bound is uniform in a block.
template <int FMT, bool PRIM>
__global__ __launch_bounds__(kGuardThreads) void k_guard_mark(const void* __restrict__ planes,
                                                              const void* __restrict__ plo,
                                                              const void* __restrict__ phi, uint64_t n, GuardParams gp,
                                                              uint32_t* __restrict__ bitmap, uint64_t words32) {
    using W = typename std::conditional<FMT == GS_FP32, uint32_t, uint16_t>::type;
    const int p = blockIdx.y;
    const int w = gp.word[p];
    const W* base = (const W*)planes + (uint64_t)w * n;
    const W* lbase = PRIM ? (const W*)plo + (uint64_t)w * n : nullptr;
    const W* hbase = PRIM ? (const W*)phi + (uint64_t)w * n : nullptr;
    auto value = [](uint32_t b) -> float {
        if (FMT == GS_FP32) return __uint_as_float(b);
        if (FMT == GS_FP16) return __half2float(__ushort_as_half((unsigned short)b));
        return __uint_as_float(b << 16);
    };
    const uint64_t span = words32 * 32u;
    for (uint64_t i0 = (uint64_t)blockIdx.x * kGuardThreads; i0 < span; i0 += (uint64_t)gridDim.x * kGuardThreads) {
        const uint64_t i = i0 + threadIdx.x;
        bool hit = false;
        if (i < n) {
            const float x = value((uint32_t)base[i]);
            const float lo = PRIM ? value((uint32_t)lbase[i]) : gp.lo[p];
            const float hi = PRIM ? value((uint32_t)hbase[i]) : gp.hi[p];
            hit = !(x >= lo && x <= hi);
        }
        const unsigned m = __ballot_sync(0xffffffffu, hit);
        const uint64_t word = i >> 5;   // lane 0: i is a multiple of 32
        if ((threadIdx.x & 31) == 0 && word < words32) bitmap[(uint64_t)w * words32 + word] = m;
    }
}

}  // namespace

int num_sms() {
    static int sms = 0;
    if (!sms) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (sms <= 0) sms = 1;
    }
    return sms;
}

gs_status launch_apply_flips(void* planes, int fmt, uint64_t n, int nwords, const gs_flip* flips, int64_t count,
                             unsigned int* err, uint64_t ecc_mask, cudaStream_t st) {
    if (count <= 0) return GS_OK;
    int64_t blocks = (count + 255) / 256;
    k_apply_flips<<<(unsigned)blocks, 256, 0, st>>>(planes, fmt, n, nwords, flips, count, err, ecc_mask);
    GS_CUDA(cudaGetLastError());
    return GS_OK;
}

gs_status launch_save_sites(const void* planes, int fmt, uint64_t n, int nwords, const gs_flip* flips, int count,
                            uint32_t* saved, cudaStream_t st) {
    if (count <= 0) return GS_OK;
    k_save_sites<<<(count + 255) / 256, 256, 0, st>>>(planes, fmt, n, nwords, flips, count, saved);
    GS_CUDA(cudaGetLastError());
    return GS_OK;
}

gs_status launch_restore_sites(void* planes, int fmt, uint64_t n, int nwords, const gs_flip* flips, int count,
                               const uint32_t* saved, cudaStream_t st) {
    if (count <= 0) return GS_OK;
    k_restore_sites<<<(count + 255) / 256, 256, 0, st>>>(planes, fmt, n, nwords, flips, count, saved);
    GS_CUDA(cudaGetLastError());
    return GS_OK;
}

gs_status launch_field_box(const void* planes, int fmt, uint64_t n, int nwords, uint32_t* dev_keys, cudaStream_t st) {
    k_box_init<<<1, 64, 0, st>>>(dev_keys, dev_keys + kMaxWords, nwords);
    GS_CUDA(cudaGetLastError());
    if (n == 0) return GS_OK;
    int bx = (int)std::min<uint64_t>(div_up(n, 256), (uint64_t)num_sms() * 4);
    dim3 grid(bx, nwords);
    k_field_box<<<grid, 256, 0, st>>>(planes, fmt, n, dev_keys, dev_keys + kMaxWords);
    GS_CUDA(cudaGetLastError());
    return GS_OK;
}

uint32_t key_to_bits(uint32_t key, int fmt) {
    uint32_t sign = fmt == GS_FP32 ? 0x80000000u : 0x8000u;
    uint32_t all = fmt == GS_FP32 ? 0xffffffffu : 0xffffu;
    return (key & sign) ? (key & ~sign & all) : (~key & all);
}

float host_word_value(uint32_t bits, int fmt) {
    if (fmt == GS_FP32) {
        float f;
        memcpy(&f, &bits, 4);
        return f;
    }
    if (fmt == GS_BF16) {
        uint32_t u = bits << 16;
        float f;
        memcpy(&f, &u, 4);
        return f;
    }
    __half_raw r;
    r.x = (unsigned short)bits;
    return __half2float(__half(r));
}

// the guarded planes of `mask` and their FIELD boxes
static gs_status guard_params(const gs_scene* s, int mode, uint64_t mask, GuardParams& gp) {
    memset(&gp, 0, sizeof(gp));
    for (int w = 0; w < s->nwords; w++) {
        if (!((mask >> w) & 1ull)) continue;
        if (mode == GS_GUARD_PRIM && w >= s->nbox_words)
            return set_error(GS_ERR_ARG, "gs_guard: PRIM mode word outside the per-primitive box planes");
        int p = gp.nplanes++;
        gp.word[p] = (uint8_t)w;
        gp.lob[p] = s->box_lo[w];
        gp.hib[p] = s->box_hi[w];
        gp.lo[p] = host_word_value(s->box_lo[w], s->fmt);
        gp.hi[p] = host_word_value(s->box_hi[w], s->fmt);
    }
    if (mode == GS_GUARD_PRIM && gp.nplanes > 0 && s->n > 0 && (!s->pbox_lo || !s->pbox_hi))
        return set_error(GS_ERR_STATE, "gs_guard: no per-primitive box set");
    return GS_OK;
}

gs_status launch_guard_mark(gs_scene* s, int mode, uint64_t mask, uint32_t* bitmap, cudaStream_t st) {
    GuardParams gp;
    GS_TRY(guard_params(s, mode, mask, gp));
    const uint64_t words32 = div_up(s->n, 32);
    if (words32 == 0) return GS_OK;
    GS_CUDA(cudaMemsetAsync(bitmap, 0, sizeof(uint32_t) * (size_t)s->nwords * (size_t)words32, st));
    if (gp.nplanes == 0) return GS_OK;
    const uint64_t want = (uint64_t)num_sms() * 16 / (uint64_t)gp.nplanes + 1;
    const uint64_t bx = std::max<uint64_t>(1, std::min<uint64_t>(div_up(words32 * 32, kGuardThreads), want));
    dim3 grid((unsigned)bx, gp.nplanes);
    const bool prim = mode == GS_GUARD_PRIM;
#define GS_MARK_LAUNCH(F, P) \
    k_guard_mark<F, P><<<grid, kGuardThreads, 0, st>>>(s->planes, s->pbox_lo, s->pbox_hi, s->n, gp, bitmap, words32)
    if (s->fmt == GS_FP32) {
        if (prim) GS_MARK_LAUNCH(GS_FP32, true); else GS_MARK_LAUNCH(GS_FP32, false);
    } else if (s->fmt == GS_FP16) {
        if (prim) GS_MARK_LAUNCH(GS_FP16, true); else GS_MARK_LAUNCH(GS_FP16, false);
    } else {
        if (prim) GS_MARK_LAUNCH(GS_BF16, true); else GS_MARK_LAUNCH(GS_BF16, false);
    }
#undef GS_MARK_LAUNCH
    GS_CUDA(cudaGetLastError());
    return GS_OK;
}

gs_status launch_guard(gs_scene* s, int mode, uint64_t mask, unsigned long long* dev_clamps, cudaStream_t st) {
    GuardParams gp;
    GS_TRY(guard_params(s, mode, mask, gp));
    if (gp.nplanes == 0 || s->n == 0) return GS_OK;
    // enough blocks for ~2 waves of 8 resident blocks per SM, spread over the planes
    uint64_t vec_per_plane = div_up(s->n, s->fmt == GS_FP32 ? 4 : 8);
    uint64_t want = (uint64_t)num_sms() * 16 / (uint64_t)gp.nplanes + 1;
    uint64_t bx = std::min<uint64_t>(div_up(vec_per_plane, (uint64_t)kGuardThreads * kGuardUnroll), want);
    if (bx < 1) bx = 1;
    dim3 grid((unsigned)bx, gp.nplanes);
    bool prim = mode == GS_GUARD_PRIM;
#define GS_GUARD_LAUNCH(F, P) \
    k_guard<F, P><<<grid, kGuardThreads, 0, st>>>(s->planes, s->pbox_lo, s->pbox_hi, s->n, gp, dev_clamps)
    if (s->fmt == GS_FP32) {
        if (prim) GS_GUARD_LAUNCH(GS_FP32, true); else GS_GUARD_LAUNCH(GS_FP32, false);
    } else if (s->fmt == GS_FP16) {
        if (prim) GS_GUARD_LAUNCH(GS_FP16, true); else GS_GUARD_LAUNCH(GS_FP16, false);
    } else {
        if (prim) GS_GUARD_LAUNCH(GS_BF16, true); else GS_GUARD_LAUNCH(GS_BF16, false);
    }
#undef GS_GUARD_LAUNCH
    GS_CUDA(cudaGetLastError());
    return GS_OK;
}

}  // namespace gs
