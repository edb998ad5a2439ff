/*
 * gs.h -- C ABI of libgs, a GB300 (sm_103a) engine for the data-parallel hot path
 * of single-event-upset (SEU) fault injection into 3D Gaussian splatting models
 * (arXiv 2606.21791, "Single-Event Upsets in 3D Gaussian Splatting Rendering").
 *
 * Every call returns a gs_status and never aborts; gs_last_error() gives a
 * thread-local message for the last failure.  Unless stated otherwise a pointer
 * argument named dev_* is CUDA device memory owned by the caller and must stay
 * valid until the work queued on `stream` completes; host_* is host memory read
 * before the call returns.  `stream` is a cudaStream_t (NULL = legacy default
 * stream).  Calls on one scene are stream-ordered: issue them on one stream, or
 * synchronise between streams.  A scene is not thread-safe.
 *
 * Parameter layout (Sec. 3 "Parameter layout"): a primitive stores mean (words
 * 0-2), logarithmic scale (3-5), quaternion w,x,y,z (6-9), opacity logit (10),
 * SH DC colour (11-13) and higher-order SH coefficients coefficient-major,
 * 3 channels each (14..): 14 words at SH degree 0, 59 at degree 3.  Scenes are
 * structure-of-arrays planes [word][primitive] in the storage format.
 */
#ifndef GS_H
#define GS_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define GS_API __attribute__((visibility("default")))
#else
#define GS_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    GS_OK = 0,
    GS_ERR_ARG = 1,      /* invalid argument (null pointer, size, format, site out of range) */
    GS_ERR_OOM = 2,      /* device allocation failed */
    GS_ERR_CUDA = 3,     /* a CUDA call failed; the message names it */
    GS_ERR_TIMEOUT = 4,  /* a bounded device-side wait gave up */
    GS_ERR_BUSY = 5,     /* admission refused (serving budget) or queue full */
    GS_ERR_STATE = 6,    /* call out of order (e.g. no views set, unknown ticket) */
    GS_ERR_CAPACITY = 7  /* an internal buffer was too small; the call can be retried */
} gs_status;

/* Storage format of the parameter words (Sec. 3 "Single-bit upset model"):
 * fp32 (sign 31, exponent 23-30, mantissa 0-22), fp16, bf16.  Math is fp32. */
typedef enum { GS_FP32 = 0, GS_FP16 = 1, GS_BF16 = 2 } gs_format;

/* Guard box modes (Algorithm 1): FIELD = one [lo, hi] per word index over all
 * primitives (the Algorithm 1 precompute); PRIM = per-primitive boxes. */
typedef enum { GS_GUARD_OFF = -1, GS_GUARD_FIELD = 0, GS_GUARD_PRIM = 1, GS_GUARD_ECC = 2 } gs_guard_mode;
/* GS_GUARD_ECC is not a clamp: it emulates an error-correcting code over the
 * sign and exponent bits of the words in word_mask (Sec. 5 "Alternative
 * defenses", Table 4): an upset on such a bit (fp32 bits 23-31, fp16 10-15,
 * bf16 7-15) is corrected and leaves the scene unchanged; other upsets apply. */

/* One single-bit upset site (Sec. 3: a fault site is (field, primitive,
 * component, bit)); `word` is the field/component word index, `bit` counts from
 * the least significant bit of the stored word (< 32 for fp32, < 16 otherwise). */
typedef struct {
    uint32_t prim;
    uint16_t word;
    uint8_t bit;
    uint8_t pad;
} gs_flip;

/* Pinhole camera: camera-space p = R * world + t (R row-major; x right, y down,
 * z forward); pixel (i, j) has centre (i + 0.5, j + 0.5); a point projects to
 * (fx x/z + cx, fy y/z + cy).  Primitives with z outside (znear, zfar) are culled. */
typedef struct {
    float R[9];
    float t[3];
    float fx, fy, cx, cy;
    int32_t width, height;
    float znear, zfar;
} gs_camera;

/* Per (variant, view) comparison against the clean frame (Definitions 1 and 2,
 * Sec. 3 "Metrics and severity"): images clamped to [0,1] (NaN counts as 0);
 * sse = sum of squared channel differences; maxabs = peak |difference|;
 * footprint = pixels whose max channel |difference| exceeds 1/255; nonfinite =
 * pixels of the corrupted render with a non-finite channel; clamps = guard
 * clamps applied to the variant (0 with the guard off). */
typedef struct {
    double sse;
    float maxabs;
    uint32_t footprint;
    uint32_t nonfinite;
    uint32_t clamps;
} gs_result;

/* One preprocessed primitive (debug/stage entry points): projected mean,
 * conic (inverse 2D covariance [[ca, cb], [cb, cc]]), colour, sigmoid opacity,
 * camera depth, half-open tile rect, pixel radius, visible flag. */
typedef struct {
    float mx, my, ca, cb, cc, r, g, b, opac, depth;
    int32_t x0, y0, x1, y1, radius, visible;
} gs_record;

typedef struct gs_scene gs_scene;

GS_API const char* gs_last_error(void);
GS_API const char* gs_version(void);

/* ---------------------------------------------------------------------------
 * Scenes.
 * gs_load_scene copies `n` primitives of `nwords(sh_degree)` storage words,
 * planes [word][prim] (uint32 words for fp32, uint16 for fp16/bf16), from host
 * or device memory (`src_on_device`) into a library-owned device scene, and runs
 * the Algorithm 1 precompute (per-word min/max box).  sh_degree 0..3.
 * ------------------------------------------------------------------------- */
GS_API gs_status gs_load_scene(const void* planes, int src_on_device, uint64_t n, int sh_degree, gs_format fmt,
                        gs_scene** out);
GS_API gs_status gs_free_scene(gs_scene* scene);
GS_API gs_status gs_scene_info(const gs_scene* scene, uint64_t* n, int* sh_degree, int* fmt, int* nwords);
/* Device pointer to the scene's resident planes (library-owned; valid until free). */
GS_API gs_status gs_scene_planes(gs_scene* scene, void** dev_planes);
/* Copy the planes back into `dst` (host or device per `dst_on_device`). */
GS_API gs_status gs_read_planes(gs_scene* scene, void* dst, int dst_on_device, void* stream);
/* Overwrite the resident planes from `src` (same layout; host or device), e.g.
 * to restore a saved clean state.  The FIELD box and any views are not
 * recomputed. */
GS_API gs_status gs_write_planes(gs_scene* scene, const void* src, int src_on_device, void* stream);

/* Read and clear the scene's sticky device error flags (bit 0: a flip site was
 * out of range and skipped; bit 1: a bounded wait of the full preprocess for
 * its staged parameter words gave up, so that render's output is incomplete --
 * the render calls that synchronise report it as GS_ERR_TIMEOUT until the
 * flags are cleared here).  Synchronises the device. */
GS_API gs_status gs_scene_errors(gs_scene* scene, uint32_t* host_flags);

/* ---------------------------------------------------------------------------
 * (a) Injection (Sec. 3 "Single-bit upset model"): XOR one bit of each listed
 * stored word, in place, persistently (the resident model keeps the upsets, as
 * in an upset storm).  Duplicate sites cancel pairwise, as sequential XOR does.
 * ------------------------------------------------------------------------- */
GS_API gs_status gs_apply_flips(gs_scene* scene, const gs_flip* dev_flips, int64_t count, void* stream);

/* ---------------------------------------------------------------------------
 * (f) Support guard (Algorithm 1; Theorems 1-2).  For every primitive and every
 * word w with bit w of `word_mask` set, a stored value that is non-finite or
 * outside [lo, hi] is replaced by the nearer endpoint's storage word (NaN goes
 * to lo) and counted; the count is ADDED to *dev_clamps (uint64, caller-owned,
 * may be NULL).  Writes happen only where a clamp fires.
 * gs_field_box reads the FIELD box (storage words widened to uint32).
 * gs_set_prim_box installs per-primitive boxes: planes [nbox_words][n] of
 * storage words (nbox_words <= nwords), host or device; PRIM mode may only
 * guard words < nbox_words.
 * ------------------------------------------------------------------------- */
GS_API gs_status gs_field_box(gs_scene* scene, uint32_t* host_lo, uint32_t* host_hi);
GS_API gs_status gs_set_prim_box(gs_scene* scene, const void* lo, const void* hi, int src_on_device, int nbox_words);
GS_API gs_status gs_guard(gs_scene* scene, int mode, uint64_t word_mask, uint64_t* dev_clamps, void* stream);
/* gs_guard with the optional bitmap of clamped words: dev_bitmap (device,
 * caller-owned, nwords * ceil(n / 32) uint32) is overwritten so that bit
 * (i % 32) of dev_bitmap[w * ceil(n / 32) + i / 32] is set iff the guard clamps
 * word w of primitive i (rows of unguarded words and the bits past n are 0).
 * The decisions are those of the clamp, taken by one extra read pass over the
 * guarded planes before it; popcount(bitmap) equals the clamps added. */
GS_API gs_status gs_guard_bitmap(gs_scene* scene, int mode, uint64_t word_mask, uint64_t* dev_clamps,
                                 uint32_t* dev_bitmap, void* stream);

/* ---------------------------------------------------------------------------
 * (b)-(d) Forward render of the scene as it is now (3DGS forward pass: EWA
 * projection, tile binning with a radix sort of (tile, depth) keys, front-to-
 * back blending over white with the 1/255 alpha and 1e-4 transmittance
 * cutoffs).  K views, each written as H*W*3 float32 (row-major, RGB) into
 * dev_rgb at offset sum_{k'<k} H_k' W_k' 3.  tile 16x16.
 * ------------------------------------------------------------------------- */
GS_API gs_status gs_render(gs_scene* scene, const gs_camera* host_cams, int K, float* dev_rgb, void* stream);

/* (e) Comparison of K image pairs (layout as gs_render), one gs_result each
 * (clamps = 0).  dev_out: K records. */
GS_API gs_status gs_compare(const float* dev_a, const float* dev_b, int H, int W, int K, gs_result* dev_out, void* stream);
/* SSIM of K image pairs (Sec. 3 "Metrics and severity", Wang et al. 2004):
 * per channel, Gaussian-weighted local means, variances and covariance over an
 * 11x11 window (sigma 1.5, normalised), SSIM = (2 mx my + C1)(2 sxy + C2) /
 * ((mx^2 + my^2 + C1)(sx^2 + sy^2 + C2)), C1 = 0.01^2, C2 = 0.03^2, on values
 * clamped to [0, 1] (NaN as 0); dev_out[k] (double) = the mean over the pixels
 * at least 5 from every edge and over the channels (1 when there are none).
 * dev_test / dev_clean: K images H*W*3 float32 (layout as gs_render).  Per-pixel
 * fp32 arithmetic with fixed rounding, summed in fixed point (2^-32). */
GS_API gs_status gs_ssim(const float* dev_test, const float* dev_clean, int H, int W, int K, double* dev_out,
                         void* stream);

/* Allocation-free variant of gs_compare (the paper has no counterpart; it is a
 * library convenience).  For callers that must not allocate device memory once
 * they are running: flight and embedded renderers that forbid dynamic
 * allocation after start-up, and processes whose allocator already owns all of
 * HBM under a fixed budget.  gs_compare takes its accumulators from the stream-
 * ordered allocator; this call instead uses one fixed device array of 64
 * accumulators compiled into the library, so it allocates nothing (no
 * cudaMalloc, cudaFree or allocating library routine).  Inputs and outputs are
 * as for gs_compare; K must be at most 64, otherwise GS_ERR_ARG.  The first call
 * on a device looks up the array's device address for that device (make that
 * first call before any stream capture).  Every call shares the one array, which
 * keeps the last call's contents; each call clears what it uses first, but calls
 * that overlap on the GPU (e.g. on two streams) race and must be serialised.
 * Every GPU that loads the library holds the array (1.5 KB) until exit. */
GS_API gs_status gs_compare_noalloc(const float* dev_a, const float* dev_b, int H, int W, int K, gs_result* dev_out,
                                    void* stream);

/* ---------------------------------------------------------------------------
 * Injection campaign (Sec. 3 "Parallel injection engine").
 * gs_set_views renders the clean frame of each view and keeps its state
 * resident (preprocessed records, sorted tile lists, clean image); the scene
 * must be clean (no persistent upsets) while a campaign runs.
 * gs_inject_and_render evaluates B variants: variant b is the clean scene with
 * flips [b*fpv, (b+1)*fpv) XOR-ed in (fpv = flips_per_variant; with
 * GS_GUARD_ECC the corrected ones are skipped), then guarded when guard_mode is
 * FIELD or PRIM, rendered in every view and compared with the clean
 * frame; dev_out gets B*K records [b][k].  Single-flip variants run on the
 * batched dirty-tile engine (only tiles the flipped primitive covers before or
 * after the upset are re-blended; bit-identical to a full re-render);
 * multi-flip variants are re-rendered in full.  The scene is left unchanged.
 * gs_inject_and_render_full is the plain loop: one variant at a time, in place,
 * full preprocess + sort + blend + compare per view, then restore.
 * ------------------------------------------------------------------------- */
GS_API gs_status gs_set_views(gs_scene* scene, const gs_camera* host_cams, int K, void* stream);
GS_API gs_status gs_clean_image(gs_scene* scene, int k, float* dev_rgb, void* stream);
GS_API gs_status gs_inject_and_render(gs_scene* scene, const gs_flip* dev_flips, int B, int flips_per_variant,
                               int guard_mode, uint64_t word_mask, gs_result* dev_out, void* stream);
GS_API gs_status gs_inject_and_render_full(gs_scene* scene, const gs_flip* dev_flips, int B, int flips_per_variant,
                                    int guard_mode, uint64_t word_mask, gs_result* dev_out, void* stream);
/* gs_inject_and_render with host buffers: host_flips (B*fpv gs_flip) and
 * host_out (B*K gs_result) are caller-owned host memory (pinned memory makes
 * the copies asynchronous DMA; pageable memory works and is slower).  The
 * library copies the upsets into device staging it owns (grown on demand,
 * freed with the scene), runs the campaign on `stream`, copies the records
 * back and synchronises the stream before returning.  Same errors as
 * gs_inject_and_render. */
GS_API gs_status gs_inject_and_render_host(gs_scene* scene, const gs_flip* host_flips, int B, int flips_per_variant,
                                    int guard_mode, uint64_t word_mask, gs_result* host_out, void* stream);
/* gs_inject_and_render for single-flip variants, also reporting how a
 * sort-first partition is contaminated (Sec. 5 "Cross-node contamination in
 * distributed rendering").  The screen is an 8x8 grid of cells, cell of pixel
 * (x, y) = (8x / W, 8y / H), bit 8 cy + cx; the 4-, 8-, 16-, 32- and 64-node
 * partitions (2x2, 4x2, 4x4, 8x4, 8x8 regions) are unions of cells.  For each
 * (variant, view), dev_regions (device, B*K*2 uint64, caller-owned) gets
 * [actual, predicted]: actual = cells holding a footprint pixel (Definition
 * 1), predicted = cells met by the flipped primitive's tile rect before or
 * after the upset when its stored words changed (0 for a corrected or
 * clamped-back upset).  Errors as gs_inject_and_render. */
GS_API gs_status gs_inject_and_render_regions(gs_scene* scene, const gs_flip* dev_flips, int B, int guard_mode,
                                              uint64_t word_mask, gs_result* dev_out, uint64_t* dev_regions,
                                              void* stream);
/* gs_inject_and_render for single-flip variants with optional extra outputs
 * (device, caller-owned, each may be NULL): dev_regions as in
 * gs_inject_and_render_regions; dev_ssim (B*K doubles) the SSIM of every
 * (variant, view) against its clean frame, as gs_ssim defines it, computed
 * from the re-blended pixels only (SSIM is exactly 1 wherever a window is
 * unchanged) and bit-identical to gs_ssim on the full re-rendered frame.  The
 * SSIM buffers (about 270 MB plus 16 B per (variant, view, tile)) are
 * allocated on first use; GS_ERR_CAPACITY if a batch has more dirty tiles
 * than they hold (retry with a smaller gs_set_batch).  The SSIM needs the
 * default 16 x 16 render tiles (GS_ERR_STATE with another gs_set_tile shape). */
GS_API gs_status gs_inject_and_render_ex(gs_scene* scene, const gs_flip* dev_flips, int B, int guard_mode,
                                         uint64_t word_mask, gs_result* dev_out, uint64_t* dev_regions,
                                         double* dev_ssim, void* stream);
/* Enable (default) or disable CUDA-graph replay of the batched dirty-tile step. */
GS_API gs_status gs_set_graphs(gs_scene* scene, int enable);
/* Work counters for measurement: while enabled, the dirty-tile kernels add
 * up, per batch: [0] pixel-primitive evaluations, [1] tiles blended, [2] list
 * entries staged, [3] dirty tiles dropped by the plan (every pixel keeps its
 * clean value), of which [4] by the stop-key test, [5] by the tile reach
 * test, [6] because no pixel is reached, [7] because every reached pixel
 * stopped before the change, [8] list entries walked by a warp of the
 * dirty-tile blend (survivors of its box cull), [9] of them blended by at
 * least one of its pixels, [10] 8x8 pixel blocks re-blended, and the SM
 * cycles the dirty-tile blend's warps spend per phase: [11] setting up a block
 * (work queue, plan item, checkpoint, sublist searches), [12] the walk over
 * its entries, [13] the comparison with the clean image and the reductions,
 * then [14] the pixels the plan left active in the re-blended blocks and [15]
 * the same weighted by the entries each block's warp walked (so [15] / [8] is
 * the mean number of a walk step's 64 pixel slots that hold an active pixel)
 * (graphs are bypassed while counting).  gs_read_work copies those 16 counts
 * into host_counts[16] and resets them (synchronises). */
GS_API gs_status gs_count_work(gs_scene* scene, int enable);
GS_API gs_status gs_read_work(gs_scene* scene, uint64_t* host_counts);
/* Kernel timing for measurement: while enabled, CUDA events bracket the two
 * dirty-tile kernels of each batch on the caller's stream (also inside the
 * captured graph).  gs_read_kernel_ms waits for the last batch and writes
 * ms[0] = the two plan kernels' time, ms[1] = the blend + compare kernel's time
 * (host array of 2 floats).  GS_ERR_STATE while timing is off. */
GS_API gs_status gs_time_kernels(gs_scene* scene, int enable);
GS_API gs_status gs_read_kernel_ms(gs_scene* scene, float* ms);
/* Stage times of the full render (the 3DGS forward pass of Sec. 3: preprocess,
 * tile binning with the radix sort, front-to-back blend) while kernel timing is
 * on: CUDA events bracket the stages of every view of gs_render.
 * gs_read_render_ms waits for the last view of the last gs_render call and
 * writes, into host arrays, ms[0] = preprocess, ms[1] = depth sort + tile
 * binning + pair sort + tile ranges, ms[2] = blend (3 floats), and counts[0] =
 * primitives, counts[1] = (tile, primitive) pairs of that view, counts[2] =
 * radix passes over the 32-bit depth keys, counts[3] = radix passes over the
 * pairs' tile keys (4 uint64).  GS_ERR_STATE while timing is off or before the
 * first gs_render after it was switched on. */
GS_API gs_status gs_read_render_ms(gs_scene* scene, float* ms, uint64_t* counts);
/* Variants per dirty-tile launch (0 = largest allowed, min(2048, 8192 / K)). */
GS_API gs_status gs_set_batch(gs_scene* scene, int batch);
/* Autotuner: times the campaign over dev_flips[0, count) at batch sizes
 * 8, 16, 32, 64, 128, 256, 512, 1024, 2048 (those <= min(2048, 8192 / K)), keeps the fastest for this scene and
 * returns it (and its time per variant in microseconds, may be NULL).
 * Synchronises the stream. */
GS_API gs_status gs_autotune(gs_scene* scene, const gs_flip* dev_flips, int count, int guard_mode, uint64_t word_mask,
                             int* best_batch, float* best_us_per_variant, void* stream);
/* Render tile shape of a scene: tile_w x tile_h pixels, each in {8, 16, 32},
 * 64 <= tile_w * tile_h <= 256 (default 16 x 16; else GS_ERR_ARG).  The tiles
 * are the bins of the tile lists and the unit of the dirty-tile engine (Sec. 6
 * of the paper names tile binning among the renderer's stages; the shape
 * itself is the renderer's, not the paper's).  Every later render, campaign
 * and plain-loop call uses it; if gs_set_views was called, its clean per-view
 * state is rebuilt for the new tiles (same errors as gs_set_views; on failure
 * the views are dropped).  Images and records do not depend on the shape
 * except through the binning: pixels are blended front to back over the same
 * primitives whatever tile holds them. */
GS_API gs_status gs_set_tile(gs_scene* scene, int tile_w, int tile_h, void* stream);
GS_API gs_status gs_get_tile(gs_scene* scene, int* tile_w, int* tile_h);
/* Autotuner over tile shape and batch: for each of the shapes 16 x 16, 8 x 8
 * and 32 x 8 it rebuilds the views (gs_set_tile) and runs gs_autotune over
 * dev_flips[0, count); the scene keeps the fastest (shape, batch), which is
 * returned with its time per variant (us, may be NULL).  On an error the scene
 * is put back to its previous shape and batch.  Synchronises the stream. */
GS_API gs_status gs_autotune_tile(gs_scene* scene, const gs_flip* dev_flips, int count, int guard_mode,
                                  uint64_t word_mask, int* best_tile_w, int* best_tile_h, int* best_batch,
                                  float* best_us_per_variant, void* stream);

/* ---------------------------------------------------------------------------
 * Stage entry points (for stage-isolated checks).
 * gs_preprocess: records of every primitive for one camera (dev_out: n).
 * gs_bin_tiles: per-tile lists front to back.  Input per primitive: depth
 * (float, > 0) and tile rect x0,y0,x1,y1 (int32, half open, clipped to the
 * grid by the call; empty = not binned).  Output: dev_offsets [tiles_x*tiles_y +
 * 1] exclusive prefix of list lengths and dev_ids [*host_total] primitive
 * indices, sorted by (tile, depth, primitive) via a stable LSD radix sort.  If
 * the total exceeds ids_cap, *host_total is set and GS_ERR_CAPACITY returned.
 * Blocks until done.
 * gs_blend_lists: blend given records and lists into H*W*3 float32.  Both
 * work on 16 x 16 tiles (gs_preprocess uses the scene's tile shape for the
 * records' tile rects).
 * ------------------------------------------------------------------------- */
GS_API gs_status gs_preprocess(gs_scene* scene, const gs_camera* host_cam, gs_record* dev_out, void* stream);
GS_API gs_status gs_bin_tiles(const float* dev_depth, const int32_t* dev_rects, uint64_t n, int tiles_x, int tiles_y,
                       uint32_t* dev_offsets, uint32_t* dev_ids, uint64_t ids_cap, uint64_t* host_total,
                       void* stream);
GS_API gs_status gs_blend_lists(const gs_record* dev_recs, uint64_t n, const uint32_t* dev_offsets, const uint32_t* dev_ids,
                         int W, int H, float* dev_rgb, void* stream);

/* ---------------------------------------------------------------------------
 * Serving loop (continuous batching).  A server owns `slots` worker slots, each
 * a CUDA stream with its own host thread and render scratch.  Scenes (owned by
 * the caller, already loaded; campaign scenes with gs_set_views done) are
 * registered with their resident device bytes, which must fit the HBM budget.
 * Requests:
 *   RENDER   render `cam` of the scene into dev_rgb (H*W*3 float32, may be
 *            NULL); with guard_mode FIELD or PRIM the guard (Algorithm 1) is
 *            applied to the resident scene first and its clamp count stored in
 *            *dev_clamps (GS_GUARD_ECC: no guard).
 *   CAMPAIGN nflips single-flip variants through gs_inject_and_render;
 *            dev_results gets nflips*K records.
 *   STORM    one frame of an upset storm: the nflips upsets are XOR-ed into the
 *            resident scene (they accumulate; with GS_GUARD_ECC the corrected
 *            ones are skipped), then guard (FIELD/PRIM) and render.
 * A free slot takes the first queued request whose scene allows it (guarded
 * renders and storm frames run alone on their scene; one campaign per scene)
 * and whose render scratch fits the budget; so requests that arrive while
 * others run are admitted as slots and memory free up, and run concurrently on
 * separate streams.  A request larger than the budget left after the resident
 * scenes is refused with GS_ERR_BUSY.  Device buffers in a request must stay
 * valid until gs_server_wait returns for it.  While a scene is registered with
 * a running server, the caller changes it only through requests: calls that
 * rebuild or free its state (gs_set_views, gs_set_tile, gs_autotune_tile,
 * gs_free_scene) race with the workers and must wait until gs_server_destroy.  Times are host milliseconds since
 * the server was created; `arrival_ms` < 0 means "now".
 * ------------------------------------------------------------------------- */
typedef struct gs_server gs_server;
typedef enum { GS_REQ_RENDER = 0, GS_REQ_CAMPAIGN = 1, GS_REQ_STORM = 2 } gs_req_kind;
typedef struct {
    int32_t kind;
    int32_t scene;
    gs_camera cam;
    int32_t guard_mode;
    int32_t nflips;
    uint64_t word_mask;
    const gs_flip* dev_flips;
    float* dev_rgb;
    gs_result* dev_results;
    uint64_t* dev_clamps;
} gs_request;
typedef struct {
    uint64_t ticket;
    int32_t status;   /* gs_status of the finished request */
    int32_t slot;
    double t_submit_ms, t_start_ms, t_done_ms;
} gs_response;

GS_API gs_status gs_server_create(uint64_t hbm_budget_bytes, int slots, gs_server** out);
GS_API gs_status gs_server_add_scene(gs_server* server, gs_scene* scene, int* scene_id);
GS_API gs_status gs_server_submit(gs_server* server, const gs_request* req, double arrival_ms, uint64_t* ticket);
/* Wait up to timeout_ms (< 0: forever) for a request; GS_ERR_TIMEOUT if not done
 * (the ticket stays valid).  On return the ticket is released. */
GS_API gs_status gs_server_wait(gs_server* server, uint64_t ticket, int timeout_ms, gs_response* out);
/* Remove a request that has not started (GS_ERR_BUSY once it has). */
GS_API gs_status gs_server_cancel(gs_server* server, uint64_t ticket);
/* host_stats[6]: [budget, resident bytes, scratch bytes held, queued, completed,
 * requests that started only after waiting for HBM budget (passed over at
 * least once because their render scratch did not fit)] */
GS_API gs_status gs_server_stats(gs_server* server, uint64_t* host_stats);
/* The server's clock: host milliseconds since gs_server_create, the time base
 * of arrival_ms and of the response times (so a caller can pass the scheduled
 * arrival of an open-loop request and have its queueing counted). */
GS_API gs_status gs_server_now(gs_server* server, double* now_ms);
/* Finishes every queued request, then stops the workers. */
GS_API gs_status gs_server_destroy(gs_server* server);

#ifdef __cplusplus
}
#endif
#endif /* GS_H */
