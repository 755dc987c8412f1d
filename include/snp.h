/*
 * snp.h -- C ABI of libsnp, a GB300 (sm_103a) tile rasterizer for splattable
 * neural primitives (arXiv 2510.08491, "Splat the Net").
 *
 * What the library computes (Sec. 3.1-3.2 of the paper):
 *   Each primitive is an ellipsoid {c + R(q) diag(s) v : |v| <= 1} with
 *   s = exp(log_s) carrying a one-hidden-layer sine density network
 *   (Eq. 5/6)  sigma(x) = w2 . cos(w0 (W1 u + b1)) + b2,  u = (x - c)/max(s).
 *   For every pixel ray o + t d that enters the ellipsoid at t_in and leaves at
 *   t_out, the closed-form line integral of sigma (Eq. 7/8) gives
 *   alpha_hat = S(t_out) - S(t_in); the kernel opacity is
 *   alpha = 1 - exp(-max(0, alpha_hat)) (Eq. 9); primitives are depth-sorted
 *   per screen tile and alpha-blended front to back (Eq. 4) with their colour.
 *
 * Around the renderer, the calls of a training step: the population-control
 * statistic, decision and scene rewrite (Sec. 3.3), the anisotropy regulariser
 * (Sec. 3.3, Sec. 5.3) and a fused Adam step; and time-conditioned (dynamic)
 * scenes (App. Applications) through snp_scene_desc.dynamic.
 *
 * Conventions fixed by this library where the paper is silent (camera model,
 * depth key, near plane, early termination, colour network) are stated at
 * each declaration below.
 *
 * Memory: every scene, image and gradient pointer passed in is DEVICE memory
 * owned by the caller; the library never frees it.  Workspace (projection
 * records, tile keys, tile ranges, per-pixel state saved for the backward pass)
 * is owned by the context.  Calls are asynchronous on the given stream unless
 * stated; `stream` is a cudaStream_t (NULL = legacy default stream).
 *
 * Errors: every call returns an snp_status; nothing is thrown across the ABI.
 * snp_last_error() returns a message for the last failing call on a context.
 * Asynchronous CUDA faults surface as SNP_ERR_CUDA on a later call.
 */
#ifndef SNP_H
#define SNP_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    SNP_OK = 0,
    SNP_ERR_INVALID_ARG = 1, /* bad pointer, size, mode or stale token */
    SNP_ERR_CUDA = 2,        /* a CUDA runtime call failed */
    SNP_ERR_CAPACITY = 3,    /* tile keys exceeded the reserved capacity (graph mode) */
    SNP_ERR_TIMEOUT = 4,     /* a bounded device wait gave up */
    SNP_ERR_UNSUPPORTED = 5  /* combination of modes not built */
} snp_status;

enum { SNP_COLOR_CONST = 0, SNP_COLOR_MLP = 1, SNP_COLOR_SH = 2 };
enum { SNP_F32 = 0, SNP_BF16 = 1 };
enum { SNP_FORM_STABLE = 0, SNP_FORM_NAIVE = 1 };

/* Number of input features of the colour MLP besides the 3-d view direction. */
#define SNP_FEAT_DIM 8
/* Floats per primitive in the geometry array. */
#define SNP_GEOM_STRIDE 16

/* Pinhole camera, OpenCV frame (x right, y down, z forward).
 *   R_wc   world -> camera rotation, row-major (rows are the camera axes).
 *   eye    camera centre in world coordinates.
 *   fx, fy, cx, cy  intrinsics in pixels; the ray of pixel (px, py) passes
 *          through its centre: d = normalize(R_wc^T ((px + .5 - cx)/fx, (py + .5 - cy)/fy, 1)).
 *   z_near a primitive is culled unless its whole bounding ellipsoid lies at
 *          camera depth > z_near (camera z of the centre minus max(s) > z_near).
 *   width, height  image size in pixels (1..32768).
 *   time   timestamp xi_t in [0, 1] of this view; read only for dynamic scenes
 *          (snp_scene_desc.dynamic), ignored otherwise. */
typedef struct {
    float R_wc[9];
    float eye[3];
    float fx, fy, cx, cy, z_near;
    int32_t width, height;
    float time;
} snp_camera;

/* Scene description (sizes and modes; no pointers).
 *   n            number of primitives (0 allowed: renders background)
 *   n_sigma      density network width N_sigma (1..64)
 *   omega0       boosting frequency w0 of Eq. 6
 *   color_mode   SNP_COLOR_CONST (rgb in the geometry array), SNP_COLOR_MLP
 *                (per-primitive colour MLP: z0 = [d, f] with d the unit ray
 *                direction of the pixel and f an 8-d feature; z1 = relu(Wc1 z0 + bc1),
 *                z2 = relu(Wc2 z1 + bc2), colour = sigmoid(Wc3 z2 + bc3); two hidden
 *                layers of width n_c, the neural colour field of App. D.2) or
 *                SNP_COLOR_SH (the view-dependent colour of Sec. 3.1: four bands of
 *                real spherical harmonics per channel, evaluated once per (view,
 *                primitive) along the unit direction v from the camera centre to
 *                the primitive centre: colour = max(0, 1/2 + sum_i Y_i(v) sh[i]);
 *                Y_i the real harmonics of degree l = 0..3, index l^2 + l + m,
 *                in the tesseral form 1/2 sqrt(1/pi); sqrt(3/(4pi)) (y, z, x); ...)
 *   n_c          colour MLP width: 32 or 64 (ignored unless SNP_COLOR_MLP)
 *   weight_dtype SNP_F32 or SNP_BF16: element type of the `net` array.  All
 *                arithmetic is FP32 either way.
 *   dynamic      0: static scene.  1: time-conditioned density of the volumetric
 *                dynamic scenes (App. Applications): every hidden unit's phase gains
 *                xi_t W_t,k, i.e. sigma(x, xi_t) = w2 . cos(w0 (W1 u + b1) + xi_t W_t) + b2
 *                with xi_t the view's camera time and W_t in R^{n_sigma} per primitive
 *                (constant along a ray, so the closed-form integral keeps its form);
 *                with SNP_COLOR_SH the degree-0 coefficient of each channel also
 *                follows the time series sh[0] + sum_{i=1..4} a_i xi^i
 *                + sum_{i=1..4} (b_i cos(i xi) + c_i sin(i xi)).  Built for
 *                SNP_COLOR_CONST and SNP_COLOR_SH (SNP_ERR_UNSUPPORTED with the MLP). */
typedef struct {
    int64_t n;
    int32_t n_sigma;
    int32_t color_mode;
    int32_t n_c;
    int32_t weight_dtype;
    float omega0;
    int32_t dynamic;
} snp_scene_desc;

/* Per-primitive network layout of the `net` array: element offsets of each
 * field inside one primitive's record and the record stride, all multiples of 8
 * elements (16 bytes in BF16, 32 in FP32).  Fields, row-major:
 *   [0] W1 [n_sigma][3]  [1] b1 [n_sigma]  [2] w2 [n_sigma]  [3] b2 [1]
 *   [4] feat [8]  [5] Wc1 [n_c][11]  [6] bc1 [n_c]  [7] Wc2 [n_c][n_c]  [8] bc2 [n_c]
 *   [9] Wc3 [3][n_c]  [10] bc3 [3]   (colour fields only with SNP_COLOR_MLP)
 *   [11] sh [16][3] (only with SNP_COLOR_SH)
 *   [12] wt [n_sigma] (only when dynamic)
 *   [13] sh_t [12][3]: a_1..a_4, b_1..b_4, c_1..c_4 per channel (only when dynamic
 *        with SNP_COLOR_SH);
 *   absent fields have offset -1.  Padding elements are ignored on input and left
 *   untouched in gradients.  Pure function; never fails for valid sizes. */
typedef struct {
    int32_t off[14];
    int32_t stride;
} snp_net_layout;
snp_status snp_get_net_layout(const snp_scene_desc *desc, snp_net_layout *out);

/* The staging chunks (primitives per shared-memory batch) the library uses for
 * this scene description at tile_size (8, 16 or 32; 0 = 16) when snp_config.chunk
 * and snp_config.bwd_chunk are 0: *fwd_chunk for the forward (Sec. 3.2's per-tile
 * blend) and *bwd_chunk for the backward, each the largest that fits its kernel's
 * shared-memory budget.  Pure host function: SNP_ERR_INVALID_ARG for a NULL
 * pointer or a bad description, SNP_ERR_UNSUPPORTED for a tile size not built. */
snp_status snp_default_chunks(const snp_scene_desc *desc, int32_t tile_size, int32_t *fwd_chunk, int32_t *bwd_chunk);

/* Scene parameters (device, caller-owned, read-only):
 *   geom  float32 [n][16]: centre xyz, log-scale xyz, quaternion (w, x, y, z; need
 *         not be normalised), constant rgb, 3 unused floats.
 *   net   [n][stride] of weight_dtype, laid out as snp_get_net_layout says.
 * Both 16-byte aligned. */
typedef struct {
    const float *geom;
    const void *net;
} snp_scene_ptrs;

/* Gradients (device, caller-owned, float32, ACCUMULATED into: zero them first
 * for a fresh gradient).  Same shapes as snp_scene_ptrs: geom [n][16] (the 3
 * unused floats are untouched), net [n][stride] in float32 even when the
 * weights are BF16.  Either pointer may be NULL to skip that group. */
typedef struct {
    float *geom;
    float *net;
} snp_grad_ptrs;

/* Renderer configuration.
 *   tile_size     screen tile edge in pixels: 8, 16 or 32 (0 = 16)
 *   chunk         primitives staged per shared-memory batch of the forward
 *                 (0 = library default)
 *   integral_form SNP_FORM_STABLE: alpha_hat = Delta_t [b2 + sum_k w2_k cos(phi_k) sinc(theta_k)]
 *                 (Eq. 8 rewritten with sin A - sin B = 2 cos((A+B)/2) sin((A-B)/2), finite
 *                 as w0 W1_k . d -> 0); SNP_FORM_NAIVE: Eq. 8 literally, a difference of
 *                 sines divided by w0 W1_k . d / max(s)
 *   t_min         early termination: after compositing a primitive a pixel stops once
 *                 its transmittance T = exp(-sum of composited alpha_hat) < t_min
 *                 (0 disables; the dropped tail is at most t_min * max colour)
 *   bg            background colour added with the final transmittance */
typedef struct {
    int32_t tile_size;
    int32_t chunk;
    int32_t integral_form;
    float t_min;
    float bg[3];
    int32_t flags; /* SNP_FLAG_* bits */
    /* primitives per shared-memory batch of the backward (0 = library default: the
     * largest that fits the backward's own shared-memory budget, which differs from
     * the forward's; a larger value is lowered to that default; < 0 is refused) */
    int32_t bwd_chunk;
} snp_config;

/* snp_config.flags: record CUDA events around every stage on the call's stream so
 * that snp_stage_times can report per-stage device time (a few microseconds of
 * event overhead per call). */
#define SNP_FLAG_STAGE_TIMING 1
/* snp_config.flags: hand tiles to the persistent raster CTAs in order of
 * decreasing list length instead of row-major order (trades L2 reuse of
 * primitive records between neighbouring tiles for a shorter tail). */
#define SNP_FLAG_LENGTH_QUEUE 2
/* snp_config.flags: keep no colour store.  By default a forward saves, for every
 * composited pair, the colour and alpha_hat (colour-MLP scenes, 16 bytes per pair)
 * or alpha_hat alone (constant or SH colour, 4 bytes per pair), in a context
 * buffer sized from the previous forward's count, so that the backward evaluates
 * neither the colour network nor the integral again; with this flag the backward
 * recomputes them (less device memory, slower backward).  Pairs that do not fit the
 * buffer are recomputed either way.  Test hook: a non-negative integer in the
 * environment variable SNP_TEST_COLSTORE_PAIRS caps the store at that many pairs
 * (read at every forward), so tests can drive the recomputation path. */
#define SNP_FLAG_REPLAY_COLOR 4

/* Stages reported by snp_stage_times. */
enum {
    SNP_STAGE_PROJECT = 0,   /* k_project: bounding, culling, projection records */
    SNP_STAGE_SCAN = 1,      /* exclusive scan of tile counts (+ key-count readback) */
    SNP_STAGE_EMIT = 2,      /* tile-key emission */
    SNP_STAGE_SORT = 3,      /* stable radix sort of (tile, depth) keys */
    SNP_STAGE_RANGES = 4,    /* per-tile ranges */
    SNP_STAGE_RASTER_FWD = 5,
    SNP_STAGE_RASTER_BWD = 6,
    SNP_STAGE_POST_BWD = 7,  /* per-primitive gradient post-passes */
    SNP_N_STAGES = 8
};

/* Work counters of the last forward (read back synchronously). */
typedef struct {
    int64_t n_keys;       /* K: (tile, primitive) pairs after culling */
    int64_t n_tiles;      /* tiles over all views */
    int64_t n_pixels;     /* pixels over all views */
    int64_t n_candidates; /* (pixel, list entry) pairs visited before termination */
    int64_t n_hits;       /* of those, rays that enter the ellipsoid */
    int64_t n_composited; /* of those, alpha_hat > 0 (colour evaluated and blended) */
    int32_t fwd_ctas_per_sm; /* CTAs per SM the last raster forward launch kept resident (its
                              * persistent grid is this times the SM count, capped by the
                              * tiles); 0 before any forward */
    int32_t bwd_ctas_per_sm; /* the same for the last raster backward; 0 before any backward */
} snp_stats;

typedef struct snp_context snp_context;

/* Create a context on CUDA device `device` (it becomes current for the calling
 * thread).  *out receives the context; free it with snp_destroy. */
snp_status snp_create(int32_t device, snp_context **out);
void snp_destroy(snp_context *ctx);

/* Thread-safe message for the last failing call on ctx ("" if none). */
const char *snp_last_error(const snp_context *ctx);

/* Pre-allocate every workspace buffer for scenes of this description, these
 * cameras and configuration, with room for max_keys tile keys (0: the estimate
 * min(4 n n_cams + 1024, 2^32 - 1); above 2^32 - 1 the call returns
 * SNP_ERR_UNSUPPORTED, since key offsets are 32-bit).  After a successful
 * reserve no render call on the same shapes allocates device memory or
 * synchronises, which stream capture requires.  A reserved forward whose keys
 * exceed max_keys drops the excess and flags it; the next snp_get_stats or
 * snp_debug_keys on it returns SNP_ERR_CAPACITY, and its image is not valid.
 * While reserved, every forward must use the reserved tile size
 * (SNP_ERR_INVALID_ARG otherwise); a later reserve replaces the reservation. */
snp_status snp_reserve(snp_context *ctx, const snp_scene_desc *desc, const snp_camera *cams, int32_t n_cams,
                       const snp_config *cfg, int64_t max_keys);

/* Forward render of n_cams views (Sec. 3.2, Eq. 4-9).
 *   cams      host array of n_cams cameras
 *   images    device float32, views concatenated, each [height][width][3] (HWC)
 *   token     out: identifies this forward for snp_render_backward (the context
 *             keeps the state of its latest forward only); may be NULL
 * Stages: projection/bounding -> tile-key emission -> stable radix sort by
 * (tile, depth) -> tile ranges -> per-tile rasterization.  Outside of a
 * reservation the call synchronises once on `stream` to read back the key
 * count.
 * Limits: n * n_cams <= 2^32 - 1 (the key value is the instance v * n + i),
 * else SNP_ERR_UNSUPPORTED before any work.  The key offsets are scanned in
 * 32 bits: a total of 2^32 or more tile keys (one per tile that a primitive's
 * rectangle covers, per view) wraps, and the instance whose keys straddle 2^32
 * then ends past the key count, so the emission flags it like a capacity
 * overflow (snp_get_stats returns SNP_ERR_CAPACITY; the image is not valid).
 * Every write stays inside the buffers either way. */
snp_status snp_render_forward(snp_context *ctx, const snp_scene_desc *desc, const snp_scene_ptrs *scene,
                              const snp_camera *cams, int32_t n_cams, const snp_config *cfg, float *images,
                              int64_t *token, void *stream);

/* Backward of the forward identified by `token` (the scene pointers and values
 * must be unchanged since that forward).
 *   dL_dimages  device float32, same layout as the forward's images
 *   grads       accumulated into (see snp_grad_ptrs)
 * Replays each tile list front to back with the forward's per-pixel state
 * (final optical depth, colour, number of entries walked); gradients flow to
 * centres, log-scales, quaternions (through the normalisation), constant
 * colours and every density and colour-MLP weight.  SNP_ERR_INVALID_ARG if a
 * later forward replaced the saved state, if desc differs from the forward's,
 * or if grads->net is not 16-byte aligned (it receives bulk reductions). */
snp_status snp_render_backward(snp_context *ctx, int64_t token, const snp_scene_desc *desc,
                               const snp_scene_ptrs *scene, const float *dL_dimages, const snp_grad_ptrs *grads,
                               void *stream);

/* Autotuner: times forward (and, when with_backward != 0, backward) of this scene
 * and these cameras for tile sizes 8, 16, 32 and two staging chunk sizes each,
 * with CUDA events on `stream`, and writes the fastest configuration to *best
 * (other fields copied from *base) and its time per call to *best_ms.
 * Allocates its own temporary image, loss-gradient and gradient buffers (an
 * offline call: not for stream capture).  Leaves the context's latest-forward
 * state undefined (render again before a backward). */
snp_status snp_autotune(snp_context *ctx, const snp_scene_desc *desc, const snp_scene_ptrs *scene,
                        const snp_camera *cams, int32_t n_cams, const snp_config *base, int32_t with_backward,
                        snp_config *best, float *best_ms, void *stream);

/* Work counters of the forward identified by token (synchronises the stream). */
snp_status snp_get_stats(snp_context *ctx, int64_t token, snp_stats *out, void *stream);

/* Copy the sorted tile keys ((global tile << 32) | float bits of the camera-frame
 * depth of the centre) and values (view * n + primitive) of the forward `token`
 * to HOST arrays of capacity cap; *k_out receives K.  Synchronous.  Used to check
 * the ordering bit for bit.  Global tile ids number the tiles of view 0 row-major,
 * then view 1, and so on. */
snp_status snp_debug_keys(snp_context *ctx, int64_t token, uint64_t *keys_host, uint32_t *vals_host, int64_t cap,
                          int64_t *k_out, void *stream);

/* Device time per stage (milliseconds, summed) and number of timed calls per
 * stage, over every call made with SNP_FLAG_STAGE_TIMING since the last reset.
 * Synchronises with the last recorded event.  reset != 0 clears the sums after
 * reading.  ms and calls may be NULL; otherwise they hold SNP_N_STAGES entries. */
snp_status snp_stage_times(snp_context *ctx, double *ms, int64_t *calls, int32_t reset);

/* Number of CUDA kernels this library has launched in this process (all
 * contexts), for accounting of work per step. */
int64_t snp_kernel_launches(void);

/* Photometric loss of the differentiation workload: the mean squared error
 *   L = (1 / n) sum_i (image_i - target_i)^2
 * over n = 3 * pixels values, and its gradient dL/dimage_i = 2 (image_i - target_i) / n,
 * which is the dL_dimages input of snp_render_backward.  (The paper trains with
 * the photometric loss of 3D Gaussian splatting (Sec. 3.3, Training); the squared
 * error is the loss of the 300k-primitive, 1280 x 720 differentiation workload.)
 *   image, target  device, n floats each (HWC, views concatenated), caller-owned
 *   dL_dimage      device, n floats, caller-owned, overwritten
 *   loss           device, one float, caller-owned, overwritten
 *   stream         cudaStream_t; asynchronous, no allocation and no host
 *                  synchronisation (capturable in a CUDA graph)
 * The sum runs in FP64 in a fixed order (deterministic).  Calls on one context
 * share its reduction slots: do not run two at once on different streams.
 * n = 0 writes loss = 0.  Errors: SNP_ERR_INVALID_ARG for a null pointer or
 * n < 0, SNP_ERR_CUDA if the launch fails. */
snp_status snp_mse_loss(snp_context *ctx, const float *image, const float *target, int64_t n, float *dL_dimage,
                        float *loss, void *stream);

/* ------------------------------------------------------------------------
 * Training-step services around the renderer (Sec. 3.3 Training and
 * Population Control, Sec. 5.3, App. hyperparameters).  All take device
 * pointers owned by the caller and run asynchronously on `stream` unless stated.
 * ------------------------------------------------------------------------ */

/* Population-control statistic (Sec. 3.3, Population Control): the paper densifies
 * on the gradient magnitude of each primitive's network weights instead of the
 * screen-space position gradient of 3D Gaussian splatting.  Per primitive i, with
 * g the network-gradient record of one step (snp_render_backward's grads->net):
 *   m_i = || (dL/dW1, dL/db1, dL/dw2, dL/db2 [, dL/dW_t]) ||_2   (the density network)
 * and, where m_i > 0 (the primitive received gradient in this step),
 *   stat_sum[i] += m_i,  stat_count[i] += 1.
 *   g_net       device float32 [n][stride], read
 *   stat_sum    device float32 [n], stat_count device int32 [n]: accumulated into
 *               (zero both to start a densification window)
 * No allocation, no host synchronisation (capturable).  SNP_ERR_INVALID_ARG for a
 * null pointer with n > 0. */
snp_status snp_popctl_accumulate(snp_context *ctx, const snp_scene_desc *desc, const float *g_net, float *stat_sum,
                                 int32_t *stat_count, void *stream);

/* Thresholds of the population-control decision.  The paper's values (App.
 * hyperparameters): grad_threshold 1e-4 (real scenes) or 1e-5 (synthetic scenes),
 * prune_threshold 2e-6 or 1e-6, grow_scale 1e-2, prune_scale 0.5. */
typedef struct {
    float grad_threshold;  /* densify where stat_sum >= grad_threshold * stat_count (count > 0) */
    float prune_threshold; /* prune where stat_sum < prune_threshold * stat_count, or count == 0 */
    float grow_scale;      /* densified primitives with max(s) <= grow_scale * extent are cloned, others split */
    float prune_scale;     /* primitives with max(s) > prune_scale * extent are pruned */
    float extent;          /* scene extent in world units (> 0) */
    int32_t reserved_;
} snp_popctl_config;

enum { SNP_POP_PRUNE = 0, SNP_POP_KEEP = 1, SNP_POP_CLONE = 2, SNP_POP_SPLIT = 3 };

/* Decide per primitive, first rule that applies (l = max of the three log-scales):
 *   l > ln(prune_scale * extent)                      -> SNP_POP_PRUNE
 *   count > 0 and sum >= grad_threshold * count       -> SNP_POP_CLONE if l <= ln(grow_scale * extent),
 *                                                        else SNP_POP_SPLIT
 *   count == 0 or sum < prune_threshold * count       -> SNP_POP_PRUNE
 *   otherwise                                         -> SNP_POP_KEEP
 * Comparisons and the two products in float32; the two logarithms are evaluated in
 * double on the host and rounded to float32.  Outputs (device, caller-owned):
 *   action      int32 [n]
 *   out_offset  uint32 [n]: first output row of primitive i, the exclusive scan of
 *               its output count (PRUNE 0, KEEP 1, CLONE 2, SPLIT 2)
 *   n_out       host int64: number of output rows (the call synchronises `stream`)
 * Errors: SNP_ERR_INVALID_ARG for null pointers or extent <= 0. */
snp_status snp_popctl_plan(snp_context *ctx, const snp_scene_desc *desc, const float *geom, const float *stat_sum,
                           const int32_t *stat_count, const snp_popctl_config *cfg, int32_t *action,
                           uint32_t *out_offset, int64_t *n_out, void *stream);

/* Write the new scene of a plan: rows out_offset[i].. of geom_out / net_out receive
 * primitive i's outputs, so survivors keep their order.
 *   KEEP   one copy;  CLONE  two copies (3D Gaussian splatting's clone: the optimiser
 *          moves them apart);
 *   SPLIT  two children j = 0, 1 centred at c + R(q) diag(s) eps_j with log-scales
 *          log s - fl(ln 1.6) per axis (float32 subtraction), all else copied;
 *   PRUNE  nothing.
 *   noise     device float32 [n][2][3]: standard normal eps_0, eps_1 per primitive
 *             (the library draws no random numbers)
 *   geom_out  device float32 [n_out][16], net_out device [n_out][stride] of the
 *             scene's weight_dtype; must not overlap the inputs.
 * Network rows are copied bit for bit.  The caller resets its optimiser moments and
 * statistics for the new rows.  Asynchronous, no allocation. */
snp_status snp_popctl_apply(snp_context *ctx, const snp_scene_desc *desc, const snp_scene_ptrs *scene,
                            const int32_t *action, const uint32_t *out_offset, const float *noise, float *geom_out,
                            void *net_out, void *stream);

/* Geometry regulariser (Sec. 3.3 Training; Sec. 5.3): penalises anisotropic
 * primitives through the standard deviation of the components of each scale vector
 * s = exp(log s):
 *   L_reg = weight * (1/n) sum_i std(s_i),  std(s) = sqrt((1/3) sum_a (s_a - mean(s))^2),
 * and adds dL_reg/dlog s_a = (weight / n) s_a (s_a - mean(s)) / (3 std(s)) (0 where
 * std(s) = 0) into the log-scale columns of g_geom [n][16].
 *   loss  device float32, overwritten (FP64 block sums added in a fixed order)
 * Shares the context's reduction slots with snp_mse_loss: do not run the two at once
 * on different streams.  No allocation (capturable).  n = 0 writes loss = 0. */
snp_status snp_geom_reg(snp_context *ctx, const snp_scene_desc *desc, const float *geom, float weight,
                        float *g_geom, float *loss, void *stream);

/* One Adam step (Kingma and Ba, Algorithm 1; the paper trains with Adam and gives
 * per-group learning rates, App. hyperparameters), per element:
 *   m = beta1 m + (1 - beta1) g,   v = beta2 v + (1 - beta2) g^2,
 *   p = p - lr * (m / (1 - beta1^t)) / (sqrt(v / (1 - beta2^t)) + eps).
 *   lr_geom  per geometry column group: centres (0-2), log-scales (3-5),
 *            quaternions (6-9), constant rgb (10-12); columns 13-15 untouched
 *   lr_net   per snp_net_layout field (index as off[]); padding elements are updated
 *            with their field's rate and, with zero gradient and moments, stay put
 *   step     t >= 1; the bias corrections 1 / (1 - beta^t) are evaluated in double on
 *            the host and rounded to float32 */
typedef struct {
    float lr_geom[4];
    float lr_net[14];
    float beta1, beta2, eps;
    int32_t step;
} snp_adam_config;

/*   geom, m_geom, v_geom        device float32 [n][16] (updated); grads->geom read
 *   net                         device [n][stride] of weight_dtype (updated)
 *   net_master                  float32 [n][stride] master weights: required with
 *                               SNP_BF16 (updated, then rounded to nearest even into
 *                               net), NULL with SNP_F32 (net updated in place)
 *   m_net, v_net                device float32 [n][stride] (updated); grads->net read
 * A group whose gradient pointer is NULL is skipped.  Asynchronous, no allocation. */
snp_status snp_adam_step(snp_context *ctx, const snp_scene_desc *desc, float *geom, void *net, float *net_master,
                         const snp_grad_ptrs *grads, float *m_geom, float *v_geom, float *m_net, float *v_net,
                         const snp_adam_config *cfg, void *stream);

/* Allocation-free sort (the paper has no counterpart: this is a library
 * service).  Sorts n (key, value) pairs in place by the low key_bits bits of the
 * key, stably (equal keys keep their input order) -- the same LSD radix sort
 * that orders the tile keys inside snp_render_forward.
 *   keys, vals  device arrays of n elements, caller-owned (read and rewritten);
 *               keys 8-byte and vals 4-byte aligned
 *   key_bits    1..64; key bits at and above key_bits do not affect the order
 *               (they are carried along unchanged)
 *   stream      cudaStream_t; the call is asynchronous on it
 * For callers that must not allocate device memory while they run (inside an
 * application whose memory pool owns the device, a plugin handed a fixed arena,
 * or loops that cannot take cudaMalloc's implicit synchronisation): it needs no
 * context and calls no cudaMalloc / cudaFree.  Its scratch is one static device
 * array of SNP_NOALLOC_SORT_BYTES that every device loading the library keeps
 * until the process exits.  The first call on a device looks up that array's
 * address (make it before any stream capture).  All calls share the array: calls
 * that overlap on the GPU race.  Returns SNP_ERR_CAPACITY when
 * n > SNP_NOALLOC_SORT_MAX, SNP_ERR_INVALID_ARG for null or misaligned pointers
 * or a bad key_bits (before any device work), SNP_ERR_CUDA if a CUDA call
 * fails. */
#define SNP_NOALLOC_SORT_MAX (1 << 20)
#define SNP_NOALLOC_SORT_BYTES (13 << 20)
snp_status snp_sort_pairs_noalloc(uint64_t *keys, uint32_t *vals, int64_t n, int32_t key_bits, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* SNP_H */
