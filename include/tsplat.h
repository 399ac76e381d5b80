/*
 * tsplat.h -- C ABI of libtsplat: latent-feature Gaussian splatting on one
 * GB300 (sm_103a).
 *
 * The calls follow the statement of the problem in Tele-Aloha (arXiv
 * 2405.14866), Sec. 4.2 "Neural Rasterization via 3DGS":
 *   - each point is a Gaussian with position x_i, latent feature f_i
 *     (d = C channels), scale s_i and opacity alpha_i (rotation identity in
 *     the paper, an input here);
 *   - positions are unprojected from the source depth maps with the camera
 *     parameters Pi, and the foreground pixels become pixel-aligned
 *     Gaussians                                           -> tsplat_build
 *   - the Gaussians are differentiably rasterized to the target view,
 *     F_novel = R_G({G}, Pi_novel), with the 3DGS rasterizer the paper
 *     cites (EWA projection, 16x16 tiles, (tile, depth) order,
 *     front-to-back alpha compositing of features)      -> tsplat_render
 *   - gradients flow through R_G because the encoder and decoder around it
 *     are trained end to end                             -> tsplat_backward
 *   - the system renders the viewer's left and right eye views every frame
 *     and is optimized with CUDA Graphs (Sec. 5.3)        -> tsplat_server_*
 *
 * General rules.
 *   - Every pointer argument documented as "device" must point to memory of
 *     the current CUDA device; "host" pointers to host memory.  The caller
 *     owns all input and output buffers; the library owns the opaque
 *     handles and their scratch memory.
 *   - `stream` is a cudaStream_t (NULL = the legacy default stream).  Calls
 *     are stream-ordered and asynchronous unless documented to synchronize.
 *   - Every call returns a tsplat_status; on failure a thread-local message
 *     is available from tsplat_last_error().  No C++ exception crosses the
 *     ABI.  Errors found by the kernels themselves (buffer capacity,
 *     invalid sizes) are written to a device status word of the context and
 *     returned by the next call that synchronizes on it (tsplat_ctx_status).
 *   - Sizes: N < 2^31 Gaussians, images up to 16383 x 16383 pixels,
 *     1 <= C <= 64 feature channels.
 */
#ifndef TSPLAT_H
#define TSPLAT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    TSPLAT_OK = 0,
    TSPLAT_ERR_INVALID_ARG = 1,  /* a size, pointer or enum is out of range */
    TSPLAT_ERR_OOM = 2,          /* device allocation failed */
    TSPLAT_ERR_CAPACITY = 3,     /* a buffer bound was exceeded (see the call) */
    TSPLAT_ERR_TIMEOUT = 4,      /* a bounded wait expired */
    TSPLAT_ERR_CUDA = 5,         /* a CUDA runtime call failed */
    TSPLAT_ERR_NOT_READY = 6,    /* asynchronous work has not finished yet */
    TSPLAT_ERR_UNSUPPORTED = 7   /* feature combination not built */
} tsplat_status;

/* feature storage types */
enum { TSPLAT_F32 = 0, TSPLAT_BF16 = 1 };

/* Pinhole camera.  R, t map world to camera coordinates, p = R x + t
 * (R row-major).  Camera frame: x right, y down, z forward.  Pixel (u, v) =
 * (column, row) is centred at image coordinate (u, v).  Only Gaussians
 * with z_near < p_z < z_far are rendered. */
typedef struct {
    float fx, fy, cx, cy;
    int32_t width, height;
    float R[9];
    float t[3];
    float z_near, z_far;
} tsplat_camera;

/* flags of tsplat_render_params */
enum {
    /* Do not synchronize to size the pair buffer: use the capacity set with
     * tsplat_ctx_reserve and report an overflow through the context status
     * (needed for CUDA-graph capture). */
    TSPLAT_RENDER_ASYNC = 1u << 0,
    /* Keep what tsplat_backward needs (final transmittance and last
     * blended index per pixel). */
    TSPLAT_RENDER_SAVE = 1u << 1,
    /* Record CUDA events between the stages of this render on its stream
     * (read back with tsplat_ctx_timings). */
    TSPLAT_RENDER_PROFILE = 1u << 2,
    /* Tight binning (a variant; the cited rasterizer keeps the whole rect).
     * A tile of a Gaussian's rect (rects of at most 32 tiles; larger ones
     * stay whole) is kept only when the smallest Q = d^T conic d over the
     * rectangle of the tile's pixel centres, clipped to the image, is at
     * most 2 ln(o / alpha_min) (1 + 2^-10) + 2^-8: dropped tiles hold no
     * pixel with alpha >= alpha_min, so the maps equal the full-rect ones up
     * to the order of FP32 accumulation, while the pairs to sort and
     * composite shrink.  Gaussians left with no tile (e.g. o < alpha_min)
     * are culled.  All of it in single precision, one rounding per
     * operation, so the tile lists are reproducible bit for bit. */
    TSPLAT_RENDER_TIGHT = 1u << 3
};

/* Rasterizer constants (the 3DGS rasterizer's; all parameters). */
typedef struct {
    float lowpass;        /* px^2 added to the diagonal of Sigma2D (0.3) */
    float alpha_max;      /* opacity clamp (0.99) */
    float alpha_min;      /* skip threshold (1/255) */
    float t_min;          /* transmittance stop threshold (1e-4) */
    float frustum_clamp;  /* Jacobian clamp in units of tan(fov/2) (1.3) */
    uint32_t flags;       /* TSPLAT_RENDER_* */
} tsplat_render_params;

/* Fill `p` with the defaults listed above (flags = 0). */
void tsplat_render_params_default(tsplat_render_params *p);

/* flags of tsplat_src_view */
enum {
    /* depth, scale, quat, opacity and feat hold only the foreground pixels
     * (mask nonzero), in row-major pixel order: n_fg rows instead of H*W.
     * The mask is required.  Background pixels carry nothing the lifting
     * reads, so this halves the bytes to move for a half-foreground view.
     * Not accepted by tsplat_build_backward (whose outputs are full maps) or
     * tsplat_build_into_noalloc (TSPLAT_ERR_UNSUPPORTED there). */
    TSPLAT_SRC_COMPACT = 1
};

/* One source view (Sec. 4.2: depth map plus the encoder's per-pixel maps).
 * All map pointers are device pointers, row-major H x W (x channels):
 *   depth    H*W   f32  camera-space z in metres
 *   mask     H*W   u8   nonzero = foreground; NULL = every pixel
 *   scale    H*W*3 f32  standard deviations along the Gaussian's axes (M_s)
 *   quat     H*W*4 f32  (w,x,y,z) rotation of the axes in the source camera
 *                       frame; NULL = identity (the paper's choice)
 *   opacity  H*W   f32  (M_alpha)
 *   feat     H*W*C      latent features (M_f), type feat_dtype
 * (with TSPLAT_SRC_COMPACT: n_fg rows of each map but the mask). */
typedef struct {
    const float *depth;
    const uint8_t *mask;
    const float *scale;
    const float *quat;
    const float *opacity;
    const void *feat;
    int32_t feat_dtype;
    int32_t flags;        /* TSPLAT_SRC_* (0: full maps) */
    tsplat_camera cam;
} tsplat_src_view;

/* ------------------------------------------------------------------------
 * Gaussians (library-owned, device-resident)
 *
 * Layout: N Gaussians in id order; positions and opacities as float4
 * (x, y, z, opacity), covariances as float4 (s00, s01, s02, s11) plus
 * float2 (s12, s22), features N x C of the storage type.  N lives in device
 * memory (so that building can be captured in a CUDA graph).
 * ---------------------------------------------------------------------- */
typedef struct tsplat_gaussians tsplat_gaussians;

/* Allocate room for `capacity` Gaussians with C channels of type
 * feat_dtype.  N starts at 0.  TSPLAT_ERR_INVALID_ARG for C outside
 * [1, 64] or an unknown type, TSPLAT_ERR_OOM / TSPLAT_ERR_CUDA when the
 * device allocation fails (no handle is returned then).  An FP32 store also
 * keeps every feature row as bf16 (hi, lo) parts (hi = bf16(f), lo =
 * bf16(f - hi); 16, 32 or 64 columns each, 4 bytes per column per
 * Gaussian), written with the features: the operands of the compositing's
 * tensor-core products. */
tsplat_status tsplat_gaussians_create(int64_t capacity, int32_t C, int32_t feat_dtype,
                                      tsplat_gaussians **out);
/* Synchronizes the device, then frees the store (NULL is a no-op).  A
 * context that rendered this store must not be asked for its statistics,
 * exports or backward afterwards: it reads the store's count and features
 * until its next render. */
tsplat_status tsplat_gaussians_destroy(tsplat_gaussians *g);

/* Load N Gaussians from caller device arrays: mean N*3 f32, cov N*6 f32
 * (s00 s01 s02 s11 s12 s22), opac N f32, feat N*C of type feat_dtype_in
 * (converted to the storage type with round-to-nearest-even).  N must not
 * exceed the capacity. */
tsplat_status tsplat_gaussians_set(tsplat_gaussians *g, int64_t n, const float *mean,
                                   const float *cov, const float *opac, const void *feat,
                                   int32_t feat_dtype_in, void *stream);

/* Copy the current Gaussians to caller device arrays (layouts as in _set;
 * feat in the storage type).  Synchronizes `stream` to learn N first. */
tsplat_status tsplat_gaussians_get(const tsplat_gaussians *g, float *mean, float *cov,
                                   float *opac, void *feat, void *stream);

/* Current N (synchronizes on the stream that last wrote it). */
tsplat_status tsplat_gaussians_count(const tsplat_gaussians *g, int64_t *n);
tsplat_status tsplat_gaussians_shape(const tsplat_gaussians *g, int64_t *capacity,
                                     int32_t *C, int32_t *feat_dtype);

/* ------------------------------------------------------------------------
 * A1 -- lifting (Sec. 4.2: foreground pixels of the source views are lifted
 * to pixel-aligned Gaussians; positions unprojected with Pi).
 *
 * For pixel (u,v) of view s with depth z:
 *   x_world = R_s^T (z ((u - cx)/fx, (v - cy)/fy, 1) - t_s)
 *   Sigma3D = R_g diag(scale)^2 R_g^T,  R_g = R_s^T R(quat)
 * Gaussian ids follow (view, row, column) order of the foreground pixels.
 * Arithmetic is single precision in a fixed operation order (no fused
 * multiply-add), identical to the oracle's key mode.
 *
 * tsplat_build allocates a new handle with capacity = sum of H*W (the
 * upper bound of N); tsplat_build_into reuses `g`, whose capacity must be at
 * least the total pixel count of the views and whose C must match.  Both
 * are asynchronous; N stays on the device.  1 <= n_views <= 16.
 * ---------------------------------------------------------------------- */
tsplat_status tsplat_build(const tsplat_src_view *views, int32_t n_views, int32_t C,
                           int32_t feat_dtype, tsplat_gaussians **out, void *stream);
tsplat_status tsplat_build_into(tsplat_gaussians *g, const tsplat_src_view *views,
                                int32_t n_views, void *stream);

/* tsplat_build_into without any device allocation (the paper has no
 * counterpart).  For callers that cannot call cudaMalloc at this point: a
 * frame loop with a fixed latency budget (device allocation and release
 * synchronize the device), or a process whose device memory is fully owned
 * by another allocator.  Same inputs, outputs and results as
 * tsplat_build_into; `g` is allocated by the caller beforehand
 * (tsplat_gaussians_create).
 * Limit: at most 64 Mi source pixels in total per call (e.g. 16 views of
 * 2048 x 2048); larger inputs return TSPLAT_ERR_CAPACITY before any work.
 * The per-block scratch of the compaction is one fixed 512 KiB device array
 * that every GPU loading the library keeps until the process exits.  The
 * first call on a device resolves that array's device address (with that
 * device current); make that first call before any stream capture.  All
 * calls share the array: calls that overlap on the GPU (other streams,
 * other threads) race and must be serialized by the caller. */
tsplat_status tsplat_build_into_noalloc(tsplat_gaussians *g, const tsplat_src_view *views,
                                        int32_t n_views, void *stream);

/* ------------------------------------------------------------------------
 * Render context: scratch memory of one render stream plus the state saved
 * for the backward pass.  One context must not be used by two streams at
 * once.  Buffers grow on demand (device allocation); tsplat_ctx_reserve
 * pre-sizes them so that later calls allocate nothing.
 * ---------------------------------------------------------------------- */
typedef struct tsplat_ctx tsplat_ctx;

/* A context with only its small state word area allocated (synchronizes
 * the legacy default stream); TSPLAT_ERR_OOM / TSPLAT_ERR_CUDA if that
 * fails, e.g. without a CUDA device. */
tsplat_status tsplat_ctx_create(tsplat_ctx **out);
/* Synchronizes the device, then frees every buffer of the context (NULL is
 * a no-op). */
tsplat_status tsplat_ctx_destroy(tsplat_ctx *ctx);
/* Grows the buffers for renders of up to max_gaussians Gaussians (instances,
 * for batches), max_pairs pairs and max_width x max_height pixels, and
 * synchronizes.  C (0 .. 64; 0 = none) sizes the staging of a
 * tsplat_rasterize call's FP32 features (their bf16 hi, lo parts); feature
 * buffers themselves belong to the caller or the store.  Needed before
 * TSPLAT_RENDER_ASYNC renders and graph capture. */
tsplat_status tsplat_ctx_reserve(tsplat_ctx *ctx, int64_t max_gaussians, int64_t max_pairs,
                                 int32_t max_width, int32_t max_height, int32_t C);

typedef struct {
    int64_t n_gaussians;   /* N of the last render */
    int64_t n_visible;     /* Gaussians with at least one tile */
    int64_t n_pairs;       /* P: (Gaussian, tile) pairs */
    int64_t pair_capacity; /* current size of the pair buffers */
    int32_t tiles_x, tiles_y;
    int32_t width, height, C;
    int32_t device_status; /* tsplat_status written by kernels (0 = OK) */
} tsplat_ctx_stats;

/* Statistics of the last render on `ctx` (synchronizes the context's last
 * stream). */
tsplat_status tsplat_ctx_stats_get(tsplat_ctx *ctx, tsplat_ctx_stats *out);

/* Device status of the last render (synchronizes); TSPLAT_ERR_CAPACITY if
 * the pair buffer overflowed in TSPLAT_RENDER_ASYNC mode. */
tsplat_status tsplat_ctx_status(tsplat_ctx *ctx);

/* Intermediate results of the last render, copied to a caller device
 * buffer of `bytes` bytes (for tests and tools).  The context reads the
 * Gaussian count of the store it last rendered: keep that store alive until
 * the exports, the statistics and the backward of that render are done.
 *   TSPLAT_EXPORT_RECT     N x 4 int32 tile rect (x0 y0 x1 y1), culled = 0
 *   TSPLAT_EXPORT_DEPTHKEY N uint32 depth key (bits of camera z), culled = 0xFFFFFFFF
 *   TSPLAT_EXPORT_MEAN2D   N x 2 f32
 *   TSPLAT_EXPORT_CONIC    N x 3 f32
 *   TSPLAT_EXPORT_RADIUS   N f32
 *   TSPLAT_EXPORT_PAIRS    P uint32 Gaussian ids in (tile, depth, id) order
 *   TSPLAT_EXPORT_RANGES   tiles x 2 uint32 [first, last) per tile
 *   TSPLAT_EXPORT_TFINAL   H x W f32 (needs TSPLAT_RENDER_SAVE)
 *   TSPLAT_EXPORT_LAST     H x W uint32 (needs TSPLAT_RENDER_SAVE)
 *   TSPLAT_EXPORT_TILE_ORDER  one uint32 per tile slot of the render (all
 *                          views of a batch): the order in which the bucket
 *                          sort, the composite and the backward take the
 *                          tiles -- a permutation of the slots, longest pair
 *                          list first (tiles bucketed by 4 log2 of their pair
 *                          count; the order within a bucket is unspecified),
 *                          then the tiles without pairs */
enum {
    TSPLAT_EXPORT_RECT = 0, TSPLAT_EXPORT_DEPTHKEY = 1, TSPLAT_EXPORT_MEAN2D = 2,
    TSPLAT_EXPORT_CONIC = 3, TSPLAT_EXPORT_RADIUS = 4, TSPLAT_EXPORT_PAIRS = 5,
    TSPLAT_EXPORT_RANGES = 6, TSPLAT_EXPORT_TFINAL = 7, TSPLAT_EXPORT_LAST = 8,
    TSPLAT_EXPORT_TILE_ORDER = 9
};
tsplat_status tsplat_ctx_export(tsplat_ctx *ctx, int32_t what, void *dst, size_t bytes, void *stream);

/* ------------------------------------------------------------------------
 * A2..A7 -- render (Sec. 4.2: F_novel = R_G({G}, Pi_novel)).
 *
 * A2 project: p = R x + t; visible iff z_near < p_z < z_far;
 *   J = [[fx/p_z, 0, -fx t_x/p_z^2], [0, fy/p_z, -fy t_y/p_z^2]] with
 *   t_x/p_z, t_y/p_z clamped to +-frustum_clamp * 0.5 W/fx (0.5 H/fy);
 *   Sigma2D = (J R) Sigma3D (J R)^T + lowpass I, det <= 0 or non-finite
 *   culls; conic = (c, -b, a)/det; r = ceil(3 sqrt(m + sqrt(max(0.1,
 *   m^2 - det)))), m = (a+c)/2; mean2D = (fx p_x/p_z + cx, fy p_y/p_z + cy);
 *   tile rect [floor((mu-r)/16), floor((mu+r+15)/16)) clamped to the grid.
 * A3-A6: one (Gaussian, tile) pair per tile of the rect, ordered by
 *   (tile, bits of p_z, Gaussian id) -- identical to a stable sort of the
 *   64-bit key tile << 32 | bits(p_z) -- and per-tile ranges.
 * A7 composite, per pixel p, front to back over its tile's list:
 *   q = -1/2 (a dx^2 + c dy^2) - b dx dy, d = p - mean2D; q > 0 skips
 *   (never, for the positive-definite conics projection keeps, but through
 *   rounding at the centre; the kernels do not test it separately);
 *   alpha = min(alpha_max, o e^q); alpha < alpha_min skips;
 *   T' = T (1 - alpha); T' < t_min stops (that Gaussian is not blended);
 *   F += f alpha T; T = T'.   A = 1 - T at the end.
 *
 * out_feat:  device, C x H x W f32 (H, W of the camera), overwritten.
 * out_alpha: device, H x W f32, overwritten; may be NULL.
 * Without TSPLAT_RENDER_ASYNC the call synchronizes once (to size the pair
 * buffer); with it the call never synchronizes and writes
 * TSPLAT_ERR_CAPACITY to the context status if P exceeds the reserved
 * capacity (outputs are then incomplete).
 * `g` must stay alive and unmodified until tsplat_backward has used `ctx`.
 * ---------------------------------------------------------------------- */
tsplat_status tsplat_render(const tsplat_gaussians *g, const tsplat_camera *cam,
                            const tsplat_render_params *params, float *out_feat,
                            float *out_alpha, tsplat_ctx *ctx, void *stream);

/* Several target views of the same Gaussians in one pass (the viewer's left
 * and right eye views, Sec. 4.2; several viewers in serving): 1 <= n_views
 * <= 8 cameras of any sizes.  Every view's Gaussians are projected in one
 * launch (each Gaussian read once), the tile ids of all views form one
 * space binned by one bucket pass over all (view, Gaussian) instances, and
 * one compositing launch covers every tile.  out_feat[v] (C x H_v x W_v) and
 * out_alpha[v] (H_v x W_v, or out_alpha == NULL) are device buffers.  Each
 * view's result is bit-identical to tsplat_render of that view alone.
 * TSPLAT_RENDER_SAVE is not supported here (TSPLAT_ERR_UNSUPPORTED).  In
 * TSPLAT_RENDER_ASYNC mode, reserve the context for n_views * N Gaussians,
 * the pairs of all views and the sum of their tiles. */
tsplat_status tsplat_render_batch(const tsplat_gaussians *g, const tsplat_camera *cams, int32_t n_views,
                                  const tsplat_render_params *params, float *const *out_feat,
                                  float *const *out_alpha, tsplat_ctx *ctx, void *stream);

/* A3..A7 from already projected 2D Gaussians (device arrays):
 *   mean2d N*2 f32, conic N*3 f32 (a, b, c), opac N f32,
 *   depth N f32 (sort key; must be > 0 for rendered Gaussians),
 *   radius N int32 (0 = not rendered), feat N*C of type feat_dtype.
 * The tile rect is derived from mean2d and radius as in A2.  Outputs as in
 * tsplat_render.  This is the forward of the differentiable rasterizer. */
tsplat_status tsplat_rasterize(int64_t n, const float *mean2d, const float *conic,
                               const float *opac, const float *depth, const int32_t *radius,
                               const void *feat, int32_t C, int32_t feat_dtype, int32_t width,
                               int32_t height, const tsplat_render_params *params,
                               float *out_feat, float *out_alpha, tsplat_ctx *ctx, void *stream);

/* ------------------------------------------------------------------------
 * Backward through the projection and the lifting (Sec. 4.2: the encoder
 * is trained end to end through R_G), continuing tsplat_backward.
 *
 * tsplat_backward_project: dL/dmean3d (N x 3, world space) and dL/dcov3d
 * (N x 6: the stored entries s00 s01 s02 s11 s12 s22) of the Gaussians in
 * `g` from dL/dmean2d (N x 2) and dL/dconic (N x 3, the raw conic (A, B, C)
 * of q = -(A dx^2 + 2 B dx dy + C dy^2) / 2, as tsplat_backward returns
 * them).  Needs the last call on `ctx` to be a tsplat_render of `g` with
 * TSPLAT_RENDER_SAVE (its camera and parameters are used).  The chain goes
 * through mu = f p / z + c, the Jacobian (x/z and y/z clamped: no gradient
 * through a clamped ratio), S = (J R) V (J R)^T + lowpass I and conic = S^-1.
 *
 * tsplat_build_backward: per source pixel gradients of the maps the store
 * `g` was built from (`views` must be those of its last build): depth
 * (H x W), scale (H x W x 3), quat (H x W x 4, w.r.t. the unnormalised
 * quaternion; ignored when the view has no quat map), opacity (H x W),
 * features (H x W x C, f32), from dL/dmean3d, dL/dcov3d, dL/dopac (N) and
 * dL/dfeat (N x C).  Background pixels get zeros.  All device f32 buffers,
 * overwritten; asynchronous on `stream`.
 * ---------------------------------------------------------------------- */
typedef struct {
    float *depth;    /* H x W */
    float *scale;    /* H x W x 3 */
    float *quat;     /* H x W x 4, 16-byte aligned, or NULL */
    float *opacity;  /* H x W */
    float *feat;     /* H x W x C */
} tsplat_src_grads;

tsplat_status tsplat_backward_project(tsplat_ctx *ctx, const tsplat_gaussians *g, const float *d_mean2d,
                                      const float *d_conic, float *d_mean3d, float *d_cov3d, void *stream);
tsplat_status tsplat_build_backward(tsplat_gaussians *g, const tsplat_src_view *views, int32_t n_views,
                                    const float *d_mean3d, const float *d_cov3d, const float *d_opac,
                                    const float *d_feat, const tsplat_src_grads *grads, void *stream);

/* ------------------------------------------------------------------------
 * Point z-buffer (Sec. 4.1: the points lifted from one view's depth map are
 * rasterized into other cameras and their z-buffer is read out; Sec. 4.3:
 * predicted depth maps are warped onto the novel view).  Each Gaussian mean
 * is projected into `cam` (the projection's single-precision operations)
 * and lands on the pixel with the nearest centre, (floor(x + 0.5),
 * floor(y + 0.5)), when its camera-space depth lies in (z_near, z_far).
 * Each pixel keeps the nearest point, the lowest Gaussian id among equal
 * depths.  out_depth: device H x W f32, 0 where no point landed;
 * out_id: device H x W int32, -1 there, or NULL.  Scratch (8 B per pixel)
 * comes from `ctx`.  Asynchronous on `stream`.
 * ---------------------------------------------------------------------- */
tsplat_status tsplat_zbuffer(const tsplat_gaussians *g, const tsplat_camera *cam, float *out_depth,
                             int32_t *out_id, tsplat_ctx *ctx, void *stream);

/* ------------------------------------------------------------------------
 * A8 -- backward of A7 (Sec. 4.2: R_G is differentiable; the encoder and
 * decoder are trained through it).  Needs a render or rasterize on `ctx`
 * with TSPLAT_RENDER_SAVE.  With g = dL/dF(p), gA = dL/dA(p), T_j the
 * transmittance before blended Gaussian j (recomputed from the saved final
 * transmittance by division, not stored) and S_j the blended features
 * behind j:
 *   dL/df_j     += alpha_j T_j g
 *   dL/dalpha_j  = T_j <f_j, g> - <S_j, g>/(1 - alpha_j) + gA T_final/(1 - alpha_j)
 * chained through alpha = o e^q (no gradient where alpha was clamped) to
 * the opacity, the conic (a, b, c) and the 2D mean.
 *   dL_dfeat  device C x H x W f32;  dL_dalpha device H x W f32 or NULL
 *   d_mean2d N*2, d_conic N*3, d_opac N, d_feat N*C: device f32 outputs,
 *   overwritten, indexed by Gaussian id.  Any output may be NULL.
 * Accumulation order across pixels is not deterministic (FP32 atomics).
 * Single precision: the sums over a warp's pixels <f_j, g> and dL/df_j are
 * tensor-core products on bf16 hi + lo parts (relative error about 2^-16);
 * the division uses the hardware reciprocal.  FP32 features are read from
 * the split rows the render used.
 * ---------------------------------------------------------------------- */
tsplat_status tsplat_backward(tsplat_ctx *ctx, const float *dL_dfeat, const float *dL_dalpha,
                              float *d_mean2d, float *d_conic, float *d_opac, float *d_feat,
                              void *stream);

/* ------------------------------------------------------------------------
 * A9 -- serving: continuous batching of target views (the viewer's left and
 * right eye views, Sec. 4.2; CUDA Graphs, Sec. 5.3).
 *
 * A worker thread admits submitted requests, in arrival order, into batches
 * of up to max_views_per_batch views of any sizes (up to max_width x
 * max_height) while the batch's estimated pairs fit one lane's pair
 * buffer.  Each lane renders one batch at a time as one
 * CUDA-graph replay of tsplat_render_batch; up to max_lanes batches overlap
 * on the device, as many as budget_bytes of scratch allow.  A batch that
 * overflows is re-run one view at a time.  Each result is bit-identical to
 * rendering that view alone.  Outputs are caller device buffers as in
 * tsplat_render; they must stay valid until the request completes, and no
 * work on them may be pending at submission (the server's streams do not
 * wait on the caller's).  Once tsplat_server_wait/poll reports completion
 * the outputs may be read on any stream.
 * ---------------------------------------------------------------------- */
typedef struct tsplat_server tsplat_server;
/* Issue each batch as plain launches instead of a CUDA-graph replay.  With
 * max_views_per_batch = 1 and max_lanes = 1 the server renders one view per
 * launch sequence, one at a time: the unbatched baseline behind the same
 * queue. */
#define TSPLAT_SERVER_NO_GRAPH 1
typedef struct {
    int32_t max_views_per_batch;  /* 1..8 (8) */
    int32_t max_lanes;            /* batches in flight at once (3) */
    int32_t max_width, max_height;/* largest view (1024 x 1024) */
    int64_t max_gaussians;        /* capacity of the frames' Gaussian stores (2^22) */
    int32_t C, feat_dtype;        /* of the frames (32, TSPLAT_BF16) */
    /* admission estimate of a view's (Gaussian, tile) pairs:
     * pairs_per_gaussian x frame capacity + pairs_per_pixel x width x height;
     * a lane's pair buffer holds max_views_per_batch maximal views' worth.
     * Once batches retire, admission scales the estimates by the running
     * ratio of their measured to estimated pairs (plus a 10 % margin) */
    float pairs_per_gaussian;     /* (2.5) */
    float pairs_per_pixel;        /* (1.0) */
    int32_t flags;                /* TSPLAT_SERVER_* (0) */
    int32_t max_inflight_views;   /* views on the device at once over all lanes; 0 = lanes x batch (0) */
    int64_t budget_bytes;         /* device memory for the lanes' scratch (8 GiB) */
    tsplat_render_params params;
} tsplat_server_config;

typedef struct {
    int64_t completed, batches, views_launched, retried, pending;
    int64_t lane_bytes;             /* device scratch of one lane */
    int32_t lanes, reserved;
    double p50_ms, p99_ms, max_ms;  /* request latency, submission to completion */
    double views_per_s;             /* completed / (last completion - first submission) */
    double pair_scale;              /* measured / estimated pairs of retired batches (running; 0 = none yet) */
} tsplat_server_stats;

void tsplat_server_config_default(tsplat_server_config *cfg);
tsplat_status tsplat_server_create(const tsplat_server_config *cfg, tsplat_server **out);
/* Waits for the batches in flight, drops pending requests. */
tsplat_status tsplat_server_destroy(tsplat_server *s);
/* Gaussians that the batches admitted from now on render (the frame; keep
 * it alive and unmodified while batches use it -- double-buffer frames).
 * Batches wait on the device for the work queued, at the time of this call,
 * on the stream that last built `g`. */
tsplat_status tsplat_server_update_frame(tsplat_server *s, const tsplat_gaussians *g);
/* Captures, on every lane, the graphs of all batch sizes for the store `g`
 * (which need not be the current frame), so that no capture happens while
 * requests wait; blocks until done or timeout_ms passed.  Graphs are kept
 * for the two most recently used stores of each lane. */
tsplat_status tsplat_server_prepare(tsplat_server *s, const tsplat_gaussians *g, double timeout_ms);
/* Blocks until no batch in flight renders `g` (a frame replaced by a later
 * tsplat_server_update_frame), so that it may be rebuilt; TSPLAT_ERR_TIMEOUT
 * after timeout_ms; TSPLAT_ERR_INVALID_ARG if `g` is the current frame. */
tsplat_status tsplat_server_release_frame(tsplat_server *s, const tsplat_gaussians *g, double timeout_ms);
tsplat_status tsplat_server_submit(tsplat_server *s, const tsplat_camera *cam, float *out_feat,
                                   float *out_alpha, uint64_t *req_id);
/* TSPLAT_OK when done (latency in ms), TSPLAT_ERR_NOT_READY before. */
tsplat_status tsplat_server_poll(tsplat_server *s, uint64_t req_id, double *latency_ms);
/* Blocks until done or timeout_ms passed (TSPLAT_ERR_TIMEOUT). */
tsplat_status tsplat_server_wait(tsplat_server *s, uint64_t req_id, double timeout_ms, double *latency_ms);
tsplat_status tsplat_server_get_stats(tsplat_server *s, tsplat_server_stats *out);
/* Clears statistics and forgets completed requests. */
tsplat_status tsplat_server_reset_stats(tsplat_server *s);

/* Mean stage durations, in milliseconds, of the renders on `ctx` that used
 * TSPLAT_RENDER_PROFILE since the previous call (at most the last 256),
 * measured with CUDA events on the render's stream; synchronizes and
 * resets.  ms[0..4] = projection with the per-tile pair counts (A2/A3),
 * scan into ranges and tile order (A4/A6), bucket fill (A4), bucket sort
 * (A5), composite (A7); *n_out = 5. */
tsplat_status tsplat_ctx_timings(tsplat_ctx *ctx, float *ms, int32_t capacity, int32_t *n_out);

/* Number of kernel launches the library has issued in this process. */
uint64_t tsplat_launch_count(void);

/* Thread-local message of the last failed call on this thread. */
const char *tsplat_last_error(void);

/* Library version string. */
const char *tsplat_version(void);

#ifdef __cplusplus
}
#endif
#endif /* TSPLAT_H */
