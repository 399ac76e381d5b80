// Host-side launchers of libtsplat's kernels (internal, C++).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <atomic>
#include <mutex>

#include "../../include/tsplat.h"

namespace tsp {

// A launch set-up value (a grid size, after any kernel attributes it needs
// are set) computed once per device, with that device current, under a
// lock; later launches on that device read it without locking.
constexpr int MAX_DEVICES = 64;
class PerDevice {
    std::mutex mu_;
    std::atomic<int> val_[MAX_DEVICES] = {};

public:
    template <class F>
    int get(F make) {
        int dev = 0;
        if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= MAX_DEVICES) return std::max(1, make(dev));
        int v = val_[dev].load(std::memory_order_acquire);
        if (v) return v;
        std::lock_guard<std::mutex> lock(mu_);
        v = val_[dev].load(std::memory_order_relaxed);
        if (!v) {
            v = std::max(1, make(dev));
            val_[dev].store(v, std::memory_order_release);
        }
        return v;
    }
};
// Streaming multiprocessors of the current device.
int sm_count();

struct Header;

constexpr int MAX_VIEWS = 16;

// ---------------------------------------------------------------- A1 build
struct ViewDesc {
    const float *depth;
    const uint8_t *mask;
    const float *scale;
    const float *quat;
    const float *opacity;
    const void *feat;
    int feat_dtype;
    int compact;      // TSPLAT_SRC_COMPACT: maps hold the foreground pixels only
    int H, W;
    int64_t blk0;     // first lifting block of this view
    tsplat_camera cam;
};

// Channels of a feature row as the compositing stages it (whole 16-column
// blocks of its tensor-core products): 16, 32 or 64.
__host__ __device__ inline int padded_channels(int C) { return C <= 16 ? 16 : (C <= 32 ? 32 : 64); }

struct BuildArgs {
    ViewDesc views[MAX_VIEWS];
    int n_views;
    int64_t total_pix;
    int C;
    int out_dtype;
    float4 *xyzo;
    float4 *cova;
    float2 *covb;
    void *feat;
    // FP32 stores: each feature row also as bf16 (hi, lo) with
    // hi = bf16(f), lo = bf16(f - hi), rows of 2 x padded_channels(C)
    // ([hi | lo], padding zero), the operands of the compositing's products
    void *fsplit;
    uint32_t *blk_cnt;  // [nblocks]
    uint32_t *blk_off;  // [nblocks]
    uint32_t *n_dev;    // N (output)
    int nblocks;
};
constexpr int BUILD_PIX_PER_BLOCK = 1024;
// Lifting blocks are laid out view by view (no block spans two views):
// sets each view's first block and returns the block count.
inline int64_t layout_build_blocks(BuildArgs &a) {
    int64_t nb = 0;
    for (int v = 0; v < a.n_views; ++v) {
        a.views[v].blk0 = nb;
        nb += ((int64_t)a.views[v].H * a.views[v].W + BUILD_PIX_PER_BLOCK - 1) / BUILD_PIX_PER_BLOCK;
    }
    return nb;
}
void launch_build(const BuildArgs &a, cudaStream_t s);

// Convert/copy caller arrays into a Gaussian store (fsplit: as in BuildArgs,
// or nullptr).
void launch_gaussians_set(int64_t n, const float *mean, const float *cov, const float *opac,
                          const void *feat, int feat_dtype_in, int C, int out_dtype, float4 *xyzo,
                          float4 *cova, float2 *covb, void *feat_out, void *fsplit, uint32_t *n_dev,
                          cudaStream_t s);
// The (hi, lo) rows of BuildArgs::fsplit from N x C FP32 features (N = *n_dev,
// n_cap >= N bounds the grid); padding columns written as zero.
void launch_feat_split(const float *feat, const uint32_t *n_dev, int64_t n_cap, int C, void *fsplit,
                       cudaStream_t s);
void launch_gaussians_get(const uint32_t *n_dev, int64_t cap, int C, int dtype, const float4 *xyzo,
                          const float4 *cova, const float2 *covb, const void *feat_in, float *mean,
                          float *cov, float *opac, void *feat_out, cudaStream_t s);

// ------------------------------------------------------------ view table
// One target view of a (possibly batched) render.  Its tiles occupy the
// global tile ids [tile_base, tile_base + tiles_x * tiles_y).
constexpr int MAX_BATCH = 8;
struct RenderView {
    tsplat_camera cam;
    uint32_t tile_base;
    int32_t tiles_x, tiles_y;
    int32_t width, height;
    int32_t pad_;
    float *out_feat;      // C x H x W
    float *out_alpha;     // H x W, may be NULL
    float *out_T;         // H x W, may be NULL
    uint32_t *out_last;   // H x W, may be NULL
};
// The table travels by value as a parameter of the first kernel of a render,
// which copies it to device memory for the kernels after it.
struct ViewBatch {
    RenderView v[MAX_BATCH];
    int32_t n_views;
    uint32_t n_tiles_total;
};

// --------------------------------------------------------------- A2 project
struct ProjectOut {
    Header *hdr;        // [N]
    uint2 *rect;        // [N] packed tile rect
    uint32_t *ntiles;   // [N]
    uint32_t *dkey;     // [N] depth key, CULLED_KEY when culled
    float *radius;      // [N]
    uint32_t *n_vis;    // [1] rendered Gaussians (pre-set to 0)
    uint32_t *tmask;    // [N] kept-tile masks (written with TSPLAT_RENDER_TIGHT)
    uint32_t *tile_cnt; // [tiles] pairs per tile (zeroed by the launcher, counted by the kernel)
};
// Rects of at most this many tiles are tested tile by tile in tight binning.
constexpr int TIGHT_MAX_TILES = 32;
// Instances: view v's copy of Gaussian g is instance v * N + g, N = *n_dev
// (n_cap >= N bounds the grid).  Also writes the view table to views_dev.
void launch_project(const float4 *xyzo, const float4 *cova, const float2 *covb,
                    const uint32_t *n_dev, int64_t n_cap, const ViewBatch &vb, RenderView *views_dev,
                    const tsplat_render_params &par, const ProjectOut &o, cudaStream_t s,
                    bool table_on_device = false);
// Same outputs from already projected 2D Gaussians (tsplat_rasterize, one view).
void launch_prepare_2d(int64_t n, const float *mean2d, const float *conic, const float *opac,
                       const float *depth, const int32_t *radius, const tsplat_render_params &par,
                       const ViewBatch &vb, RenderView *views_dev, const ProjectOut &o, cudaStream_t s);

// ------------------------------------------------------ A3..A6 bins
// The (Gaussian, tile) pairs of a render in (tile, depth key, instance id)
// order, and each tile's [first, last) range, through tile buckets (see
// k_bin.cu).  Instances: view v's copy of Gaussian g is instance v N + g.
struct BinArgs {
    const uint32_t *n_inst;      // instances (device)
    const uint32_t *n_stride;    // N (device)
    int64_t inst_cap;            // bound of the instance count (grid sizing)
    const uint32_t *ntiles;      // [inst] kept tiles per instance (0: culled)
    const uint2 *rect;           // [inst] packed tile rects
    const uint32_t *tmask;       // [inst] tight-binning masks, or nullptr
    const uint32_t *dkey;        // [inst] depth keys
    const RenderView *views;     // device view table
    int n_views;
    uint32_t n_slots;            // tile slots of the launch (>= the views' tiles)
    uint32_t *tile_cnt;          // [n_slots] per-tile pair counts
    uint32_t *cursor;            // [n_slots] fill cursors
    uint2 *ranges;               // [n_slots] output
    uint32_t *p_dev;             // P (written by the scan)
    uint32_t *p_eff;             // P, or 0 when the pairs do not fit (written by the fill)
    int64_t p_cap;               // pair buffer capacity
    uint32_t *bk_key, *bk_id;    // [p_cap] buckets: depth keys, instance ids
    uint32_t *tmp_key, *tmp_id;  // [p_cap] scratch of buckets too large for shared memory
    uint32_t *ids_out;           // [p_cap] instance ids in (tile, depth, id) order
    const uint32_t *tile_order;  // [n_slots] order the sort takes the tiles in
    uint32_t *tile_order_out;    // the same array, written by the scan
    uint4 *tile_info_out;        // [n_slots] per position of that order: (tile, first, end, 0)
    uint32_t *tile_ctr;          // persistent-sort tile counter
    uint32_t *status;            // TSPLAT_ERR_CAPACITY when P > p_cap
    int sort_wide;               // bucket sort with twelve-warp blocks (buckets near the shared-memory size)
};
// Ranges, fill cursors and P from the per-tile counts the projection made.
void launch_bin_scan(const BinArgs &a, cudaStream_t s);
// Buckets filled with (depth key, id); P > p_cap: nothing written, empty ranges.
void launch_bin_fill(const BinArgs &a, cudaStream_t s);
// Each bucket sorted by (depth key, id) into ids_out (tiles in tile_order).
void launch_bin_sort(const BinArgs &a, cudaStream_t s);
// One-time kernel attributes of the bucket sort (called outside any stream
// capture, when a context is created); returns its grid.
int bin_sort_setup();

// ------------------------------------------------------------ A7 composite
struct CompositeArgs {
    const uint2 *ranges;       // per global tile
    const uint32_t *ids;       // sorted pairs: instance ids
    const Header *hdr;         // per instance
    const void *feat;          // per Gaussian (instance % N)
    const void *fsplit;        // FP32 features: their (hi, lo) bf16 rows (see BuildArgs)
    const uint32_t *n_stride;  // N (device)
    int C;
    int feat_dtype;
    const RenderView *views;   // device view table
    int n_views;
    uint32_t n_tiles_total;
    float alpha_max, alpha_min, t_min;
    float log2_alpha_min;  // blend test: log2(o) + q log2(e) >= log2(alpha_min)
    uint32_t *status;      // TSPLAT_ERR_TIMEOUT if a bounded wait expired
    uint32_t *tile_counter;  // next tile to hand out (0 at launch)
    int save;                // record T_final and the last blended index (backward)
    const uint4 *tile_info;  // per ticket (longest lists first): (tile, first, end, 0)
};
void launch_composite(const CompositeArgs &a, cudaStream_t s);

// ------------------------------------------------------------- A8 backward
struct BackwardArgs {
    const uint2 *ranges;
    const uint32_t *ids;
    const Header *hdr;
    const void *feat;
    int C;
    int feat_dtype;
    int W, H, tiles_x, tiles_y;
    float alpha_max, alpha_min;
    float log2_alpha_min;
    const float *T_final;
    const uint32_t *last;
    const float *dF;
    const float *dA;
    float *d_mean2d;
    float *d_conic;
    float *d_opac;
    float *d_feat;
    uint32_t *unit_counter;  // next (tile, warp block) unit to hand out (0 at launch)
    const uint32_t *tile_order;  // the forward's tile order (longest lists first), or NULL
    const void *fsplit;          // FP32 features: their (hi, lo) bf16 rows, as the forward read them
};
void launch_backward(const BackwardArgs &a, cudaStream_t s);

// every launcher reports its launches here (tsplat_launch_count)
void note_launches(int n);

// Device arrays of a Gaussian store (for entry points outside api.cu).
struct GaussianStore {
    int64_t cap;
    int C, dtype;
    float4 *xyzo;
    float4 *cova;
    float2 *covb;
    void *feat;
    void *fsplit;  // FP32 stores: (hi, lo) rows (see BuildArgs), else nullptr
    uint32_t *n_dev;
};
void gaussians_store(tsplat_gaussians *g, GaussianStore &out, cudaStream_t writer);
// Read-only view of the store; *last_writer = the stream that last wrote it.
void gaussians_peek(const tsplat_gaussians *g, GaussianStore &out, cudaStream_t *last_writer);
// Record the thread-local message returned by tsplat_last_error; returns st.
tsplat_status record_error(tsplat_status st, const char *msg);

// Serving support: size a context for batched renders (instances, pairs,
// tiles over all views); its device view table; its pair capacity and
// status word.
tsplat_status ctx_reserve_batch(tsplat_ctx *c, int64_t instances, int64_t pairs, int64_t tiles);
RenderView *ctx_view_table(tsplat_ctx *c);
int64_t ctx_pair_capacity(const tsplat_ctx *c);
uint32_t *ctx_status_word(tsplat_ctx *c);  // device word written by the kernels of a render
uint32_t *ctx_pairs_word(tsplat_ctx *c);   // device word: the last render's pair count P (all its views)
// tsplat_render_batch; with table_on_device the projection reads the view
// table from ctx_view_table(ctx), written there by the caller before the
// launch (so that a captured graph can be replayed for other views).
tsplat_status render_batch_impl(const tsplat_gaussians *g, const tsplat_camera *cams, int32_t n_views,
                                const tsplat_render_params *params, float *const *out_feat,
                                float *const *out_alpha, tsplat_ctx *ctx, void *stream, bool table_on_device);
// The view table of a batch: views laid out in order, tile ids concatenated.
void make_view_batch(const tsplat_camera *cams, int32_t n_views, float *const *out_feat, float *const *out_alpha,
                     ViewBatch &vb);

// Adjoint of the projection (FP32, per Gaussian): d_mean3d (N x 3) and
// d_cov3d (N x 6) from d_mean2d (N x 2) and d_conic (N x 3, raw conic).
void launch_project_backward(const float4 *xyzo, const float4 *cova, const float2 *covb, const uint32_t *n_dev,
                             int64_t n_cap, const tsplat_camera &cam, const tsplat_render_params &par,
                             const float *d_mean2d, const float *d_conic, float *d_mean3d, float *d_cov3d,
                             cudaStream_t s);

// Adjoint of the lifting: per source pixel gradients of the maps.
struct SrcGrads {
    float *depth;    // H x W
    float *scale;    // H x W x 3
    float *quat;     // H x W x 4, or NULL
    float *opacity;  // H x W
    float *feat;     // H x W x C
};
struct LiftBwdArgs {
    BuildArgs b;  // views, blk_cnt / blk_off scratch, n_dev
    const float *d_mean;
    const float *d_cov;
    const float *d_opac;
    const float *d_feat;
    SrcGrads g[MAX_VIEWS];
};
void launch_build_backward(const LiftBwdArgs &a, cudaStream_t s);

// Point z-buffer of the Gaussian means into `cam`: keys = W*H scratch words,
// depth / id = W*H outputs (id may be NULL).
void launch_zbuffer(const float4 *xyzo, const uint32_t *n_dev, int64_t n_cap, const tsplat_camera &cam,
                    unsigned long long *keys, float *depth, int32_t *id, cudaStream_t s);

// small utilities
void launch_fill_u32(uint32_t *p, uint32_t v, int64_t n, cudaStream_t s);
void launch_scale_u32(const uint32_t *src, uint32_t k, uint32_t *dst, cudaStream_t s);  // *dst = *src * k
void launch_zero_f32_n(float *p, const uint32_t *n_dev, int mult, int64_t n_cap, cudaStream_t s);  // p[0 .. n*mult)
void launch_export_rect(const uint2 *rect, const uint32_t *n_dev, int64_t n_cap, int32_t *dst, cudaStream_t s);
void launch_export_header(const Header *hdr, const uint32_t *n_dev, int64_t n_cap, int what, void *dst,
                          cudaStream_t s);

}  // namespace tsp
