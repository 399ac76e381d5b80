// Host-side launchers of libtsplat's kernels (internal, C++).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/tsplat.h"

namespace tsp {

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
    int H, W;
    int64_t pix_off;  // first global pixel index of this view
    tsplat_camera cam;
};

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
    uint32_t *blk_cnt;  // [nblocks]
    uint32_t *blk_off;  // [nblocks]
    uint32_t *n_dev;    // N (output)
    int nblocks;
};
constexpr int BUILD_PIX_PER_BLOCK = 4096;
void launch_build(const BuildArgs &a, cudaStream_t s);

// Convert/copy caller arrays into a Gaussian store.
void launch_gaussians_set(int64_t n, const float *mean, const float *cov, const float *opac,
                          const void *feat, int feat_dtype_in, int C, int out_dtype, float4 *xyzo,
                          float4 *cova, float2 *covb, void *feat_out, uint32_t *n_dev, cudaStream_t s);
void launch_gaussians_get(const uint32_t *n_dev, int64_t cap, int C, int dtype, const float4 *xyzo,
                          const float4 *cova, const float2 *covb, const void *feat_in, float *mean,
                          float *cov, float *opac, void *feat_out, cudaStream_t s);

// --------------------------------------------------------------- A2 project
struct ProjectOut {
    Header *hdr;        // [N]
    uint2 *rect;        // [N] packed tile rect
    uint32_t *ntiles;   // [N]
    uint32_t *dkey;     // [N] depth key, CULLED_KEY when culled
    float *radius;      // [N]
    uint32_t *kminmax;  // [2] min / max depth key of rendered Gaussians (pre-set to ~0u / 0)
    uint32_t *n_vis;    // [1] rendered Gaussians (pre-set to 0)
};
void launch_project(const float4 *xyzo, const float4 *cova, const float2 *covb,
                    const uint32_t *n_dev, int64_t n_cap, const tsplat_camera &cam,
                    const tsplat_render_params &par, int tiles_x, int tiles_y,
                    const ProjectOut &o, cudaStream_t s);
// Same outputs from already projected 2D Gaussians (tsplat_rasterize).
void launch_prepare_2d(int64_t n, const float *mean2d, const float *conic, const float *opac,
                       const float *depth, const int32_t *radius, const tsplat_render_params &par,
                       int tiles_x, int tiles_y, const ProjectOut &o, cudaStream_t s);

// ------------------------------------------------------ A3..A6 sort / bins
constexpr int RS_THREADS = 256;
constexpr int RS_ITEMS = 16;
constexpr int RS_TILE = RS_THREADS * RS_ITEMS;  // keys per radix block

// Stable LSD radix sort of (u32 key, u32 value) pairs, 8-bit digits.
// Pass p reads pass p-1's output (pass 0 reads keys_in / vals_in, vals_in
// NULL meaning 0..n-1, and maps key k to k - *kmin, CULLED_KEY to 0, when
// kmin is given) and writes keys[p & 1] / vals[p & 1].  The number of
// passes is *npass_dev when given, else npass_host; passes beyond it do
// nothing, so the result lives in buffer (npass-1) & 1, or is the input
// when npass is 0.
struct RadixSort {
    const uint32_t *keys_in;
    const uint32_t *vals_in;
    uint32_t *keys[2];
    uint32_t *vals[2];
    const uint32_t *n_dev;
    const uint32_t *npass_dev;
    int npass_host;
    const uint32_t *kmin;
    uint32_t *hist;    // [256 * nblocks]
    uint32_t *totals;  // [4 * 256], zeroed by the launcher
    int nblocks;       // ceil(n_cap / RS_TILE)
};
void launch_radix_sort(const RadixSort &rs, int max_passes, cudaStream_t s);
void launch_depth_npass(const uint32_t *kminmax, uint32_t *npass, cudaStream_t s);

// Where a sort left its values: buffer (npass - 1) & 1, or the input.
struct SortedVals {
    const uint32_t *vals_in;  // NULL = identity
    const uint32_t *vals[2];
    const uint32_t *npass_dev;
    int npass_host;
};

// A3/A4: exclusive scan of n_tiles in depth order and emission of
// (tile, Gaussian id) pairs.  Two launches: reduce (+ total P), then
// scan + emit.  P_cap bounds the emission; overflow sets TSPLAT_ERR_CAPACITY.
struct EmitArgs {
    SortedVals order;          // depth order (values = Gaussian ids)
    const uint32_t *n_dev;
    int64_t n_cap;
    const uint32_t *ntiles;
    const uint2 *rect;
    int tiles_x;
    uint32_t tile_base;        // added to tile ids (batched views)
    uint32_t *blk_sum;         // [nblocks]
    uint32_t *p_dev;           // total pairs (output)
    uint32_t *pair_tile;       // [P_cap]
    uint32_t *pair_id;         // [P_cap]
    int64_t p_cap;
    uint32_t *status;
};
void launch_emit_count(const EmitArgs &a, cudaStream_t s);
void launch_emit_write(const EmitArgs &a, cudaStream_t s);

// A6: per-tile [first, last) of the tile-sorted pairs (ranges zeroed first).
void launch_ranges(const uint32_t *tiles_sorted, const uint32_t *p_dev, int64_t p_cap, uint2 *ranges,
                   int n_tiles, cudaStream_t s);

// ------------------------------------------------------------ A7 composite
struct CompositeArgs {
    const uint2 *ranges;
    const uint32_t *ids;
    const Header *hdr;
    const void *feat;
    int C;
    int feat_dtype;
    int W, H, tiles_x, tiles_y;
    float alpha_max, alpha_min, t_min;
    float log2_alpha_min;  // blend test: log2(o) + q log2(e) >= log2(alpha_min)
    uint32_t *status;      // TSPLAT_ERR_TIMEOUT if a bounded wait expired
    uint32_t *tile_counter;  // next tile to hand out (0 at launch)
    float *out_feat;
    float *out_alpha;
    float *out_T;        // may be NULL
    uint32_t *out_last;  // may be NULL
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
    uint32_t *n_dev;
};
void gaussians_store(tsplat_gaussians *g, GaussianStore &out, cudaStream_t writer);
// Record the thread-local message returned by tsplat_last_error; returns st.
tsplat_status record_error(tsplat_status st, const char *msg);

// small utilities
void launch_fill_u32(uint32_t *p, uint32_t v, int64_t n, cudaStream_t s);
// *dst = *src if it fits in cap, else 0 (an overflowing render emits no pairs)
void launch_pairs_effective(const uint32_t *src, uint32_t cap, uint32_t *dst, cudaStream_t s);
void launch_zero_f32_n(float *p, const uint32_t *n_dev, int mult, int64_t n_cap, cudaStream_t s);  // p[0 .. n*mult)
void launch_export_rect(const uint2 *rect, const uint32_t *n_dev, int64_t n_cap, int32_t *dst, cudaStream_t s);
void launch_export_header(const Header *hdr, const uint32_t *n_dev, int64_t n_cap, int what, void *dst,
                          cudaStream_t s);

}  // namespace tsp
