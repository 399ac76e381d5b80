// A2: EWA projection of 3D Gaussians into the target camera (the cited
// 3DGS rasterizer's preprocessing, Tele-Aloha Sec. 4.2).
//
// Every quantity that decides an integer -- visibility, radius, tile rect,
// depth key -- is evaluated in single precision one correctly rounded
// operation at a time (__f*_rn), in a fixed order, so that an independent
// implementation following the same order obtains the same bits.
#include <math.h>
#include <string.h>

#include <algorithm>

#include "bins.cuh"
#include "common.cuh"
#include "internal.h"

namespace tsp {

namespace {

// Half extents of the box around mean2d outside which alpha < alpha_min:
// o e^q >= alpha_min  <=>  d^T Q d <= kappa = 2 ln(o / alpha_min), whose
// bounding box has half widths sqrt(kappa Q^-1_00), sqrt(kappa Q^-1_11).
// Padded by 1% + 0.01 px so that the kernel's own rounding never reaches
// it; unbounded when Q is too ill-conditioned to evaluate safely.
__device__ __forceinline__ void cull_extents(float a, float b, float c, float o, float alpha_min,
                                             float &ex, float &ey) {
    if (!(o >= alpha_min)) {  // alpha <= o < alpha_min everywhere (or NaN)
        ex = ey = -INFINITY;
        return;
    }
    const float kappa = 2.0f * logf(o / alpha_min);
    const float detq = a * c - b * b;
    if (!(detq > 1e-4f * a * c) || !isfinite(detq)) {
        ex = ey = INFINITY;
        return;
    }
    ex = sqrtf(kappa * c / detq) * 1.01f + 0.01f;
    ey = sqrtf(kappa * a / detq) * 1.01f + 0.01f;
    if (!isfinite(ex) || !isfinite(ey)) ex = ey = INFINITY;
}

// floor(v) clamped to [0, hi] and converted (v may be +-inf)
__device__ __forceinline__ int clamp_floor(float v, int hi) {
    return (int)fminf((float)hi, fmaxf(0.0f, floorf(v)));
}

__device__ __forceinline__ void write_culled(const ProjectOut &o, uint64_t i) {
    o.hdr[i].h0 = make_float4(0.f, 0.f, 0.f, 0.f);
    o.hdr[i].h1 = make_float4(0.f, 0.f, -INFINITY, -INFINITY);
    o.rect[i] = make_uint2(0u, 0u);
    o.ntiles[i] = 0u;
    o.dkey[i] = CULLED_KEY;
    o.radius[i] = 0.0f;
}

// Count of rendered Gaussians, reduced per block before one atomic.
// Called by every thread of a 256-thread block.
__device__ __forceinline__ void account_n(const ProjectOut &o, uint32_t tn) {
    __shared__ uint32_t s_n[8];
    const uint32_t nv = __reduce_add_sync(0xffffffffu, tn);
    const int warp = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0) s_n[warp] = nv;
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t bn = 0;
        for (int w = 0; w < 8; ++w) bn += s_n[w];
        if (bn) atomicAdd(o.n_vis, bn);
    }
}

// Tile rect from mean2d and radius, as the cited rasterizer defines it.
__device__ __forceinline__ int tile_rect(float mx, float my, float r, int tiles_x, int tiles_y, int &x0,
                                         int &y0, int &x1, int &y1) {
    // v / 16 == v * 0.0625 exactly (power-of-two scaling)
    x0 = clamp_floor(fmul(fsub(mx, r), 0.0625f), tiles_x);
    x1 = clamp_floor(fmul(fadd(fadd(mx, r), 15.0f), 0.0625f), tiles_x);
    y0 = clamp_floor(fmul(fsub(my, r), 0.0625f), tiles_y);
    y1 = clamp_floor(fmul(fadd(fadd(my, r), 15.0f), 0.0625f), tiles_y);
    return (x1 - x0) * (y1 - y0);
}

// ---- tight binning (TSPLAT_RENDER_TIGHT) --------------------------------
// Single precision, one rounding per operation, in a fixed order, so that
// an independent implementation of the same steps keeps the same tiles.

// ln x for finite x >= 1: x = 2^e m with m in [sqrt(1/2), sqrt(2)),
// ln x = e ln 2 + 2 atanh(t), t = (m - 1)/(m + 1), with atanh summed as its
// odd power series up to t^9 (|t| < 0.172: the rest is below 1e-9).
__device__ __forceinline__ float key_ln(float x) {
    const uint32_t u = __float_as_uint(x);
    int e = (int)((u >> 23) & 0xffu) - 127;
    float m = __uint_as_float((u & 0x7fffffu) | 0x3f800000u);
    if (m > 1.41421354f) {
        m = fmul(m, 0.5f);
        e += 1;
    }
    const float t = fdiv(fsub(m, 1.0f), fadd(m, 1.0f));
    const float t2 = fmul(t, t);
    float sr = 0.111111111f;
    sr = fadd(fmul(sr, t2), 0.142857143f);
    sr = fadd(fmul(sr, t2), 0.2f);
    sr = fadd(fmul(sr, t2), 0.333333333f);
    sr = fadd(fmul(sr, t2), 1.0f);
    return fadd(fmul(__int2float_rn(e), 0.693147182f), fmul(2.0f, fmul(t, sr)));
}

// Q = a dx^2 + 2b dx dy + c dy^2 as dx (a dx + 2b dy) + (c dy) dy
__device__ __forceinline__ float tight_q(float a, float b2, float c, float dx, float dy) {
    return fadd(fmul(dx, fadd(fmul(a, dx), fmul(b2, dy))), fmul(fmul(c, dy), dy));
}

// Smallest Q over [dx0, dx1] x [dy0, dy1] when the mean lies outside it:
// the least of the four edge minima (each edge: the parabola's clamped
// vertex).  (With the mean inside, the smallest Q is 0.)
__device__ __forceinline__ float tight_qmin_outside(float a, float b2, float c, float ra, float rc, float dx0,
                                                    float dx1, float dy0, float dy1) {
    float q = INFINITY;
    q = fminf(q, tight_q(a, b2, c, fminf(dx1, fmaxf(dx0, -fmul(ra, dy0))), dy0));
    q = fminf(q, tight_q(a, b2, c, fminf(dx1, fmaxf(dx0, -fmul(ra, dy1))), dy1));
    q = fminf(q, tight_q(a, b2, c, dx0, fminf(dy1, fmaxf(dy0, -fmul(rc, dx0)))));
    q = fminf(q, tight_q(a, b2, c, dx1, fminf(dy1, fmaxf(dy0, -fmul(rc, dx1)))));
    return q;
}

// Kept tiles of the rect [x0, x1) x [y0, y1) (at most 32 tiles): bit
// (ty - y0) * (x1 - x0) + (tx - x0) is set when the tile's pixel-centre
// rectangle (clipped to the W x H image) reaches Q <= 2 ln(o / alpha_min)
// (1 + 2^-10) + 2^-8.  Conic (a, b, c) of the inverse 2D covariance.
__device__ uint32_t tight_mask(float mx, float my, float a, float b, float c, float o, float alpha_min, int x0,
                               int y0, int x1, int y1, int W, int H) {
    const float ratio = fdiv(o, alpha_min);
    if (!(ratio >= 1.0f)) return 0u;
    const int w = x1 - x0;
    if (w == 1 && y1 - y0 == 1) {  // one tile holding the mean: kept (Q = 0 < threshold)
        const float dx0 = fsub((float)(16 * x0), mx), dx1 = fsub((float)min(16 * x0 + 15, W - 1), mx);
        const float dy0 = fsub((float)(16 * y0), my), dy1 = fsub((float)min(16 * y0 + 15, H - 1), my);
        if (dx0 <= 0.0f && dx1 >= 0.0f && dy0 <= 0.0f && dy1 >= 0.0f) return 1u;
    }
    const float kappa = fmul(2.0f, key_ln(ratio));
    const float thr = fadd(fmul(kappa, 1.0009765625f), 0.00390625f);
    const float b2 = fmul(2.0f, b), ra = fdiv(b, a), rc = fdiv(b, c);
    uint32_t m = 0u;
    for (int ty = y0; ty < y1; ++ty) {
        const float dy0 = fsub((float)(16 * ty), my), dy1 = fsub((float)min(16 * ty + 15, H - 1), my);
        for (int tx = x0; tx < x1; ++tx) {
            const float dx0 = fsub((float)(16 * tx), mx), dx1 = fsub((float)min(16 * tx + 15, W - 1), mx);
            if ((dx0 <= 0.0f && dx1 >= 0.0f && dy0 <= 0.0f && dy1 >= 0.0f) ||
                tight_qmin_outside(a, b2, c, ra, rc, dx0, dx1, dy0, dy1) <= thr)
                m |= 1u << ((ty - y0) * w + (tx - x0));
        }
    }
    return m;
}

// Applies tight binning to a visible Gaussian's tile count: writes its mask
// and returns the tiles kept (0 culls).  Whole rects above 32 tiles.
__device__ __forceinline__ int tighten(const ProjectOut &o, uint64_t i, int nt, float mx, float my, float a,
                                       float b, float c, float op, float alpha_min, int x0, int y0, int x1, int y1,
                                       int W, int H, uint32_t &mask) {
    if (nt > TIGHT_MAX_TILES) {
        mask = 0xffffffffu;
        o.tmask[i] = mask;
        return nt;
    }
    mask = tight_mask(mx, my, a, b, c, op, alpha_min, x0, y0, x1, y1, W, H);
    o.tmask[i] = mask;
    return __popc(mask);
}

// Copy the view table to device memory for the kernels after this one.
__device__ __forceinline__ void publish_views(const ViewBatch &vb, RenderView *views_dev) {
    if (blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x < (unsigned)vb.n_views) views_dev[threadIdx.x] = vb.v[threadIdx.x];
}

// grid (gx, n_views): view blockIdx.y; blocks stride over the Gaussians gi
// (gx is at most a few waves, whatever the capacity); instance i = view * N + gi.
__global__ __launch_bounds__(256, 4) void k_project(const float4 *__restrict__ xyzo,
                                                 const float4 *__restrict__ cova,
                                                 const float2 *__restrict__ covb,
                                                 const uint32_t *n_dev,
                                                 const __grid_constant__ ViewBatch vb, RenderView *views_dev,
                                                 int table_on_device, tsplat_render_params par, ProjectOut o) {
    // the view table comes with the launch and is published for the later
    // kernels, or (graph replays) it is already in device memory
    if (!table_on_device) publish_views(vb, views_dev);
    const RenderView &view = table_on_device ? views_dev[blockIdx.y] : vb.v[blockIdx.y];
    const tsplat_camera &cam = view.cam;
    const int tiles_x = view.tiles_x, tiles_y = view.tiles_y;
    const uint64_t n = *n_dev;
    uint32_t tn = 0u;
    // warps stride over 32-Gaussian chunks (the tile count is warp-synchronous)
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t g0 = (uint64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31u); g0 < n; g0 += stride) {
    const uint64_t gi = g0 + (threadIdx.x & 31);
    const uint64_t i = (uint64_t)blockIdx.y * n + gi;
    bool vis = false;
    uint32_t key = CULLED_KEY;
    uint32_t cnt = 0;
    TileWalk tw;
    tw.clear();
    if (gi < n) {
    const float4 g = xyzo[gi];
    const float *R = cam.R;
    const float px = fadd(fadd(fadd(fmul(R[0], g.x), fmul(R[1], g.y)), fmul(R[2], g.z)), cam.t[0]);
    const float py = fadd(fadd(fadd(fmul(R[3], g.x), fmul(R[4], g.y)), fmul(R[5], g.z)), cam.t[1]);
    const float pz = fadd(fadd(fadd(fmul(R[6], g.x), fmul(R[7], g.y)), fmul(R[8], g.z)), cam.t[2]);
    vis = pz > cam.z_near && pz < cam.z_far;
    if (vis) {
        const float limx = fmul(par.frustum_clamp, fdiv(fmul(0.5f, (float)cam.width), cam.fx));
        const float limy = fmul(par.frustum_clamp, fdiv(fmul(0.5f, (float)cam.height), cam.fy));
        const float txz = fminf(limx, fmaxf(-limx, fdiv(px, pz)));
        const float tyz = fminf(limy, fmaxf(-limy, fdiv(py, pz)));
        const float tx = fmul(txz, pz), ty = fmul(tyz, pz);
        const float pz2 = fmul(pz, pz);
        const float j00 = fdiv(cam.fx, pz), j02 = -fdiv(fmul(cam.fx, tx), pz2);
        const float j11 = fdiv(cam.fy, pz), j12 = -fdiv(fmul(cam.fy, ty), pz2);
        float T0[3], T1[3];
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            T0[j] = fadd(fmul(j00, R[0 * 3 + j]), fmul(j02, R[2 * 3 + j]));
            T1[j] = fadd(fmul(j11, R[1 * 3 + j]), fmul(j12, R[2 * 3 + j]));
        }
        const float4 ca = cova[gi];
        const float2 cb = covb[gi];
        const float V[3][3] = {{ca.x, ca.y, ca.z}, {ca.y, ca.w, cb.x}, {ca.z, cb.x, cb.y}};
        float U0[3], U1[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            U0[k] = fadd(fadd(fmul(T0[0], V[0][k]), fmul(T0[1], V[1][k])), fmul(T0[2], V[2][k]));
            U1[k] = fadd(fadd(fmul(T1[0], V[0][k]), fmul(T1[1], V[1][k])), fmul(T1[2], V[2][k]));
        }
        const float s00 = fadd(fadd(fmul(U0[0], T0[0]), fmul(U0[1], T0[1])), fmul(U0[2], T0[2]));
        const float s01 = fadd(fadd(fmul(U0[0], T1[0]), fmul(U0[1], T1[1])), fmul(U0[2], T1[2]));
        const float s11 = fadd(fadd(fmul(U1[0], T1[0]), fmul(U1[1], T1[1])), fmul(U1[2], T1[2]));
        const float a = fadd(s00, par.lowpass), b = s01, c = fadd(s11, par.lowpass);
        const float det = fsub(fmul(a, c), fmul(b, b));
        if (!(det > 0.0f) || !isfinite(det)) {
            vis = false;
        } else {
            const float mid = fmul(0.5f, fadd(a, c));
            const float disc = fmaxf(0.1f, fsub(fmul(mid, mid), det));
            const float lam = fadd(mid, fsqrt(disc));
            const float r = ceilf(fmul(3.0f, fsqrt(lam)));
            const float mx = fadd(fdiv(fmul(cam.fx, px), pz), cam.cx);
            const float my = fadd(fdiv(fmul(cam.fy, py), pz), cam.cy);
            int x0, y0, x1, y1;
            int nt = tile_rect(mx, my, r, tiles_x, tiles_y, x0, y0, x1, y1);
            const float ca_ = fdiv(c, det), cb_ = -fdiv(b, det), cc_ = fdiv(a, det);
            uint32_t mask = 0xffffffffu;
            if (nt > 0 && (par.flags & TSPLAT_RENDER_TIGHT))
                nt = tighten(o, i, nt, mx, my, ca_, cb_, cc_, g.w, par.alpha_min, x0, y0, x1, y1, cam.width,
                             cam.height, mask);
            if (nt <= 0) {
                vis = false;
            } else {
                float ex, ey;
                cull_extents(ca_, cb_, cc_, g.w, par.alpha_min, ex, ey);
                o.hdr[i].h0 = make_float4(mx, my, -0.5f * ca_, -cb_);
                o.hdr[i].h1 = make_float4(-0.5f * cc_, log2f(g.w), ex, ey);
                o.rect[i] = pack_rect(x0, y0, x1, y1);
                o.ntiles[i] = (uint32_t)nt;
                key = __float_as_uint(pz);
                o.dkey[i] = key;
                o.radius[i] = r;
                cnt = (uint32_t)nt;
                tw.init(view.tile_base, tiles_x, x0, y0, x1, mask);
            }
        }
    }
    if (!vis) {
        write_culled(o, i);
    } else {
        ++tn;
    }
    }
    warp_count_tiles(tw, cnt, o.tile_cnt);
    }
    account_n(o, tn);
}

__global__ __launch_bounds__(256) void k_prepare_2d(uint64_t n, const float *__restrict__ mean2d,
                                                    const float *__restrict__ conic,
                                                    const float *__restrict__ opac,
                                                    const float *__restrict__ depth,
                                                    const int32_t *__restrict__ radius,
                                                    tsplat_render_params par,
                                                    const __grid_constant__ ViewBatch vb,
                                                    RenderView *views_dev, ProjectOut o) {
    publish_views(vb, views_dev);
    const int tiles_x = vb.v[0].tiles_x, tiles_y = vb.v[0].tiles_y;
    const uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const bool active = i < n;
    bool vis = false;
    uint32_t key = CULLED_KEY;
    uint32_t cnt = 0;
    TileWalk tw;
    tw.clear();
    if (active) {
    const int32_t ri = radius[i];
    const float z = depth[i];
    vis = ri > 0 && z > 0.0f;
    if (vis) {
        const float mx = mean2d[2 * i], my = mean2d[2 * i + 1];
        const float r = (float)ri;
        int x0, y0, x1, y1;
        int nt = tile_rect(mx, my, r, tiles_x, tiles_y, x0, y0, x1, y1);
        const float a = conic[3 * i], b = conic[3 * i + 1], c = conic[3 * i + 2];
        uint32_t mask = 0xffffffffu;
        if (nt > 0 && (par.flags & TSPLAT_RENDER_TIGHT))
            nt = tighten(o, i, nt, mx, my, a, b, c, opac[i], par.alpha_min, x0, y0, x1, y1, vb.v[0].cam.width,
                         vb.v[0].cam.height, mask);
        if (nt <= 0) {
            vis = false;
        } else {
            float ex, ey;
            cull_extents(a, b, c, opac[i], par.alpha_min, ex, ey);
            o.hdr[i].h0 = make_float4(mx, my, -0.5f * a, -b);
            o.hdr[i].h1 = make_float4(-0.5f * c, log2f(opac[i]), ex, ey);
            o.rect[i] = pack_rect(x0, y0, x1, y1);
            o.ntiles[i] = (uint32_t)nt;
            key = __float_as_uint(z);
            o.dkey[i] = key;
            o.radius[i] = r;
            cnt = (uint32_t)nt;
            tw.init(0u, tiles_x, x0, y0, x1, mask);
        }
    }
    if (!vis) write_culled(o, i);
    }
    warp_count_tiles(tw, cnt, o.tile_cnt);
    account_n(o, vis ? 1u : 0u);
}

// export of header fields: 2 = mean2d, 3 = conic
__global__ void k_export_header(const Header *hdr, const uint32_t *n_dev, int what, float *dst) {
    const uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= *n_dev) return;
    const Header h = hdr[i];
    if (what == TSPLAT_EXPORT_MEAN2D) {
        dst[2 * i] = h.h0.x;
        dst[2 * i + 1] = h.h0.y;
    } else {
        dst[3 * i] = -2.0f * h.h0.z;  // the record keeps (-a/2, -b, -c/2)
        dst[3 * i + 1] = -h.h0.w;
        dst[3 * i + 2] = -2.0f * h.h1.x;
    }
}

__global__ void k_export_rect(const uint2 *rect, const uint32_t *n_dev, int32_t *dst) {
    const uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= *n_dev) return;
    int x0, y0, x1, y1;
    unpack_rect(rect[i], x0, y0, x1, y1);
    dst[4 * i] = x0;
    dst[4 * i + 1] = y0;
    dst[4 * i + 2] = x1;
    dst[4 * i + 3] = y1;
}

}  // namespace

// Adjoint of the projection (Sec. 4.2, trained end to end): per Gaussian,
// dL/dmean and dL/dcov from dL/dmu and dL/d(conic) (raw conic (A, B, C) of
// q = -(A dx^2 + 2 B dx dy + C dy^2) / 2).  Chain: p = R x + t;
// mu = f p_xy / p_z + c; J from p with x/z and y/z clamped (no gradient
// through a clamped ratio); S = (J R) V (J R)^T + lowpass I; conic = S^-1.
__global__ __launch_bounds__(256) void k_project_backward(const float4 *__restrict__ xyzo,
                                                          const float4 *__restrict__ cova,
                                                          const float2 *__restrict__ covb, const uint32_t *n_dev,
                                                          const __grid_constant__ tsplat_camera cam,
                                                          tsplat_render_params par, const float *d_mu,
                                                          const float *d_conic, float *d_mean, float *d_cov) {
    const uint64_t n = *n_dev;
    const float *R = cam.R;
    const float limx = par.frustum_clamp * (0.5f * (float)cam.width / cam.fx);
    const float limy = par.frustum_clamp * (0.5f * (float)cam.height / cam.fy);
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
        float gp[3] = {0.0f, 0.0f, 0.0f};
        float gc[6] = {0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f};
        const float4 g = xyzo[i];
        const float px = R[0] * g.x + R[1] * g.y + R[2] * g.z + cam.t[0];
        const float py = R[3] * g.x + R[4] * g.y + R[5] * g.z + cam.t[1];
        const float z = R[6] * g.x + R[7] * g.y + R[8] * g.z + cam.t[2];
        if (z > 0.0f) {
            const float gmx = d_mu[2 * i], gmy = d_mu[2 * i + 1];
            const float iz = 1.0f / z, iz2 = iz * iz;
            gp[0] = cam.fx * iz * gmx;
            gp[1] = cam.fy * iz * gmy;
            gp[2] = -(cam.fx * px * gmx + cam.fy * py * gmy) * iz2;
            const float rx = px * iz, ry = py * iz;
            const bool inx = rx > -limx && rx < limx, iny = ry > -limy && ry < limy;
            const float txz = fminf(limx, fmaxf(-limx, rx)), tyz = fminf(limy, fmaxf(-limy, ry));
            const float J00 = cam.fx * iz, J02 = -cam.fx * txz * iz, J11 = cam.fy * iz, J12 = -cam.fy * tyz * iz;
            float T0[3], T1[3];
#pragma unroll
            for (int j = 0; j < 3; ++j) {
                T0[j] = J00 * R[0 * 3 + j] + J02 * R[2 * 3 + j];
                T1[j] = J11 * R[1 * 3 + j] + J12 * R[2 * 3 + j];
            }
            const float4 ca = cova[i];
            const float2 cb = covb[i];
            const float V[3][3] = {{ca.x, ca.y, ca.z}, {ca.y, ca.w, cb.x}, {ca.z, cb.x, cb.y}};
            float VT0[3], VT1[3];
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                VT0[k] = V[k][0] * T0[0] + V[k][1] * T0[1] + V[k][2] * T0[2];
                VT1[k] = V[k][0] * T1[0] + V[k][1] * T1[1] + V[k][2] * T1[2];
            }
            const float a = T0[0] * VT0[0] + T0[1] * VT0[1] + T0[2] * VT0[2] + par.lowpass;
            const float b = T0[0] * VT1[0] + T0[1] * VT1[1] + T0[2] * VT1[2];
            const float c = T1[0] * VT1[0] + T1[1] * VT1[1] + T1[2] * VT1[2] + par.lowpass;
            const float D = a * c - b * b;
            if (D > 0.0f && isfinite(D)) {
                const float gA = d_conic[3 * i], gB = d_conic[3 * i + 1], gC = d_conic[3 * i + 2];
                const float iD = 1.0f / D, iD2 = iD * iD;
                const float ga = -gA * c * c * iD2 + gB * b * c * iD2 + gC * (iD - a * c * iD2);
                const float gb = 2.0f * gA * b * c * iD2 - gB * (iD + 2.0f * b * b * iD2) + 2.0f * gC * a * b * iD2;
                const float gcc = gA * (iD - a * c * iD2) + gB * a * b * iD2 - gC * a * a * iD2;
                const int ii[6] = {0, 0, 0, 1, 1, 2}, jj[6] = {0, 1, 2, 1, 2, 2};
#pragma unroll
                for (int e = 0; e < 6; ++e) {
                    const int u = ii[e], v = jj[e];
                    float d00 = T0[u] * T0[v], d01 = T0[u] * T1[v], d11 = T1[u] * T1[v];
                    if (u != v) {
                        d00 += T0[v] * T0[u];
                        d01 += T0[v] * T1[u];
                        d11 += T1[v] * T1[u];
                    }
                    gc[e] = ga * d00 + gb * d01 + gcc * d11;
                }
                float gJ00 = 0.0f, gJ02 = 0.0f, gJ11 = 0.0f, gJ12 = 0.0f;
#pragma unroll
                for (int k = 0; k < 3; ++k) {
                    const float gt0 = 2.0f * ga * VT0[k] + gb * VT1[k];
                    const float gt1 = gb * VT0[k] + 2.0f * gcc * VT1[k];
                    gJ00 += gt0 * R[0 * 3 + k];
                    gJ02 += gt0 * R[2 * 3 + k];
                    gJ11 += gt1 * R[1 * 3 + k];
                    gJ12 += gt1 * R[2 * 3 + k];
                }
                gp[2] -= (cam.fx * gJ00 + cam.fy * gJ11) * iz2;
                if (inx) {
                    gp[0] -= cam.fx * iz2 * gJ02;
                    gp[2] += 2.0f * cam.fx * px * iz2 * iz * gJ02;
                } else {
                    gp[2] += cam.fx * txz * iz2 * gJ02;
                }
                if (iny) {
                    gp[1] -= cam.fy * iz2 * gJ12;
                    gp[2] += 2.0f * cam.fy * py * iz2 * iz * gJ12;
                } else {
                    gp[2] += cam.fy * tyz * iz2 * gJ12;
                }
            }
        }
#pragma unroll
        for (int k = 0; k < 3; ++k) d_mean[3 * i + k] = R[0 * 3 + k] * gp[0] + R[1 * 3 + k] * gp[1] + R[2 * 3 + k] * gp[2];
#pragma unroll
        for (int e = 0; e < 6; ++e) d_cov[6 * i + e] = gc[e];
    }
}

void launch_project_backward(const float4 *xyzo, const float4 *cova, const float2 *covb, const uint32_t *n_dev,
                             int64_t n_cap, const tsplat_camera &cam, const tsplat_render_params &par,
                             const float *d_mean2d, const float *d_conic, float *d_mean3d, float *d_cov3d,
                             cudaStream_t s) {
    if (n_cap <= 0) return;
    const int64_t blocks = std::min<int64_t>((n_cap + 255) / 256, 152 * 16);
    k_project_backward<<<(unsigned)blocks, 256, 0, s>>>(xyzo, cova, covb, n_dev, cam, par, d_mean2d, d_conic, d_mean3d,
                                                       d_cov3d);
    note_launches(1);
}

void launch_export_rect(const uint2 *rect, const uint32_t *n_dev, int64_t n_cap, int32_t *dst, cudaStream_t s) {
    if (n_cap <= 0) return;
    k_export_rect<<<(unsigned)((n_cap + 255) / 256), 256, 0, s>>>(rect, n_dev, dst);
    note_launches(1);
}

void launch_project(const float4 *xyzo, const float4 *cova, const float2 *covb, const uint32_t *n_dev,
                    int64_t n_cap, const ViewBatch &vb, RenderView *views_dev,
                    const tsplat_render_params &par, const ProjectOut &o, cudaStream_t s, bool table_on_device) {
    const int sms = sm_count();
    // about four waves of 256-thread blocks over all views
    const int64_t gx = std::max<int64_t>(1, std::min<int64_t>((n_cap + 255) / 256, (int64_t)sms * 32 / vb.n_views));
    const dim3 grid((unsigned)gx, (unsigned)vb.n_views);
    cudaMemsetAsync(o.tile_cnt, 0, sizeof(uint32_t) * std::max<uint32_t>(vb.n_tiles_total, 1u), s);
    k_project<<<grid, 256, 0, s>>>(xyzo, cova, covb, n_dev, vb, views_dev, table_on_device ? 1 : 0, par, o);
    note_launches(1);
}

void launch_prepare_2d(int64_t n, const float *mean2d, const float *conic, const float *opac,
                       const float *depth, const int32_t *radius, const tsplat_render_params &par,
                       const ViewBatch &vb, RenderView *views_dev, const ProjectOut &o, cudaStream_t s) {
    const unsigned blocks = (unsigned)std::max<int64_t>(1, (n + 255) / 256);
    cudaMemsetAsync(o.tile_cnt, 0, sizeof(uint32_t) * std::max<uint32_t>(vb.n_tiles_total, 1u), s);
    k_prepare_2d<<<blocks, 256, 0, s>>>((uint64_t)n, mean2d, conic, opac, depth, radius, par, vb, views_dev, o);
    note_launches(1);
}

void launch_export_header(const Header *hdr, const uint32_t *n_dev, int64_t n_cap, int what, void *dst,
                          cudaStream_t s) {
    if (n_cap <= 0) return;
    k_export_header<<<(unsigned)((n_cap + 255) / 256), 256, 0, s>>>(hdr, n_dev, what, (float *)dst);
    note_launches(1);
}

}  // namespace tsp
