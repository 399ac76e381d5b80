// A1: lifting of foreground source pixels to 3D Gaussians (Tele-Aloha
// Sec. 4.2: positions unprojected from the depth maps with the camera
// parameters; scale, opacity and latent feature from the encoder maps).
//
// Three launches: per-block foreground counts, a scan of those counts, and
// the lift itself, which numbers Gaussians in (view, row, column) order of
// the foreground pixels.  Single precision, one rounding per operation in a
// fixed order (the oracle's key mode follows the same order).
#include <algorithm>

#include "common.cuh"
#include "internal.h"
#include "ptx.cuh"

namespace tsp {

namespace {

constexpr int BT = 256;                             // threads per block
constexpr int BI = BUILD_PIX_PER_BLOCK / BT;        // pixels per thread (4)
static_assert(BI == 4, "k_build_count reads the block's pixels four at a time");
constexpr uint32_t FULL = 0xffffffffu;

// Blocks are laid out view by view: view v owns blocks [blk0, blk0 +
// ceil(H W / 1024)), and block b of it covers the view's pixels
// [(b - blk0) * 1024, (b - blk0 + 1) * 1024).
__device__ __forceinline__ int view_of_block(const BuildArgs &a, int64_t b) {
    int v = 0;
    for (int k = 1; k < a.n_views; ++k)
        if (b >= a.views[k].blk0) v = k;
    return v;
}

__device__ __forceinline__ bool is_fg(const ViewDesc &vd, int64_t p) {
    if (p >= (int64_t)vd.H * vd.W) return false;
    return vd.mask == nullptr || vd.mask[p] != 0;
}

template <int NW>
__device__ __forceinline__ uint32_t block_excl_scan(uint32_t v, uint32_t *sw, uint32_t &total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(FULL, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) sw[warp] = x;
    __syncthreads();
    if (warp == 0) {
        uint32_t w = lane < NW ? sw[lane] : 0u;
#pragma unroll
        for (int o = 1; o < NW; o <<= 1) {
            uint32_t y = __shfl_up_sync(FULL, w, o);
            if (lane >= o) w += y;
        }
        if (lane < NW) sw[lane] = w;
    }
    __syncthreads();
    total = sw[NW - 1];
    const uint32_t pre = warp ? sw[warp - 1] : 0u;
    __syncthreads();
    return pre + x - v;
}

__device__ __forceinline__ uint32_t lanemask_lt() {
    uint32_t m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

// Pixels of a block are visited in 4 rounds of 256 consecutive pixels
// (thread t takes pixel round * 256 + t).
__global__ __launch_bounds__(BT) void k_build_count(BuildArgs a) {
    // the block's 1024 pixels, 4 consecutive ones per thread (one 32-bit mask
    // load where aligned); the same pixels the lift visits in its 4 rounds
    __shared__ uint32_t sw[BT / 32];
    const ViewDesc &vd = a.views[view_of_block(a, blockIdx.x)];
    const int64_t hw = (int64_t)vd.H * vd.W;
    const int64_t p0 = ((int64_t)blockIdx.x - vd.blk0) * BUILD_PIX_PER_BLOCK + 4 * (int64_t)threadIdx.x;
    uint32_t c = 0;
    if (!vd.mask) {
        c = (uint32_t)max((int64_t)0, min((int64_t)4, hw - p0));
    } else if (p0 + 3 < hw && (reinterpret_cast<uintptr_t>(vd.mask + p0) & 3u) == 0) {
        const uint32_t w = *reinterpret_cast<const uint32_t *>(vd.mask + p0);
        c = (uint32_t)((w & 0xffu) != 0) + (uint32_t)((w & 0xff00u) != 0) + (uint32_t)((w & 0xff0000u) != 0) +
            (uint32_t)((w >> 24) != 0);
    } else {
        for (int k = 0; k < 4; ++k) c += (p0 + k < hw && vd.mask[p0 + k] != 0) ? 1u : 0u;
    }
    c = __reduce_add_sync(FULL, c);
    if ((threadIdx.x & 31) == 0) sw[threadIdx.x >> 5] = c;
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t t = 0;
        for (int w = 0; w < BT / 32; ++w) t += sw[w];
        a.blk_cnt[blockIdx.x] = t;
    }
}

__global__ __launch_bounds__(1024) void k_build_scan(BuildArgs a) {
    __shared__ uint32_t sw[32];
    const int nb = a.nblocks;
    const int per = (nb + 1023) / 1024;
    const int b0 = min((int)threadIdx.x * per, nb), b1 = min(b0 + per, nb);
    uint32_t local = 0;
    for (int b = b0; b < b1; ++b) local += a.blk_cnt[b];
    uint32_t tot;
    uint32_t run = block_excl_scan<32>(local, sw, tot);
    for (int b = b0; b < b1; ++b) {
        a.blk_off[b] = run;
        run += a.blk_cnt[b];
    }
    if (threadIdx.x == 0) *a.n_dev = tot;
}

__device__ __forceinline__ void copy_feat(const void *src, int src_dtype, int64_t src_row, void *dst,
                                          int dst_dtype, int64_t dst_row, int C) {
    if (src_dtype == TSPLAT_F32) {
        const float *s = (const float *)src + src_row * C;
        if (dst_dtype == TSPLAT_F32) {
            float *d = (float *)dst + dst_row * C;
            for (int c = 0; c < C; ++c) d[c] = s[c];
        } else {
            __nv_bfloat16 *d = (__nv_bfloat16 *)dst + dst_row * C;
            for (int c = 0; c < C; ++c) d[c] = __float2bfloat16_rn(s[c]);
        }
    } else {
        const __nv_bfloat16 *s = (const __nv_bfloat16 *)src + src_row * C;
        if (dst_dtype == TSPLAT_F32) {
            float *d = (float *)dst + dst_row * C;
            for (int c = 0; c < C; ++c) d[c] = __bfloat162float(s[c]);
        } else {
            __nv_bfloat16 *d = (__nv_bfloat16 *)dst + dst_row * C;
            for (int c = 0; c < C; ++c) d[c] = s[c];
        }
    }
}

// The (hi, lo) bf16 parts of FP32 features (hi = bf16(v), lo = bf16(v - hi),
// both rounded to nearest even): four at a time, and one at a time.
__device__ __forceinline__ void split4(const float (&v)[4], uint2 &hi, uint2 &lo) {
    hi.x = pack_bf16x2(v[0], v[1]);
    hi.y = pack_bf16x2(v[2], v[3]);
    lo.x = pack_bf16x2(v[0] - bf16_lo_f(hi.x), v[1] - bf16_hi_f(hi.x));
    lo.y = pack_bf16x2(v[2] - bf16_lo_f(hi.y), v[3] - bf16_hi_f(hi.y));
}
__device__ __forceinline__ void split1(float v, int C, int64_t row, int c, void *fsplit) {
    const int cp = padded_channels(C);
    __nv_bfloat16 *r = (__nv_bfloat16 *)fsplit + row * 2 * cp;
    const __nv_bfloat16 h = __float2bfloat16_rn(v);
    r[c] = h;
    r[cp + c] = __float2bfloat16_rn(v - __bfloat162float(h));
}

// Lift pixel p (row v, column u) of view vd into Gaussian `id`; its maps
// are read at index k (k = p, or the pixel's foreground rank for compact maps).
__device__ __forceinline__ void lift_one(const BuildArgs &a, const ViewDesc &vd, int64_t p, int64_t k, int64_t id) {
    const int u = (int)(p % vd.W), v = (int)(p / vd.W);
    const tsplat_camera &cam = vd.cam;
    const float *R = cam.R;
    const float z = vd.depth[k];
    const float rx = fdiv(fsub((float)u, cam.cx), cam.fx);
    const float ry = fdiv(fsub((float)v, cam.cy), cam.fy);
    const float d0 = fsub(fmul(rx, z), cam.t[0]);
    const float d1 = fsub(fmul(ry, z), cam.t[1]);
    const float d2 = fsub(z, cam.t[2]);
    float m[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) m[i] = fadd(fadd(fmul(R[0 * 3 + i], d0), fmul(R[1 * 3 + i], d1)), fmul(R[2 * 3 + i], d2));

    float w = 1.0f, x = 0.0f, y = 0.0f, zq = 0.0f;
    if (vd.quat) {
        const float4 q = reinterpret_cast<const float4 *>(vd.quat)[k];
        w = q.x; x = q.y; y = q.z; zq = q.w;
    }
    const float nn = fadd(fadd(fadd(fmul(w, w), fmul(x, x)), fmul(y, y)), fmul(zq, zq));
    const float nq = fsqrt(nn);
    w = fdiv(w, nq); x = fdiv(x, nq); y = fdiv(y, nq); zq = fdiv(zq, nq);
    float Rq[3][3];
    Rq[0][0] = fsub(1.0f, fmul(2.0f, fadd(fmul(y, y), fmul(zq, zq))));
    Rq[0][1] = fmul(2.0f, fsub(fmul(x, y), fmul(w, zq)));
    Rq[0][2] = fmul(2.0f, fadd(fmul(x, zq), fmul(w, y)));
    Rq[1][0] = fmul(2.0f, fadd(fmul(x, y), fmul(w, zq)));
    Rq[1][1] = fsub(1.0f, fmul(2.0f, fadd(fmul(x, x), fmul(zq, zq))));
    Rq[1][2] = fmul(2.0f, fsub(fmul(y, zq), fmul(w, x)));
    Rq[2][0] = fmul(2.0f, fsub(fmul(x, zq), fmul(w, y)));
    Rq[2][1] = fmul(2.0f, fadd(fmul(y, zq), fmul(w, x)));
    Rq[2][2] = fsub(1.0f, fmul(2.0f, fadd(fmul(x, x), fmul(y, y))));
    const float s[3] = {vd.scale[3 * k], vd.scale[3 * k + 1], vd.scale[3 * k + 2]};
    float M[3][3];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            const float rg = fadd(fadd(fmul(R[0 * 3 + i], Rq[0][j]), fmul(R[1 * 3 + i], Rq[1][j])), fmul(R[2 * 3 + i], Rq[2][j]));
            M[i][j] = fmul(rg, s[j]);
        }
    auto cv = [&](int i, int j) {
        return fadd(fadd(fmul(M[i][0], M[j][0]), fmul(M[i][1], M[j][1])), fmul(M[i][2], M[j][2]));
    };
    a.xyzo[id] = make_float4(m[0], m[1], m[2], vd.opacity[k]);
    a.cova[id] = make_float4(cv(0, 0), cv(0, 1), cv(0, 2), cv(1, 1));
    a.covb[id] = make_float2(cv(1, 2), cv(2, 2));
}

// Copy `rows` feature rows (Gaussian ids first .. first + rows - 1, rows
// s_src[] of view vd's feature map) cooperatively: consecutive threads take
// consecutive 4-wide chunks, so both the reads and the writes are coalesced.
__device__ __forceinline__ void copy_rows(const BuildArgs &a, const ViewDesc &vd, const int64_t *s_src, int rows,
                                          int64_t first) {
    const int C = a.C;
    if (vd.feat_dtype == TSPLAT_BF16 && a.out_dtype == TSPLAT_BF16 && (C & 7) == 0 &&
        (reinterpret_cast<uintptr_t>(vd.feat) & 15u) == 0) {
        // BF16 rows stored as they come: 16-byte chunks, no conversion
        const int cpr = C >> 3;
        const bool pow2 = (cpr & (cpr - 1)) == 0;
        const int sh = __ffs(cpr) - 1;
        for (int ch = threadIdx.x; ch < rows * cpr; ch += BT) {
            const int row = pow2 ? ch >> sh : ch / cpr, part = ch - row * cpr;
            const uint4 x = __ldg(reinterpret_cast<const uint4 *>((const __nv_bfloat16 *)vd.feat + s_src[row] * C) + part);
            reinterpret_cast<uint4 *>((__nv_bfloat16 *)a.feat + (first + row) * C)[part] = x;
        }
        return;
    }
    const bool vec = (C & 3) == 0;
    const int cpr = vec ? C / 4 : C;  // chunks per row
    const bool pow2 = (cpr & (cpr - 1)) == 0;
    const int sh = __ffs(cpr) - 1;
    for (int ch = threadIdx.x; ch < rows * cpr; ch += BT) {
        const int row = pow2 ? ch >> sh : ch / cpr, part = ch - row * cpr;
        const int64_t p = s_src[row], id = first + row;
        if (vec) {
            const int c0 = part * 4;
            float v[4];
            if (vd.feat_dtype == TSPLAT_F32) {
                const float4 x = *reinterpret_cast<const float4 *>((const float *)vd.feat + p * C + c0);
                v[0] = x.x; v[1] = x.y; v[2] = x.z; v[3] = x.w;
            } else {
                const uint2 x = *reinterpret_cast<const uint2 *>((const __nv_bfloat16 *)vd.feat + p * C + c0);
                v[0] = __uint_as_float(x.x << 16); v[1] = __uint_as_float(x.x & 0xffff0000u);
                v[2] = __uint_as_float(x.y << 16); v[3] = __uint_as_float(x.y & 0xffff0000u);
            }
            if (a.out_dtype == TSPLAT_F32) {
                *reinterpret_cast<float4 *>((float *)a.feat + id * C + c0) = make_float4(v[0], v[1], v[2], v[3]);
                if (a.fsplit) {
                    uint2 hi, lo;
                    split4(v, hi, lo);
                    const int cp = padded_channels(C);
                    __nv_bfloat16 *row = (__nv_bfloat16 *)a.fsplit + id * 2 * cp;
                    *reinterpret_cast<uint2 *>(row + c0) = hi;
                    *reinterpret_cast<uint2 *>(row + cp + c0) = lo;
                }
            } else {
                __nv_bfloat162 lo = __floats2bfloat162_rn(v[0], v[1]), hi = __floats2bfloat162_rn(v[2], v[3]);
                uint2 o;
                o.x = *reinterpret_cast<uint32_t *>(&lo);
                o.y = *reinterpret_cast<uint32_t *>(&hi);
                *reinterpret_cast<uint2 *>((__nv_bfloat16 *)a.feat + id * C + c0) = o;
            }
        } else {
            float v = vd.feat_dtype == TSPLAT_F32 ? ((const float *)vd.feat)[p * C + part]
                                                  : __bfloat162float(((const __nv_bfloat16 *)vd.feat)[p * C + part]);
            if (a.out_dtype == TSPLAT_F32) {
                ((float *)a.feat)[id * C + part] = v;
                if (a.fsplit) split1(v, C, id, part, a.fsplit);
            } else {
                ((__nv_bfloat16 *)a.feat)[id * C + part] = __float2bfloat16_rn(v);
            }
        }
    }
}

__global__ __launch_bounds__(BT) void k_build_lift(BuildArgs a) {
    __shared__ uint32_t s_wn[BT / 32];
    __shared__ int64_t s_src[BT];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const ViewDesc &vd = a.views[view_of_block(a, blockIdx.x)];
    const int64_t base = ((int64_t)blockIdx.x - vd.blk0) * BUILD_PIX_PER_BLOCK;
    int64_t running = a.blk_off[blockIdx.x];
    // compact maps: a foreground pixel's row is its Gaussian id minus the view's first id
    const int64_t goff = vd.compact ? (int64_t)a.blk_off[vd.blk0] : 0;
    for (int r = 0; r < BI; ++r) {
        const int64_t g = base + (int64_t)r * BT + threadIdx.x;  // pixel of the view
        const bool fg = is_fg(vd, g);
        const uint32_t bal = __ballot_sync(FULL, fg);
        if (lane == 0) s_wn[warp] = __popc(bal);
        __syncthreads();
        uint32_t woff = 0, tot = 0;
#pragma unroll
        for (int w = 0; w < BT / 32; ++w) {
            const uint32_t c = s_wn[w];
            woff += w < warp ? c : 0u;
            tot += c;
        }
        const uint32_t local = woff + __popc(bal & lanemask_lt());
        if (fg) {
            const int64_t id = running + local;
            const int64_t k = vd.compact ? id - goff : g;
            lift_one(a, vd, g, k, id);
            s_src[local] = k;
        }
        __syncthreads();
        copy_rows(a, vd, s_src, (int)tot, running);
        running += tot;
        __syncthreads();
    }
}

// Adjoint of the lifting (Tele-Aloha trains the encoder through R_G, Sec.
// 4.2): same striping and Gaussian numbering as k_build_lift; each
// foreground pixel turns its Gaussian's gradients into gradients of the
// depth, scale, quaternion, opacity and feature maps; background pixels get
// zeros.  mean = Rs^T (z ray - ts) gives dL/dz = (Rs^T ray) . dL/dmean;
// cov = M M^T with M = Rs^T R(q / |q|) diag(s) gives dL/dM = 2 G M for the
// symmetric gradient G of the covariance, then the scales, the rotation and
// the quaternion through its normalisation.
__global__ __launch_bounds__(BT) void k_build_backward(LiftBwdArgs a) {
    __shared__ uint32_t s_wn[BT / 32];
    const BuildArgs &b = a.b;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int vi = view_of_block(b, blockIdx.x);
    const ViewDesc &vd = b.views[vi];
    const SrcGrads &out = a.g[vi];
    const int64_t base = ((int64_t)blockIdx.x - vd.blk0) * BUILD_PIX_PER_BLOCK;
    const int C = b.C;
    int64_t running = b.blk_off[blockIdx.x];
    for (int r = 0; r < BI; ++r) {
        const int64_t p = base + (int64_t)r * BT + threadIdx.x;  // pixel of the view
        const bool fg = is_fg(vd, p);
        const uint32_t bal = __ballot_sync(FULL, fg);
        if (lane == 0) s_wn[warp] = __popc(bal);
        __syncthreads();
        uint32_t woff = 0, tot = 0;
#pragma unroll
        for (int w = 0; w < BT / 32; ++w) {
            const uint32_t c = s_wn[w];
            woff += w < warp ? c : 0u;
            tot += c;
        }
        if (p < (int64_t)vd.H * vd.W) {
            if (!fg) {
                out.depth[p] = 0.0f;
                out.opacity[p] = 0.0f;
                for (int k = 0; k < 3; ++k) out.scale[3 * p + k] = 0.0f;
                if (out.quat) for (int k = 0; k < 4; ++k) out.quat[4 * p + k] = 0.0f;
                for (int c = 0; c < C; ++c) out.feat[p * C + c] = 0.0f;
            } else {
                const int64_t n = running + woff + __popc(bal & lanemask_lt());
                const tsplat_camera &cam = vd.cam;
                const float *Rs = cam.R;
                const int u = (int)(p % vd.W), v = (int)(p / vd.W);
                const float ray[3] = {(u - cam.cx) / cam.fx, (v - cam.cy) / cam.fy, 1.0f};
                const float *gm = a.d_mean + 3 * n;
                float gz = 0.0f;
#pragma unroll
                for (int i = 0; i < 3; ++i) gz += (Rs[0 * 3 + i] * ray[0] + Rs[1 * 3 + i] * ray[1] + Rs[2 * 3 + i] * ray[2]) * gm[i];
                out.depth[p] = gz;
                float w = 1.0f, x = 0.0f, y = 0.0f, z = 0.0f;
                if (vd.quat) {
                    const float4 q = *reinterpret_cast<const float4 *>(vd.quat + 4 * p);
                    w = q.x; x = q.y; y = q.z; z = q.w;
                }
                const float nq = sqrtf(w * w + x * x + y * y + z * z);
                w /= nq; x /= nq; y /= nq; z /= nq;
                const float Rq[3][3] = {{1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)},
                                        {2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)},
                                        {2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)}};
                const float s3[3] = {vd.scale[3 * p], vd.scale[3 * p + 1], vd.scale[3 * p + 2]};
                float Rg[3][3], M[3][3];
#pragma unroll
                for (int i = 0; i < 3; ++i)
#pragma unroll
                    for (int j = 0; j < 3; ++j) {
                        Rg[i][j] = Rs[0 * 3 + i] * Rq[0][j] + Rs[1 * 3 + i] * Rq[1][j] + Rs[2 * 3 + i] * Rq[2][j];
                        M[i][j] = Rg[i][j] * s3[j];
                    }
                const float *gc = a.d_cov + 6 * n;
                const float G[3][3] = {{gc[0], 0.5f * gc[1], 0.5f * gc[2]},
                                       {0.5f * gc[1], gc[3], 0.5f * gc[4]},
                                       {0.5f * gc[2], 0.5f * gc[4], gc[5]}};
                float gM[3][3];
#pragma unroll
                for (int i = 0; i < 3; ++i)
#pragma unroll
                    for (int j = 0; j < 3; ++j) gM[i][j] = 2.0f * (G[i][0] * M[0][j] + G[i][1] * M[1][j] + G[i][2] * M[2][j]);
#pragma unroll
                for (int j = 0; j < 3; ++j) out.scale[3 * p + j] = gM[0][j] * Rg[0][j] + gM[1][j] * Rg[1][j] + gM[2][j] * Rg[2][j];
                if (out.quat) {
                    float gR[3][3];
#pragma unroll
                    for (int k = 0; k < 3; ++k)
#pragma unroll
                        for (int j = 0; j < 3; ++j)
                            gR[k][j] = (Rs[k * 3 + 0] * gM[0][j] + Rs[k * 3 + 1] * gM[1][j] + Rs[k * 3 + 2] * gM[2][j]) * s3[j];
                    const float gw = 2 * (-z * gR[0][1] + y * gR[0][2] + z * gR[1][0] - x * gR[1][2] - y * gR[2][0] + x * gR[2][1]);
                    const float gx = 2 * (y * gR[0][1] + z * gR[0][2] + y * gR[1][0] - 2 * x * gR[1][1] - w * gR[1][2] +
                                          z * gR[2][0] + w * gR[2][1] - 2 * x * gR[2][2]);
                    const float gy = 2 * (-2 * y * gR[0][0] + x * gR[0][1] + w * gR[0][2] + x * gR[1][0] + z * gR[1][2] -
                                          w * gR[2][0] + z * gR[2][1] - 2 * y * gR[2][2]);
                    const float gzq = 2 * (-2 * z * gR[0][0] - w * gR[0][1] + x * gR[0][2] + w * gR[1][0] - 2 * z * gR[1][1] +
                                           y * gR[1][2] + x * gR[2][0] + y * gR[2][1]);
                    const float dot = gw * w + gx * x + gy * y + gzq * z;
                    *reinterpret_cast<float4 *>(out.quat + 4 * p) =
                        make_float4((gw - w * dot) / nq, (gx - x * dot) / nq, (gy - y * dot) / nq, (gzq - z * dot) / nq);
                }
                out.opacity[p] = a.d_opac[n];
                for (int c = 0; c < C; ++c) out.feat[p * C + c] = a.d_feat[n * C + c];
            }
        }
        running += tot;
        __syncthreads();
    }
}

__global__ void k_gaussians_set(uint64_t n, const float *mean, const float *cov, const float *opac,
                                const void *feat, int dtype_in, int C, int dtype_out, float4 *xyzo,
                                float4 *cova, float2 *covb, void *feat_out, void *fsplit, uint32_t *n_dev) {
    const uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i == 0) *n_dev = (uint32_t)n;
    if (i >= n) return;
    xyzo[i] = make_float4(mean[3 * i], mean[3 * i + 1], mean[3 * i + 2], opac[i]);
    cova[i] = make_float4(cov[6 * i], cov[6 * i + 1], cov[6 * i + 2], cov[6 * i + 3]);
    covb[i] = make_float2(cov[6 * i + 4], cov[6 * i + 5]);
    copy_feat(feat, dtype_in, (int64_t)i, feat_out, dtype_out, (int64_t)i, C);
    if (fsplit && dtype_out == TSPLAT_F32)
        for (int c = 0; c < C; ++c) split1(((const float *)feat_out)[i * C + c], C, (int64_t)i, c, fsplit);
}

// (hi, lo) rows of N x C FP32 features: thread t of Gaussian i writes
// columns 4t .. 4t + 3 of both halves, zero beyond C.
__global__ void k_feat_split(const float *feat, const uint32_t *n_dev, int C, void *fsplit) {
    const int cp = padded_channels(C), q = cp / 4;
    const uint64_t n = *n_dev;
    for (uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n * q; t += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t i = t / q;
        const int c0 = (int)(t - i * q) * 4;
        float v[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) v[k] = c0 + k < C ? feat[i * C + c0 + k] : 0.0f;
        uint2 hi, lo;
        split4(v, hi, lo);
        __nv_bfloat16 *row = (__nv_bfloat16 *)fsplit + i * 2 * cp;
        *reinterpret_cast<uint2 *>(row + c0) = hi;
        *reinterpret_cast<uint2 *>(row + cp + c0) = lo;
    }
}

__global__ void k_gaussians_get(const uint32_t *n_dev, int C, int dtype, const float4 *xyzo,
                                const float4 *cova, const float2 *covb, const void *feat_in, float *mean,
                                float *cov, float *opac, void *feat_out) {
    const uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= *n_dev) return;
    const float4 g = xyzo[i];
    const float4 ca = cova[i];
    const float2 cb = covb[i];
    if (mean) { mean[3 * i] = g.x; mean[3 * i + 1] = g.y; mean[3 * i + 2] = g.z; }
    if (opac) opac[i] = g.w;
    if (cov) {
        cov[6 * i] = ca.x; cov[6 * i + 1] = ca.y; cov[6 * i + 2] = ca.z;
        cov[6 * i + 3] = ca.w; cov[6 * i + 4] = cb.x; cov[6 * i + 5] = cb.y;
    }
    if (feat_out) copy_feat(feat_in, dtype, (int64_t)i, feat_out, dtype, (int64_t)i, C);
}

}  // namespace

void launch_build(const BuildArgs &a, cudaStream_t s) {
    if (a.nblocks <= 0) {
        cudaMemsetAsync(a.n_dev, 0, sizeof(uint32_t), s);
        return;
    }
    k_build_count<<<a.nblocks, BT, 0, s>>>(a);
    note_launches(1);
    k_build_scan<<<1, 1024, 0, s>>>(a);
    note_launches(1);
    k_build_lift<<<a.nblocks, BT, 0, s>>>(a);
    note_launches(1);
}

void launch_build_backward(const LiftBwdArgs &a, cudaStream_t s) {
    if (a.b.nblocks <= 0) return;
    k_build_count<<<a.b.nblocks, BT, 0, s>>>(a.b);
    k_build_scan<<<1, 1024, 0, s>>>(a.b);
    k_build_backward<<<a.b.nblocks, BT, 0, s>>>(a);
    note_launches(3);
}

void launch_gaussians_set(int64_t n, const float *mean, const float *cov, const float *opac, const void *feat,
                          int feat_dtype_in, int C, int out_dtype, float4 *xyzo, float4 *cova, float2 *covb,
                          void *feat_out, void *fsplit, uint32_t *n_dev, cudaStream_t s) {
    const int64_t blocks = n > 0 ? (n + 255) / 256 : 1;
    k_gaussians_set<<<(unsigned)blocks, 256, 0, s>>>((uint64_t)n, mean, cov, opac, feat, feat_dtype_in, C,
                                                     out_dtype, xyzo, cova, covb, feat_out, fsplit, n_dev);
    note_launches(1);
}

void launch_feat_split(const float *feat, const uint32_t *n_dev, int64_t n_cap, int C, void *fsplit,
                       cudaStream_t s) {
    if (n_cap <= 0) return;
    const int64_t work = n_cap * (padded_channels(C) / 4);
    const int blocks = (int)std::min<int64_t>((work + 255) / 256, (int64_t)sm_count() * 16);
    k_feat_split<<<blocks, 256, 0, s>>>(feat, n_dev, C, fsplit);
    note_launches(1);
}

void launch_gaussians_get(const uint32_t *n_dev, int64_t cap, int C, int dtype, const float4 *xyzo,
                          const float4 *cova, const float2 *covb, const void *feat_in, float *mean, float *cov,
                          float *opac, void *feat_out, cudaStream_t s) {
    if (cap <= 0) return;
    k_gaussians_get<<<(unsigned)((cap + 255) / 256), 256, 0, s>>>(n_dev, C, dtype, xyzo, cova, covb, feat_in,
                                                                  mean, cov, opac, feat_out);
    note_launches(1);
}

}  // namespace tsp
