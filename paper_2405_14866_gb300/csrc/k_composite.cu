// A7: front-to-back alpha compositing of C-channel latent features per
// 16x16 tile, and A8: its adjoint (Tele-Aloha Sec. 4.2: the rasterizer
// splats latent features instead of colours and is differentiated end to
// end).
//
// One CTA of 256 threads per tile; warp w owns an 8x4 pixel block.  The
// tile's depth-ordered Gaussians are staged 256 at a time into shared
// memory (32-byte projected record + feature row).  Each warp first tests
// the 32-wide chunks of the batch against its block with the Gaussians'
// alpha_min boxes (exact: outside its box a Gaussian's alpha is provably
// below alpha_min, so skipping it is what the per-pixel test would do) and
// iterates only over the survivors, in order.  A warp stops computing when
// all its pixels are saturated; the CTA stops staging when all warps have.
// No tensor cores: blending is a per-pixel sequential recurrence, not a
// dense contraction.
#include <algorithm>

#include "common.cuh"
#include "internal.h"

namespace tsp {

namespace {

constexpr int CT = 256;  // threads per CTA = pixels per tile
constexpr uint32_t FULL = 0xffffffffu;

template <typename FT>
struct FeatIO;

template <>
struct FeatIO<float> {
    static constexpr int VEC = 4;  // elements per 16-byte vector
    template <int CP>
    __device__ static __forceinline__ void axpy(float (&F)[CP], const float *row, float w) {
        const float4 *r4 = reinterpret_cast<const float4 *>(row);
#pragma unroll
        for (int i = 0; i < CP / 4; ++i) {
            const float4 v = r4[i];
            F[4 * i] = fmaf(v.x, w, F[4 * i]);
            F[4 * i + 1] = fmaf(v.y, w, F[4 * i + 1]);
            F[4 * i + 2] = fmaf(v.z, w, F[4 * i + 2]);
            F[4 * i + 3] = fmaf(v.w, w, F[4 * i + 3]);
        }
    }
    template <int CP>
    __device__ static __forceinline__ void load(float (&f)[CP], const float *row) {
        const float4 *r4 = reinterpret_cast<const float4 *>(row);
#pragma unroll
        for (int i = 0; i < CP / 4; ++i) {
            const float4 v = r4[i];
            f[4 * i] = v.x; f[4 * i + 1] = v.y; f[4 * i + 2] = v.z; f[4 * i + 3] = v.w;
        }
    }
};

__device__ __forceinline__ float bf_lo(uint32_t u) { return __uint_as_float(u << 16); }
__device__ __forceinline__ float bf_hi(uint32_t u) { return __uint_as_float(u & 0xffff0000u); }

template <>
struct FeatIO<__nv_bfloat16> {
    static constexpr int VEC = 8;
    template <int CP>
    __device__ static __forceinline__ void axpy(float (&F)[CP], const __nv_bfloat16 *row, float w) {
        const uint4 *r4 = reinterpret_cast<const uint4 *>(row);
#pragma unroll
        for (int i = 0; i < CP / 8; ++i) {
            const uint4 v = r4[i];
            F[8 * i + 0] = fmaf(bf_lo(v.x), w, F[8 * i + 0]);
            F[8 * i + 1] = fmaf(bf_hi(v.x), w, F[8 * i + 1]);
            F[8 * i + 2] = fmaf(bf_lo(v.y), w, F[8 * i + 2]);
            F[8 * i + 3] = fmaf(bf_hi(v.y), w, F[8 * i + 3]);
            F[8 * i + 4] = fmaf(bf_lo(v.z), w, F[8 * i + 4]);
            F[8 * i + 5] = fmaf(bf_hi(v.z), w, F[8 * i + 5]);
            F[8 * i + 6] = fmaf(bf_lo(v.w), w, F[8 * i + 6]);
            F[8 * i + 7] = fmaf(bf_hi(v.w), w, F[8 * i + 7]);
        }
    }
    template <int CP>
    __device__ static __forceinline__ void load(float (&f)[CP], const __nv_bfloat16 *row) {
        const uint4 *r4 = reinterpret_cast<const uint4 *>(row);
#pragma unroll
        for (int i = 0; i < CP / 8; ++i) {
            const uint4 v = r4[i];
            f[8 * i + 0] = bf_lo(v.x); f[8 * i + 1] = bf_hi(v.x);
            f[8 * i + 2] = bf_lo(v.y); f[8 * i + 3] = bf_hi(v.y);
            f[8 * i + 4] = bf_lo(v.z); f[8 * i + 5] = bf_hi(v.z);
            f[8 * i + 6] = bf_lo(v.w); f[8 * i + 7] = bf_hi(v.w);
        }
    }
};

// Stage record + feature row of Gaussian `id` into slot `slot` (C real
// channels; the padding channels of the shared rows stay zero).
template <int CP, typename FT>
__device__ __forceinline__ void stage(const Header *__restrict__ hdr, const FT *__restrict__ feat, int C,
                                      bool vec_ok, uint32_t id, Header *s_hdr, FT *s_feat, int slot) {
    s_hdr[slot] = hdr[id];
    FT *dst = s_feat + (size_t)slot * CP;
    const FT *src = feat + (size_t)id * C;
    if (vec_ok) {
        constexpr int V = FeatIO<FT>::VEC;
        const uint4 *s4 = reinterpret_cast<const uint4 *>(src);
        uint4 *d4 = reinterpret_cast<uint4 *>(dst);
        for (int i = 0; i < C / V; ++i) d4[i] = __ldg(s4 + i);
    } else {
        for (int c = 0; c < C; ++c) dst[c] = src[c];
    }
}

template <int CP, typename FT>
__global__ __launch_bounds__(CT, 2) void k_composite(CompositeArgs a) {
    extern __shared__ __align__(16) unsigned char smem[];
    Header *s_hdr = reinterpret_cast<Header *>(smem);
    FT *s_feat = reinterpret_cast<FT *>(smem + CT * sizeof(Header));
    const FT *feat = reinterpret_cast<const FT *>(a.feat);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int tile = blockIdx.x;
    const int tx = tile % a.tiles_x, ty = tile / a.tiles_x;
    const int bx0 = tx * TILE + (warp & 1) * 8, by0 = ty * TILE + (warp >> 1) * 4;
    const int px = bx0 + (lane & 7), py = by0 + (lane >> 3);
    const bool inside = px < a.W && py < a.H;
    const float fpx = (float)px, fpy = (float)py;
    const float fbx0 = (float)bx0, fbx1 = (float)(bx0 + 7), fby0 = (float)by0, fby1 = (float)(by0 + 3);

    if (a.C < CP) {
        // zero the padding channels once; staging writes only the first C
        for (int i = tid; i < CT * CP; i += CT) s_feat[i] = FT(0.0f);
    }
    const uint2 rg = a.ranges[tile];
    const int n = (int)(rg.y - rg.x);
    const bool vec_ok = (a.C % FeatIO<FT>::VEC) == 0;

    float F[CP];
#pragma unroll
    for (int c = 0; c < CP; ++c) F[c] = 0.0f;
    float T = 1.0f;
    uint32_t last = 0;
    bool done = !inside;

    for (int b0 = 0; b0 < n; b0 += CT) {
        if (__syncthreads_and(done)) break;  // also guards the staging buffers
        if (b0 + tid < n) stage<CP, FT>(a.hdr, feat, a.C, vec_ok, a.ids[rg.x + b0 + tid], s_hdr, s_feat, tid);
        __syncthreads();
        const int cnt = min(CT, n - b0);
        if (__all_sync(FULL, done)) continue;
        for (int c0 = 0; c0 < cnt; c0 += 32) {
            bool rel = false;
            if (c0 + lane < cnt) {
                const Header h = s_hdr[c0 + lane];
                rel = (h.h0.x + h.h1.z >= fbx0) && (h.h0.x - h.h1.z <= fbx1) && (h.h0.y + h.h1.w >= fby0) &&
                      (h.h0.y - h.h1.w <= fby1);
            }
            uint32_t m = __ballot_sync(FULL, rel);
            while (m) {
                const int j = c0 + __ffs(m) - 1;
                m &= m - 1;
                const float4 h0 = s_hdr[j].h0;
                const float4 h1 = s_hdr[j].h1;
                const float q = gauss_q(fpx - h0.x, fpy - h0.y, h0.z, h0.w, h1.x);
                float w = 0.0f;
                if (!done && q <= 0.0f) {
                    const float al = fminf(a.alpha_max, gauss_alpha_raw(q, h1.y));
                    if (al >= a.alpha_min) {
                        const float Tn = T * (1.0f - al);
                        if (Tn < a.t_min) {
                            done = true;
                        } else {
                            w = al * T;
                            T = Tn;
                            last = (uint32_t)(b0 + j + 1);
                        }
                    }
                }
                if (__any_sync(FULL, w != 0.0f)) FeatIO<FT>::template axpy<CP>(F, s_feat + (size_t)j * CP, w);
            }
            if (__all_sync(FULL, done)) break;
        }
    }
    if (inside) {
        const size_t HW = (size_t)a.W * a.H, pix = (size_t)py * a.W + px;
#pragma unroll
        for (int c = 0; c < CP; ++c)
            if (c < a.C) a.out_feat[c * HW + pix] = F[c];
        if (a.out_alpha) a.out_alpha[pix] = 1.0f - T;
        if (a.out_T) a.out_T[pix] = T;
        if (a.out_last) a.out_last[pix] = last;
    }
}

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
    return v;
}

// A8: reverse traversal from each pixel's last blended Gaussian, with the
// transmittance in front of each Gaussian recomputed by division from the
// saved final transmittance.
template <int CP, typename FT>
__global__ __launch_bounds__(CT, 2) void k_backward(BackwardArgs a) {
    extern __shared__ __align__(16) unsigned char smem[];
    Header *s_hdr = reinterpret_cast<Header *>(smem);
    FT *s_feat = reinterpret_cast<FT *>(smem + CT * sizeof(Header));
    __shared__ uint32_t s_max[CT / 32];
    __shared__ uint32_t s_id[CT];
    const FT *feat = reinterpret_cast<const FT *>(a.feat);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int tile = blockIdx.x;
    const int tx = tile % a.tiles_x, ty = tile / a.tiles_x;
    const int bx0 = tx * TILE + (warp & 1) * 8, by0 = ty * TILE + (warp >> 1) * 4;
    const int px = bx0 + (lane & 7), py = by0 + (lane >> 3);
    const bool inside = px < a.W && py < a.H;
    const float fpx = (float)px, fpy = (float)py;
    const float fbx0 = (float)bx0, fbx1 = (float)(bx0 + 7), fby0 = (float)by0, fby1 = (float)(by0 + 3);
    const size_t HW = (size_t)a.W * a.H, pix = (size_t)py * a.W + px;

    if (a.C < CP)
        for (int i = tid; i < CT * CP; i += CT) s_feat[i] = FT(0.0f);
    const uint2 rg = a.ranges[tile];
    const bool vec_ok = (a.C % FeatIO<FT>::VEC) == 0;

    float g[CP];
    float T = 1.0f, Tfin = 1.0f, gA = 0.0f;
    uint32_t lastk = 0;
#pragma unroll
    for (int c = 0; c < CP; ++c) g[c] = 0.0f;
    if (inside) {
        Tfin = a.T_final[pix];
        T = Tfin;
        lastk = a.last[pix];
        gA = a.dA ? a.dA[pix] : 0.0f;
#pragma unroll
        for (int c = 0; c < CP; ++c)
            if (c < a.C) g[c] = a.dF[c * HW + pix];
    }
    // the tile's deepest blended position
    uint32_t wmax = __reduce_max_sync(FULL, lastk);
    if (lane == 0) s_max[warp] = wmax;
    __syncthreads();
    uint32_t nmax = 0;
#pragma unroll
    for (int w = 0; w < CT / 32; ++w) nmax = max(nmax, s_max[w]);
    float sg = 0.0f;  // <S, g>: blended features behind the current Gaussian

    for (int hi = (int)nmax; hi > 0; hi -= CT) {
        const int lo = max(0, hi - CT);
        __syncthreads();
        if (lo + tid < hi) {
            const uint32_t id = a.ids[rg.x + lo + tid];
            s_id[tid] = id;
            stage<CP, FT>(a.hdr, feat, a.C, vec_ok, id, s_hdr, s_feat, tid);
        }
        __syncthreads();
        const int cnt = hi - lo;
        const uint32_t wl = __reduce_max_sync(FULL, lastk);
        if (wl <= (uint32_t)lo) continue;  // nothing of this batch blended in this warp
        for (int c1 = cnt; c1 > 0; c1 -= 32) {
            const int c0 = max(0, c1 - 32);
            bool rel = false;
            const int jj = c0 + lane;
            if (jj < c1) {
                const Header h = s_hdr[jj];
                rel = (h.h0.x + h.h1.z >= fbx0) && (h.h0.x - h.h1.z <= fbx1) && (h.h0.y + h.h1.w >= fby0) &&
                      (h.h0.y - h.h1.w <= fby1);
            }
            uint32_t m = __ballot_sync(FULL, rel);
            while (m) {
                const int j = c0 + 31 - __clz(m);  // highest first: back to front
                m &= ~(1u << (j - c0));
                const uint32_t k = (uint32_t)(lo + j);
                const float4 h0 = s_hdr[j].h0;
                const float4 h1 = s_hdr[j].h1;
                const float dx = fpx - h0.x, dy = fpy - h0.y;
                const float q = gauss_q(dx, dy, h0.z, h0.w, h1.x);
                bool contrib = false;
                float al = 0.0f, eq = 0.0f, raw = 0.0f;
                if (k < lastk && q <= 0.0f) {
                    eq = __expf(q);
                    raw = __fmul_rn(h1.y, eq);
                    al = fminf(a.alpha_max, raw);
                    contrib = al >= a.alpha_min;
                }
                if (!__any_sync(FULL, contrib)) continue;
                float f[CP];
                FeatIO<FT>::template load<CP>(f, s_feat + (size_t)j * CP);
                float wgt = 0.0f, d_o = 0.0f, dq = 0.0f;
                if (contrib) {
                    const float inv = 1.0f / (1.0f - al);
                    const float Tj = T * inv;
                    float fg = 0.0f;
#pragma unroll
                    for (int c = 0; c < CP; ++c) fg = fmaf(f[c], g[c], fg);
                    wgt = al * Tj;
                    const float dal = Tj * fg - sg * inv + gA * Tfin * inv;
                    sg = fmaf(wgt, fg, sg);
                    T = Tj;
                    if (raw < a.alpha_max) {
                        d_o = eq * dal;
                        dq = al * dal;
                    }
                }
                // per-Gaussian sums over the warp's pixels
                if (a.d_feat) {
#pragma unroll
                    for (int c = 0; c < CP; ++c) {
                        const float v = warp_sum(wgt * g[c]);
                        if (lane == 0 && c < a.C) atomicAdd(&a.d_feat[(size_t)s_id[j] * a.C + c], v);
                    }
                }
                const float gx = dq * (h0.z * dx + h0.w * dy);
                const float gy = dq * (h0.w * dx + h1.x * dy);
                const float ga = dq * (-0.5f * dx * dx);
                const float gb = dq * (-dx * dy);
                const float gc = dq * (-0.5f * dy * dy);
                const float so = warp_sum(d_o), sx = warp_sum(gx), sy = warp_sum(gy);
                const float sa = warp_sum(ga), sb = warp_sum(gb), sc = warp_sum(gc);
                if (lane == 0) {
                    const uint32_t id = s_id[j];
                    if (a.d_opac) atomicAdd(&a.d_opac[id], so);
                    if (a.d_mean2d) {
                        atomicAdd(&a.d_mean2d[2 * id], sx);
                        atomicAdd(&a.d_mean2d[2 * id + 1], sy);
                    }
                    if (a.d_conic) {
                        atomicAdd(&a.d_conic[3 * id], sa);
                        atomicAdd(&a.d_conic[3 * id + 1], sb);
                        atomicAdd(&a.d_conic[3 * id + 2], sc);
                    }
                }
            }
        }
    }
}

template <int CP, typename FT>
void run_composite(const CompositeArgs &a, cudaStream_t s) {
    const size_t smem = CT * sizeof(Header) + (size_t)CT * CP * sizeof(FT);
    static bool attr = false;
    if (!attr) {
        cudaFuncSetAttribute(k_composite<CP, FT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        attr = true;
    }
    k_composite<CP, FT><<<a.tiles_x * a.tiles_y, CT, smem, s>>>(a);
}

template <int CP, typename FT>
void run_backward(const BackwardArgs &a, cudaStream_t s) {
    const size_t smem = CT * sizeof(Header) + (size_t)CT * CP * sizeof(FT);
    static bool attr = false;
    if (!attr) {
        cudaFuncSetAttribute(k_backward<CP, FT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        attr = true;
    }
    k_backward<CP, FT><<<a.tiles_x * a.tiles_y, CT, smem, s>>>(a);
}

}  // namespace

void launch_composite(const CompositeArgs &a, cudaStream_t s) {
    if (a.tiles_x * a.tiles_y == 0) return;
    const bool bf = a.feat_dtype == TSPLAT_BF16;
    if (a.C <= 8) { if (bf) run_composite<8, __nv_bfloat16>(a, s); else run_composite<8, float>(a, s); }
    else if (a.C <= 16) { if (bf) run_composite<16, __nv_bfloat16>(a, s); else run_composite<16, float>(a, s); }
    else if (a.C <= 32) { if (bf) run_composite<32, __nv_bfloat16>(a, s); else run_composite<32, float>(a, s); }
    else { if (bf) run_composite<64, __nv_bfloat16>(a, s); else run_composite<64, float>(a, s); }
}

void launch_backward(const BackwardArgs &a, cudaStream_t s) {
    if (a.tiles_x * a.tiles_y == 0) return;
    const bool bf = a.feat_dtype == TSPLAT_BF16;
    if (a.C <= 8) { if (bf) run_backward<8, __nv_bfloat16>(a, s); else run_backward<8, float>(a, s); }
    else if (a.C <= 16) { if (bf) run_backward<16, __nv_bfloat16>(a, s); else run_backward<16, float>(a, s); }
    else if (a.C <= 32) { if (bf) run_backward<32, __nv_bfloat16>(a, s); else run_backward<32, float>(a, s); }
    else { if (bf) run_backward<64, __nv_bfloat16>(a, s); else run_backward<64, float>(a, s); }
}

}  // namespace tsp
