// A8: adjoint of the front-to-back compositing (Tele-Aloha Sec. 4.2: the
// rasterizer is differentiated end to end).  Persistent warps take
// (tile, 8x4 pixel block) units from a counter; each walks its pixels' list
// range back to front from their last blended Gaussian, recomputing the
// transmittance in front of each Gaussian by division from the saved final
// one, and repeats the forward's blend decisions with the forward's
// arithmetic, so the contributor set is the forward's.
#include <algorithm>

#include "common.cuh"
#include "internal.h"
#include "ptx.cuh"

namespace tsp {

namespace {

constexpr uint32_t FULL = 0xffffffffu;
constexpr float LOG2E = 1.4426950408889634f;

constexpr int CT = 256;

template <typename FT>
struct FeatIO;

template <>
struct FeatIO<float> {
    static constexpr int VEC = 4;
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

template <>
struct FeatIO<__nv_bfloat16> {
    static constexpr int VEC = 8;
    template <int CP>
    __device__ static __forceinline__ void load(float (&f)[CP], const __nv_bfloat16 *row) {
        const uint4 *r4 = reinterpret_cast<const uint4 *>(row);
#pragma unroll
        for (int i = 0; i < CP / 8; ++i) {
            const uint4 v = r4[i];
            f[8 * i + 0] = bf16_lo_f(v.x); f[8 * i + 1] = bf16_hi_f(v.x);
            f[8 * i + 2] = bf16_lo_f(v.y); f[8 * i + 3] = bf16_hi_f(v.y);
            f[8 * i + 4] = bf16_lo_f(v.z); f[8 * i + 5] = bf16_hi_f(v.z);
            f[8 * i + 6] = bf16_lo_f(v.w); f[8 * i + 7] = bf16_hi_f(v.w);
        }
    }
};

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

// Warp totals of NV per-lane values (NV a power of two) with NV - 1 + ...
// shuffles instead of 5 NV: at each level a lane keeps one half of its
// values and receives the partner's partial sums of that half.  Afterwards,
// for NV >= 32, lane l holds in v[i] the total of value l * (NV / 32) + i;
// for NV < 32, lanes with (l & (32 / NV - 1)) == 0 hold in v[0] the total of
// value l / (32 / NV).
template <int NV>
__device__ __forceinline__ void warp_transpose_sum(float (&v)[NV], int lane) {
    int n = NV;
#pragma unroll
    for (int b = 16; b > 0; b >>= 1) {
        if (n > 1) {
            const int half = n / 2;
            const bool upper = (lane & b) != 0;
#pragma unroll
            for (int i = 0; i < NV / 2; ++i) {
                if (i < half) {
                    const float keep = upper ? v[i + half] : v[i];
                    const float send = upper ? v[i] : v[i + half];
                    v[i] = keep + __shfl_xor_sync(FULL, send, b);
                }
            }
            n = half;
        } else {
            v[0] += __shfl_xor_sync(FULL, v[0], b);
        }
    }
}

// Feature gradients of a group of up to 16 contributing Gaussians of one
// warp as a tensor-core product: dF_j[c] = sum over the warp's 32 pixels of
// w_j(p) g_p[c], i.e. D (16 x C) = W^T (16 x 32) G (32 x C), with W and G
// split into bf16 hi + lo parts (three products, FP32 accumulation).
// W is stored per pixel row ([32][BWROW]), G likewise ([32][CP16 + 8]).
constexpr int BWROW = 24;
template <int CP>
struct BwdGroup {
    static constexpr int GP = CP < 16 ? 16 : CP;  // channels padded to whole k16 / n16 blocks
    __nv_bfloat16 wh[CT / 32][32][BWROW];
    __nv_bfloat16 wl[CT / 32][32][BWROW];
    __nv_bfloat16 gh[CT / 32][32][GP + 8];
    __nv_bfloat16 gl[CT / 32][32][GP + 8];
    uint32_t gid[CT / 32][16];
};

template <int CP>
__device__ __forceinline__ void flush_feat_grads(BwdGroup<CP> &B, int warp, int lane, int cnt, int C,
                                                 float *d_feat) {
    constexpr int GP = BwdGroup<CP>::GP;
    for (int k = cnt; k < 16; ++k) {  // unused columns contribute nothing
        B.wh[warp][lane][k] = __float2bfloat16_rn(0.0f);
        B.wl[warp][lane][k] = __float2bfloat16_rn(0.0f);
    }
    __syncwarp();
    float acc[GP / 8][4];
#pragma unroll
    for (int t = 0; t < GP / 8; ++t)
#pragma unroll
        for (int e = 0; e < 4; ++e) acc[t][e] = 0.0f;
    const int kl = ((lane >> 3) & 1) * 8 + (lane & 7);        // B: pixel row this lane addresses
    const int arow = ((lane >> 4) & 1) * 8 + (lane & 7);      // A (transposed load): pixel row
    const int acol = ((lane >> 3) & 1) * 8, bcol = (lane >> 4) * 8;
#pragma unroll
    for (int ks = 0; ks < 2; ++ks) {  // two k-steps of 16 pixels
        uint32_t ah[4], al[4];
        ldsm_x4_t(ah[0], ah[1], ah[2], ah[3], &B.wh[warp][ks * 16 + arow][acol]);
        ldsm_x4_t(al[0], al[1], al[2], al[3], &B.wl[warp][ks * 16 + arow][acol]);
#pragma unroll
        for (int p = 0; p < GP / 16; ++p) {
            uint32_t bh[4], bl[4];
            ldsm_x4_t(bh[0], bh[1], bh[2], bh[3], &B.gh[warp][ks * 16 + kl][p * 16 + bcol]);
            ldsm_x4_t(bl[0], bl[1], bl[2], bl[3], &B.gl[warp][ks * 16 + kl][p * 16 + bcol]);
            mma_bf16(acc[2 * p], ah[0], ah[1], ah[2], ah[3], bh[0], bh[1]);
            mma_bf16(acc[2 * p], al[0], al[1], al[2], al[3], bh[0], bh[1]);
            mma_bf16(acc[2 * p], ah[0], ah[1], ah[2], ah[3], bl[0], bl[1]);
            mma_bf16(acc[2 * p + 1], ah[0], ah[1], ah[2], ah[3], bh[2], bh[3]);
            mma_bf16(acc[2 * p + 1], al[0], al[1], al[2], al[3], bh[2], bh[3]);
            mma_bf16(acc[2 * p + 1], ah[0], ah[1], ah[2], ah[3], bl[2], bl[3]);
        }
    }
    // D fragment: Gaussian rows lane/4 (+8), channel columns 2(lane%4) (+1)
#pragma unroll
    for (int t = 0; t < GP / 8; ++t)
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const int j = (lane >> 2) + ((e >> 1) << 3), c = t * 8 + 2 * (lane & 3) + (e & 1);
            if (j < cnt && c < C) atomicAdd(&d_feat[(size_t)B.gid[warp][j] * C + c], acc[t][e]);
        }
    __syncwarp();
}

// A8: reverse traversal from each pixel's last blended Gaussian, with the
// transmittance in front of each Gaussian recomputed by division from the
// saved final transmittance.  The blend decisions repeat the forward's
// arithmetic exactly (same instructions), so the contributor set is the
// forward's.
template <int CP, typename FT>
__global__ __launch_bounds__(CT, 2) void k_backward(BackwardArgs a) {
    extern __shared__ __align__(16) unsigned char smem[];
    Header *s_hdr = reinterpret_cast<Header *>(smem);
    FT *s_feat = reinterpret_cast<FT *>(smem + CT * sizeof(Header));
    BwdGroup<CP> &BG = *reinterpret_cast<BwdGroup<CP> *>(smem + CT * sizeof(Header) + (size_t)CT * CP * sizeof(FT));
    __shared__ uint32_t s_id[CT];
    const FT *feat = reinterpret_cast<const FT *>(a.feat);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    // each warp zeroes the channel padding of its own staging rows
    if (a.C < CP)
        for (int i = lane; i < 32 * CP; i += 32) s_feat[(size_t)warp * 32 * CP + i] = FT(0.0f);
    __syncwarp();
    const int n_units = a.tiles_x * a.tiles_y * 8;
    // Persistent: every warp takes (tile, 8x4 block) units from a counter, so
    // the load balances at warp granularity whatever the tiles' list lengths.
    for (;;) {
    uint32_t unit = 0;
    if (lane == 0) unit = atomicAdd(a.unit_counter, 1u);
    unit = __shfl_sync(FULL, unit, 0);
    if (unit >= (uint32_t)n_units) break;
    const int tile = a.tile_order ? (int)a.tile_order[unit >> 3] : (int)(unit >> 3), wb = (int)(unit & 7);
    const int tx = tile % a.tiles_x, ty = tile / a.tiles_x;
    const int bx0 = tx * TILE + (wb & 1) * 8, by0 = ty * TILE + (wb >> 1) * 4;
    const int px = bx0 + (lane & 7), py = by0 + (lane >> 3);
    const bool inside = px < a.W && py < a.H;
    const float fpx = (float)px, fpy = (float)py;
    const float fbx0 = (float)bx0, fbx1 = (float)(bx0 + 7), fby0 = (float)by0, fby1 = (float)(by0 + 3);
    const size_t HW = (size_t)a.W * a.H, pix = (size_t)py * a.W + px;
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
    // this pixel's row of G for the feature-gradient products (hi + lo)
#pragma unroll
    for (int c = 0; c < BwdGroup<CP>::GP; ++c) {
        const float v = c < CP ? g[c] : 0.0f;
        const __nv_bfloat16 h = __float2bfloat16_rn(v);
        BG.gh[warp][lane][c] = h;
        BG.gl[warp][lane][c] = __float2bfloat16_rn(v - __bfloat162float(h));
    }
    unsigned long long g2[CP / 2];  // g in (even, odd) channel pairs, for the packed <f, g>
#pragma unroll
    for (int c = 0; c < CP / 2; ++c) g2[c] = f2pack(g[2 * c], g[2 * c + 1]);
    const unsigned long long fp2 = f2pack(fpx, fpy);
    int gs = 0;  // contributing Gaussians collected in this warp's current group
    const uint32_t wmax = __reduce_max_sync(FULL, lastk);
    float sg = 0.0f;  // <S, g>: blended features behind the current Gaussian
    // Each warp walks its own list range [0, wmax) back to front in chunks of
    // 32, staged into its own slice of shared memory: no block-wide barrier,
    // so a warp whose pixels stopped early does not wait for the others.
    Header *w_hdr = s_hdr + warp * 32;
    FT *w_feat = s_feat + (size_t)warp * 32 * CP;
    uint32_t *w_id = s_id + warp * 32;
    {
        for (int c1 = (int)wmax; c1 > 0; c1 -= 32) {
            const int c0 = max(0, c1 - 32);
            __syncwarp();
            if (c0 + lane < c1) {
                const uint32_t gid = a.ids[rg.x + c0 + lane];
                w_id[lane] = gid;
                stage<CP, FT>(a.hdr, feat, a.C, vec_ok, gid, w_hdr, w_feat, lane);
            }
            __syncwarp();
            bool rel = false;
            if (c0 + lane < c1) {
                const Header h = w_hdr[lane];
                rel = (h.h0.x + h.h1.z >= fbx0) && (h.h0.x - h.h1.z <= fbx1) && (h.h0.y + h.h1.w >= fby0) &&
                      (h.h0.y - h.h1.w <= fby1);
            }
            uint32_t m = __ballot_sync(FULL, rel);
            while (m) {
                const int j = 31 - __clz(m);  // highest first: back to front
                m &= ~(1u << j);
                const uint32_t k = (uint32_t)(c0 + j);
                const float4 h0 = w_hdr[j].h0;
                const float4 h1 = w_hdr[j].h1;
                float dx, dy;
                f2unpack(f2sub(fp2, *reinterpret_cast<const unsigned long long *>(&w_hdr[j].h0.x)), dx, dy);
                const float q = gauss_q(dx, dy, h0.z, h0.w, h1.x);
                bool contrib = false;
                float al = 0.0f, raw = 0.0f;
                if (k < lastk) {  // the forward's tests, in the same order
                    const float e2 = fmaf(q, LOG2E, h1.y);
                    if (e2 >= a.log2_alpha_min) {
                        raw = ex2(e2);
                        al = fminf(a.alpha_max, raw);
                        contrib = true;
                    }
                }
                if (!__any_sync(FULL, contrib)) continue;
                float f[CP];
                FeatIO<FT>::template load<CP>(f, w_feat + (size_t)j * CP);
                float wgt = 0.0f, d_o = 0.0f, dq = 0.0f;
                if (contrib) {
                    const float inv = __frcp_rn(1.0f - al);
                    const float Tj = T * inv;
                    unsigned long long fg2 = 0;  // even and odd channels' partial sums, packed
#pragma unroll
                    for (int c = 0; c < CP / 2; ++c) fg2 = f2fma(f2pack(f[2 * c], f[2 * c + 1]), g2[c], fg2);
                    float fge, fgo;
                    f2unpack(fg2, fge, fgo);
                    const float fg = fge + fgo;
                    wgt = al * Tj;
                    const float dal = Tj * fg - sg * inv + gA * Tfin * inv;
                    sg = fmaf(wgt, fg, sg);
                    T = Tj;
                    if (raw < a.alpha_max) {
                        d_o = ex2(q * LOG2E) * dal;  // d alpha / d o = e^q
                        dq = al * dal;
                    }
                }
                const uint32_t id = w_id[j];
                if (a.d_feat) {  // collect w for the group's tensor-core product
                    const __nv_bfloat16 wh = __float2bfloat16_rn(wgt);
                    BG.wh[warp][lane][gs] = wh;
                    BG.wl[warp][lane][gs] = __float2bfloat16_rn(wgt - __bfloat162float(wh));
                    if (lane == 0) BG.gid[warp][gs] = id;
                    if (++gs == 16) {
                        flush_feat_grads<CP>(BG, warp, lane, 16, a.C, a.d_feat);
                        gs = 0;
                    }
                }
                const float ca = -2.0f * h0.z, cb = -h0.w, cc = -2.0f * h1.x;  // conic from the record
                float gv[8] = {d_o, dq * (ca * dx + cb * dy), dq * (cb * dx + cc * dy), dq * (-0.5f * dx * dx),
                               dq * (-dx * dy), dq * (-0.5f * dy * dy), 0.0f, 0.0f};
                warp_transpose_sum<8>(gv, lane);
                if ((lane & 3) == 0) {  // lane 4k holds value k: opacity, mean x, y, conic a, b, c
                    const int k = lane >> 2;
                    float *dst = nullptr;
                    if (k == 0) dst = a.d_opac ? a.d_opac + id : nullptr;
                    else if (k <= 2) dst = a.d_mean2d ? a.d_mean2d + 2 * (size_t)id + (k - 1) : nullptr;
                    else if (k <= 5) dst = a.d_conic ? a.d_conic + 3 * (size_t)id + (k - 3) : nullptr;
                    if (dst) atomicAdd(dst, gv[0]);
                }
            }
        }
    }
    if (gs > 0) flush_feat_grads<CP>(BG, warp, lane, gs, a.C, a.d_feat);
    }
}

template <int CP, typename FT>
void run_backward(const BackwardArgs &a, cudaStream_t s) {
    const size_t smem = CT * sizeof(Header) + (size_t)CT * CP * sizeof(FT) + sizeof(BwdGroup<CP>);
    static PerDevice cache;
    const int grid = cache.get([smem](int) {
        cudaFuncSetAttribute(k_backward<CP, FT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        int per_sm = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_backward<CP, FT>, CT, smem);
        return sm_count() * std::max(1, per_sm);
    });
    k_backward<CP, FT><<<std::min(grid, std::max(1, a.tiles_x * a.tiles_y)), CT, smem, s>>>(a);
    note_launches(1);
}

}  // namespace

void launch_backward(const BackwardArgs &a, cudaStream_t s) {
    if (a.tiles_x * a.tiles_y == 0) return;
    const bool bf = a.feat_dtype == TSPLAT_BF16;
    if (a.C <= 8) { if (bf) run_backward<8, __nv_bfloat16>(a, s); else run_backward<8, float>(a, s); }
    else if (a.C <= 16) { if (bf) run_backward<16, __nv_bfloat16>(a, s); else run_backward<16, float>(a, s); }
    else if (a.C <= 32) { if (bf) run_backward<32, __nv_bfloat16>(a, s); else run_backward<32, float>(a, s); }
    else { if (bf) run_backward<64, __nv_bfloat16>(a, s); else run_backward<64, float>(a, s); }
}

}  // namespace tsp
