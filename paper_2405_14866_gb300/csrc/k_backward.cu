// A8: adjoint of the front-to-back compositing (Tele-Aloha Sec. 4.2: the
// rasterizer is differentiated end to end).  Persistent warps take
// (tile, 8x4 pixel block) units from a counter; each walks its pixels' list
// range back to front from their last blended Gaussian, recomputing the
// transmittance in front of each Gaussian by division from the saved final
// one, and repeats the forward's blend decisions with the forward's
// arithmetic, so the contributor set is the forward's.
#include <algorithm>
#include <type_traits>

#include "common.cuh"
#include "internal.h"
#include "ptx.cuh"

namespace tsp {

namespace {

constexpr uint32_t FULL = 0xffffffffu;
constexpr float LOG2E = 1.4426950408889634f;

constexpr int CT = 256;

// Per-warp shared state of the gradient reductions.
//
// Feature gradients of a group of up to 16 contributing Gaussians as a
// tensor-core product: dF_j[c] = sum over the warp's 32 pixels of
// w_j(p) g_p[c], i.e. D (16 x C) = W^T (16 x 32) G (32 x C), with W and G
// split into bf16 hi + lo parts (three products, FP32 accumulation).  W^T is
// stored row per Gaussian (each lane writes its pixel's column: no bank
// conflicts), G row per pixel.
//
// Geometric gradients of a batch of MB Gaussians from per-pixel moments:
// with dq the gradient of the exponent at a pixel and (dx, dy) its offset
// from the mean, sum_p dq (a dx + b dy) = a M1 + b M2 for the mean and
// -M3/2, -M4, -M5/2 for the conic, where M1 = sum dq dx, M2 = sum dq dy,
// M3 = sum dq dx^2, M4 = sum dq dx dy, M5 = sum dq dy^2 (M0 = sum of the
// opacity terms).  The batch's 6 MB moment terms are stored column-major, a
// column of 32 pixels per term: each lane writes its pixel's entry of six
// columns (consecutive words: conflict-free), and a flush sums the columns,
// one per lane, with 16-byte loads (column stride 36 words: the eight lanes
// of a load phase fall into distinct bank groups), instead of a chain of
// shuffles per Gaussian.
constexpr int NB = 8;      // survivors per batch of the reverse walk (the n of one MMA)
constexpr int WTROW = 40;  // bf16 per W^T row (32 used; 80-byte stride spreads ldmatrix rows over the banks)
constexpr int MSTRIDE = 36;  // floats per moment column (32 used)
constexpr int FGSTRIDE = 36; // floats per <f, g> row (32 used; the stride keeps the D fragment stores free of bank conflicts)
template <int CP>
struct BwdGroup {
    static constexpr int GP = CP < 16 ? 16 : CP;  // channels padded to whole k16 / n16 blocks
    static constexpr int MB = CP <= 16 ? 5 : 2;   // Gaussians per geometric batch (6 MB columns <= 32 lanes)
    __nv_bfloat16 wth[CT / 32][16][WTROW];
    __nv_bfloat16 wtl[CT / 32][16][WTROW];
    __nv_bfloat16 gh[CT / 32][32][GP + 8];
    __nv_bfloat16 gl[CT / 32][32][GP + 8];
    uint32_t gid[CT / 32][16];
    float mom[CT / 32][6 * MB][MSTRIDE];  // per moment term of the pending batch: its 32 pixels
    float4 mrec[CT / 32][MB];              // the batch's Gaussians: conic (a, b, c) and id (bits)
    float fg[CT / 32][NB][FGSTRIDE];       // <f_j, g_p> of a survivor batch: a row of 32 pixels per survivor
};

template <int CP>
__device__ __forceinline__ void flush_feat_grads(BwdGroup<CP> &B, int warp, int lane, int cnt, int C,
                                                 float *d_feat, bool vec4) {
    constexpr int GP = BwdGroup<CP>::GP;
    for (int k = cnt; k < 16; ++k) {  // unused rows contribute nothing
        B.wth[warp][k][lane] = __float2bfloat16_rn(0.0f);
        B.wtl[warp][k][lane] = __float2bfloat16_rn(0.0f);
    }
    __syncwarp();
    float acc[GP / 8][4];
#pragma unroll
    for (int t = 0; t < GP / 8; ++t)
#pragma unroll
        for (int e = 0; e < 4; ++e) acc[t][e] = 0.0f;
    const int kl = ((lane >> 3) & 1) * 8 + (lane & 7);        // B: pixel row this lane addresses
    const int arow = ((lane >> 3) & 1) * 8 + (lane & 7);      // A: Gaussian row this lane addresses
    const int acol = (lane >> 4) * 8, bcol = (lane >> 4) * 8;
#pragma unroll
    for (int ks = 0; ks < 2; ++ks) {  // two k-steps of 16 pixels
        uint32_t ah[4], al[4];
        ldsm_x4(ah[0], ah[1], ah[2], ah[3], &B.wth[warp][arow][ks * 16 + acol]);
        ldsm_x4(al[0], al[1], al[2], al[3], &B.wtl[warp][arow][ks * 16 + acol]);
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
    if (vec4) {
        // lanes 2i and 2i + 1 swap halves: the even lane then holds four
        // consecutive channels of row lane/4, the odd lane those of row
        // lane/4 + 8, each added by one 16-byte atomic
        const bool odd = lane & 1;
        const int j = (lane >> 2) + (odd ? 8 : 0);
#pragma unroll
        for (int t = 0; t < GP / 8; ++t) {
            const float sx = odd ? acc[t][0] : acc[t][2], sy = odd ? acc[t][1] : acc[t][3];
            const float rx = __shfl_xor_sync(FULL, sx, 1), ry = __shfl_xor_sync(FULL, sy, 1);
            const float4 v = odd ? make_float4(rx, ry, acc[t][2], acc[t][3]) : make_float4(acc[t][0], acc[t][1], rx, ry);
            const int c = t * 8 + 4 * ((lane >> 1) & 1);
            if (j < cnt && c < C) atomicAdd(reinterpret_cast<float4 *>(&d_feat[(size_t)B.gid[warp][j] * C + c]), v);
        }
    } else {
#pragma unroll
        for (int t = 0; t < GP / 8; ++t)
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const int j = (lane >> 2) + ((e >> 1) << 3), c = t * 8 + 2 * (lane & 3) + (e & 1);
                if (j < cnt && c < C) atomicAdd(&d_feat[(size_t)B.gid[warp][j] * C + c], acc[t][e]);
            }
    }
    __syncwarp();
}

// Geometric gradients of the nb pending Gaussians: lane 6 g + k sums moment
// column k of Gaussian g over the 32 pixels and adds its gradient (k = 0:
// opacity; 1, 2: mean x, y; 3, 4, 5: conic a, b, c).
template <int CP>
__device__ __forceinline__ void flush_geo_grads(BwdGroup<CP> &B, int warp, int lane, int nb, const BackwardArgs &a) {
    __syncwarp();
    const int col = lane < 6 * nb ? lane : 0;
    // pixels p = 4 i + r summed per r in pixel order, two r at a time
    const float4 *cv = reinterpret_cast<const float4 *>(&B.mom[warp][col][0]);
    float4 v = cv[0];
    unsigned long long s01 = f2pack(v.x, v.y), s23 = f2pack(v.z, v.w);
#pragma unroll
    for (int i = 1; i < 8; ++i) {
        v = cv[i];
        s01 = f2add(s01, f2pack(v.x, v.y));
        s23 = f2add(s23, f2pack(v.z, v.w));
    }
    float s0, s1, s2, s3;
    f2unpack(s01, s0, s1);
    f2unpack(s23, s2, s3);
    const float S = (s0 + s1) + (s2 + s3);
    // mean x needs M2 of the next lane, mean y M1 of the previous one
    const float next = __shfl_down_sync(FULL, S, 1), prev = __shfl_up_sync(FULL, S, 1);
    if (lane < 6 * nb) {
        const int g = lane / 6, k = lane - 6 * g;
        const float4 r = B.mrec[warp][g];
        const size_t id = __float_as_uint(r.w);
        const float v = k == 0 ? S
                      : k == 1 ? fmaf(r.x, S, r.y * next)
                      : k == 2 ? fmaf(r.y, prev, r.z * S)
                      : k == 4 ? -S
                               : -0.5f * S;
        float *dst = k == 0 ? (a.d_opac ? a.d_opac + id : nullptr)
                   : k <= 2 ? (a.d_mean2d ? a.d_mean2d + 2 * id + (k - 1) : nullptr)
                            : (a.d_conic ? a.d_conic + 3 * id + (k - 3) : nullptr);
        if (dst) atomicAdd(dst, v);
    }
    __syncwarp();
}

// A8: reverse traversal from each pixel's last blended Gaussian, with the
// transmittance in front of each Gaussian recomputed by division from the
// saved final transmittance.  The blend decisions repeat the forward's
// arithmetic exactly (same instructions), so the contributor set is the
// forward's.
//
// The box survivors of a staged chunk are taken in batches of NB, back to
// front.  Per batch: <f_j, g_p> for the warp's 32 pixels and the NB
// Gaussians as one tensor-core product G (32 x GP) F^T (GP x NB) on bf16
// hi + lo parts (feature rows staged as bf16 rows: BF16 features as stored,
// FP32 features as the split (hi, lo) rows the forward reads); then each
// lane's terms of the NB Gaussians, which are independent of one another;
// then the two recurrences that are not (the transmittance T and the
// suffix <S, g>), one multiply and one FMA per Gaussian.
// Staged feature rows keep their 16-byte chunks XOR-permuted by the row, so
// that the eight rows one ldmatrix phase reads (a batch's survivors, mostly
// consecutive entries) fall into distinct bank groups whatever the row
// length: chunk c of row r sits at chunk c ^ row_swz<NCH>(r).
template <int NCH>
__device__ __forceinline__ int row_swz(int r) {
    return NCH >= 8 ? (r & 7) : ((r / (8 / NCH)) & (NCH - 1));
}

// 1 / x with the hardware approximation (rcp.approx, relative error ~2^-23)
__device__ __forceinline__ float rcp_approx(float x) {
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

template <int CP, typename FT>
__global__ __launch_bounds__(CT, 2) void k_backward(BackwardArgs a) {
    constexpr bool F32 = std::is_same<FT, float>::value;
    constexpr int GP = BwdGroup<CP>::GP;
    constexpr int RW = (F32 ? 2 : 1) * GP;  // bf16 per staged feature row: hi (then lo)
    constexpr int NCH = RW / 8;             // its 16-byte chunks
    extern __shared__ __align__(16) unsigned char smem[];
    // records staged as two arrays of 16-byte halves (h0, h1): a warp's
    // per-lane reads and writes of one half then cover consecutive words
    float4 *s_h0 = reinterpret_cast<float4 *>(smem), *s_h1 = s_h0 + CT;
    __nv_bfloat16 *s_row = reinterpret_cast<__nv_bfloat16 *>(smem + CT * sizeof(Header));
    BwdGroup<CP> &BG = *reinterpret_cast<BwdGroup<CP> *>(smem + CT * sizeof(Header) + (size_t)CT * RW * 2);
    __shared__ uint32_t s_id[CT];

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    // BF16 rows of fewer than GP channels: the padding columns stay zero
    if (!F32 && a.C < GP)
        for (int i = lane; i < 32 * RW; i += 32) s_row[(size_t)warp * 32 * RW + i] = __float2bfloat16_rn(0.0f);
    __syncwarp();
    const int n_units = a.tiles_x * a.tiles_y * 8;
    const bool bvec = !F32 && a.C == GP;  // BF16 rows of exactly GP channels: 16-byte copies
    // feature gradients by 16-byte atomics: rows of a multiple of 4 channels on a 16-byte boundary
    const bool vec4 = (a.C % 4) == 0 && (reinterpret_cast<uintptr_t>(a.d_feat) & 15u) == 0;
    const int arow = ((lane >> 3) & 1) * 8 + (lane & 7), acol = (lane >> 4) * 8;  // A fragment rows / columns
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

    float T = 1.0f, Tfin = 1.0f, gA = 0.0f;
    uint32_t lastk = 0;
    if (inside) {
        Tfin = a.T_final[pix];
        T = Tfin;
        lastk = a.last[pix];
        gA = a.dA ? a.dA[pix] : 0.0f;
    }
    // this pixel's row of G = dL/dF (hi + lo), the operand of both products,
    // written eight channels per 16-byte store
#pragma unroll
    for (int c8 = 0; c8 < GP / 8; ++c8) {
        uint32_t hw[4], lw[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const int c = 8 * c8 + 2 * e;
            const float v0 = (inside && c < a.C) ? a.dF[c * HW + pix] : 0.0f;
            const float v1 = (inside && c + 1 < a.C) ? a.dF[(c + 1) * HW + pix] : 0.0f;
            hw[e] = pack_bf16x2(v0, v1);
            lw[e] = pack_bf16x2(v0 - bf16_lo_f(hw[e]), v1 - bf16_hi_f(hw[e]));
        }
        *reinterpret_cast<uint4 *>(&BG.gh[warp][lane][8 * c8]) = make_uint4(hw[0], hw[1], hw[2], hw[3]);
        *reinterpret_cast<uint4 *>(&BG.gl[warp][lane][8 * c8]) = make_uint4(lw[0], lw[1], lw[2], lw[3]);
    }
    const unsigned long long fp2 = f2pack(fpx, fpy);
    int gs = 0;  // contributing Gaussians collected in this warp's current feature group
    int bs = 0;  // and in its current geometric batch
    const uint32_t wmax = __reduce_max_sync(FULL, lastk);
    float sg = 0.0f;  // <S, g>: blended features behind the current Gaussian
    // Each warp walks its own list range [0, wmax) back to front in chunks of
    // 32, staged into its own slice of shared memory: no block-wide barrier,
    // so a warp whose pixels stopped early does not wait for the others.
    float4 *w_h0 = s_h0 + warp * 32, *w_h1 = s_h1 + warp * 32;
    __nv_bfloat16 *w_row = s_row + (size_t)warp * 32 * RW;
    uint32_t *w_id = s_id + warp * 32;
    uint32_t nid = 0;  // ids of the next chunk, loaded one chunk ahead
    {
        const int c0 = max(0, (int)wmax - 32);
        if (c0 + lane < (int)wmax) nid = a.ids[rg.x + c0 + lane];
    }
    for (int c1 = (int)wmax; c1 > 0; c1 -= 32) {
        const int c0 = max(0, c1 - 32);
        const uint32_t gid = nid;
        if (c0 > 0) {
            const int n0 = max(0, c0 - 32);
            nid = n0 + lane < c0 ? a.ids[rg.x + n0 + lane] : 0u;
        }
        __syncwarp();
        if (c0 + lane < c1) w_id[lane] = gid;
        // records: two lanes per record (its 16-byte halves), so that the two
        // halves of a 32-byte sector are requested by one load
#pragma unroll
        for (int r = 0; r < 2; ++r) {
            const int j = 16 * r + (lane >> 1), h = lane & 1;
            const uint32_t gj = __shfl_sync(FULL, gid, j);
            if (c0 + j < c1) (h ? w_h1 : w_h0)[j] = __ldg(reinterpret_cast<const float4 *>(a.hdr + gj) + h);
        }
        // rows: NCH lanes per row, 32 / NCH rows per load (a warp's load then
        // touches 32 / NCH rows, not 32)
        if (F32 || bvec) {
            constexpr int GPI = 32 / NCH;
            const __nv_bfloat16 *rows = reinterpret_cast<const __nv_bfloat16 *>(F32 ? a.fsplit : a.feat);
#pragma unroll
            for (int r = 0; r < NCH; ++r) {
                const int j = GPI * r + lane / NCH, i = lane % NCH;
                const uint32_t gj = __shfl_sync(FULL, gid, j);
                if (c0 + j < c1)
                    reinterpret_cast<uint4 *>(w_row + (size_t)j * RW)[i ^ row_swz<NCH>(j)] =
                        __ldg(reinterpret_cast<const uint4 *>(rows + (size_t)gj * RW) + i);
            }
        } else if (c0 + lane < c1) {  // BF16 rows of fewer than GP channels: one lane per row
            __nv_bfloat16 *dst = w_row + (size_t)lane * RW;
            const __nv_bfloat16 *src = reinterpret_cast<const __nv_bfloat16 *>(a.feat) + (size_t)gid * a.C;
            for (int c = 0; c < a.C; ++c) dst[8 * ((c >> 3) ^ row_swz<NCH>(lane)) + (c & 7)] = src[c];
        }
        __syncwarp();
        bool rel = false;
        if (c0 + lane < c1) {
            const float4 h0 = w_h0[lane], h1 = w_h1[lane];
            rel = (h0.x + h1.z >= fbx0) && (h0.x - h1.z <= fbx1) && (h0.y + h1.w >= fby0) && (h0.y - h1.w <= fby1);
        }
        uint32_t m = __ballot_sync(FULL, rel);
        while (m) {
            // the next batch: up to NB survivors, highest list position first
            uint32_t mb = 0;
#pragma unroll
            for (int s = 0; s < NB; ++s)
                if (m) {
                    const uint32_t top = 1u << (31 - __clz(m));
                    mb |= top;
                    m &= ~top;
                }
            // <f_j, g_p> of the batch: D (32 px x NB) = G (32 x GP) F^T (GP x NB) on the
            // tensor cores (hi/lo parts); lane l addresses the B row of survivor l % 8
            {
                uint32_t t = mb;
                for (int i = 0; i < (lane & 7) && t; ++i) t &= ~(1u << (31 - __clz(t)));
                const int jr = t ? 31 - __clz(t) : 0;
                float d[2][4];
#pragma unroll
                for (int mt = 0; mt < 2; ++mt)
#pragma unroll
                    for (int e = 0; e < 4; ++e) d[mt][e] = 0.0f;
#pragma unroll
                for (int ks = 0; ks < GP / 16; ++ks) {
                    uint32_t bh0, bh1, bl0 = 0u, bl1 = 0u;
                    // chunk of this lane's row: hi k 0-7, 8-15 (lanes 0-15), lo k 0-7, 8-15 (lanes 16-31)
                    const int ch = 2 * ks + ((lane >> 3) & 1) + (F32 ? (lane >> 4) * (GP / 8) : 0);
                    const __nv_bfloat16 *rowp = w_row + (size_t)jr * RW + 8 * (ch ^ row_swz<NCH>(jr));
                    if (F32) ldsm_x4(bh0, bh1, bl0, bl1, rowp);
                    else ldsm_x2(bh0, bh1, rowp);
#pragma unroll
                    for (int mt = 0; mt < 2; ++mt) {
                        uint32_t ah[4], al[4];
                        ldsm_x4(ah[0], ah[1], ah[2], ah[3], &BG.gh[warp][mt * 16 + arow][ks * 16 + acol]);
                        ldsm_x4(al[0], al[1], al[2], al[3], &BG.gl[warp][mt * 16 + arow][ks * 16 + acol]);
                        mma_bf16(d[mt], ah[0], ah[1], ah[2], ah[3], bh0, bh1);
                        mma_bf16(d[mt], al[0], al[1], al[2], al[3], bh0, bh1);
                        if (F32) mma_bf16(d[mt], ah[0], ah[1], ah[2], ah[3], bl0, bl1);
                    }
                }
                // D fragment: pixel rows 16 mt + lane/4 (+8), survivor columns 2(lane%4) (+1),
                // stored survivor-major so that each survivor's step reads its row by lane
#pragma unroll
                for (int mt = 0; mt < 2; ++mt)
#pragma unroll
                    for (int hh = 0; hh < 2; ++hh)
#pragma unroll
                        for (int e = 0; e < 2; ++e)
                            BG.fg[warp][2 * (lane & 3) + e][mt * 16 + hh * 8 + (lane >> 2)] = d[mt][2 * hh + e];
                __syncwarp();
            }
            for (int s = 0; mb; ++s) {
                const int j = 31 - __clz(mb);  // highest first: back to front
                mb &= ~(1u << j);
                const uint32_t k = (uint32_t)(c0 + j);
                const float4 h0 = w_h0[j];
                const float4 h1 = w_h1[j];
                float dx, dy;
                f2unpack(f2sub(fp2, f2pack(h0.x, h0.y)), dx, dy);
                const float q = gauss_q(dx, dy, h0.z, h0.w, h1.x);
                // the forward's tests, in the same order
                const float e2 = fmaf(q, LOG2E, h1.y);
                const bool contrib = k < lastk && e2 >= a.log2_alpha_min;
                if (!__any_sync(FULL, contrib)) continue;
                const float raw = ex2(e2);
                const float al = contrib ? fminf(a.alpha_max, raw) : 0.0f;
                // a lane that does not blend this Gaussian has al = 0: inv = 1 and
                // wgt = 0, so its T and sg stay as they are
                const float inv = rcp_approx(1.0f - al);
                const float fg = BG.fg[warp][s][lane];
                const float Tj = T * inv;
                const float wgt = al * Tj;
                const float dal = Tj * fg - sg * inv + gA * Tfin * inv;
                sg = fmaf(wgt, fg, sg);
                T = Tj;
                // a clamped alpha (= alpha_max) passes no gradient to o or q
                const bool g_ok = contrib && raw < a.alpha_max;
                const float d_o = g_ok ? ex2(q * LOG2E) * dal : 0.0f;  // d alpha / d o = e^q
                const float dq = g_ok ? al * dal : 0.0f;
                const uint32_t id = w_id[j];
                if (a.d_feat) {  // collect w for the group's tensor-core product
                    const __nv_bfloat16 wh = __float2bfloat16_rn(wgt);
                    BG.wth[warp][gs][lane] = wh;
                    BG.wtl[warp][gs][lane] = __float2bfloat16_rn(wgt - __bfloat162float(wh));
                    if (lane == 0) BG.gid[warp][gs] = id;
                    if (++gs == 16) {
                        flush_feat_grads<CP>(BG, warp, lane, 16, a.C, a.d_feat, vec4);
                        gs = 0;
                    }
                }
                // this pixel's moment terms (zero where it does not contribute)
                float *mm = &BG.mom[warp][6 * bs][lane];
                const float m1 = dq * dx, m2 = dq * dy;
                mm[0 * MSTRIDE] = d_o;
                mm[1 * MSTRIDE] = m1;
                mm[2 * MSTRIDE] = m2;
                mm[3 * MSTRIDE] = m1 * dx;
                mm[4 * MSTRIDE] = m1 * dy;
                mm[5 * MSTRIDE] = m2 * dy;
                if (lane == 0)  // the conic (a, b, c) from the record, and the id
                    BG.mrec[warp][bs] = make_float4(-2.0f * h0.z, -h0.w, -2.0f * h1.x, __uint_as_float(id));
                if (++bs == BwdGroup<CP>::MB) {
                    flush_geo_grads<CP>(BG, warp, lane, bs, a);
                    bs = 0;
                }
            }
            __syncwarp();  // the batch's <f, g> tile is read before the next batch rewrites it
        }
    }
    if (gs > 0) flush_feat_grads<CP>(BG, warp, lane, gs, a.C, a.d_feat, vec4);
    if (bs > 0) flush_geo_grads<CP>(BG, warp, lane, bs, a);
    }
}

template <int CP, typename FT>
void run_backward(const BackwardArgs &a, cudaStream_t s) {
    const size_t smem = CT * sizeof(Header) + (size_t)CT * (std::is_same<FT, float>::value ? 2 : 1) * BwdGroup<CP>::GP * 2 +
                        sizeof(BwdGroup<CP>);
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
