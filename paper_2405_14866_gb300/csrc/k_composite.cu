// A7: front-to-back alpha compositing of C-channel latent features per
// 16x16 tile (Tele-Aloha Sec. 4.2: the rasterizer splats latent features
// instead of colours; the adjoint is in k_backward.cu).
//
// Persistent CTAs take tiles from a counter.  Per tile: 8 consumer warps,
// each owning an 8x4 pixel block, and 1 producer warp.  The producer
// streams the tile's depth-ordered
// Gaussians through a ring of shared-memory slots (128 Gaussians each with
// BF16 features, 64 with FP32),
// gathering each Gaussian's 32-byte projected record and feature row with
// 16-byte asynchronous copies (cp.async; adjacent lanes copy adjacent chunks
// of one record or row) whose completion arrives on the slot's mbarrier;
// consumer warps advance at their own pace and release slots, so no CTA-wide
// barrier couples them.  (Gathers through the TMA
// engine measured slower for these 32- and 64-byte rows: one bulk copy per
// row, and tensor-map gathers of four rows per instruction alike.)  The ids
// of the next two slots are loaded ahead.
//
// Per slot a warp tests the slot's records against its block with each
// Gaussian's alpha_min box (exact: outside it alpha < alpha_min, so skipping
// is what the per-pixel test would do) and walks the survivors in order.
// Each lane runs the per-pixel recurrence (alpha, T, stop) and produces the
// blending weight w = alpha T; groups of 16 weights are applied to the
// features as a warp-level bf16 tensor-core product
//     F(32 px x C) += W(32 px x 16) * Feat(16 x C),
// with W split into bf16 hi + lo parts (and FP32 features likewise), so the
// product keeps ~2^-16 relative precision with FP32 accumulation.  A warp
// stops when all its pixels are saturated; the producer stops when all
// warps have.
#include <algorithm>

#include "common.cuh"
#include "internal.h"
#include "ptx.cuh"

namespace tsp {

namespace {

constexpr uint32_t FULL = 0xffffffffu;
constexpr float LOG2E = 1.4426950408889634f;

constexpr int NCW = 8;               // consumer warps
constexpr int NTHR = (NCW + 1) * 32; // + 1 producer warp
// Gaussians per ring slot: 128 with BF16 rows (fewer slots per tile, so
// less per-slot work and less padding of the survivor groups; 0.334 ->
// 0.309 ms on the 1024x1024 headline against 64), 64 with FP32 features,
// whose split rows take twice the space (a ring of two 128-slots measured
// slower than six 64-slots)
template <bool F32F>
struct Slot {
    static constexpr int SB = F32F ? 64 : 128;
    static constexpr int NQ = SB / 32;  // entries per lane in the producer's and the box test's loops
};
constexpr int WROW = 24;             // bf16 per W row (16 used; 48-byte stride avoids bank conflicts)

// Ring slots: as deep as two CTAs per SM allow (the ring is the slack that
// lets a warp with little work in a slot run ahead of the slowest one).
template <int CP, bool F32F>
struct Ring {
    static constexpr int N = F32F ? (CP <= 16 ? 8 : (CP <= 32 ? 6 : 3)) : (CP <= 32 ? 4 : 2);
};

constexpr uint32_t FINAL_TILE = 0xffffffffu;  // slot tile id of the last slot a CTA produces

// Two consecutive survivors' records, interleaved so that one 64-bit
// register holds a field of both: a = (mx0, mx1, my0, my1), b = (-a/2 x2,
// -b x2), c = (-c/2 x2, log2 o x2).
struct RecPair {
    float4 a, b, c;
};

template <int CP, bool F32F>
struct CompSmem {
    static constexpr int RING = Ring<CP, F32F>::N;
    static constexpr int SB = Slot<F32F>::SB;
    Header hdr[RING][SB + 1];  // entry SB of each slot: an empty record (alpha = 0 everywhere)
    __nv_bfloat16 fhi[RING][SB][CP + 8];  // rows padded by 16 B: spreads ldmatrix row reads over the banks
    __nv_bfloat16 flo[F32F ? RING : 1][F32F ? SB : 1][CP + 8];
    __nv_bfloat16 whi[NCW][32][WROW];
    __nv_bfloat16 wlo[NCW][32][WROW];
    __nv_bfloat16 zero[CP];
    uint64_t full[RING];
    uint64_t empty[RING];
    uint32_t cnt[RING];        // Gaussians in the slot; 0 marks the end of a tile (or of the CTA's work)
    uint32_t tile[RING];       // tile the slot belongs to, FINAL_TILE after the last tile
    uint32_t base[RING];       // list position of the slot's first Gaussian
    int32_t done_seq[NCW];     // per consumer warp: sequence number of the last tile it is done with
    uint8_t list[NCW][SB];     // per consumer warp: slot indices of its surviving Gaussians, in order
    RecPair wpair[NCW][SB / 2];  // per consumer warp: the survivors' records, compacted in pairs
    RenderView views[MAX_BATCH];
};

// Entry k of a slot keeps h0 in its first 16 bytes and h1 in its second,
// swapped when (k >> 2) is odd: the h0 (or h1) halves of eight consecutive
// entries then fall into eight distinct groups of four banks, so a warp's
// 16-byte reads of one half per lane are free of bank conflicts.
__device__ __forceinline__ int hsw(int k) { return (k >> 2) & 1; }
__device__ __forceinline__ float4 *hdr_h0(Header *slot_hdr, int k) {
    return reinterpret_cast<float4 *>(slot_hdr + k) + hsw(k);
}
__device__ __forceinline__ float4 *hdr_h1(Header *slot_hdr, int k) {
    return reinterpret_cast<float4 *>(slot_hdr + k) + (1 - hsw(k));
}

__device__ __forceinline__ void cp_async16(void *dst, const void *src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}

// Producer side of one Gaussian of a slot with BF16 rows of fewer than CP
// channels: its record by two 16-byte asynchronous copies, its feature row
// loaded and zero-padded by the producer lane itself.
template <int CP, bool F32F>
__device__ __forceinline__ void produce_one_padded(CompSmem<CP, F32F> &S, const CompositeArgs &a, int slot, int k,
                                                   uint32_t id, uint32_t ns) {
    const uint4 *hs = reinterpret_cast<const uint4 *>(a.hdr + id);
    cp_async16(hdr_h0(S.hdr[slot], k), hs);
    cp_async16(hdr_h1(S.hdr[slot], k), hs + 1);
    const size_t gi = id % ns;  // features are stored once per Gaussian, records per (view, Gaussian)
    const __nv_bfloat16 *src = reinterpret_cast<const __nv_bfloat16 *>(a.feat) + gi * a.C;
    for (int c = 0; c < CP; ++c) S.fhi[slot][k][c] = c < a.C ? src[c] : __float2bfloat16_rn(0.0f);
}

// Producer side of 32 Gaussians of a slot (entries k0 .. k0 + 31, id of
// entry k0 + j held by lane j): records and feature rows -- BF16 rows of
// exactly CP channels as stored, FP32 rows as their pre-split bf16 (hi, lo)
// rows of CP columns each (zero-padded) -- by 16-byte asynchronous copies,
// made chunk-cooperatively: two lanes per record (its two halves) and RC
// lanes per row, so that the lanes of one copy instruction that share a
// 32-byte sector request it once (one lane per Gaussian measured 1 % slower
// on BF16 rows and 4 % on FP32 rows).
template <int CP, bool F32F>
__device__ __forceinline__ void produce_group(CompSmem<CP, F32F> &S, const CompositeArgs &a, int slot, int k0,
                                              int cnt, uint32_t id, uint32_t ns, int lane) {
    const uint32_t gi = id % ns;  // features are stored once per Gaussian, records per (view, Gaussian)
#pragma unroll
    for (int r = 0; r < 2; ++r) {
        const int j = 16 * r + (lane >> 1), h = lane & 1;
        const uint32_t idj = __shfl_sync(FULL, id, j);
        const int k = k0 + j;
        if (k < cnt)
            cp_async16(h ? hdr_h1(S.hdr[slot], k) : hdr_h0(S.hdr[slot], k),
                       reinterpret_cast<const uint4 *>(a.hdr + idj) + h);
    }
    constexpr int NC = CP / 8;
    constexpr int RC = (F32F ? 2 : 1) * NC;
    constexpr int GPI = 32 / RC;
    const __nv_bfloat16 *rows = reinterpret_cast<const __nv_bfloat16 *>(F32F ? a.fsplit : a.feat);
#pragma unroll
    for (int r = 0; r < RC; ++r) {
        const int j = GPI * r + lane / RC, c = lane % RC;
        const uint32_t gj = __shfl_sync(FULL, gi, j);
        const int k = k0 + j;
        if (k < cnt) {
            const uint4 *fs = reinterpret_cast<const uint4 *>(rows + (size_t)gj * (RC * 8));
            __nv_bfloat16 *dst = (!F32F || c < NC) ? &S.fhi[slot][k][8 * c]
                                                   : &S.flo[F32F ? slot : 0][F32F ? k : 0][8 * (c - NC)];
            cp_async16(dst, fs + c);
        }
    }
}

// The producer warp takes tiles from the grid-wide counter until none are
// left and streams each tile's list through the ring, followed by an
// end-of-tile slot; a final slot tells the consumers to leave.  The full
// barrier of a slot expects one regular arrival (lane 0, after the slot's
// metadata is written) plus, per producer lane, the asynchronous arrival that
// fires once that lane's copies have landed.  A tile whose consumer warps
// are all saturated is cut short.
template <int CP, bool F32F>
__device__ void producer(CompSmem<CP, F32F> &S, const CompositeArgs &a, int lane) {
    constexpr int RING = CompSmem<CP, F32F>::RING;
    constexpr int SB = Slot<F32F>::SB, NQ = Slot<F32F>::NQ;
    // the tile count comes from the view table in device memory, so a replayed
    // graph may render a different mix of view sizes
    const RenderView &lastv = S.views[a.n_views - 1];
    const uint32_t n_tiles = lastv.tile_base + (uint32_t)(lastv.tiles_x * lastv.tiles_y);
    const uint32_t ns = *a.n_stride;
    uint32_t i = 0;  // slots produced so far (ring position and phase)
    bool timed_out = false;
    for (int32_t seq = 0;; ++seq) {
        uint32_t tk = 0;
        if (lane == 0) tk = atomicAdd(a.tile_counter, 1u);
        tk = __shfl_sync(FULL, tk, 0);
        const bool last_tile = tk >= n_tiles;
        // the scan's table: tile and list range of each ticket in one load
        const uint4 info = last_tile ? make_uint4(0u, 0u, 0u, 0u) : a.tile_info[tk];
        const uint32_t t = info.x, first = info.y;
        const int n = (int)(info.z - info.y);
        // ids of the next two slots' Gaussians (NQ per lane each), loaded ahead
        uint32_t nid[NQ], mid[NQ];
#pragma unroll
        for (int q = 0; q < NQ; ++q) {
            nid[q] = lane + 32 * q < n ? a.ids[first + lane + 32 * q] : 0u;
            mid[q] = SB + lane + 32 * q < n ? a.ids[first + SB + lane + 32 * q] : 0u;
        }
        for (int b = 0;; b += SB, ++i) {
            const int slot = (int)(i % RING);
            if (!mbar_wait(&S.empty[slot], ((i / RING) & 1) ^ 1, a.status)) {
                timed_out = true;
                break;
            }
            bool all_done = true;
#pragma unroll
            for (int w = 0; w < NCW; ++w) all_done &= *reinterpret_cast<volatile int32_t *>(&S.done_seq[w]) >= seq;
            const bool end = last_tile || b >= n || all_done;
            const int cnt = end ? 0 : min(SB, n - b);
            if (!end) {
                uint32_t id[NQ];
                const int nb = b + 2 * SB;
#pragma unroll
                for (int q = 0; q < NQ; ++q) {
                    id[q] = nid[q];
                    nid[q] = mid[q];
                    mid[q] = nb + lane + 32 * q < n ? a.ids[first + nb + lane + 32 * q] : 0u;
                }
                if (F32F || a.C == CP) {  // rows of exactly CP columns: chunk-cooperative copies
#pragma unroll
                    for (int q = 0; q < NQ; ++q) produce_group<CP, F32F>(S, a, slot, 32 * q, cnt, id[q], ns, lane);
                } else {
#pragma unroll
                    for (int q = 0; q < NQ; ++q)
                        if (lane + 32 * q < cnt) produce_one_padded<CP, F32F>(S, a, slot, lane + 32 * q, id[q], ns);
                }
            }
            // every lane, every slot: counts against the barrier's expected
            // arrivals (.noinc) and fires once this lane's copies have landed
            asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];" ::"r"(smem_u32(&S.full[slot])) : "memory");
            __syncwarp();
            if (lane == 0) {
                S.cnt[slot] = cnt;
                S.tile[slot] = last_tile ? FINAL_TILE : t;
                S.base[slot] = b;
                mbar_arrive(&S.full[slot]);
            }
            if (end) {
                ++i;
                break;
            }
        }
        if (timed_out || last_tile) break;
    }
    if (timed_out) {
        set_status(a.status, TSPLAT_ERR_TIMEOUT);
        asm volatile("cp.async.wait_all;" ::: "memory");  // copies already issued land before the CTA exits
    }
}

// The record's alpha_min box (mean2d +- (ex, ey)) meets [bx0, bx1] x [by0, by1]:
// x and y of each bound by one packed addition or subtraction.
__device__ __forceinline__ bool box_hit(Header *slot_hdr, int k, float bx0, float bx1, float by0, float by1) {
    const ulonglong2 p0 = *reinterpret_cast<const ulonglong2 *>(hdr_h0(slot_hdr, k));  // (mx, my), (-a/2, -b)
    const ulonglong2 p1 = *reinterpret_cast<const ulonglong2 *>(hdr_h1(slot_hdr, k));  // (-c/2, log2 o), (ex, ey)
    const unsigned long long mu = p0.x, ext = p1.y;
    float hx, hy, lx, ly;
    f2unpack(f2add(mu, ext), hx, hy);
    f2unpack(f2sub(mu, ext), lx, ly);
    return (hx >= bx0) && (lx <= bx1) && (hy >= by0) && (ly <= by1);
}

// Persistent: gridDim.x CTAs (a few per SM) share the tiles through
// a.tile_counter, which must be 0 at launch.
// SAVE: track each pixel's last blended list position (for the backward).
template <int CP, bool F32F, bool SAVE>
__global__ __launch_bounds__(NTHR, 2) void k_composite(CompositeArgs a) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    CompSmem<CP, F32F> &S = *reinterpret_cast<CompSmem<CP, F32F> *>(smem_raw);
    constexpr int NT8 = CP / 8;  // n8 tiles of the MMA
    constexpr int RING = CompSmem<CP, F32F>::RING;
    constexpr int SB = Slot<F32F>::SB, NQ = Slot<F32F>::NQ;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (tid == 0) {
        for (int r = 0; r < RING; ++r) {
            mbar_init(&S.full[r], 1 + 32);  // lane 0's arrival + one asynchronous arrival per producer lane
            mbar_init(&S.empty[r], NCW);
            *hdr_h0(S.hdr[r], SB) = make_float4(0.f, 0.f, 0.f, 0.f);
            *hdr_h1(S.hdr[r], SB) = make_float4(0.f, -INFINITY, -INFINITY, -INFINITY);
        }
        mbar_init_fence();
    }
    if (tid < NCW) S.done_seq[tid] = -1;
    if (tid < a.n_views) S.views[tid] = a.views[tid];
    for (int c = tid; c < CP; c += NTHR) S.zero[c] = __float2bfloat16_rn(0.0f);
    __syncthreads();

    if (warp == NCW) {
        producer<CP, F32F>(S, a, lane);
        return;
    }

    // ---------------------------------------------------------- consumers
    const float amax = a.alpha_max, l2min = a.log2_alpha_min, tmin = a.t_min;
    // ldmatrix address pattern: lane supplies row (lane & 7) of matrix lane / 8
    const int kl = ((lane >> 3) & 1) * 8 + (lane & 7);  // group entry whose B row this lane addresses
    const int arow = kl, acol = (lane >> 4) * 8, bcol = (lane >> 4) * 8;
    const uint32_t lt = (1u << lane) - 1u;

    float acc[2][NT8][4];
    float T = 1.0f;
    uint32_t last = 0;
    bool done = true, wdone = true;
    int bx0 = 0, by0 = 0;          // this warp's 8x4 block in the current tile
    int cv = 0, W = 0, H = 0;      // view of the current tile and its size
    unsigned long long fpx2 = 0, fpy2 = 0;  // this lane's pixel centre, x and y in both halves
    const unsigned long long log2e2 = f2pack(LOG2E, LOG2E);
    uint32_t cur = FINAL_TILE;     // tile in progress
    int32_t seq = -1;

    for (uint32_t i = 0;; ++i) {
        const int slot = (int)(i % RING);
        if (!mbar_wait(&S.full[slot], (i / RING) & 1, a.status)) {
            set_status(a.status, TSPLAT_ERR_TIMEOUT);
            break;
        }
        const uint32_t t = S.tile[slot];
        const int cnt = (int)S.cnt[slot];
        if (t == FINAL_TILE) break;
        if (t != cur) {  // first slot of a new tile: reset the per-pixel state
            cur = t;
            ++seq;
            cv = 0;
            for (int k = 1; k < a.n_views; ++k) cv = t >= S.views[k].tile_base ? k : cv;
            const uint32_t local = t - S.views[cv].tile_base;
            W = S.views[cv].width;
            H = S.views[cv].height;
            const int tx = (int)(local % (uint32_t)S.views[cv].tiles_x), ty = (int)(local / (uint32_t)S.views[cv].tiles_x);
            bx0 = tx * TILE + (warp & 1) * 8;
            by0 = ty * TILE + (warp >> 1) * 4;
            const float fpx = (float)(bx0 + (lane & 7)), fpy = (float)(by0 + (lane >> 3));
            fpx2 = f2pack(fpx, fpx);
            fpy2 = f2pack(fpy, fpy);
#pragma unroll
            for (int m = 0; m < 2; ++m)
#pragma unroll
                for (int u = 0; u < NT8; ++u)
#pragma unroll
                    for (int e = 0; e < 4; ++e) acc[m][u][e] = 0.0f;
            T = 1.0f;
            last = 0;
            done = !(bx0 + (lane & 7) < W && by0 + (lane >> 3) < H);
            wdone = __all_sync(FULL, done);
            if (wdone && lane == 0) *reinterpret_cast<volatile int32_t *>(&S.done_seq[warp]) = seq;
        }
        if (cnt == 0) {
            // end of the tile: write this warp's block (the accumulator of lane l
            // holds pixels l/4 (+8, +16, +24) and channels 8u + 2(l%4) (+1))
            const RenderView &vw = S.views[cv];
            const size_t HW = (size_t)W * H;
#pragma unroll
            for (int m = 0; m < 2; ++m)
#pragma unroll
                for (int hh = 0; hh < 2; ++hh) {
                    const int p = m * 16 + hh * 8 + (lane >> 2);
                    const int x = bx0 + (p & 7), y = by0 + (p >> 3);
                    if (x < W && y < H) {
                        float *dst = vw.out_feat + (size_t)y * W + x;
#pragma unroll
                        for (int u = 0; u < NT8; ++u) {
                            const int c = u * 8 + 2 * (lane & 3);
                            if (c < a.C) dst[c * HW] = acc[m][u][2 * hh];
                            if (c + 1 < a.C) dst[(c + 1) * HW] = acc[m][u][2 * hh + 1];
                        }
                    }
                }
            const int px = bx0 + (lane & 7), py = by0 + (lane >> 3);
            if (px < W && py < H) {
                const size_t pix = (size_t)py * W + px;
                if (vw.out_alpha) vw.out_alpha[pix] = 1.0f - T;
                if (vw.out_T) vw.out_T[pix] = T;
                if (SAVE && vw.out_last) vw.out_last[pix] = last;
            }
            if (lane == 0) *reinterpret_cast<volatile int32_t *>(&S.done_seq[warp]) = seq;
            cur = FINAL_TILE;
        } else if (!wdone) {
            const int base = (int)S.base[slot];
            // survivors of the alpha_min box test, in list order, against the
            // bounding box of the block's pixels that are still blending (a
            // Gaussian that reaches only saturated pixels changes nothing)
            const uint32_t live = __ballot_sync(FULL, !done);  // bit 8 r + c: pixel (c, r) of the block
            const uint32_t rows = ((live & 0xffu) ? 1u : 0u) | ((live & 0xff00u) ? 2u : 0u) |
                                  ((live & 0xff0000u) ? 4u : 0u) | ((live & 0xff000000u) ? 8u : 0u);
            const uint32_t cols = (live | (live >> 8) | (live >> 16) | (live >> 24)) & 0xffu;
            const float fbx0 = (float)(bx0 + __ffs(cols) - 1), fbx1 = (float)(bx0 + 31 - __clz(cols));
            const float fby0 = (float)(by0 + __ffs(rows) - 1), fby1 = (float)(by0 + 31 - __clz(rows));
            int nrel = 0;
#pragma unroll
            for (int q = 0; q < NQ; ++q) {
                const bool rq = lane + 32 * q < cnt && box_hit(S.hdr[slot], lane + 32 * q, fbx0, fbx1, fby0, fby1);
                const uint32_t mq = __ballot_sync(FULL, rq);
                if (rq) S.list[warp][nrel + __popc(mq & lt)] = (uint8_t)(lane + 32 * q);
                nrel += __popc(mq);
            }
            // pad the list to a multiple of 16 with the empty record
            if (lane < 16 && nrel + lane < ((nrel + 15) & ~15)) S.list[warp][nrel + lane] = (uint8_t)SB;
            __syncwarp();
            // the survivors' records, copied in order, so that the recurrence
            // reads them at fixed offsets
            for (int k = lane; k < ((nrel + 15) & ~15); k += 32) {
                const int e = S.list[warp][k];
                const float4 k0 = *hdr_h0(S.hdr[slot], e), k1 = *hdr_h1(S.hdr[slot], e);
                float *f = reinterpret_cast<float *>(&S.wpair[warp][k >> 1]) + (k & 1);
                f[0] = k0.x;
                f[2] = k0.y;
                f[4] = k0.z;
                f[6] = k0.w;
                f[8] = k1.x;
                f[10] = k1.y;
            }
            __syncwarp();
            for (int g0 = 0; g0 < nrel && !wdone; g0 += 16) {
                uint32_t wh[8], wl[8];
#pragma unroll
                for (int g4 = 0; g4 < 16; g4 += 4) {
                    if (g0 + g4 >= nrel) {  // warp-uniform: only padding left (weight 0, no state change)
                        wh[g4 / 2] = wh[g4 / 2 + 1] = wl[g4 / 2] = wl[g4 / 2 + 1] = 0u;
                        continue;
                    }
#pragma unroll
                    for (int g = g4; g < g4 + 4; g += 2) {
                        // exponents of the pair: the scalar path's operations
                        // (gauss_q, then q log2 e + log2 o), two lanes at a time
                        const RecPair &rp = S.wpair[warp][(g0 + g) >> 1];
                        const ulonglong2 pa = *reinterpret_cast<const ulonglong2 *>(&rp.a);
                        const ulonglong2 pb = *reinterpret_cast<const ulonglong2 *>(&rp.b);
                        const ulonglong2 pc = *reinterpret_cast<const ulonglong2 *>(&rp.c);
                        const unsigned long long dx = f2sub(fpx2, pa.x), dy = f2sub(fpy2, pa.y);
                        const unsigned long long tq = f2fma(pb.x, dx, f2mul(pb.y, dy));
                        const unsigned long long qq = f2fma(dx, tq, f2mul(f2mul(pc.x, dy), dy));
                        float e2v[2];
                        f2unpack(f2fma(qq, log2e2, pc.y), e2v[0], e2v[1]);
                        float w2[2];
#pragma unroll
                        for (int h = 0; h < 2; ++h) {
                            // straight-line recurrence: only T / done / last carry a
                            // dependency; padded entries are the empty record (e2 = -inf)
                            const int j = SAVE ? (int)S.list[warp][g0 + g + h] : 0;
                            const float e2 = e2v[h];
                            const float al = fminf(amax, ex2(e2));
                            // (q <= 0 for a positive-definite conic; its rounding near the
                            // centre is one of the oracle's ambiguous decisions)
                            const bool ok = !done & (e2 >= l2min);
                            const float wr = al * T;
                            const float Tn = T - wr;
                            const bool stop = ok & (Tn < tmin);
                            const bool blend = ok & !stop;
                            w2[h] = blend ? wr : 0.0f;
                            T = blend ? Tn : T;
                            if (SAVE) last = blend ? (uint32_t)(base + j + 1) : last;
                            done = done | stop;
                        }
                        wh[g / 2] = pack_bf16x2(w2[0], w2[1]);
                        wl[g / 2] = pack_bf16x2(w2[0] - bf16_lo_f(wh[g / 2]), w2[1] - bf16_hi_f(wh[g / 2]));
                    }
                }
                // this lane's row of W (pixel = lane), hi and lo parts
                uint4 *rh = reinterpret_cast<uint4 *>(&S.whi[warp][lane][0]);
                uint4 *rl = reinterpret_cast<uint4 *>(&S.wlo[warp][lane][0]);
                rh[0] = make_uint4(wh[0], wh[1], wh[2], wh[3]);
                rh[1] = make_uint4(wh[4], wh[5], wh[6], wh[7]);
                rl[0] = make_uint4(wl[0], wl[1], wl[2], wl[3]);
                rl[1] = make_uint4(wl[4], wl[5], wl[6], wl[7]);
                __syncwarp();
                uint32_t ah[2][4], aw[2][4];
#pragma unroll
                for (int m = 0; m < 2; ++m) {
                    ldsm_x4(ah[m][0], ah[m][1], ah[m][2], ah[m][3], &S.whi[warp][m * 16 + arow][acol]);
                    ldsm_x4(aw[m][0], aw[m][1], aw[m][2], aw[m][3], &S.wlo[warp][m * 16 + arow][acol]);
                }
                const int my_j = g0 + kl < nrel ? (int)S.list[warp][g0 + kl] : -1;
                const __nv_bfloat16 *browh = my_j >= 0 ? &S.fhi[slot][my_j][0] : &S.zero[0];
#pragma unroll
                for (int p = 0; p < NT8 / 2; ++p) {
                    uint32_t bb[4];
                    ldsm_x4_t(bb[0], bb[1], bb[2], bb[3], browh + p * 16 + bcol);
#pragma unroll
                    for (int m = 0; m < 2; ++m) {
                        mma_bf16(acc[m][2 * p], ah[m][0], ah[m][1], ah[m][2], ah[m][3], bb[0], bb[1]);
                        mma_bf16(acc[m][2 * p], aw[m][0], aw[m][1], aw[m][2], aw[m][3], bb[0], bb[1]);
                        mma_bf16(acc[m][2 * p + 1], ah[m][0], ah[m][1], ah[m][2], ah[m][3], bb[2], bb[3]);
                        mma_bf16(acc[m][2 * p + 1], aw[m][0], aw[m][1], aw[m][2], aw[m][3], bb[2], bb[3]);
                    }
                    if (F32F) {
                        const __nv_bfloat16 *browl =
                            my_j >= 0 ? &S.flo[F32F ? slot : 0][F32F ? my_j : 0][0] : &S.zero[0];
                        ldsm_x4_t(bb[0], bb[1], bb[2], bb[3], browl + p * 16 + bcol);
#pragma unroll
                        for (int m = 0; m < 2; ++m) {
                            mma_bf16(acc[m][2 * p], ah[m][0], ah[m][1], ah[m][2], ah[m][3], bb[0], bb[1]);
                            mma_bf16(acc[m][2 * p], aw[m][0], aw[m][1], aw[m][2], aw[m][3], bb[0], bb[1]);
                            mma_bf16(acc[m][2 * p + 1], ah[m][0], ah[m][1], ah[m][2], ah[m][3], bb[2], bb[3]);
                            mma_bf16(acc[m][2 * p + 1], aw[m][0], aw[m][1], aw[m][2], aw[m][3], bb[2], bb[3]);
                        }
                    }
                }
                __syncwarp();
                wdone = __all_sync(FULL, done);
            }
            if (wdone && lane == 0) *reinterpret_cast<volatile int32_t *>(&S.done_seq[warp]) = seq;
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(&S.empty[slot]);
    }
}

template <int CP, bool F32F, bool SAVE>
void run_composite(const CompositeArgs &a, cudaStream_t s) {
    const size_t smem = sizeof(CompSmem<CP, F32F>);
    static PerDevice cache;
    const int grid = cache.get([smem](int) {
        cudaFuncSetAttribute(k_composite<CP, F32F, SAVE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        int per_sm = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_composite<CP, F32F, SAVE>, NTHR, smem);
        return sm_count() * std::max(1, per_sm);
    });
    k_composite<CP, F32F, SAVE><<<std::min(grid, std::max(1, (int)a.n_tiles_total)), NTHR, smem, s>>>(a);
    note_launches(1);
}

}  // namespace

void launch_composite(const CompositeArgs &a, cudaStream_t s) {
    if (a.n_tiles_total == 0) return;
    const bool f32 = a.feat_dtype == TSPLAT_F32;  // then a.fsplit holds the split rows
    if (a.save) {
        if (a.C <= 16) { if (f32) run_composite<16, true, true>(a, s); else run_composite<16, false, true>(a, s); }
        else if (a.C <= 32) { if (f32) run_composite<32, true, true>(a, s); else run_composite<32, false, true>(a, s); }
        else { if (f32) run_composite<64, true, true>(a, s); else run_composite<64, false, true>(a, s); }
    } else {
        if (a.C <= 16) { if (f32) run_composite<16, true, false>(a, s); else run_composite<16, false, false>(a, s); }
        else if (a.C <= 32) { if (f32) run_composite<32, true, false>(a, s); else run_composite<32, false, false>(a, s); }
        else { if (f32) run_composite<64, true, false>(a, s); else run_composite<64, false, false>(a, s); }
    }
}

}  // namespace tsp
