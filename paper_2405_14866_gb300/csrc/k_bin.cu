// A3..A6: the (Gaussian, tile) pairs of a render ordered by (tile, depth,
// id) -- the order the cited 3DGS rasterizer (Tele-Aloha Sec. 4.2) gets from
// one stable sort of the 64-bit keys tile << 32 | bits(depth) over pairs
// emitted in Gaussian-id order -- and each tile's [first, last) range.
//
// Built from tile buckets instead of device-wide sorts:
//   1. (in the projection) every instance, in id order, walks its kept
//                         tiles; lanes of a warp that meet the same tile add
//                         their count with one atomic (match_any);
//   2. k_bin_scan         one block: exclusive scan of the tile counts: each
//                         tile's range and fill cursor, and the total P; then
//                         the tile order, longest lists first;
//   3. k_bin_fill         the same walk; each (warp, tile) group reserves a run
//                         of its tile's bucket with one atomic and writes
//                         (depth key, instance id) into it;
//   4. k_bin_sort         persistent blocks take tiles in that order and sort
//                         each bucket by (depth key, id): in shared memory,
//                         an LSD radix sort with 8-bit digits over the
//                         highest 16 (or 24) bits in which the tile's depth
//                         keys differ (its lowest pass unstable), then runs
//                         that agree on those bits put in (key, id) order
//                         (runs longer than 32: id digits, then depth digits
//                         again); buckets larger than shared memory are
//                         first split into depth slabs by a pass over global
//                         memory.
// A bucket's order after step 3 depends on the atomics; after step 5 it does
// not: (depth key, id) is unique within a tile.
#include <algorithm>

#include "bins.cuh"
#include "common.cuh"
#include "internal.h"

namespace tsp {

namespace {

constexpr uint32_t FULL = 0xffffffffu;

__device__ __forceinline__ uint32_t lanemask_lt() {
    uint32_t m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

// Exclusive scan across a block of NW warps; `sw` holds NW words.
template <int NW, typename T>
__device__ __forceinline__ T block_excl_scan(T v, T *sw, T &total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    T x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const T y = __shfl_up_sync(FULL, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) sw[warp] = x;
    __syncthreads();
    if (warp == 0) {
        T w = lane < NW ? sw[lane] : T(0);
#pragma unroll
        for (int o = 1; o < NW; o <<= 1) {
            const T y = __shfl_up_sync(FULL, w, o);
            if (lane >= o) w += y;
        }
        if (lane < NW) sw[lane] = w;
    }
    __syncthreads();
    total = sw[NW - 1];
    const T pre = warp ? sw[warp - 1] : T(0);
    __syncthreads();
    return pre + x - v;
}

// Step 3.  Warps stride over 32-instance chunks in id order; the loop over
// a chunk's tiles runs to the chunk's largest count, lanes past their own
// count sitting out.  (Step 1 runs inside the projection, which walks the
// same tiles with warp_count_tiles.)
__global__ __launch_bounds__(256) void k_bin_fill(BinArgs a) {
    const uint32_t n = *a.n_inst;
    if (blockIdx.x == 0 && threadIdx.x == 0) *a.p_eff = *a.p_dev <= a.p_cap ? *a.p_dev : 0u;
    if (*a.p_dev > a.p_cap) {
        // the pairs do not fit: nothing is written and every tile is empty
        if (blockIdx.x == 0 && threadIdx.x == 0) set_status(a.status, TSPLAT_ERR_CAPACITY);
        for (uint32_t t = blockIdx.x * blockDim.x + threadIdx.x; t < a.n_slots; t += gridDim.x * blockDim.x) {
            a.ranges[t] = make_uint2(0u, 0u);
            uint32_t *info = reinterpret_cast<uint32_t *>(a.tile_info_out + t);  // (tile, first, end, 0)
            info[1] = 0u;
            info[2] = 0u;
        }
        return;
    }
    const uint32_t ns = *a.n_stride;
    const int lane = threadIdx.x & 31;
    const uint32_t lt = lanemask_lt();
    const uint64_t wstride = (uint64_t)gridDim.x * (blockDim.x >> 5) * 32;
    for (uint64_t c0 = ((uint64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5)) * 32; c0 < n; c0 += wstride) {
        const uint64_t i = c0 + lane;
        uint32_t cnt = 0, key = 0;
        TileWalk tw;
        tw.clear();
        if (i < n) {
            cnt = a.ntiles[i];
            if (cnt) {
                int x0, y0, x1, y1;
                unpack_rect(a.rect[i], x0, y0, x1, y1);
                const RenderView &vw = a.views[a.n_views > 1 ? (uint32_t)(i / ns) : 0u];
                tw.init(vw.tile_base, vw.tiles_x, x0, y0, x1, a.tmask ? a.tmask[i] : FULL);
                key = a.dkey[i];
            }
        }
        const uint32_t maxc = __reduce_max_sync(FULL, cnt);
        for (uint32_t k = 0; k < maxc; ++k) {
            const bool act = k < cnt;
            const uint32_t am = __ballot_sync(FULL, act);
            if (act) {
                const uint32_t t = tw.next();
                const uint32_t peers = __match_any_sync(am, t);
                const int leader = __ffs(peers) - 1;
                uint32_t b = 0;
                if (lane == leader) b = atomicAdd(&a.cursor[t], (uint32_t)__popc(peers));
                b = __shfl_sync(peers, b, leader);
                const uint32_t slot = b + (uint32_t)__popc(peers & lt);
                a.bk_key[slot] = key;
                a.bk_id[slot] = (uint32_t)i;
            }
        }
    }
}

// Step 4, inside the scan kernel: tile order, longest lists first
// (largest-processing-time-first scheduling shortens the tail of the
// persistent kernels).  Tiles are bucketed by 4 log2(pair count); tiles with
// no pairs follow, then the slots beyond the views' T tiles (graph replays
// size the launch for their largest batch).  The order within a bucket
// depends on atomics, which changes no output: every tile is processed
// independently.
constexpr int TO_BUCKETS = 64;
__device__ __forceinline__ uint32_t order_bucket(uint32_t c, uint32_t t, uint32_t T) {
    if (t >= T) return TO_BUCKETS + 1;  // not a tile of this batch
    if (c == 0) return TO_BUCKETS;
    const int lg = (int)(4.0f * __log2f((float)c));
    return TO_BUCKETS - 1 - min(TO_BUCKETS - 1, max(0, lg));  // descending count
}

// Counts of 4 consecutive slots t0..t0+3 (0 past the batch's T tiles);
// one 16-byte load when all four are tiles (t0 is a multiple of 4).
__device__ __forceinline__ void load_counts4(const uint32_t *cnt, uint32_t t0, uint32_t T, uint32_t c[4]) {
    if (t0 + 4 <= T) {
        const uint4 v = *reinterpret_cast<const uint4 *>(cnt + t0);
        c[0] = v.x; c[1] = v.y; c[2] = v.z; c[3] = v.w;
    } else {
#pragma unroll
        for (int k = 0; k < 4; ++k) c[k] = t0 + k < T ? cnt[t0 + k] : 0u;
    }
}

// One block of 1024 threads, slots in chunks of 4096 (4 consecutive per
// thread).  The loop over chunks scans the counts into ranges and cursors,
// carrying the running total, and counts the tiles of each order bucket; a
// second loop over the chunks places every slot at its bucket's cursor.
// Each warp stages its 128 first offsets and counts in shared memory and
// writes ranges and cursors lane by lane (whole 32-byte sectors: one SM's
// store throughput bounds the kernel otherwise).
__global__ __launch_bounds__(1024) void k_bin_scan(BinArgs a) {
    __shared__ unsigned long long sw[32];
    __shared__ uint32_t bc[TO_BUCKETS + 2];
    __shared__ uint4 sf[1024], sc[1024];  // per thread: first offsets and counts of its 4 slots
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const RenderView &lv = a.views[a.n_views - 1];
    const uint32_t T = min(a.n_slots, lv.tile_base + (uint32_t)(lv.tiles_x * lv.tiles_y));
    if (threadIdx.x < TO_BUCKETS + 2) bc[threadIdx.x] = 0;
    unsigned long long carry = 0;
    for (uint32_t c0 = 0; c0 < a.n_slots; c0 += 4096u) {
        const uint32_t t0 = c0 + 4u * threadIdx.x;
        uint32_t c[4], f[4];
        load_counts4(a.tile_cnt, t0, T, c);
        const unsigned long long local = (unsigned long long)c[0] + c[1] + c[2] + c[3];
        unsigned long long tot;
        unsigned long long run = carry + block_excl_scan<32>(local, sw, tot);  // its barriers also order bc's zeroing
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            f[k] = (uint32_t)min(run, 0xffffffffull);
            run += c[k];
            if (t0 + k < a.n_slots) atomicAdd(&bc[order_bucket(c[k], t0 + k, T)], 1u);
        }
        sf[threadIdx.x] = make_uint4(f[0], f[1], f[2], f[3]);
        sc[threadIdx.x] = make_uint4(c[0], c[1], c[2], c[3]);
        __syncwarp();
        const uint32_t *wf = reinterpret_cast<const uint32_t *>(sf + 32 * warp);
        const uint32_t *wc = reinterpret_cast<const uint32_t *>(sc + 32 * warp);
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const uint32_t t = c0 + 128u * warp + 32u * j + lane;
            if (t < a.n_slots) {
                const uint32_t fj = wf[32 * j + lane], cj = wc[32 * j + lane];
                const uint32_t ej = (uint32_t)min((unsigned long long)fj + cj, 0xffffffffull);  // saturates as the offsets do
                a.ranges[t] = cj ? make_uint2(fj, ej) : make_uint2(0u, 0u);  // empty: [0, 0)
                a.cursor[t] = fj;
            }
        }
        __syncwarp();
        carry += tot;
    }
    if (threadIdx.x == 0) *a.p_dev = (uint32_t)min(carry, 0xffffffffull);
    __syncthreads();
    // bucket offsets: warp 0 scans the TO_BUCKETS + 2 counts, 3 per lane
    static_assert(TO_BUCKETS + 2 <= 96, "three buckets per lane");
    if (threadIdx.x < 32) {
        uint32_t v[3], sum = 0;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const int b = 3 * lane + k;
            v[k] = b < TO_BUCKETS + 2 ? bc[b] : 0u;
            sum += v[k];
        }
        uint32_t x = sum;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(FULL, x, o);
            if (lane >= o) x += y;
        }
        uint32_t off = x - sum;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const int b = 3 * lane + k;
            if (b < TO_BUCKETS + 2) bc[b] = off;
            off += v[k];
        }
    }
    __syncthreads();
    for (uint32_t c0 = 0; c0 < a.n_slots; c0 += 4096u) {
        const uint32_t t0 = c0 + 4u * threadIdx.x;
        uint32_t c[4];
        load_counts4(a.tile_cnt, t0, T, c);
#pragma unroll
        for (int k = 0; k < 4; ++k)
            if (t0 + k < a.n_slots) {
                const uint32_t pos = atomicAdd(&bc[order_bucket(c[k], t0 + k, T)], 1u);
                a.tile_order_out[pos] = t0 + k;
                // the tile's range (written by this block's first loop, before the barriers)
                const uint2 rg = a.ranges[t0 + k];
                a.tile_info_out[pos] = make_uint4(t0 + k, rg.x, rg.y, 0u);
            }
    }
}

// ---------------------------------------------------------------- step 5
// The bucket sort in two block shapes (bin_sort.cuh): eight warps, three
// blocks per SM, for views whose tiles hold up to a couple of thousand pairs
// (more tiles in flight per SM); twelve warps, two blocks per SM, where most
// buckets approach the shared-memory size (more warps per tile).
#define BS_NS sort8
#define BS_NT 256
#define BS_OCC 3
#include "bin_sort.cuh"
#undef BS_NS
#undef BS_NT
#undef BS_OCC
#define BS_NS sort12
#define BS_NT 384
#define BS_OCC 2
#include "bin_sort.cuh"
#undef BS_NS
#undef BS_NT
#undef BS_OCC

__global__ void k_fill_u32(uint32_t *p, uint32_t v, uint64_t n) {
    const uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) p[i] = v;
}

__global__ void k_scale_u32(const uint32_t *src, uint32_t k, uint32_t *dst) { *dst = *src * k; }

__global__ void k_zero_f32_n(float *p, const uint32_t *n_dev, int mult) {
    const uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < (uint64_t)*n_dev * mult) p[i] = 0.0f;
}

// Grid of the instance walks: at most a few waves, whatever the capacity is
// (warps stride over the instance count on the device).
int walk_blocks(int64_t inst_cap) {
    const int64_t want = (std::max<int64_t>(inst_cap, 1) + 255) / 256;
    return (int)std::max<int64_t>(1, std::min<int64_t>(want, (int64_t)sm_count() * 8));
}

}  // namespace

void launch_bin_scan(const BinArgs &a, cudaStream_t s) {
    k_bin_scan<<<1, 1024, 0, s>>>(a);
    note_launches(1);
}

void launch_bin_fill(const BinArgs &a, cudaStream_t s) {
    k_bin_fill<<<walk_blocks(a.inst_cap), 256, 0, s>>>(a);
    note_launches(1);
}

int sm_count() {
    static PerDevice cache;
    return cache.get([](int dev) {
        int sms = 0;
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        return sms;
    });
}

int bin_sort_setup() {
    sort12::setup();
    return sort8::setup();
}

void launch_bin_sort(const BinArgs &a, cudaStream_t s) {
    if (a.sort_wide) sort12::launch(a, s);
    else sort8::launch(a, s);
    note_launches(1);
}

void launch_fill_u32(uint32_t *p, uint32_t v, int64_t n, cudaStream_t s) {
    if (n <= 0) return;
    k_fill_u32<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(p, v, (uint64_t)n);
    note_launches(1);
}

void launch_scale_u32(const uint32_t *src, uint32_t k, uint32_t *dst, cudaStream_t s) {
    k_scale_u32<<<1, 1, 0, s>>>(src, k, dst);
    note_launches(1);
}

void launch_zero_f32_n(float *p, const uint32_t *n_dev, int mult, int64_t n_cap, cudaStream_t s) {
    if (n_cap <= 0) return;
    const int64_t n = n_cap * mult;
    k_zero_f32_n<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(p, n_dev, mult);
    note_launches(1);
}

}  // namespace tsp
