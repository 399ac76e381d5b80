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
//                         each bucket by (depth key, id): an LSD radix sort
//                         with 8-bit digits over the bits in which the tile's
//                         depth keys differ, then runs of equal depth keys
//                         put in id order (runs longer than 32: id digits,
//                         then depth digits again); in shared memory, or for
//                         buckets larger than it, by the same passes over
//                         global memory.
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
constexpr int BS_THREADS = 256;                  // = the 256 digits: thread d owns digit d in the scans
constexpr int BS_WARPS = BS_THREADS / 32;
constexpr int BS_MAX = 3840;                     // bucket size sorted in shared memory (3 blocks per SM)
constexpr int BS_ROUNDS = BS_MAX / BS_THREADS;   // rounds of 32 per warp for a full chunk
constexpr int BS_RUN_MAX = 32;                   // longest run of equal depth keys fixed in place

struct BinSortSmem {
    uint2 kv[2][BS_MAX];           // (depth key - the tile's smallest, instance id)
    uint32_t wcnt[BS_WARPS][256];  // per warp and digit: counts, then offsets within the digit
    uint32_t dbase[256];           // first position of each digit
    uint32_t run[256];             // global path: next position of each digit
    uint32_t slab[256];            // large buckets: end of each depth slab
    uint32_t sw[BS_WARPS];
    uint32_t red[4];
    uint32_t tile, flag;
};

// Digit `shift` of an entry: of its remapped depth key, or of its id - vmin.
__device__ __forceinline__ uint32_t digit_of(uint2 e, bool by_id, uint32_t vmin, int shift) {
    return ((by_id ? e.y - vmin : e.x) >> shift) & 255u;
}

// Elements per warp for a chunk of m: the chunk is split evenly, in
// multiples of 32 (a warp's round), warp w owning [w pw, (w + 1) pw).
__device__ __forceinline__ int per_warp(int m) { return ((m + BS_THREADS - 1) / BS_THREADS) * 32; }

// Stable ranking of the chunk kv[0, m) on one 8-bit digit: warp w owns
// elements [w pw, (w + 1) pw), 32 per round in order (R >= pw / 32 rounds
// unrolled); on return S.wcnt[w][d] is warp w's first position within digit
// d, and thread d holds digit d's count in `count`.
template <int R>
__device__ __forceinline__ void rank_chunk(BinSortSmem &S, const uint2 *kv, int m, bool by_id, uint32_t vmin,
                                           int shift, uint32_t (&dig)[R], uint32_t (&rank)[R], uint32_t &count) {
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const uint32_t lt = lanemask_lt();
    for (int i = tid; i < BS_WARPS * 256; i += BS_THREADS) (&S.wcnt[0][0])[i] = 0u;
    __syncthreads();
    const int pw = per_warp(m), wb = warp * pw;
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int j = wb + r * 32 + lane;
        const bool valid = r * 32 < pw && j < m;
        uint32_t d = 0;
        if (valid) d = digit_of(kv[j], by_id, vmin, shift);
        uint32_t peers = __ballot_sync(FULL, valid);
        uint32_t rk = 0;
        if (peers) {  // warp-uniform
#pragma unroll
            for (int b = 0; b < 8; ++b) {
                const uint32_t bal = __ballot_sync(FULL, (d >> b) & 1u);
                peers &= ((d >> b) & 1u) ? bal : ~bal;
            }
            uint32_t before = 0;
            if (valid) before = S.wcnt[warp][d];
            __syncwarp();
            if (valid && (peers & lt) == 0) S.wcnt[warp][d] = before + (uint32_t)__popc(peers);
            __syncwarp();
            rk = before + (uint32_t)__popc(peers & lt);
        }
        dig[r] = d;
        rank[r] = rk;
    }
    __syncthreads();
    count = 0;
#pragma unroll
    for (int w = 0; w < BS_WARPS; ++w) {
        const uint32_t c = S.wcnt[w][tid];
        S.wcnt[w][tid] = count;
        count += c;
    }
}

// One stable pass over the chunk in shared memory: kv[src] -> kv[src ^ 1].
template <int R>
__device__ __forceinline__ void smem_pass(BinSortSmem &S, int src, int m, bool by_id, uint32_t vmin, int shift) {
    uint32_t dig[R], rank[R], count;
    rank_chunk<R>(S, S.kv[src], m, by_id, vmin, shift, dig, rank, count);
    uint32_t tot;
    const uint32_t base = block_excl_scan<BS_WARPS>(count, S.sw, tot);
    S.dbase[threadIdx.x] = base;
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, pw = per_warp(m), wb = warp * pw;
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int j = wb + r * 32 + lane;
        if (r * 32 < pw && j < m) S.kv[src ^ 1][S.dbase[dig[r]] + S.wcnt[warp][dig[r]] + rank[r]] = S.kv[src][j];
    }
    __syncthreads();
}

// The pass with the fewest unrolled rounds that cover m.
__device__ __forceinline__ void smem_pass_any(BinSortSmem &S, int src, int m, bool by_id, uint32_t vmin, int shift) {
    const int rounds = per_warp(m) / 32;
    if (rounds <= 1) smem_pass<1>(S, src, m, by_id, vmin, shift);
    else if (rounds <= 2) smem_pass<2>(S, src, m, by_id, vmin, shift);
    else if (rounds <= 4) smem_pass<4>(S, src, m, by_id, vmin, shift);
    else if (rounds <= 8) smem_pass<8>(S, src, m, by_id, vmin, shift);
    else if (rounds <= 12) smem_pass<12>(S, src, m, by_id, vmin, shift);
    else smem_pass<BS_ROUNDS>(S, src, m, by_id, vmin, shift);
}

constexpr int LD_BATCH = 8;  // global loads per thread issued together in the streaming loops

// (k - kmin, v) of entries [0, m), m <= BS_MAX, into dst: all loads of a
// thread issued before its first store, so that they are in flight together.
__device__ __forceinline__ void load_chunk(uint2 *dst, const uint32_t *k, const uint32_t *v, uint32_t m, uint32_t kmin) {
    const uint32_t tid = threadIdx.x;
    uint32_t kr[BS_ROUNDS], vr[BS_ROUNDS];
#pragma unroll
    for (int r = 0; r < BS_ROUNDS; ++r) {
        const uint32_t j = tid + r * BS_THREADS;
        kr[r] = j < m ? k[j] : 0u;
        vr[r] = j < m ? v[j] : 0u;
    }
#pragma unroll
    for (int r = 0; r < BS_ROUNDS; ++r) {
        const uint32_t j = tid + r * BS_THREADS;
        if (j < m) dst[j] = make_uint2(kr[r] - kmin, vr[r]);
    }
}

// This thread's share of the minimum and maximum of k[0, n) (and of v[0, n)
// when v is given), LD_BATCH loads in flight per step.
__device__ __forceinline__ void range_minmax(const uint32_t *k, const uint32_t *v, uint32_t n, uint32_t &kmn,
                                             uint32_t &kmx, uint32_t &vmn, uint32_t &vmx) {
    kmn = FULL; kmx = 0u; vmn = FULL; vmx = 0u;
    for (uint32_t j0 = 0; j0 < n; j0 += LD_BATCH * BS_THREADS) {
        uint32_t kr[LD_BATCH], vr[LD_BATCH];
#pragma unroll
        for (int r = 0; r < LD_BATCH; ++r) {
            const uint32_t j = j0 + threadIdx.x + r * BS_THREADS;
            kr[r] = j < n ? k[j] : FULL;
            vr[r] = (v && j < n) ? v[j] : FULL;
        }
#pragma unroll
        for (int r = 0; r < LD_BATCH; ++r) {
            const bool ok = j0 + threadIdx.x + r * BS_THREADS < n;
            if (ok) {
                kmn = min(kmn, kr[r]); kmx = max(kmx, kr[r]);
                vmn = min(vmn, vr[r]); vmx = max(vmx, vr[r]);
            }
        }
    }
    if (!v) { vmn = 0u; vmx = 0u; }
}

// One stable pass over a bucket in global memory, chunk by chunk:
// (ka, va)[0, n) -> (kb, vb)[0, n); keys are remapped by kmin while in
// shared memory.
__device__ void global_pass(BinSortSmem &S, const uint32_t *ka, const uint32_t *va, uint32_t *kb, uint32_t *vb,
                            uint32_t n, bool by_id, uint32_t kmin, uint32_t vmin, int shift) {
    const int tid = threadIdx.x;
    S.dbase[tid] = 0u;
    __syncthreads();
    for (uint32_t j0 = 0; j0 < n; j0 += LD_BATCH * BS_THREADS) {  // LD_BATCH loads per thread in flight
        uint32_t d[LD_BATCH];
#pragma unroll
        for (int r = 0; r < LD_BATCH; ++r) {
            const uint32_t j = j0 + tid + r * BS_THREADS;
            d[r] = j < n ? digit_of(make_uint2(ka[j] - kmin, by_id ? va[j] : 0u), by_id, vmin, shift) : 256u;
        }
#pragma unroll
        for (int r = 0; r < LD_BATCH; ++r)
            if (d[r] < 256u) atomicAdd(&S.dbase[d[r]], 1u);
    }
    __syncthreads();
    {
        uint32_t tot;
        const uint32_t e = block_excl_scan<BS_WARPS>(S.dbase[tid], S.sw, tot);
        S.run[tid] = e;
    }
    __syncthreads();
    const int warp = tid >> 5, lane = tid & 31;
    for (uint32_t c0 = 0; c0 < n; c0 += BS_MAX) {
        const int m = (int)min((uint32_t)BS_MAX, n - c0);
        load_chunk(S.kv[0], ka + c0, va + c0, (uint32_t)m, kmin);
        __syncthreads();
        uint32_t dig[BS_ROUNDS], rank[BS_ROUNDS], count;
        rank_chunk<BS_ROUNDS>(S, S.kv[0], m, by_id, vmin, shift, dig, rank, count);
        __syncthreads();
        const int pw = per_warp(m), wb = warp * pw;
#pragma unroll
        for (int r = 0; r < BS_ROUNDS; ++r) {
            const int j = wb + r * 32 + lane;
            if (r * 32 < pw && j < m) {
                const uint32_t pos = S.run[dig[r]] + S.wcnt[warp][dig[r]] + rank[r];
                const uint2 e = S.kv[0][j];
                kb[pos] = e.x + kmin;
                vb[pos] = e.y;
            }
        }
        __syncthreads();
        S.run[tid] += count;
        __syncthreads();
    }
}

__device__ __forceinline__ int sig_bits(uint32_t lo, uint32_t hi) { return hi > lo ? 32 - __clz(hi - lo) : 0; }

// Block-wide min and max of two words (results in S.red: kmin, kmax, vmin, vmax).
__device__ __forceinline__ void block_minmax(BinSortSmem &S, uint32_t kmn, uint32_t kmx, uint32_t vmn, uint32_t vmx) {
    kmn = __reduce_min_sync(FULL, kmn);
    kmx = __reduce_max_sync(FULL, kmx);
    vmn = __reduce_min_sync(FULL, vmn);
    vmx = __reduce_max_sync(FULL, vmx);
    if (threadIdx.x == 0) {
        S.red[0] = FULL;
        S.red[1] = 0u;
        S.red[2] = FULL;
        S.red[3] = 0u;
    }
    __syncthreads();
    if ((threadIdx.x & 31) == 0) {
        atomicMin(&S.red[0], kmn);
        atomicMax(&S.red[1], kmx);
        atomicMin(&S.red[2], vmn);
        atomicMax(&S.red[3], vmx);
    }
    __syncthreads();
}

// Entries in global memory (two arrays).
struct GlobalEntries {
    const uint32_t *k;
    uint32_t *v;
    __device__ uint32_t key(uint32_t j) const { return k[j]; }
    __device__ uint32_t id(uint32_t j) const { return v[j]; }
    __device__ void set_id(uint32_t j, uint32_t x) const { v[j] = x; }
};

// Puts the ids of each run of equal keys of entries [0, n) (sorted by key)
// in ascending order, in place, when the run holds at most 32 entries (one
// thread per run); returns true (block-uniform) when a longer run exists,
// leaving the entries sorted by key only.
template <class E>
__device__ bool fix_ties(BinSortSmem &S, const E &e, uint32_t n) {
    const int tid = threadIdx.x;
    if (tid == 0) S.flag = 0u;
    __syncthreads();
    for (uint32_t j = tid; j + 1 < n; j += BS_THREADS) {
        const uint32_t kj = e.key(j);
        if ((j == 0 || e.key(j - 1) != kj) && e.key(j + 1) == kj) {
            uint32_t end = j + 1;
            while (end < n && e.key(end) == kj && end - j <= (uint32_t)BS_RUN_MAX) ++end;
            if (end - j > (uint32_t)BS_RUN_MAX) {
                atomicOr(&S.flag, 1u);
            } else {
                for (uint32_t x = j + 1; x < end; ++x) {  // insertion sort of the run's ids
                    const uint32_t vx = e.id(x);
                    uint32_t y = x;
                    while (y > j && e.id(y - 1) > vx) {
                        e.set_id(y, e.id(y - 1));
                        --y;
                    }
                    e.set_id(y, vx);
                }
            }
        }
    }
    __syncthreads();
    const bool longrun = S.flag != 0u;
    __syncthreads();
    return longrun;
}

// Puts each run of entries with equal key >> lo (entries [0, n) in shared
// memory, sorted by key >> lo) in (key, id) order, in place, when the run
// holds at most BS_RUN_MAX entries (one thread per run, insertion); returns
// true (block-uniform) when a longer run exists, leaving it as it was.
__device__ bool fix_runs(BinSortSmem &S, uint2 *kv, uint32_t n, int lo) {
    const int tid = threadIdx.x;
    if (tid == 0) S.flag = 0u;
    __syncthreads();
    for (uint32_t j = tid; j + 1 < n; j += BS_THREADS) {
        const uint32_t hj = kv[j].x >> lo;
        if ((j == 0 || (kv[j - 1].x >> lo) != hj) && (kv[j + 1].x >> lo) == hj) {
            uint32_t end = j + 1;
            while (end < n && (kv[end].x >> lo) == hj && end - j <= (uint32_t)BS_RUN_MAX) ++end;
            if (end - j > (uint32_t)BS_RUN_MAX) {
                atomicOr(&S.flag, 1u);
            } else {
                for (uint32_t x = j + 1; x < end; ++x) {
                    const uint2 vx = kv[x];
                    uint32_t y = x;
                    while (y > j && (kv[y - 1].x > vx.x || (kv[y - 1].x == vx.x && kv[y - 1].y > vx.y))) {
                        kv[y] = kv[y - 1];
                        --y;
                    }
                    kv[y] = vx;
                }
            }
        }
    }
    __syncthreads();
    const bool longrun = S.flag != 0u;
    __syncthreads();
    return longrun;
}

// Sorts n <= BS_MAX entries (keys k, ids v in global memory) by (key, id)
// in shared memory and writes the ids to out (which may alias v).  The radix
// passes cover the highest 8 * npass significant key bits (npass = 2 up to
// 24 significant bits, else 3); runs of entries that agree on those bits are
// then put in (key, id) order by insertion, which completes the order.
__device__ void sort_range_smem(BinSortSmem &S, const uint32_t *k, const uint32_t *v, uint32_t n, uint32_t *out) {
    const int tid = threadIdx.x;
    if (n <= 1) {
        if (n == 1 && tid == 0) out[0] = v[0];
        __syncthreads();
        return;
    }
    // the whole bucket in registers first (BS_ROUNDS loads per thread in flight together)
    uint32_t kr[BS_ROUNDS], vr[BS_ROUNDS];
#pragma unroll
    for (int r = 0; r < BS_ROUNDS; ++r) {
        const uint32_t j = tid + r * BS_THREADS;
        kr[r] = j < n ? k[j] : 0u;
        vr[r] = j < n ? v[j] : 0u;
    }
    uint32_t kmn = FULL, kmx = 0u, vmn = FULL, vmx = 0u;
#pragma unroll
    for (int r = 0; r < BS_ROUNDS; ++r)
        if (tid + r * BS_THREADS < n) {
            kmn = min(kmn, kr[r]); kmx = max(kmx, kr[r]); vmn = min(vmn, vr[r]); vmx = max(vmx, vr[r]);
        }
    block_minmax(S, kmn, kmx, vmn, vmx);
    const uint32_t kmin = S.red[0], vmin = S.red[2];
    const int kb = sig_bits(kmin, S.red[1]), vb = sig_bits(vmin, S.red[3]);
    const int m = (int)n;
#pragma unroll
    for (int r = 0; r < BS_ROUNDS; ++r) {
        const uint32_t j = tid + r * BS_THREADS;
        if (j < n) S.kv[0][j] = make_uint2(kr[r] - kmin, vr[r]);
    }
    __syncthreads();
    int src = 0;
    const int npass = kb <= 16 ? (kb + 7) / 8 : (kb <= 24 ? 2 : 3);
    const int lo = max(0, kb - 8 * npass);  // key bits below the passes
    for (int sh = lo; sh < kb; sh += 8) {
        smem_pass_any(S, src, m, false, vmin, sh);
        src ^= 1;
    }
    // runs that agree on the passes' bits: (key, id) order (short runs in place)
    if (fix_runs(S, S.kv[src], n, lo)) {  // a long run: the full (depth key, id) order
        for (int sh = 0; sh < vb; sh += 8) {
            smem_pass_any(S, src, m, true, vmin, sh);
            src ^= 1;
        }
        for (int sh = 0; sh < kb; sh += 8) {
            smem_pass_any(S, src, m, false, vmin, sh);
            src ^= 1;
        }
    }
    for (int j = tid; j < m; j += BS_THREADS) out[j] = S.kv[src][j].y;
    __syncthreads();
}

// Sorts n entries by radix passes over global memory: (k0, v0) with the
// scratch (k1, v1); ids to out (which may alias v0 or v1).
__device__ void sort_range_global(BinSortSmem &S, uint32_t *k0, uint32_t *v0, uint32_t *k1, uint32_t *v1, uint32_t n,
                                  uint32_t *out) {
    const int tid = threadIdx.x;
    uint32_t kmn, kmx, vmn, vmx;
    range_minmax(k0, v0, n, kmn, kmx, vmn, vmx);
    block_minmax(S, kmn, kmx, vmn, vmx);
    const uint32_t kmin = S.red[0], vmin = S.red[2];
    const int kb = sig_bits(kmin, S.red[1]), vb = sig_bits(vmin, S.red[3]);
    for (int sh = 0; sh < kb; sh += 8) {
        global_pass(S, k0, v0, k1, v1, n, false, kmin, vmin, sh);
        uint32_t *t = k0; k0 = k1; k1 = t;
        t = v0; v0 = v1; v1 = t;
    }
    if (fix_ties(S, GlobalEntries{k0, v0}, n)) {  // a long run of equal depth keys: ids, then depth
        for (int sh = 0; sh < vb; sh += 8) {
            global_pass(S, k0, v0, k1, v1, n, true, kmin, vmin, sh);
            uint32_t *t = k0; k0 = k1; k1 = t;
            t = v0; v0 = v1; v1 = t;
        }
        for (int sh = 0; sh < kb; sh += 8) {
            global_pass(S, k0, v0, k1, v1, n, false, kmin, vmin, sh);
            uint32_t *t = k0; k0 = k1; k1 = t;
            t = v0; v0 = v1; v1 = t;
        }
    }
    if (out != v0) {  // the result is in (k0, v0)
        for (uint32_t j0 = 0; j0 < n; j0 += LD_BATCH * BS_THREADS) {
            uint32_t vr[LD_BATCH];
#pragma unroll
            for (int r = 0; r < LD_BATCH; ++r) {
                const uint32_t j = j0 + tid + r * BS_THREADS;
                vr[r] = j < n ? v0[j] : 0u;
            }
#pragma unroll
            for (int r = 0; r < LD_BATCH; ++r) {
                const uint32_t j = j0 + tid + r * BS_THREADS;
                if (j < n) out[j] = vr[r];
            }
        }
    }
    __syncthreads();
}

__global__ __launch_bounds__(BS_THREADS, 3) void k_bin_sort(BinArgs a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    BinSortSmem &S = *reinterpret_cast<BinSortSmem *>(smem_raw);
    const int tid = threadIdx.x;
    if (*a.p_dev > a.p_cap) return;  // nothing was filled (the ranges are empty)
    for (;;) {
        if (tid == 0) S.tile = atomicAdd(a.tile_ctr, 1u);
        __syncthreads();
        const uint32_t q = S.tile;
        __syncthreads();
        if (q >= a.n_slots) break;
        const uint2 rg = a.ranges[a.tile_order[q]];
        const uint32_t first = rg.x, n = rg.y - rg.x;
        if (n == 0) continue;
        uint32_t *bk = a.bk_key + first, *bi = a.bk_id + first;
        uint32_t *tk = a.tmp_key + first, *ti = a.tmp_id + first;
        uint32_t *out = a.ids_out + first;
        if (n <= (uint32_t)BS_MAX) {
            sort_range_smem(S, bk, bi, n, out);
            continue;
        }
        // A bucket beyond shared memory: one pass over global memory on the
        // highest significant digit splits it into depth slabs; runs of
        // consecutive slabs of at most BS_MAX entries are then sorted in
        // shared memory, and a slab larger than that by global passes.
        uint32_t kmn, kmx, vmn, vmx;
        range_minmax(bk, nullptr, n, kmn, kmx, vmn, vmx);
        block_minmax(S, kmn, kmx, vmn, vmx);
        const uint32_t kmin = S.red[0];
        const int kb = sig_bits(kmin, S.red[1]);
        if (kb == 0) {  // one depth key: the id order, by global passes
            sort_range_global(S, bk, bi, tk, ti, n, out);
            continue;
        }
        global_pass(S, bk, bi, tk, ti, n, false, kmin, 0u, ((kb - 1) / 8) * 8);
        S.slab[tid] = S.run[tid];  // end of each slab (the passes below reuse S.run)
        __syncthreads();
        uint32_t c0 = 0;  // start of the pending run of slabs (the same in every thread)
        for (int d = 0; d < 256; ++d) {
            const uint32_t beg = d ? S.slab[d - 1] : 0u, end = S.slab[d];
            if (end - c0 <= (uint32_t)BS_MAX) continue;
            if (beg > c0) sort_range_smem(S, tk + c0, ti + c0, beg - c0, out + c0);
            c0 = beg;
            if (end - beg > (uint32_t)BS_MAX) {
                sort_range_global(S, tk + beg, ti + beg, bk + beg, bi + beg, end - beg, out + beg);
                c0 = end;
            }
        }
        if (n > c0) sort_range_smem(S, tk + c0, ti + c0, n - c0, out + c0);
    }
}

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
    static PerDevice cache;
    return cache.get([](int) {
        const size_t smem = sizeof(BinSortSmem);
        cudaFuncSetAttribute(k_bin_sort, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        int per_sm = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_bin_sort, BS_THREADS, smem);
        return sm_count() * std::max(1, per_sm);
    });
}

void launch_bin_sort(const BinArgs &a, cudaStream_t s) {
    const int grid = bin_sort_setup();
    cudaMemsetAsync(a.tile_ctr, 0, sizeof(uint32_t), s);
    k_bin_sort<<<std::min(grid, (int)std::max<uint32_t>(a.n_slots, 1)), BS_THREADS, sizeof(BinSortSmem), s>>>(a);
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
