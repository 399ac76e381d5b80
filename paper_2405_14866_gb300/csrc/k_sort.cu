// A3..A6: ordering of (Gaussian, tile) pairs by (tile, depth, id).
//
// The order the rasterizer needs is that of a stable sort of the 64-bit key
// tile << 32 | bits(depth) over pairs emitted in Gaussian-id order (3DGS,
// cited in Tele-Aloha Sec. 4.2).  An LSD radix sort processes the depth
// digits first; since all pairs of one Gaussian share its depth, those
// passes are run once over the N Gaussians instead of the P ~ 2.4 N pairs:
//   1. stable radix sort of (depth key, id) over Gaussians, only over the
//      bytes in which the rendered depths differ;
//   2. exclusive scan of tiles-per-Gaussian in that order and emission of
//      (tile, id) pairs in that order;
//   3. stable radix sort of the pairs on the tile digits;
//   4. per-tile [first, last) ranges.
// Each radix pass is a single launch: blocks take key tiles in ticket order
// and chain their per-digit offsets through published counts (decoupled
// look-back), after one launch that counts the digits of all passes.
#include <algorithm>

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

// Exclusive scan across a block of NW warps (warp-shuffle inside warps,
// one warp over the warp totals).  `sw` holds NW words of shared memory.
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

__device__ __forceinline__ int rs_passes(const RadixSort &rs) {
    return min(rs.npass_dev ? (int)*rs.npass_dev : rs.npass_host, RS_MAX_PASSES);
}

__device__ __forceinline__ uint32_t rs_remap(uint32_t k, bool remap, uint32_t kmin) {
    return remap ? (k == CULLED_KEY ? 0u : k - kmin) : k;
}

// Digit counts of every pass in one read of the keys.  Blocks stride over
// the key tiles; equal digits within a warp are combined before the shared
// atomic (depth keys share their high bytes, so lanes collide often).  The
// launch also clears the look-back words of the active tiles and the tile
// tickets of the passes that follow.
__global__ __launch_bounds__(RS_THREADS) void k_radix_hist(RadixSort rs) {
    const int np = rs_passes(rs);
    if (np == 0) return;
    __shared__ uint32_t h[RS_MAX_PASSES][256];
    const int tid = threadIdx.x, lane = tid & 31;
    for (int i = tid; i < RS_MAX_PASSES * 256; i += RS_THREADS) (&h[0][0])[i] = 0;
    if (blockIdx.x == 0 && tid < RS_MAX_PASSES) rs.tile_ctr[tid] = 0;
    __syncthreads();
    const uint32_t n = *rs.n_dev;
    const uint32_t n_tiles = (n + RS_TILE - 1) / RS_TILE;
    const bool remap = rs.kmin != nullptr;
    const uint32_t kmin = remap ? *rs.kmin : 0u;
    for (uint32_t t = blockIdx.x; t < n_tiles; t += gridDim.x) {
        for (int p = 0; p < np; ++p) rs.status[((size_t)p * rs.nblocks + t) * 256 + tid] = 0u;
        const uint32_t base = t * RS_TILE + tid;
        uint32_t key[RS_ITEMS];
#pragma unroll
        for (int i = 0; i < RS_ITEMS; ++i) {  // all loads in flight before any use
            const uint32_t idx = base + i * RS_THREADS;
            key[i] = idx < n ? rs.keys_in[idx] : 0u;
        }
#pragma unroll
        for (int i = 0; i < RS_ITEMS; ++i) {
            const bool valid = base + i * RS_THREADS < n;
            const uint32_t k = rs_remap(key[i], remap, kmin);
            const uint32_t nval = __popc(__ballot_sync(FULL, valid));
            for (int p = 0; p < np; ++p) {
                const uint32_t d = (k >> (8 * p)) & 255u;
                // a warp whose valid keys share the digit adds once (common in
                // the high bytes); otherwise one shared atomic per key
                const uint32_t d0 = __shfl_sync(FULL, d, 0);
                if (__all_sync(FULL, !valid || d == d0)) {  // valid lanes are a prefix: lane 0 is valid if any is
                    if (lane == 0 && nval) atomicAdd(&h[p][d0], nval);
                } else if (valid) {
                    atomicAdd(&h[p][d], 1u);
                }
            }
        }
    }
    __syncthreads();
    for (int p = 0; p < np; ++p)
        if (h[p][tid]) atomicAdd(&rs.totals[p * 256 + tid], h[p][tid]);
}

// One pass of the sort: a block takes key tiles in order from the pass's
// ticket counter; ranks its 4096 keys per digit (per warp, one ballot per
// digit bit); publishes its per-digit counts, marked AGGREGATE, then walks
// back over earlier tiles, adding their counts until it meets a tile marked
// PREFIX (whose count already includes everything before it), and
// publishes its own inclusive prefix; places its keys in digit order in
// shared memory and writes each digit's run contiguously at the digit's
// global offset.  Every earlier ticket belongs to a running block that
// publishes its aggregate before it waits on anything, so the walk always
// ends; it is nevertheless bounded.
constexpr int DS_THREADS = 512;
constexpr uint32_t LB_AGG = 1u << 30, LB_PREFIX = 2u << 30, LB_COUNT = (1u << 30) - 1u;

__global__ __launch_bounds__(DS_THREADS, 2) void k_radix_onesweep(RadixSort rs, int pass) {
    if (pass >= rs_passes(rs)) return;
    constexpr int NW = DS_THREADS / 32;
    constexpr int PER_WARP = RS_TILE / NW;  // 256 keys, 8 rounds of 32
    constexpr int ROUNDS = PER_WARP / 32;
    __shared__ uint32_t wcnt[NW][256];      // per-warp digit counts, then per-warp digit offsets
    __shared__ uint32_t lbase[256];         // first local position of each digit
    __shared__ uint32_t gbase[256];         // global offset of each digit for this tile
    __shared__ uint32_t dbase[256];         // global start of each digit (all tiles)
    __shared__ uint32_t sw[NW];
    __shared__ uint32_t s_tile;
    __shared__ uint32_t skey[RS_TILE];
    __shared__ uint32_t sval[RS_TILE];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const uint32_t n = *rs.n_dev;
    const uint32_t n_tiles = (n + RS_TILE - 1) / RS_TILE;
    const bool remap = pass == 0 && rs.kmin;
    const uint32_t kmin = remap ? *rs.kmin : 0u;
    const int shift = 8 * pass;
    const bool odd = (pass & 1) != 0;
    const uint32_t *ksrc = pass == 0 ? rs.keys_in : (odd ? rs.keys[0] : rs.keys[1]);
    const uint32_t *vsrc = pass == 0 ? rs.vals_in : (odd ? rs.vals[0] : rs.vals[1]);
    uint32_t *kdst = odd ? rs.keys[1] : rs.keys[0];
    uint32_t *vdst = odd ? rs.vals[1] : rs.vals[0];
    volatile uint32_t *lb = rs.status + (size_t)pass * rs.nblocks * 256;
    {   // global start of each digit: exclusive scan of the pass's digit totals
        const uint32_t c = tid < 256 ? rs.totals[pass * 256 + tid] : 0u;
        uint32_t tot;
        const uint32_t e = block_excl_scan<NW>(c, sw, tot);
        if (tid < 256) dbase[tid] = e;
    }
    const uint32_t lt = lanemask_lt();
    for (;;) {
        if (tid == 0) s_tile = atomicAdd(&rs.tile_ctr[pass], 1u);
        for (int i = tid; i < NW * 256; i += DS_THREADS) (&wcnt[0][0])[i] = 0;
        __syncthreads();
        const uint32_t tile = s_tile;
        if (tile >= n_tiles) break;
        const uint32_t bbase = tile * RS_TILE;
        const uint32_t wbase = bbase + warp * PER_WARP;
        uint32_t key[ROUNDS], val[ROUNDS], rank[ROUNDS];
#pragma unroll
        for (int r = 0; r < ROUNDS; ++r) {  // all loads in flight before any use
            const uint32_t idx = wbase + r * 32 + lane;
            key[r] = idx < n ? ksrc[idx] : 0u;
            val[r] = idx < n ? (vsrc ? vsrc[idx] : idx) : 0u;
        }
#pragma unroll
        for (int r = 0; r < ROUNDS; ++r) {
            const bool valid = wbase + r * 32 + lane < n;
            const uint32_t k = valid ? rs_remap(key[r], remap, kmin) : 0u;
            key[r] = k;
            const uint32_t d = (k >> shift) & 255u;
            uint32_t peers = __ballot_sync(FULL, valid);
#pragma unroll
            for (int b = 0; b < 8; ++b) {
                const uint32_t bal = __ballot_sync(FULL, (d >> b) & 1u);
                peers &= ((d >> b) & 1u) ? bal : ~bal;
            }
            uint32_t before = 0;
            if (valid) before = wcnt[warp][d];
            __syncwarp();
            if (valid && (peers & lt) == 0) wcnt[warp][d] = before + __popc(peers);
            __syncwarp();
            rank[r] = before + __popc(peers & lt);
        }
        __syncthreads();
        uint32_t run = 0;  // this tile's count of digit tid
        if (tid < 256) {
#pragma unroll
            for (int w = 0; w < NW; ++w) {
                const uint32_t c = wcnt[w][tid];
                wcnt[w][tid] = run;
                run += c;
            }
            // publish, then look back for the exclusive prefix over earlier tiles
            volatile uint32_t *mine = lb + (size_t)tile * 256 + tid;
            if (tile == 0) {
                *mine = LB_PREFIX | run;
                gbase[tid] = dbase[tid];
            } else {
                *mine = LB_AGG | run;
                // walk back 8 tiles at a time (their words are read together)
                constexpr int LA = 8;
                uint32_t excl = 0;
                bool ok = true, found = false;
                for (int64_t t = (int64_t)tile - 1; t >= 0 && ok && !found; t -= LA) {
                    uint32_t v[LA];
#pragma unroll
                    for (int j = 0; j < LA; ++j) v[j] = t - j >= 0 ? (uint32_t)lb[(size_t)(t - j) * 256 + tid] : (uint32_t)LB_PREFIX;
#pragma unroll
                    for (int j = 0; j < LA; ++j) {
                        if (found || !ok) break;
                        volatile const uint32_t *w = lb + (size_t)(t - j) * 256 + tid;
                        for (uint32_t it = 0; (v[j] & ~LB_COUNT) == 0; ++it) {  // t - j >= 0 here
                            if (it >= (1u << 22)) {
                                ok = false;
                                break;
                            }
                            __nanosleep(32);
                            v[j] = *w;
                        }
                        if (!ok) break;
                        excl += v[j] & LB_COUNT;
                        found = (v[j] & LB_PREFIX) != 0;
                    }
                }
                if (!ok) set_status(rs.err, TSPLAT_ERR_TIMEOUT);
                *mine = LB_PREFIX | ((excl + run) & LB_COUNT);
                gbase[tid] = dbase[tid] + excl;
            }
        }
        uint32_t tot;
        const uint32_t lbv = block_excl_scan<NW>(run, sw, tot);
        if (tid < 256) lbase[tid] = lbv;
        __syncthreads();
#pragma unroll
        for (int r = 0; r < ROUNDS; ++r) {
            if (wbase + r * 32 + lane < n) {
                const uint32_t d = (key[r] >> shift) & 255u;
                const uint32_t pos = lbase[d] + wcnt[warp][d] + rank[r];
                skey[pos] = key[r];
                sval[pos] = val[r];
            }
        }
        __syncthreads();
        const uint32_t cnt = min((uint32_t)RS_TILE, n - bbase);
        for (uint32_t p = tid; p < cnt; p += DS_THREADS) {
            const uint32_t k = skey[p];
            const uint32_t d = (k >> shift) & 255u;
            const uint32_t pos = gbase[d] + (p - lbase[d]);
            kdst[pos] = k;
            vdst[pos] = sval[p];
        }
        __syncthreads();
    }
}

__global__ void k_depth_npass(const uint32_t *kminmax, uint32_t *npass) {
    const uint32_t lo = kminmax[0], hi = kminmax[1];
    uint32_t np = 0;
    if (lo != CULLED_KEY && hi >= lo) {
        const uint32_t r = hi - lo;
        const int bits = 32 - __clz(r);
        np = (uint32_t)((bits + 7) / 8);
    }
    *npass = np;
}

// ---------------------------------------------------------------- emit
constexpr int EM_THREADS = 256;
constexpr int EM_ITEMS = 16;
constexpr int EM_TILE = EM_THREADS * EM_ITEMS;

__device__ __forceinline__ uint32_t sorted_val(const SortedVals &s, int np, uint64_t k) {
    if (np == 0) return s.vals_in ? s.vals_in[k] : (uint32_t)k;
    return (((np - 1) & 1) ? s.vals[1] : s.vals[0])[k];
}

__device__ __forceinline__ int sv_passes(const SortedVals &s) {
    return s.npass_dev ? (int)*s.npass_dev : s.npass_host;
}

// Blocks stride over the item tiles [b * 4096, (b + 1) * 4096) of the n
// depth-ordered Gaussians; blk_sum[b] = pairs of tile b.
__global__ __launch_bounds__(EM_THREADS) void k_emit_count(EmitArgs a) {
    __shared__ uint32_t sw[EM_THREADS / 32];
    const uint64_t n = *a.n_dev;
    const uint32_t n_items = (uint32_t)((n + EM_TILE - 1) / EM_TILE);
    const int np = sv_passes(a.order);
    for (uint32_t b = blockIdx.x; b < n_items; b += gridDim.x) {
        const uint64_t base = (uint64_t)b * EM_TILE + threadIdx.x;
        uint32_t s = 0;
        for (int i = 0; i < EM_ITEMS; ++i) {
            const uint64_t k = base + (uint64_t)i * EM_THREADS;
            if (k < n) s += a.ntiles[sorted_val(a.order, np, k)];
        }
        uint32_t tot;
        block_excl_scan<EM_THREADS / 32>(s, sw, tot);
        if (threadIdx.x == 0) a.blk_sum[b] = tot;
    }
}

// single block: exclusive scan of the item tiles' sums in place, total pairs
__global__ __launch_bounds__(1024) void k_emit_scan_blocks(EmitArgs a) {
    __shared__ uint32_t sw[32];
    const int nblocks = (int)((*a.n_dev + EM_TILE - 1) / EM_TILE);
    const int per = (nblocks + 1023) / 1024;
    const int b0 = min((int)threadIdx.x * per, nblocks), b1 = min(b0 + per, nblocks);
    uint32_t local = 0;
    for (int b = b0; b < b1; ++b) local += a.blk_sum[b];
    uint32_t tot;
    uint32_t run = block_excl_scan<32>(local, sw, tot);
    for (int b = b0; b < b1; ++b) {
        const uint32_t c = a.blk_sum[b];
        a.blk_sum[b] = run;
        run += c;
    }
    if (threadIdx.x == 0) *a.p_dev = tot;
}

// Items (depth-ordered Gaussians) of block b: [b * 4096, (b + 1) * 4096) in
// 16 rounds of 256.  Per round a block scan gives each item its pair offset;
// the 32 items of a warp own one contiguous run of pairs, which the warp
// writes cooperatively (lane e of the run finds its Gaussian by binary
// search over the lanes' offsets), so the stores are coalesced.
__global__ __launch_bounds__(EM_THREADS) void k_emit_write(EmitArgs a) {
    __shared__ uint32_t sw[EM_THREADS / 32];
    if ((uint64_t)*a.p_dev > (uint64_t)a.p_cap) {  // nothing is emitted when the pairs do not fit
        if (blockIdx.x == 0 && threadIdx.x == 0) set_status(a.status, TSPLAT_ERR_CAPACITY);
        return;
    }
    const uint64_t n = *a.n_dev;
    const uint32_t n_items = (uint32_t)((n + EM_TILE - 1) / EM_TILE);
    const uint32_t ns = *a.n_stride;
    const int np = sv_passes(a.order);
    const int lane = threadIdx.x & 31;
    for (uint32_t b = blockIdx.x; b < n_items; b += gridDim.x) {
    uint64_t running = a.blk_sum[b];
    const uint64_t base = (uint64_t)b * EM_TILE;
    for (int r = 0; r < EM_ITEMS; ++r) {
        const uint64_t k = base + (uint64_t)r * EM_THREADS + threadIdx.x;
        uint32_t id = 0, cnt = 0, vbase = 0, msk = 0xffffffffu;
        int x0 = 0, y0 = 0, x1 = 0, y1 = 0, vtx = 0;
        if (k < n) {
            id = sorted_val(a.order, np, k);
            cnt = a.ntiles[id];
            if (cnt) {
                unpack_rect(a.rect[id], x0, y0, x1, y1);
                if (a.tmask) msk = a.tmask[id];
                const RenderView &vw = a.views[id / ns];
                vbase = vw.tile_base;
                vtx = vw.tiles_x;
            }
        }
        uint32_t tot;
        const uint32_t excl = block_excl_scan<EM_THREADS / 32>(cnt, sw, tot);
        const uint64_t my_off = running + excl;
        const uint64_t wfirst = __shfl_sync(FULL, my_off, 0);
        const uint32_t start = (uint32_t)(my_off - wfirst);           // run-relative start of this lane
        const uint32_t wtot = __shfl_sync(FULL, start + cnt, 31);     // the warp's run length
        const int w = x1 - x0;
        for (uint32_t e0 = 0; e0 < wtot; e0 += 32) {  // warp-uniform trip count
            const uint32_t e = e0 + lane;
            int o = 0;  // owner: the last lane whose start <= e
#pragma unroll
            for (int step = 16; step > 0; step >>= 1) {
                const int cand = o + step;
                const uint32_t sc = __shfl_sync(FULL, start, cand & 31);
                if (cand < 32 && sc <= e) o = cand;
            }
            const uint32_t so = __shfl_sync(FULL, start, o);
            const int ox0 = __shfl_sync(FULL, x0, o), oy0 = __shfl_sync(FULL, y0, o), ow = __shfl_sync(FULL, w, o);
            const uint32_t oid = __shfl_sync(FULL, id, o);
            const uint32_t ovb = __shfl_sync(FULL, vbase, o);
            const int otx = __shfl_sync(FULL, vtx, o);
            const uint32_t omsk = __shfl_sync(FULL, msk, o);
            if (e < wtot) {
                int loc = (int)(e - so);
                if (omsk != 0xffffffffu) {  // tight binning: the loc-th kept tile of the rect
                    uint32_t mm = omsk;
                    for (int j = 0; j < loc; ++j) mm &= mm - 1u;
                    loc = __ffs(mm) - 1;
                }
                const int ty = oy0 + loc / ow, tx = ox0 + loc % ow;
                a.pair_tile[wfirst + e] = ovb + (uint32_t)(ty * otx + tx);
                a.pair_id[wfirst + e] = oid;
            }
        }
        running += tot;
    }
    }
}

// Grid-stride over the P sorted pairs: a pair that starts or ends a tile's
// run sets that tile's range bound.
__global__ void k_ranges(const uint32_t *tiles, const uint32_t *p_dev, uint64_t p_cap, uint2 *ranges,
                         uint32_t n_tiles) {
    const uint64_t P = min((uint64_t)*p_dev, p_cap);
    for (uint64_t k = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; k < P; k += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t t = tiles[k];
        if (t >= n_tiles) continue;
        if (k == 0 || tiles[k - 1] != t) ranges[t].x = (uint32_t)k;
        if (k == P - 1 || tiles[k + 1] != t) ranges[t].y = (uint32_t)(k + 1);
    }
}

// Order in which the persistent composite takes the tiles: longest lists
// first (largest-processing-time-first scheduling shortens the tail of the
// grid).  One block buckets the tiles by 4 log2(pair count); tiles with no
// pairs follow, then tile slots beyond the views' tile count (graph replays
// size the launch for their largest batch).  The order within a bucket
// depends on atomics, which changes nothing in the output: every tile is
// composited independently.
constexpr int TO_BUCKETS = 64;
__global__ __launch_bounds__(1024) void k_tile_order(const uint2 *ranges, const RenderView *views, int n_views,
                                                     uint32_t n_slots, uint32_t *order) {
    __shared__ uint32_t cnt[TO_BUCKETS + 2], off[TO_BUCKETS + 2];
    const RenderView &lv = views[n_views - 1];
    const uint32_t n_tiles = min(n_slots, lv.tile_base + (uint32_t)(lv.tiles_x * lv.tiles_y));
    for (int i = threadIdx.x; i < TO_BUCKETS + 2; i += blockDim.x) cnt[i] = 0;
    __syncthreads();
    auto bucket = [&](uint32_t t) -> int {
        if (t >= n_tiles) return TO_BUCKETS + 1;  // not a tile of this batch
        const uint32_t c = ranges[t].y - ranges[t].x;
        if (c == 0) return TO_BUCKETS;
        const int lg = (int)(4.0f * __log2f((float)c));
        return TO_BUCKETS - 1 - min(TO_BUCKETS - 1, max(0, lg));  // descending count
    };
    for (uint32_t t = threadIdx.x; t < n_slots; t += blockDim.x) atomicAdd(&cnt[bucket(t)], 1u);
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t run = 0;
        for (int b = 0; b < TO_BUCKETS + 2; ++b) {
            off[b] = run;
            run += cnt[b];
        }
    }
    __syncthreads();
    for (uint32_t t = threadIdx.x; t < n_slots; t += blockDim.x) order[atomicAdd(&off[bucket(t)], 1u)] = t;
}

__global__ void k_scale_u32(const uint32_t *src, uint32_t k, uint32_t *dst) { *dst = *src * k; }

__global__ void k_fill_u32(uint32_t *p, uint32_t v, uint64_t n) {
    const uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) p[i] = v;
}

__global__ void k_pairs_effective(const uint32_t *src, uint32_t cap, uint32_t *dst) { *dst = *src <= cap ? *src : 0u; }

__global__ void k_zero_f32_n(float *p, const uint32_t *n_dev, int mult) {
    const uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < (uint64_t)*n_dev * mult) p[i] = 0.0f;
}

}  // namespace

void launch_radix_sort(const RadixSort &rs, int max_passes, cudaStream_t s) {
    static int grid_hist = 0, grid_pass = 0;
    if (!grid_pass) {
        int dev = 0, sms = 0, per_h = 0, per_p = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_h, k_radix_hist, RS_THREADS, 0);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_p, k_radix_onesweep, DS_THREADS, 0);
        grid_hist = std::max(1, sms) * std::max(1, per_h);
        grid_pass = std::max(1, sms) * std::max(1, per_p);
    }
    max_passes = std::min(max_passes, RS_MAX_PASSES);
    if (max_passes <= 0 || rs.nblocks <= 0) return;
    cudaMemsetAsync(rs.totals, 0, sizeof(uint32_t) * 256 * max_passes, s);
    k_radix_hist<<<std::min(grid_hist, rs.nblocks), RS_THREADS, 0, s>>>(rs);
    note_launches(1);
    for (int p = 0; p < max_passes; ++p) {
        k_radix_onesweep<<<std::min(grid_pass, rs.nblocks), DS_THREADS, 0, s>>>(rs, p);
        note_launches(1);
    }
}

void launch_depth_npass(const uint32_t *kminmax, uint32_t *npass, cudaStream_t s) {
    k_depth_npass<<<1, 1, 0, s>>>(kminmax, npass);
    note_launches(1);
}

// Grids of the capacity-sized launches: at most a few waves, whatever n_cap
// is (blocks stride over the work counted on the device).
static int sm_count() {
    static int sms = 0;
    if (!sms) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        sms = std::max(sms, 1);
    }
    return sms;
}

static int emit_blocks(int64_t n_cap) {
    return (int)std::min<int64_t>((n_cap + EM_TILE - 1) / EM_TILE, (int64_t)sm_count() * 8);
}

void launch_emit_count(const EmitArgs &a, cudaStream_t s) {
    const int nb = emit_blocks(a.n_cap);
    if (nb == 0) {
        cudaMemsetAsync(a.p_dev, 0, sizeof(uint32_t), s);
        return;
    }
    k_emit_count<<<nb, EM_THREADS, 0, s>>>(a);
    note_launches(1);
    k_emit_scan_blocks<<<1, 1024, 0, s>>>(a);
    note_launches(1);
}

void launch_emit_write(const EmitArgs &a, cudaStream_t s) {
    const int nb = emit_blocks(a.n_cap);
    if (nb == 0) return;
    k_emit_write<<<nb, EM_THREADS, 0, s>>>(a);
    note_launches(1);
}

void launch_ranges(const uint32_t *tiles_sorted, const uint32_t *p_dev, int64_t p_cap, uint2 *ranges,
                   int n_tiles, cudaStream_t s) {
    cudaMemsetAsync(ranges, 0, sizeof(uint2) * (size_t)n_tiles, s);
    if (p_cap <= 0) return;
    const int threads = 256;
    const int64_t blocks = std::min<int64_t>((p_cap + threads - 1) / threads, (int64_t)sm_count() * 16);
    k_ranges<<<(unsigned)blocks, threads, 0, s>>>(tiles_sorted, p_dev, (uint64_t)p_cap, ranges, (uint32_t)n_tiles);
    note_launches(1);
}

void launch_tile_order(const uint2 *ranges, const RenderView *views, int n_views, int n_slots, uint32_t *order,
                       cudaStream_t s) {
    if (n_slots <= 0) return;
    k_tile_order<<<1, 1024, 0, s>>>(ranges, views, n_views, (uint32_t)n_slots, order);
    note_launches(1);
}

void launch_pairs_effective(const uint32_t *src, uint32_t cap, uint32_t *dst, cudaStream_t s) {
    k_pairs_effective<<<1, 1, 0, s>>>(src, cap, dst);
    note_launches(1);
}

void launch_zero_f32_n(float *p, const uint32_t *n_dev, int mult, int64_t n_cap, cudaStream_t s) {
    if (!p || n_cap <= 0) return;
    const int64_t tot = n_cap * mult;
    k_zero_f32_n<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(p, n_dev, mult);
    note_launches(1);
}

void launch_scale_u32(const uint32_t *src, uint32_t k, uint32_t *dst, cudaStream_t s) {
    k_scale_u32<<<1, 1, 0, s>>>(src, k, dst);
    note_launches(1);
}

void launch_fill_u32(uint32_t *p, uint32_t v, int64_t n, cudaStream_t s) {
    if (n <= 0) return;
    k_fill_u32<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(p, v, (uint64_t)n);
    note_launches(1);
}

}  // namespace tsp
