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
// The radix sort is reduce-then-scan (per-block digit histograms, a scan
// over them, a stable scatter ranked with warp match): no kernel waits on
// another block, so nothing can spin.
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
    return rs.npass_dev ? (int)*rs.npass_dev : rs.npass_host;
}

__device__ __forceinline__ uint32_t rs_remap(uint32_t k, bool remap, uint32_t kmin) {
    return remap ? (k == CULLED_KEY ? 0u : k - kmin) : k;
}

__global__ __launch_bounds__(RS_THREADS) void k_radix_upsweep(RadixSort rs, int pass) {
    if (pass >= rs_passes(rs)) return;
    __shared__ uint32_t h[RS_THREADS / 32][256];
    const int tid = threadIdx.x, warp = tid >> 5;
    for (int i = tid; i < (RS_THREADS / 32) * 256; i += RS_THREADS) (&h[0][0])[i] = 0;
    __syncthreads();
    const uint64_t n = *rs.n_dev;
    const bool remap = pass == 0 && rs.kmin;
    const uint32_t kmin = remap ? *rs.kmin : 0u;
    const int shift = 8 * pass;
    const uint32_t *src = pass == 0 ? rs.keys_in : (((pass - 1) & 1) ? rs.keys[1] : rs.keys[0]);
    const uint64_t base = (uint64_t)blockIdx.x * RS_TILE;
#pragma unroll 4
    for (int i = 0; i < RS_ITEMS; ++i) {
        const uint64_t idx = base + (uint64_t)i * RS_THREADS + tid;
        if (idx < n) {
            const uint32_t k = rs_remap(src[idx], remap, kmin);
            atomicAdd(&h[warp][(k >> shift) & 255u], 1u);
        }
    }
    __syncthreads();
    uint32_t sum = 0;
#pragma unroll
    for (int w = 0; w < RS_THREADS / 32; ++w) sum += h[w][tid];
    rs.hist[(size_t)tid * rs.nblocks + blockIdx.x] = sum;
    if (sum) atomicAdd(&rs.totals[pass * 256 + tid], sum);
}

// One block per digit: global offset of every (digit, block) = the counts
// of all smaller digits plus this digit's counts in earlier blocks.
__global__ __launch_bounds__(256) void k_radix_scan(RadixSort rs, int pass) {
    if (pass >= rs_passes(rs)) return;
    __shared__ uint32_t sw[8];
    const int d = blockIdx.x, tid = threadIdx.x;
    uint32_t tot;
    const uint32_t smaller = (tid < d) ? rs.totals[pass * 256 + tid] : 0u;
    block_excl_scan<8>(smaller, sw, tot);
    const uint32_t base = tot;
    const int nb = rs.nblocks;
    const int per = (nb + 255) / 256;
    const int b0 = min(tid * per, nb), b1 = min(b0 + per, nb);
    uint32_t *row = rs.hist + (size_t)d * nb;
    uint32_t local = 0;
    for (int b = b0; b < b1; ++b) local += row[b];
    uint32_t dummy;
    uint32_t run = base + block_excl_scan<8>(local, sw, dummy);
    for (int b = b0; b < b1; ++b) {
        const uint32_t c = row[b];
        row[b] = run;
        run += c;
    }
}

// Stable scatter of one block's 4096 keys: (1) each warp ranks its 512 keys
// (16 rounds of 32) among equal digits with a ballot per digit bit;
// (2) digit offsets inside the block follow from the per-warp counts;
// (3) keys and values are placed in shared memory in digit order;
// (4) consecutive threads write consecutive entries, so each digit's run is
// stored contiguously (coalesced) at its global offset.
constexpr int DS_THREADS = 512;

__global__ __launch_bounds__(DS_THREADS, 2) void k_radix_downsweep(RadixSort rs, int pass) {
    if (pass >= rs_passes(rs)) return;
    constexpr int NW = DS_THREADS / 32;
    constexpr int PER_WARP = RS_TILE / NW;  // 256 keys, 8 rounds of 32
    constexpr int ROUNDS = PER_WARP / 32;
    __shared__ uint32_t wcnt[NW][256];      // per-warp digit counts, then per-warp digit offsets
    __shared__ uint32_t lbase[256];         // first local position of each digit
    __shared__ uint32_t gbase[256];         // global offset of each digit for this block
    __shared__ uint32_t sw[NW];
    __shared__ uint32_t skey[RS_TILE];
    __shared__ uint32_t sval[RS_TILE];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    for (int i = tid; i < NW * 256; i += DS_THREADS) (&wcnt[0][0])[i] = 0;
    __syncthreads();
    const uint64_t n = *rs.n_dev;
    const bool remap = pass == 0 && rs.kmin;
    const uint32_t kmin = remap ? *rs.kmin : 0u;
    const int shift = 8 * pass;
    const bool odd = (pass & 1) != 0;
    const uint32_t *ksrc = pass == 0 ? rs.keys_in : (odd ? rs.keys[0] : rs.keys[1]);
    const uint32_t *vsrc = pass == 0 ? rs.vals_in : (odd ? rs.vals[0] : rs.vals[1]);
    uint32_t *kdst = odd ? rs.keys[1] : rs.keys[0];
    uint32_t *vdst = odd ? rs.vals[1] : rs.vals[0];
    const uint64_t bbase = (uint64_t)blockIdx.x * RS_TILE;
    const uint64_t wbase = bbase + (uint64_t)warp * PER_WARP;
    const uint32_t lt = lanemask_lt();
    uint32_t key[ROUNDS], val[ROUNDS], rank[ROUNDS];
#pragma unroll
    for (int r = 0; r < ROUNDS; ++r) {
        const uint64_t idx = wbase + (uint64_t)r * 32 + lane;
        const bool valid = idx < n;
        uint32_t k = 0, v = 0;
        if (valid) {
            k = rs_remap(ksrc[idx], remap, kmin);
            v = vsrc ? vsrc[idx] : (uint32_t)idx;
        }
        key[r] = k;
        val[r] = v;
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
    {   // thread d < 256 owns digit d: offsets of each warp inside the digit, digit base inside the block
        uint32_t run = 0;
        if (tid < 256) {
#pragma unroll
            for (int w = 0; w < NW; ++w) {
                const uint32_t c = wcnt[w][tid];
                wcnt[w][tid] = run;
                run += c;
            }
        }
        uint32_t tot;
        const uint32_t lb = block_excl_scan<NW>(run, sw, tot);
        if (tid < 256) {
            lbase[tid] = lb;
            gbase[tid] = rs.hist[(size_t)tid * rs.nblocks + blockIdx.x];
        }
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < ROUNDS; ++r) {
        const uint64_t idx = wbase + (uint64_t)r * 32 + lane;
        if (idx < n) {
            const uint32_t d = (key[r] >> shift) & 255u;
            const uint32_t pos = lbase[d] + wcnt[warp][d] + rank[r];
            skey[pos] = key[r];
            sval[pos] = val[r];
        }
    }
    __syncthreads();
    const uint32_t cnt = (uint32_t)min((uint64_t)RS_TILE, n > bbase ? n - bbase : 0);
    for (uint32_t p = tid; p < cnt; p += DS_THREADS) {
        const uint32_t k = skey[p];
        const uint32_t d = (k >> shift) & 255u;
        const uint32_t pos = gbase[d] + (p - lbase[d]);
        kdst[pos] = k;
        vdst[pos] = sval[p];
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

__global__ __launch_bounds__(EM_THREADS) void k_emit_count(EmitArgs a) {
    __shared__ uint32_t sw[EM_THREADS / 32];
    const uint64_t n = *a.n_dev;
    const int np = sv_passes(a.order);
    const uint64_t base = (uint64_t)blockIdx.x * EM_TILE + threadIdx.x;
    uint32_t s = 0;
    for (int i = 0; i < EM_ITEMS; ++i) {
        const uint64_t k = base + (uint64_t)i * EM_THREADS;
        if (k < n) s += a.ntiles[sorted_val(a.order, np, k)];
    }
    uint32_t tot;
    block_excl_scan<EM_THREADS / 32>(s, sw, tot);
    if (threadIdx.x == 0) a.blk_sum[blockIdx.x] = tot;
}

// single block: exclusive scan of the block sums in place, total pairs
__global__ __launch_bounds__(1024) void k_emit_scan_blocks(EmitArgs a, int nblocks) {
    __shared__ uint32_t sw[32];
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
    const uint32_t ns = *a.n_stride;
    const int np = sv_passes(a.order);
    const int lane = threadIdx.x & 31;
    uint64_t running = a.blk_sum[blockIdx.x];
    const uint64_t base = (uint64_t)blockIdx.x * EM_TILE;
    for (int r = 0; r < EM_ITEMS; ++r) {
        const uint64_t k = base + (uint64_t)r * EM_THREADS + threadIdx.x;
        uint32_t id = 0, cnt = 0, vbase = 0;
        int x0 = 0, y0 = 0, x1 = 0, y1 = 0, vtx = 0;
        if (k < n) {
            id = sorted_val(a.order, np, k);
            cnt = a.ntiles[id];
            if (cnt) {
                unpack_rect(a.rect[id], x0, y0, x1, y1);
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
            if (e < wtot) {
                const int loc = (int)(e - so);
                const int ty = oy0 + loc / ow, tx = ox0 + loc % ow;
                a.pair_tile[wfirst + e] = ovb + (uint32_t)(ty * otx + tx);
                a.pair_id[wfirst + e] = oid;
            }
        }
        running += tot;
    }
}

__global__ void k_ranges(const uint32_t *tiles, const uint32_t *p_dev, uint64_t p_cap, uint2 *ranges,
                         uint32_t n_tiles) {
    const uint64_t P = min((uint64_t)*p_dev, p_cap);
    const uint64_t k = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= P) return;
    const uint32_t t = tiles[k];
    if (t >= n_tiles) return;
    if (k == 0 || tiles[k - 1] != t) ranges[t].x = (uint32_t)k;
    if (k == P - 1 || tiles[k + 1] != t) ranges[t].y = (uint32_t)(k + 1);
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
    cudaMemsetAsync(rs.totals, 0, sizeof(uint32_t) * 256 * max_passes, s);
    for (int p = 0; p < max_passes; ++p) {
        k_radix_upsweep<<<rs.nblocks, RS_THREADS, 0, s>>>(rs, p);
    note_launches(1);
        k_radix_scan<<<256, 256, 0, s>>>(rs, p);
    note_launches(1);
        k_radix_downsweep<<<rs.nblocks, DS_THREADS, 0, s>>>(rs, p);
    note_launches(1);
    }
}

void launch_depth_npass(const uint32_t *kminmax, uint32_t *npass, cudaStream_t s) {
    k_depth_npass<<<1, 1, 0, s>>>(kminmax, npass);
    note_launches(1);
}

static int emit_blocks(int64_t n_cap) { return (int)((n_cap + EM_TILE - 1) / EM_TILE); }

void launch_emit_count(const EmitArgs &a, cudaStream_t s) {
    const int nb = emit_blocks(a.n_cap);
    if (nb == 0) {
        cudaMemsetAsync(a.p_dev, 0, sizeof(uint32_t), s);
        return;
    }
    k_emit_count<<<nb, EM_THREADS, 0, s>>>(a);
    note_launches(1);
    k_emit_scan_blocks<<<1, 1024, 0, s>>>(a, nb);
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
    const int64_t blocks = (p_cap + threads - 1) / threads;
    k_ranges<<<(unsigned)blocks, threads, 0, s>>>(tiles_sorted, p_dev, (uint64_t)p_cap, ranges, (uint32_t)n_tiles);
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
