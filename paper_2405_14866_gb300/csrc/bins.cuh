// Device helpers shared by the projection (which counts each tile's pairs)
// and the bucket fill (which places them): the walk over an instance's kept
// tiles, and the warp-aggregated count.
#pragma once
#include <stdint.h>

namespace tsp {

// The kept tiles of one instance, in row-major order of its rect: the whole
// rect, or the set bits of its tight-binning mask.
struct TileWalk {
    uint32_t row0;   // global id of tile (0, y0) of the rect's view
    int tiles_x, x0, w;
    uint32_t rest;   // masked: kept tiles not visited yet (bit = index in the rect)
    uint32_t inv_w;  // masked: ceil(2^16 / w); loc * inv_w >> 16 = loc / w for loc < 32
    int lx, ly;      // whole rect: the next tile
    bool masked;

    __device__ __forceinline__ void clear() {
        row0 = 0; tiles_x = 1; x0 = 0; w = 1; rest = 0; inv_w = 0; lx = 0; ly = 0; masked = false;
    }
    // rect [x0, x1) x [y0, ...) of a view whose tile (0, 0) is tile_base; mask
    // 0xFFFFFFFF = the whole rect (then any size), else at most 32 tiles
    __device__ __forceinline__ void init(uint32_t tile_base, int tx, int x0_, int y0, int x1, uint32_t mask) {
        tiles_x = tx;
        x0 = x0_;
        w = x1 - x0_;
        row0 = tile_base + (uint32_t)(y0 * tx);
        masked = mask != 0xffffffffu;
        rest = mask;
        inv_w = (65535u + (uint32_t)w) / (uint32_t)w;
        lx = 0;
        ly = 0;
    }
    __device__ __forceinline__ uint32_t next() {
        int x, y;
        if (masked) {
            const int loc = __ffs(rest) - 1;
            rest &= rest - 1u;
            y = (int)(((uint32_t)loc * inv_w) >> 16);
            x = loc - y * w;
        } else {
            x = lx;
            y = ly;
            if (++lx == w) {
                lx = 0;
                ++ly;
            }
        }
        return row0 + (uint32_t)(y * tiles_x + x0 + x);
    }
};

// Called by all 32 lanes: each lane's `cnt` tiles of `tw` are added to
// tile_cnt, lanes that meet the same tile adding with one atomic.
__device__ __forceinline__ void warp_count_tiles(TileWalk &tw, uint32_t cnt, uint32_t *tile_cnt) {
    const uint32_t maxc = __reduce_max_sync(0xffffffffu, cnt);
    const int lane = threadIdx.x & 31;
    for (uint32_t k = 0; k < maxc; ++k) {
        const bool act = k < cnt;
        const uint32_t am = __ballot_sync(0xffffffffu, act);
        if (act) {
            const uint32_t t = tw.next();
            const uint32_t peers = __match_any_sync(am, t);
            if (lane == __ffs(peers) - 1) atomicAdd(&tile_cnt[t], (uint32_t)__popc(peers));
        }
    }
}

}  // namespace tsp
