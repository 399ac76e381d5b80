// Point z-buffer: Tele-Aloha lifts one view's depth map to points and
// rasterizes them into other cameras, reading the z-buffer out (Sec. 4.1,
// initial disparities of the cascade), and warps the predicted depth maps
// onto the novel view (Sec. 4.3, fused depth).  A point is a Gaussian's
// mean.  Its camera-space depth pz and image position (mx, my) are computed
// with the single-precision operation order of the projection (k_project);
// it lands on the pixel whose centre is nearest, (floor(mx + 0.5),
// floor(my + 0.5)).  Each pixel keeps the smallest (depth bits, Gaussian id)
// pair through a 64-bit atomicMin, so the nearest point wins and equal
// depths resolve to the lowest id, independent of the arrival order.
#include <algorithm>

#include "common.cuh"
#include "internal.h"

namespace tsp {

namespace {

constexpr unsigned long long ZB_EMPTY = ~0ull;

__global__ void k_zbuf_clear(unsigned long long *keys, uint64_t n) {
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x)
        keys[i] = ZB_EMPTY;
}

__global__ __launch_bounds__(256) void k_zbuf_splat(const float4 *__restrict__ xyzo, const uint32_t *n_dev,
                                                    const __grid_constant__ tsplat_camera cam,
                                                    unsigned long long *keys) {
    const uint64_t n = *n_dev;
    const float *R = cam.R;
    for (uint64_t gi = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; gi < n;
         gi += (uint64_t)gridDim.x * blockDim.x) {
        const float4 g = xyzo[gi];
        const float px = fadd(fadd(fadd(fmul(R[0], g.x), fmul(R[1], g.y)), fmul(R[2], g.z)), cam.t[0]);
        const float py = fadd(fadd(fadd(fmul(R[3], g.x), fmul(R[4], g.y)), fmul(R[5], g.z)), cam.t[1]);
        const float pz = fadd(fadd(fadd(fmul(R[6], g.x), fmul(R[7], g.y)), fmul(R[8], g.z)), cam.t[2]);
        if (!(pz > cam.z_near && pz < cam.z_far)) continue;
        const float mx = fadd(fdiv(fmul(cam.fx, px), pz), cam.cx);
        const float my = fadd(fdiv(fmul(cam.fy, py), pz), cam.cy);
        const float fu = floorf(fadd(mx, 0.5f)), fv = floorf(fadd(my, 0.5f));
        if (!(fu >= 0.0f && fu < (float)cam.width && fv >= 0.0f && fv < (float)cam.height)) continue;
        const uint64_t p = (uint64_t)fv * (uint64_t)cam.width + (uint64_t)fu;
        const unsigned long long key = ((unsigned long long)__float_as_uint(pz) << 32) | (uint32_t)gi;
        atomicMin(&keys[p], key);
    }
}

__global__ void k_zbuf_resolve(const unsigned long long *keys, uint64_t n, float *depth, int32_t *id) {
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
        const unsigned long long k = keys[i];
        const bool empty = k == ZB_EMPTY;
        depth[i] = empty ? 0.0f : __uint_as_float((uint32_t)(k >> 32));
        if (id) id[i] = empty ? -1 : (int32_t)(uint32_t)k;
    }
}

int zb_grid(uint64_t n) {
    const int sms = sm_count();
    return (int)std::max<uint64_t>(1, std::min<uint64_t>((n + 255) / 256, (uint64_t)sms * 16));
}

}  // namespace

void launch_zbuffer(const float4 *xyzo, const uint32_t *n_dev, int64_t n_cap, const tsplat_camera &cam,
                    unsigned long long *keys, float *depth, int32_t *id, cudaStream_t s) {
    const uint64_t pix = (uint64_t)cam.width * (uint64_t)cam.height;
    k_zbuf_clear<<<zb_grid(pix), 256, 0, s>>>(keys, pix);
    if (n_cap > 0) k_zbuf_splat<<<zb_grid((uint64_t)n_cap), 256, 0, s>>>(xyzo, n_dev, cam, keys);
    k_zbuf_resolve<<<zb_grid(pix), 256, 0, s>>>(keys, pix, depth, id);
    note_launches(n_cap > 0 ? 3 : 2);
}

}  // namespace tsp
