// Internal definitions shared by the CUDA translation units of libtsplat.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/tsplat.h"

namespace tsp {

constexpr int TILE = 16;            // tile edge in pixels (the 3DGS rasterizer's)
constexpr int TILE_PIX = TILE * TILE;
constexpr uint32_t CULLED_KEY = 0xFFFFFFFFu;

// Projected record of one Gaussian instance, 32 bytes (one DRAM sector),
// read by the compositing once per (Gaussian, tile) pair, which evaluates
// alpha = min(alpha_max, 2^(q log2(e) + log2(o))):
//   h0 = (mu_x, mu_y, -a/2, -b), h1 = (-c/2, log2 o, ex, ey)
// where [[a, b], [b, c]] is the conic (inverse 2D covariance) and (ex, ey)
// the half extents of the box outside which o e^q < alpha_min.  The conic is
// kept pre-scaled for the quadratic form (the scalings are exact in FP32).
struct __align__(16) Header {
    float4 h0;
    float4 h1;
};

// Single-precision operations with one rounding each (no contraction), for
// the quantities that decide integers (key mode).
__device__ __forceinline__ float fadd(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float fsub(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ float fmul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float fdiv(float a, float b) { return __fdiv_rn(a, b); }
__device__ __forceinline__ float fsqrt(float a) { return __fsqrt_rn(a); }

// Exponent q of the Gaussian at offset d = p - mean2d,
//   q = -(a dx^2 + 2 b dx dy + c dy^2) / 2,
// from the pre-scaled conic (ha, nb, hc) = (-a/2, -b, -c/2) as
// q = dx (ha dx + nb dy) + hc dy^2.  The backward calls this function; the
// forward composite evaluates the same operations two Gaussians at a time
// (packed f32x2, rounded as the scalar ones), so both take identical skip
// decisions.
__device__ __forceinline__ float gauss_q(float dx, float dy, float ha, float nb, float hc) {
    const float t = __fmaf_rn(ha, dx, __fmul_rn(nb, dy));
    return __fmaf_rn(dx, t, __fmul_rn(__fmul_rn(hc, dy), dy));
}

// alpha before the alpha_max clamp: o e^q
__device__ __forceinline__ float gauss_alpha_raw(float q, float o) { return __fmul_rn(o, __expf(q)); }

// Pack / unpack a tile rect [x0,x1) x [y0,y1) (each < 65536) into 64 bits.
__device__ __forceinline__ uint2 pack_rect(int x0, int y0, int x1, int y1) {
    return make_uint2((uint32_t)x0 | ((uint32_t)y0 << 16), (uint32_t)x1 | ((uint32_t)y1 << 16));
}
__device__ __forceinline__ void unpack_rect(uint2 r, int &x0, int &y0, int &x1, int &y1) {
    x0 = r.x & 0xFFFF; y0 = r.x >> 16; x1 = r.y & 0xFFFF; y1 = r.y >> 16;
}

// Status word written by kernels (first error wins).
__device__ __forceinline__ void set_status(uint32_t *st, uint32_t code) {
    if (st) atomicCAS(st, 0u, code);
}

}  // namespace tsp
