// tsplat_build_into_noalloc: lifting (tsplat_build_into) without any device
// allocation.  The paper has no counterpart; this exists for callers that
// must not allocate device memory at call time -- a frame loop with a fixed
// latency budget (cudaMalloc/cudaFree synchronize the device), or a host
// whose device memory is fully owned by another allocator.  Its only scratch, the per-block foreground counts
// and offsets of the stream compaction, lives in a fixed device array below.
#include <stdio.h>
#include <string.h>

#include <mutex>

#include "common.cuh"
#include "internal.h"

namespace {

// Largest total source-pixel count one call may lift: 64 Mi pixels (e.g.
// 16 views of 2048 x 2048).  Scratch: 2 words per 1024-pixel block = 512 KiB,
// held by every GPU that loads the library until the process exits.
constexpr int64_t NOALLOC_MAX_PIXELS = int64_t(64) << 20;
constexpr int NOALLOC_MAX_BLOCKS = (int)(NOALLOC_MAX_PIXELS / tsp::BUILD_PIX_PER_BLOCK);

static __device__ __align__(256) uint32_t g_build_scratch[2 * NOALLOC_MAX_BLOCKS];

// Device address of g_build_scratch per device, resolved once per device
// with that device current (the host-side name is only a stand-in).
constexpr int MAX_DEVICES = 64;
std::mutex g_mu;
uint32_t *g_scratch_ptr[MAX_DEVICES] = {};

tsplat_status scratch_for_current_device(uint32_t **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return tsp::record_error(TSPLAT_ERR_CUDA, cudaGetErrorString(e));
    if (dev < 0 || dev >= MAX_DEVICES) return tsp::record_error(TSPLAT_ERR_UNSUPPORTED, "build_into_noalloc: device index >= 64");
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_scratch_ptr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_build_scratch);
        if (e != cudaSuccess || p == nullptr) {
            char msg[256];
            snprintf(msg, sizeof(msg), "build_into_noalloc: cudaGetSymbolAddress failed: %s", cudaGetErrorString(e));
            return tsp::record_error(TSPLAT_ERR_CUDA, msg);
        }
        g_scratch_ptr[dev] = static_cast<uint32_t *>(p);
    }
    *out = g_scratch_ptr[dev];
    return TSPLAT_OK;
}

}  // namespace

extern "C" tsplat_status tsplat_build_into_noalloc(tsplat_gaussians *g, const tsplat_src_view *views,
                                                   int32_t n_views, void *stream) {
    using namespace tsp;
    char msg[256];
    if (!g || !views) return record_error(TSPLAT_ERR_INVALID_ARG, "build_into_noalloc: NULL argument");
    if (n_views < 1 || n_views > MAX_VIEWS) return record_error(TSPLAT_ERR_INVALID_ARG, "build_into_noalloc: n_views not in [1, 16]");
    GaussianStore st;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    BuildArgs a;
    memset(&a, 0, sizeof(a));
    int64_t total = 0;
    for (int v = 0; v < n_views; ++v) {
        const tsplat_src_view &sv = views[v];
        const int H = sv.cam.height, W = sv.cam.width;
        if (H <= 0 || W <= 0 || H > 16383 || W > 16383) {
            snprintf(msg, sizeof(msg), "build_into_noalloc: view %d: size %dx%d", v, W, H);
            return record_error(TSPLAT_ERR_INVALID_ARG, msg);
        }
        if (!sv.depth || !sv.scale || !sv.opacity || !sv.feat) return record_error(TSPLAT_ERR_INVALID_ARG, "build_into_noalloc: NULL map");
        if (sv.quat && ((uintptr_t)sv.quat & 15)) return record_error(TSPLAT_ERR_INVALID_ARG, "build_into_noalloc: quat not 16-byte aligned");
        if (sv.feat_dtype != TSPLAT_F32 && sv.feat_dtype != TSPLAT_BF16) return record_error(TSPLAT_ERR_INVALID_ARG, "build_into_noalloc: feat_dtype");
        if (sv.flags != 0) return record_error(TSPLAT_ERR_UNSUPPORTED, "build_into_noalloc: source view flags are not supported here");
        ViewDesc &d = a.views[v];
        d.depth = sv.depth; d.mask = sv.mask; d.scale = sv.scale; d.quat = sv.quat; d.opacity = sv.opacity;
        d.feat = sv.feat; d.feat_dtype = sv.feat_dtype; d.H = H; d.W = W; d.cam = sv.cam;
        total += (int64_t)H * W;
    }
    if (total > NOALLOC_MAX_PIXELS) {
        snprintf(msg, sizeof(msg), "build_into_noalloc: %lld source pixels exceed the fixed scratch limit of %lld",
                 (long long)total, (long long)NOALLOC_MAX_PIXELS);
        return record_error(TSPLAT_ERR_CAPACITY, msg);
    }
    // every check runs before the store records this stream as its last writer
    gaussians_peek(g, st, nullptr);
    if (total > st.cap) {
        snprintf(msg, sizeof(msg), "build_into_noalloc: %lld pixels exceed capacity %lld", (long long)total, (long long)st.cap);
        return record_error(TSPLAT_ERR_CAPACITY, msg);
    }
    for (int v = 0; v < n_views; ++v)
        if ((st.C % 4) == 0 && ((uintptr_t)views[v].feat & 15)) return record_error(TSPLAT_ERR_INVALID_ARG, "build_into_noalloc: feat not 16-byte aligned");
    uint32_t *scratch = nullptr;
    tsplat_status rc = scratch_for_current_device(&scratch);
    if (rc != TSPLAT_OK) return rc;
    a.n_views = n_views;
    a.total_pix = total;
    a.C = st.C;
    a.out_dtype = st.dtype;
    a.xyzo = st.xyzo;
    a.cova = st.cova;
    a.covb = st.covb;
    a.feat = st.feat;
    a.fsplit = st.fsplit;
    const int64_t nblocks = layout_build_blocks(a);
    if (nblocks > NOALLOC_MAX_BLOCKS) return record_error(TSPLAT_ERR_CAPACITY, "build_into_noalloc: too many lifting blocks for the fixed scratch");
    a.nblocks = (int)nblocks;
    gaussians_store(g, st, s);
    // every entry of the scratch that the kernels read is written earlier in the same call
    a.blk_cnt = scratch;
    a.blk_off = scratch + NOALLOC_MAX_BLOCKS;
    a.n_dev = st.n_dev;
    launch_build(a, s);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return record_error(TSPLAT_ERR_CUDA, cudaGetErrorString(e));
    return TSPLAT_OK;
}
