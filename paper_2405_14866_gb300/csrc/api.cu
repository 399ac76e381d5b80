// Host side of the C ABI declared in include/tsplat.h: handles, scratch
// management and the ordering of the kernel launches.  No arithmetic of the
// method happens here; every step runs in the kernels of k_*.cu.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <new>
#include <string>

#include "common.cuh"
#include "internal.h"

using namespace tsp;

namespace {

thread_local std::string g_err;
std::atomic<uint64_t> g_launches{0};

tsplat_status fail(tsplat_status st, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_err = buf;
    return st;
}

#define TRY_CUDA(expr)                                                                                \
    do {                                                                                              \
        cudaError_t e_ = (expr);                                                                      \
        if (e_ != cudaSuccess)                                                                        \
            return fail(e_ == cudaErrorMemoryAllocation ? TSPLAT_ERR_OOM : TSPLAT_ERR_CUDA, "%s: %s (%s:%d)", \
                        #expr, cudaGetErrorString(e_), __FILE__, __LINE__);                          \
    } while (0)

#define TRY(expr)                                  \
    do {                                           \
        tsplat_status s_ = (expr);                 \
        if (s_ != TSPLAT_OK) return s_;            \
    } while (0)

tsplat_status check_launch(const char *what) {
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail(TSPLAT_ERR_CUDA, "%s: kernel launch failed: %s", what, cudaGetErrorString(e));
    return TSPLAT_OK;
}

inline cudaStream_t S(void *s) { return reinterpret_cast<cudaStream_t>(s); }

// A device buffer that grows (stream-ordered) and never shrinks.
struct DBuf {
    void *p = nullptr;
    size_t bytes = 0;
    template <typename T>
    T *as() const { return reinterpret_cast<T *>(p); }
};

tsplat_status grow(DBuf &b, size_t bytes, cudaStream_t s) {
    if (bytes == 0) bytes = 16;
    if (b.bytes >= bytes) return TSPLAT_OK;
    if (b.p) TRY_CUDA(cudaFreeAsync(b.p, s));
    b.p = nullptr;
    b.bytes = 0;
    const size_t nb = bytes + bytes / 8 + 256;
    TRY_CUDA(cudaMallocAsync(&b.p, nb, s));
    b.bytes = nb;
    return TSPLAT_OK;
}

void release(DBuf &b) {
    if (b.p) cudaFree(b.p);
    b.p = nullptr;
    b.bytes = 0;
}

size_t feat_size(int dtype) { return dtype == TSPLAT_BF16 ? 2 : 4; }

}  // namespace

namespace tsp {
void note_launches(int n) { g_launches.fetch_add((uint64_t)n, std::memory_order_relaxed); }
}  // namespace tsp

// ------------------------------------------------------------------ handles

struct tsplat_gaussians {
    int64_t cap = 0;
    int C = 0;
    int dtype = TSPLAT_F32;
    DBuf xyzo, cova, covb, feat, fsplit, n_dev, blk;
    cudaStream_t last_stream = nullptr;
};

struct tsplat_ctx {
    // N-sized
    DBuf hdr, rect, ntiles, tmask, dkey, radius;
    // P-sized
    DBuf pk0, pk1, pv0, pv1, tcnt;
    // tiles / pixels / view table
    DBuf ranges, tfinal, last, views;
    DBuf zkeys;  // point z-buffer scratch
    DBuf torder; // composite tile order
    DBuf tinfo;  // per position of that order: tile and list range
    DBuf fsplit; // (hi, lo) rows of a rasterize call's FP32 features
    // small words (SM_*): visible count, P, effective P, status, tile and unit counters, N
    DBuf small;
    uint32_t *host_small = nullptr;  // pinned mirror
    int64_t p_cap = 0;

    // last render
    cudaStream_t stream = nullptr;
    int64_t n_cap = 0;
    const uint32_t *n_dev = nullptr;
    int W = 0, H = 0, C = 0, dtype = TSPLAT_F32, tiles_x = 0, tiles_y = 0;
    int n_slots = 0;  // tile slots of the last render (all its views)
    const void *feat = nullptr;
    const void *feat_split = nullptr;  // FP32 features: their split rows
    const uint32_t *pairs = nullptr;  // sorted Gaussian ids
    bool saved = false;
    bool has_cam = false;        // the last render had a camera (tsplat_render)
    tsplat_camera cam;
    tsplat_render_params par;
    float alpha_max = 0, alpha_min = 0;
    // stage events of profiled renders (TSPLAT_RENDER_PROFILE): a ring of
    // the last RING renders, averaged and reset by tsplat_ctx_timings
    static constexpr int N_EV = 6, RING = 256;
    cudaEvent_t ev[RING][N_EV] = {};
    int64_t n_prof = 0;
};

namespace {
enum { SM_NVIS = 2, SM_P = 4, SM_PEFF = 5, SM_STATUS = 6, SM_TILECTR = 7,
       SM_N = 8, SM_NINST = 9, SM_BINCTR = 10, SM_BWDCTR = 14, SM_WORDS = 16 };
uint32_t *small_ptr(tsplat_ctx *c, int w) { return c->small.as<uint32_t>() + w; }
}  // namespace

namespace tsp {
void gaussians_store(tsplat_gaussians *g, GaussianStore &out, cudaStream_t writer) {
    out.cap = g->cap;
    out.C = g->C;
    out.dtype = g->dtype;
    out.xyzo = g->xyzo.as<float4>();
    out.cova = g->cova.as<float4>();
    out.covb = g->covb.as<float2>();
    out.feat = g->feat.p;
    out.fsplit = g->fsplit.p;
    out.n_dev = g->n_dev.as<uint32_t>();
    g->last_stream = writer;
}
void gaussians_peek(const tsplat_gaussians *g, GaussianStore &out, cudaStream_t *last_writer) {
    out.cap = g->cap;
    out.C = g->C;
    out.dtype = g->dtype;
    out.xyzo = g->xyzo.as<float4>();
    out.cova = g->cova.as<float4>();
    out.covb = g->covb.as<float2>();
    out.feat = g->feat.p;
    out.fsplit = g->fsplit.p;
    out.n_dev = g->n_dev.as<uint32_t>();
    if (last_writer) *last_writer = g->last_stream;
}
tsplat_status record_error(tsplat_status st, const char *msg) { return fail(st, "%s", msg); }
}  // namespace tsp



extern "C" {

void tsplat_render_params_default(tsplat_render_params *p) {
    if (!p) return;
    p->lowpass = 0.3f;
    p->alpha_max = 0.99f;
    p->alpha_min = 1.0f / 255.0f;
    p->t_min = 1e-4f;
    p->frustum_clamp = 1.3f;
    p->flags = 0;
}

const char *tsplat_last_error(void) { return g_err.c_str(); }

const char *tsplat_version(void) { return "tsplat 0.1 (sm_103a)"; }

tsplat_status tsplat_gaussians_create(int64_t capacity, int32_t C, int32_t feat_dtype, tsplat_gaussians **out) {
    if (!out) return fail(TSPLAT_ERR_INVALID_ARG, "gaussians_create: out is NULL");
    *out = nullptr;
    if (capacity < 0 || capacity >= (int64_t)1 << 31) return fail(TSPLAT_ERR_INVALID_ARG, "capacity %lld out of range", (long long)capacity);
    if (C < 1 || C > 64) return fail(TSPLAT_ERR_INVALID_ARG, "C = %d not in [1, 64]", C);
    if (feat_dtype != TSPLAT_F32 && feat_dtype != TSPLAT_BF16) return fail(TSPLAT_ERR_INVALID_ARG, "feat_dtype %d", feat_dtype);
    tsplat_gaussians *g = new (std::nothrow) tsplat_gaussians();
    if (!g) return fail(TSPLAT_ERR_OOM, "host allocation failed");
    g->cap = capacity;
    g->C = C;
    g->dtype = feat_dtype;
    const size_t n = (size_t)std::max<int64_t>(capacity, 1);
    cudaStream_t s = nullptr;
    tsplat_status st = TSPLAT_OK;
    if ((st = grow(g->xyzo, n * 16, s)) || (st = grow(g->cova, n * 16, s)) || (st = grow(g->covb, n * 8, s)) ||
        (st = grow(g->feat, n * C * feat_size(feat_dtype), s)) || (st = grow(g->n_dev, 16, s)) ||
        (feat_dtype == TSPLAT_F32 && (st = grow(g->fsplit, n * 4 * padded_channels(C), s)))) {
        tsplat_gaussians_destroy(g);
        return st;
    }
    // the split rows' padding columns are never written: zero once
    if (cudaMemsetAsync(g->n_dev.p, 0, 4, s) != cudaSuccess ||
        (g->fsplit.p && cudaMemsetAsync(g->fsplit.p, 0, g->fsplit.bytes, s) != cudaSuccess) ||
        cudaStreamSynchronize(s) != cudaSuccess) {
        tsplat_gaussians_destroy(g);
        return fail(TSPLAT_ERR_CUDA, "gaussians_create: %s", cudaGetErrorString(cudaGetLastError()));
    }
    *out = g;
    return TSPLAT_OK;
}

tsplat_status tsplat_gaussians_destroy(tsplat_gaussians *g) {
    if (!g) return TSPLAT_OK;
    cudaDeviceSynchronize();
    release(g->xyzo); release(g->cova); release(g->covb); release(g->feat); release(g->fsplit); release(g->n_dev);
    release(g->blk);
    delete g;
    return TSPLAT_OK;
}

tsplat_status tsplat_gaussians_set(tsplat_gaussians *g, int64_t n, const float *mean, const float *cov,
                                   const float *opac, const void *feat, int32_t feat_dtype_in, void *stream) {
    if (!g) return fail(TSPLAT_ERR_INVALID_ARG, "gaussians_set: g is NULL");
    if (n < 0 || n > g->cap) return fail(TSPLAT_ERR_CAPACITY, "gaussians_set: n = %lld exceeds capacity %lld", (long long)n, (long long)g->cap);
    if (n > 0 && (!mean || !cov || !opac || !feat)) return fail(TSPLAT_ERR_INVALID_ARG, "gaussians_set: NULL array");
    if (feat_dtype_in != TSPLAT_F32 && feat_dtype_in != TSPLAT_BF16) return fail(TSPLAT_ERR_INVALID_ARG, "feat_dtype %d", feat_dtype_in);
    launch_gaussians_set(n, mean, cov, opac, feat, feat_dtype_in, g->C, g->dtype, g->xyzo.as<float4>(),
                         g->cova.as<float4>(), g->covb.as<float2>(), g->feat.p, g->fsplit.p, g->n_dev.as<uint32_t>(),
                         S(stream));
    g->last_stream = S(stream);
    return check_launch("gaussians_set");
}

tsplat_status tsplat_gaussians_count(const tsplat_gaussians *g, int64_t *n) {
    if (!g || !n) return fail(TSPLAT_ERR_INVALID_ARG, "gaussians_count: NULL argument");
    uint32_t v = 0;
    TRY_CUDA(cudaStreamSynchronize(g->last_stream));
    TRY_CUDA(cudaMemcpy(&v, g->n_dev.p, 4, cudaMemcpyDeviceToHost));
    *n = v;
    return TSPLAT_OK;
}

tsplat_status tsplat_gaussians_shape(const tsplat_gaussians *g, int64_t *capacity, int32_t *C, int32_t *feat_dtype) {
    if (!g) return fail(TSPLAT_ERR_INVALID_ARG, "gaussians_shape: g is NULL");
    if (capacity) *capacity = g->cap;
    if (C) *C = g->C;
    if (feat_dtype) *feat_dtype = g->dtype;
    return TSPLAT_OK;
}

tsplat_status tsplat_gaussians_get(const tsplat_gaussians *g, float *mean, float *cov, float *opac, void *feat,
                                   void *stream) {
    if (!g) return fail(TSPLAT_ERR_INVALID_ARG, "gaussians_get: g is NULL");
    TRY_CUDA(cudaStreamSynchronize(g->last_stream));
    launch_gaussians_get(g->n_dev.as<uint32_t>(), g->cap, g->C, g->dtype, g->xyzo.as<float4>(), g->cova.as<float4>(),
                         g->covb.as<float2>(), g->feat.p, mean, cov, opac, feat, S(stream));
    return check_launch("gaussians_get");
}

// The lifting's launch arguments for `views` into the store g (also used by
// the adjoint, which walks the same pixels in the same order).
static tsplat_status build_args(tsplat_gaussians *g, const tsplat_src_view *views, int32_t n_views, BuildArgs &a,
                                cudaStream_t s) {
    if (n_views < 1 || n_views > MAX_VIEWS) return fail(TSPLAT_ERR_INVALID_ARG, "n_views = %d not in [1, %d]", n_views, MAX_VIEWS);
    memset(&a, 0, sizeof(a));
    int64_t total = 0;
    for (int v = 0; v < n_views; ++v) {
        const tsplat_src_view &sv = views[v];
        const int H = sv.cam.height, W = sv.cam.width;
        if (H <= 0 || W <= 0 || H > 16383 || W > 16383) return fail(TSPLAT_ERR_INVALID_ARG, "view %d: size %dx%d", v, W, H);
        if (!sv.depth || !sv.scale || !sv.opacity || !sv.feat) return fail(TSPLAT_ERR_INVALID_ARG, "view %d: NULL map", v);
        if (sv.quat && ((uintptr_t)sv.quat & 15)) return fail(TSPLAT_ERR_INVALID_ARG, "view %d: quat not 16-byte aligned", v);
        if ((g->C % 4) == 0 && ((uintptr_t)sv.feat & 15)) return fail(TSPLAT_ERR_INVALID_ARG, "view %d: feat not 16-byte aligned", v);
        if (sv.feat_dtype != TSPLAT_F32 && sv.feat_dtype != TSPLAT_BF16) return fail(TSPLAT_ERR_INVALID_ARG, "view %d: feat_dtype", v);
        if (sv.flags & ~(int32_t)TSPLAT_SRC_COMPACT) return fail(TSPLAT_ERR_INVALID_ARG, "view %d: unknown flags 0x%x", v, sv.flags);
        if ((sv.flags & TSPLAT_SRC_COMPACT) && !sv.mask) return fail(TSPLAT_ERR_INVALID_ARG, "view %d: TSPLAT_SRC_COMPACT needs a mask", v);
        ViewDesc &d = a.views[v];
        d.depth = sv.depth; d.mask = sv.mask; d.scale = sv.scale; d.quat = sv.quat; d.opacity = sv.opacity;
        d.feat = sv.feat; d.feat_dtype = sv.feat_dtype; d.compact = (sv.flags & TSPLAT_SRC_COMPACT) != 0;
        d.H = H; d.W = W; d.cam = sv.cam;
        total += (int64_t)H * W;
    }
    if (total > g->cap) return fail(TSPLAT_ERR_CAPACITY, "build: %lld pixels exceed capacity %lld", (long long)total, (long long)g->cap);
    a.n_views = n_views;
    a.total_pix = total;
    a.C = g->C;
    a.out_dtype = g->dtype;
    a.xyzo = g->xyzo.as<float4>();
    a.cova = g->cova.as<float4>();
    a.covb = g->covb.as<float2>();
    a.feat = g->feat.p;
    a.fsplit = g->fsplit.p;
    a.nblocks = (int)layout_build_blocks(a);
    TRY(grow(g->blk, (size_t)a.nblocks * 8, s));
    a.blk_cnt = g->blk.as<uint32_t>();
    a.blk_off = a.blk_cnt + a.nblocks;
    a.n_dev = g->n_dev.as<uint32_t>();
    return TSPLAT_OK;
}

static tsplat_status build_into(tsplat_gaussians *g, const tsplat_src_view *views, int32_t n_views, cudaStream_t s) {
    BuildArgs a;
    TRY(build_args(g, views, n_views, a, s));
    launch_build(a, s);
    g->last_stream = s;
    return check_launch("build");
}

tsplat_status tsplat_build(const tsplat_src_view *views, int32_t n_views, int32_t C, int32_t feat_dtype,
                           tsplat_gaussians **out, void *stream) {
    if (!views || !out) return fail(TSPLAT_ERR_INVALID_ARG, "build: NULL argument");
    if (n_views < 1 || n_views > MAX_VIEWS) return fail(TSPLAT_ERR_INVALID_ARG, "n_views = %d not in [1, %d]", n_views, MAX_VIEWS);
    int64_t total = 0;
    for (int v = 0; v < n_views; ++v) total += (int64_t)std::max(views[v].cam.height, 0) * std::max(views[v].cam.width, 0);
    TRY(tsplat_gaussians_create(total, C, feat_dtype, out));
    tsplat_status st = build_into(*out, views, n_views, S(stream));
    if (st != TSPLAT_OK) {
        tsplat_gaussians_destroy(*out);
        *out = nullptr;
    }
    return st;
}

tsplat_status tsplat_build_into(tsplat_gaussians *g, const tsplat_src_view *views, int32_t n_views, void *stream) {
    if (!g || !views) return fail(TSPLAT_ERR_INVALID_ARG, "build_into: NULL argument");
    return build_into(g, views, n_views, S(stream));
}

// ---------------------------------------------------------------- contexts

tsplat_status tsplat_ctx_create(tsplat_ctx **out) {
    if (!out) return fail(TSPLAT_ERR_INVALID_ARG, "ctx_create: out is NULL");
    tsplat_ctx *c = new (std::nothrow) tsplat_ctx();
    if (!c) return fail(TSPLAT_ERR_OOM, "host allocation failed");
    tsplat_status st = grow(c->small, SM_WORDS * 4, nullptr);
    if (st == TSPLAT_OK && cudaMallocHost(&c->host_small, SM_WORDS * 4) != cudaSuccess) st = fail(TSPLAT_ERR_OOM, "pinned allocation failed");
    if (st == TSPLAT_OK && (cudaMemset(c->small.p, 0, SM_WORDS * 4) != cudaSuccess)) st = fail(TSPLAT_ERR_CUDA, "memset");
    if (st == TSPLAT_OK && cudaStreamSynchronize(nullptr) != cudaSuccess) st = fail(TSPLAT_ERR_CUDA, "sync");
    if (st == TSPLAT_OK) bin_sort_setup();
    if (st != TSPLAT_OK) {
        tsplat_ctx_destroy(c);
        return st;
    }
    *out = c;
    return TSPLAT_OK;
}

tsplat_status tsplat_ctx_destroy(tsplat_ctx *c) {
    if (!c) return TSPLAT_OK;
    cudaDeviceSynchronize();
    DBuf *bufs[] = {&c->hdr, &c->rect, &c->ntiles, &c->tmask, &c->dkey, &c->radius, &c->pk0, &c->pk1, &c->pv0,
                    &c->pv1, &c->tcnt,
                    &c->ranges, &c->tfinal, &c->last, &c->views, &c->zkeys, &c->torder, &c->tinfo, &c->fsplit,
                    &c->small};
    for (DBuf *b : bufs) release(*b);
    for (auto &row : c->ev)
        for (cudaEvent_t e : row)
            if (e) cudaEventDestroy(e);
    if (c->host_small) cudaFreeHost(c->host_small);
    delete c;
    return TSPLAT_OK;
}

static tsplat_status ensure_n(tsplat_ctx *c, int64_t n, cudaStream_t s) {
    const size_t N = (size_t)std::max<int64_t>(n, 1);
    TRY(grow(c->hdr, N * sizeof(Header), s));
    TRY(grow(c->rect, N * 8, s));
    TRY(grow(c->ntiles, N * 4, s));
    TRY(grow(c->tmask, N * 4, s));
    TRY(grow(c->dkey, N * 4, s));
    TRY(grow(c->radius, N * 4, s));
    return TSPLAT_OK;
}

static tsplat_status ensure_p(tsplat_ctx *c, int64_t p, cudaStream_t s) {
    if (p <= c->p_cap && c->pk0.p) return TSPLAT_OK;
    const int64_t cap = std::min<int64_t>(std::max<int64_t>(p + p / 8, 4096), 0xfffffffell);
    if (p > cap) return fail(TSPLAT_ERR_CAPACITY, "render: %lld pairs exceed the 32-bit pair index", (long long)p);
    TRY(grow(c->pk0, (size_t)cap * 4, s));
    TRY(grow(c->pk1, (size_t)cap * 4, s));
    TRY(grow(c->pv0, (size_t)cap * 4, s));
    TRY(grow(c->pv1, (size_t)cap * 4, s));
    c->p_cap = cap;
    return TSPLAT_OK;
}

// Per-tile buffers of a render over n_tiles tile slots (all views of a batch).
static tsplat_status ensure_tiles(tsplat_ctx *c, int64_t n_tiles, cudaStream_t s) {
    const size_t T = (size_t)std::max<int64_t>(n_tiles, 1);
    TRY(grow(c->ranges, T * 8, s));
    TRY(grow(c->torder, T * 4, s));
    TRY(grow(c->tinfo, T * 16, s));
    TRY(grow(c->tcnt, T * 8, s));  // counts, then fill cursors
    TRY(grow(c->views, sizeof(RenderView) * MAX_BATCH, s));
    return TSPLAT_OK;
}

static bool tiles_fit(const tsplat_ctx *c, int64_t n_tiles) {
    const size_t T = (size_t)std::max<int64_t>(n_tiles, 1);
    return c->ranges.bytes >= T * 8 && c->torder.bytes >= T * 4 && c->tinfo.bytes >= T * 16 && c->tcnt.bytes >= T * 8 &&
           c->views.bytes >= sizeof(RenderView) * MAX_BATCH;
}

static tsplat_status ensure_pix(tsplat_ctx *c, int W, int H, int n_tiles, bool save, cudaStream_t s) {
    TRY(ensure_tiles(c, n_tiles, s));
    if (save) {
        TRY(grow(c->tfinal, (size_t)W * H * 4, s));
        TRY(grow(c->last, (size_t)W * H * 4, s));
    }
    return TSPLAT_OK;
}

tsplat_status tsplat_ctx_reserve(tsplat_ctx *c, int64_t max_gaussians, int64_t max_pairs, int32_t max_width,
                                 int32_t max_height, int32_t C) {
    if (!c) return fail(TSPLAT_ERR_INVALID_ARG, "ctx_reserve: ctx is NULL");
    if (max_gaussians < 0 || max_pairs < 0 || max_width < 0 || max_height < 0) return fail(TSPLAT_ERR_INVALID_ARG, "ctx_reserve: negative size");
    if (C < 0 || C > 64) return fail(TSPLAT_ERR_INVALID_ARG, "ctx_reserve: C = %d not in [0, 64]", C);
    cudaStream_t s = nullptr;
    TRY(ensure_n(c, max_gaussians, s));
    // tsplat_rasterize with FP32 features stages their (hi, lo) rows here
    if (C > 0) TRY(grow(c->fsplit, (size_t)std::max<int64_t>(max_gaussians, 1) * 4 * padded_channels(C), s));
    TRY(ensure_p(c, max_pairs, s));
    const int tx = (max_width + TILE - 1) / TILE, ty = (max_height + TILE - 1) / TILE;
    TRY(ensure_pix(c, max_width, max_height, tx * ty, true, s));
    TRY_CUDA(cudaStreamSynchronize(s));
    return TSPLAT_OK;
}

static tsplat_status mark(tsplat_ctx *c, bool prof, int i, cudaStream_t s) {
    if (!prof) return TSPLAT_OK;
    cudaEvent_t &e = c->ev[c->n_prof % tsplat_ctx::RING][i];
    if (!e) TRY_CUDA(cudaEventCreate(&e));
    TRY_CUDA(cudaEventRecord(e, s));
    if (i == tsplat_ctx::N_EV - 1) ++c->n_prof;
    return TSPLAT_OK;
}

// A2 (done by the caller of this function) .. A7
// n_cap: Gaussian count bound (grid sizing); n_dev: Gaussian count N on
// the device; the render has n_views * N instances (instance i = view * N + id).
static tsplat_status render_tail(tsplat_ctx *c, int64_t n_cap, const uint32_t *n_dev,
                                 const ViewBatch &vb, const void *feat, const void *fsplit, int C, int dtype,
                                 const tsplat_render_params &par, cudaStream_t s) {
    const int n_tiles = (int)vb.n_tiles_total;
    const int W = vb.v[0].width, H = vb.v[0].height;
    const int tiles_x = vb.v[0].tiles_x, tiles_y = vb.v[0].tiles_y;
    const bool async_mode = (par.flags & TSPLAT_RENDER_ASYNC) != 0;
    const bool save = (par.flags & TSPLAT_RENDER_SAVE) != 0;
    const bool prof = (par.flags & TSPLAT_RENDER_PROFILE) != 0;
    uint32_t *sm = c->small.as<uint32_t>();
    if (dtype == TSPLAT_F32 && !fsplit) return fail(TSPLAT_ERR_INVALID_ARG, "render: FP32 features without their split rows");
    if (!tiles_fit(c, n_tiles)) return fail(TSPLAT_ERR_CAPACITY, "render: the context holds fewer than %d tile slots", n_tiles);
    const int64_t inst_cap = n_cap * vb.n_views;
    const uint32_t *n_inst = n_dev;
    if (vb.n_views > 1) {
        launch_scale_u32(n_dev, (uint32_t)vb.n_views, sm + SM_NINST, s);
        n_inst = sm + SM_NINST;
    }
    TRY(mark(c, prof, 1, s));

    // (tile, depth, id) order of the pairs through per-tile buckets
    BinArgs bn;
    memset(&bn, 0, sizeof(bn));
    bn.n_inst = n_inst;
    bn.n_stride = n_dev;
    bn.inst_cap = inst_cap;
    bn.ntiles = c->ntiles.as<uint32_t>();
    bn.rect = c->rect.as<uint2>();
    bn.tmask = (par.flags & TSPLAT_RENDER_TIGHT) ? c->tmask.as<uint32_t>() : nullptr;
    bn.dkey = c->dkey.as<uint32_t>();
    bn.views = c->views.as<RenderView>();
    bn.n_views = vb.n_views;
    bn.n_slots = (uint32_t)n_tiles;
    bn.tile_cnt = c->tcnt.as<uint32_t>();
    bn.cursor = bn.tile_cnt + std::max(n_tiles, 1);
    bn.ranges = c->ranges.as<uint2>();
    bn.p_dev = sm + SM_P;
    bn.p_eff = sm + SM_PEFF;
    bn.tile_order = c->torder.as<uint32_t>();
    bn.tile_order_out = c->torder.as<uint32_t>();
    bn.tile_info_out = c->tinfo.as<uint4>();
    bn.tile_ctr = sm + SM_BINCTR;
    bn.status = sm + SM_STATUS;
    launch_bin_scan(bn, s);
    TRY(check_launch("render: scan"));
    TRY(mark(c, prof, 2, s));

    if (!async_mode) {
        TRY_CUDA(cudaMemcpyAsync(c->host_small + SM_P, sm + SM_P, 4, cudaMemcpyDeviceToHost, s));
        TRY_CUDA(cudaStreamSynchronize(s));
        TRY(ensure_p(c, (int64_t)c->host_small[SM_P], s));
    } else if (!c->pk0.p) {
        return fail(TSPLAT_ERR_CAPACITY, "render: TSPLAT_RENDER_ASYNC needs tsplat_ctx_reserve first");
    }
    bn.p_cap = c->p_cap;
    bn.bk_key = c->pk0.as<uint32_t>();
    bn.bk_id = c->pv0.as<uint32_t>();
    bn.tmp_key = c->pk1.as<uint32_t>();
    bn.tmp_id = c->pv1.as<uint32_t>();
    bn.ids_out = c->pv1.as<uint32_t>();  // the scratch of a bucket ends before its output is written
    launch_bin_fill(bn, s);
    TRY(mark(c, prof, 3, s));
    // instances per tile slot, from the store's capacity: about 4 K for a
    // 512x512 and 1.8 K for a 768x768 view of a 4 Mi-pixel frame, whose
    // buckets sort faster with more warps per tile; 1 K at 1024x1024, where
    // more tiles in flight per SM pay more
    bn.sort_wide = (double)inst_cap > 1500.0 * (double)std::max(n_tiles, 1);
    launch_bin_sort(bn, s);
    TRY(check_launch("render: bins"));
    TRY(mark(c, prof, 4, s));
    const uint32_t *ids_sorted = bn.ids_out;

    CompositeArgs ca;
    memset(&ca, 0, sizeof(ca));
    ca.ranges = c->ranges.as<uint2>();
    ca.ids = ids_sorted;
    ca.hdr = c->hdr.as<Header>();
    ca.feat = feat;
    ca.fsplit = fsplit;
    ca.n_stride = n_dev;
    ca.C = C;
    ca.feat_dtype = dtype;
    ca.views = c->views.as<RenderView>();
    ca.n_views = vb.n_views;
    ca.n_tiles_total = vb.n_tiles_total;
    ca.alpha_max = par.alpha_max;
    ca.alpha_min = par.alpha_min;
    ca.t_min = par.t_min;
    ca.log2_alpha_min = (float)log2((double)par.alpha_min);
    ca.status = sm + SM_STATUS;
    ca.tile_counter = sm + SM_TILECTR;
    ca.save = save ? 1 : 0;
    ca.tile_info = c->tinfo.as<uint4>();
    launch_composite(ca, s);
    TRY(check_launch("render: composite"));
    TRY(mark(c, prof, 5, s));

    c->stream = s;
    c->n_cap = n_cap;
    c->n_dev = n_dev;
    c->W = W; c->H = H; c->C = C; c->dtype = dtype;
    c->tiles_x = tiles_x; c->tiles_y = tiles_y;
    c->n_slots = n_tiles;
    c->feat = feat;
    c->feat_split = fsplit;
    c->pairs = ids_sorted;
    c->saved = save;
    c->alpha_max = par.alpha_max;
    c->alpha_min = par.alpha_min;
    return TSPLAT_OK;
}

static tsplat_status check_common(tsplat_ctx *c, int W, int H, int C, int dtype, const tsplat_render_params *p,
                                  const float *out_feat) {
    if (!c || !p || !out_feat) return fail(TSPLAT_ERR_INVALID_ARG, "render: NULL argument");
    if (W <= 0 || H <= 0 || W > 16383 || H > 16383) return fail(TSPLAT_ERR_INVALID_ARG, "render: image %dx%d", W, H);
    if (C < 1 || C > 64) return fail(TSPLAT_ERR_INVALID_ARG, "render: C = %d", C);
    if (dtype != TSPLAT_F32 && dtype != TSPLAT_BF16) return fail(TSPLAT_ERR_INVALID_ARG, "render: feat_dtype %d", dtype);
    return TSPLAT_OK;
}

static RenderView make_view(const tsplat_camera &cam, uint32_t tile_base, float *out_feat, float *out_alpha,
                            float *out_T, uint32_t *out_last) {
    RenderView v;
    memset(&v, 0, sizeof(v));
    v.cam = cam;
    v.tile_base = tile_base;
    v.tiles_x = (cam.width + TILE - 1) / TILE;
    v.tiles_y = (cam.height + TILE - 1) / TILE;
    v.width = cam.width;
    v.height = cam.height;
    v.out_feat = out_feat;
    v.out_alpha = out_alpha;
    v.out_T = out_T;
    v.out_last = out_last;
    return v;
}

static ProjectOut project_out(tsplat_ctx *c) {
    ProjectOut o;
    o.hdr = c->hdr.as<Header>();
    o.rect = c->rect.as<uint2>();
    o.ntiles = c->ntiles.as<uint32_t>();
    o.tmask = c->tmask.as<uint32_t>();
    o.tile_cnt = c->tcnt.as<uint32_t>();
    o.dkey = c->dkey.as<uint32_t>();
    o.radius = c->radius.as<float>();
    o.n_vis = small_ptr(c, SM_NVIS);
    return o;
}

static void init_small(tsplat_ctx *c, cudaStream_t s) {
    uint32_t *sm = c->small.as<uint32_t>();
    cudaMemsetAsync(sm + SM_NVIS, 0, sizeof(uint32_t) * 6, s);  // n_vis, (unused), P, P_eff, status, tile counter
}

tsplat_status tsplat_render(const tsplat_gaussians *g, const tsplat_camera *cam, const tsplat_render_params *params,
                            float *out_feat, float *out_alpha, tsplat_ctx *ctx, void *stream) {
    if (!g || !cam) return fail(TSPLAT_ERR_INVALID_ARG, "render: NULL argument");
    TRY(check_common(ctx, cam->width, cam->height, g->C, g->dtype, params, out_feat));
    cudaStream_t s = S(stream);
    const int W = cam->width, H = cam->height;
    const int tiles_x = (W + TILE - 1) / TILE, tiles_y = (H + TILE - 1) / TILE;
    const bool async_mode = (params->flags & TSPLAT_RENDER_ASYNC) != 0;
    if (async_mode) {
        if (ctx->hdr.bytes < (size_t)std::max<int64_t>(g->cap, 1) * sizeof(Header) ||
            !tiles_fit(ctx, (int64_t)tiles_x * tiles_y) ||
            ((params->flags & TSPLAT_RENDER_SAVE) && ctx->tfinal.bytes < (size_t)W * H * 4))
            return fail(TSPLAT_ERR_CAPACITY, "render: TSPLAT_RENDER_ASYNC needs tsplat_ctx_reserve for these sizes");
    } else {
        TRY(ensure_n(ctx, g->cap, s));
        TRY(ensure_pix(ctx, W, H, tiles_x * tiles_y, (params->flags & TSPLAT_RENDER_SAVE) != 0, s));
    }
    init_small(ctx, s);
    TRY(mark(ctx, (params->flags & TSPLAT_RENDER_PROFILE) != 0, 0, s));
    const bool save = (params->flags & TSPLAT_RENDER_SAVE) != 0;
    ViewBatch vb;
    memset(&vb, 0, sizeof(vb));
    vb.n_views = 1;
    vb.n_tiles_total = (uint32_t)(tiles_x * tiles_y);
    vb.v[0] = make_view(*cam, 0, out_feat, out_alpha, save ? ctx->tfinal.as<float>() : nullptr,
                        save ? ctx->last.as<uint32_t>() : nullptr);
    ProjectOut o = project_out(ctx);
    launch_project(g->xyzo.as<float4>(), g->cova.as<float4>(), g->covb.as<float2>(), g->n_dev.as<uint32_t>(), g->cap,
                   vb, ctx->views.as<RenderView>(), *params, o, s);
    TRY(check_launch("render: project"));
    TRY(render_tail(ctx, g->cap, g->n_dev.as<uint32_t>(), vb, g->feat.p, g->fsplit.p, g->C, g->dtype, *params, s));
    ctx->has_cam = true;
    ctx->cam = *cam;
    ctx->par = *params;
    return TSPLAT_OK;
}

tsplat_status tsplat_render_batch(const tsplat_gaussians *g, const tsplat_camera *cams, int32_t n_views,
                                  const tsplat_render_params *params, float *const *out_feat,
                                  float *const *out_alpha, tsplat_ctx *ctx, void *stream) {
    return render_batch_impl(g, cams, n_views, params, out_feat, out_alpha, ctx, stream, false);
}
}  // extern "C"

namespace tsp {
void make_view_batch(const tsplat_camera *cams, int32_t n_views, float *const *out_feat, float *const *out_alpha,
                     ViewBatch &vb) {
    memset(&vb, 0, sizeof(vb));
    vb.n_views = n_views;
    uint32_t tiles = 0;
    for (int v = 0; v < n_views; ++v) {
        vb.v[v] = make_view(cams[v], tiles, out_feat[v], out_alpha ? out_alpha[v] : nullptr, nullptr, nullptr);
        tiles += (uint32_t)(vb.v[v].tiles_x * vb.v[v].tiles_y);
    }
    vb.n_tiles_total = tiles;
}

tsplat_status render_batch_impl(const tsplat_gaussians *g, const tsplat_camera *cams, int32_t n_views,
                                const tsplat_render_params *params, float *const *out_feat,
                                float *const *out_alpha, tsplat_ctx *ctx, void *stream, bool table_on_device) {
    if (!g || !cams || !out_feat) return fail(TSPLAT_ERR_INVALID_ARG, "render_batch: NULL argument");
    if (n_views < 1 || n_views > MAX_BATCH) return fail(TSPLAT_ERR_INVALID_ARG, "render_batch: n_views = %d not in [1, %d]", n_views, MAX_BATCH);
    if (params && (params->flags & TSPLAT_RENDER_SAVE)) return fail(TSPLAT_ERR_UNSUPPORTED, "render_batch: TSPLAT_RENDER_SAVE is single-view only");
    for (int v = 0; v < n_views; ++v)
        TRY(check_common(ctx, cams[v].width, cams[v].height, g->C, g->dtype, params, out_feat[v]));
    ViewBatch vb;
    make_view_batch(cams, n_views, out_feat, out_alpha, vb);
    const uint32_t tiles = vb.n_tiles_total;
    cudaStream_t s = S(stream);
    const int64_t inst = std::max<int64_t>(g->cap, 1) * n_views;
    if (params->flags & TSPLAT_RENDER_ASYNC) {
        if (ctx->hdr.bytes < (size_t)inst * sizeof(Header) || !tiles_fit(ctx, tiles))
            return fail(TSPLAT_ERR_CAPACITY, "render_batch: TSPLAT_RENDER_ASYNC needs tsplat_ctx_reserve for these sizes");
    } else {
        TRY(ensure_n(ctx, inst, s));
        TRY(ensure_pix(ctx, 0, 0, (int)tiles, false, s));
    }
    init_small(ctx, s);
    TRY(mark(ctx, (params->flags & TSPLAT_RENDER_PROFILE) != 0, 0, s));
    ProjectOut o = project_out(ctx);
    launch_project(g->xyzo.as<float4>(), g->cova.as<float4>(), g->covb.as<float2>(), g->n_dev.as<uint32_t>(), g->cap,
                   vb, ctx->views.as<RenderView>(), *params, o, s, table_on_device);
    TRY(check_launch("render_batch: project"));
    ctx->has_cam = false;
    return render_tail(ctx, g->cap, g->n_dev.as<uint32_t>(), vb, g->feat.p, g->fsplit.p, g->C, g->dtype, *params, s);
}
}  // namespace tsp

extern "C" {

tsplat_status tsplat_backward_project(tsplat_ctx *c, const tsplat_gaussians *g, const float *d_mean2d,
                                      const float *d_conic, float *d_mean3d, float *d_cov3d, void *stream) {
    if (!c || !g || !d_mean2d || !d_conic || !d_mean3d || !d_cov3d)
        return fail(TSPLAT_ERR_INVALID_ARG, "backward_project: NULL argument");
    if (!c->saved || !c->has_cam)
        return fail(TSPLAT_ERR_INVALID_ARG, "backward_project: the last render on this context was not a tsplat_render with TSPLAT_RENDER_SAVE");
    if (c->n_dev != g->n_dev.as<uint32_t>())
        return fail(TSPLAT_ERR_INVALID_ARG, "backward_project: g is not the store of the last render");
    launch_project_backward(g->xyzo.as<float4>(), g->cova.as<float4>(), g->covb.as<float2>(), g->n_dev.as<uint32_t>(),
                            g->cap, c->cam, c->par, d_mean2d, d_conic, d_mean3d, d_cov3d, S(stream));
    return check_launch("backward_project");
}

tsplat_status tsplat_build_backward(tsplat_gaussians *g, const tsplat_src_view *views, int32_t n_views,
                                    const float *d_mean3d, const float *d_cov3d, const float *d_opac,
                                    const float *d_feat, const tsplat_src_grads *grads, void *stream) {
    if (!g || !views || !d_mean3d || !d_cov3d || !d_opac || !d_feat || !grads)
        return fail(TSPLAT_ERR_INVALID_ARG, "build_backward: NULL argument");
    cudaStream_t s = S(stream);
    LiftBwdArgs a;
    memset(&a, 0, sizeof(a));
    TRY(build_args(g, views, n_views, a.b, s));
    for (int v = 0; v < n_views; ++v)
        if (a.b.views[v].compact)
            return fail(TSPLAT_ERR_UNSUPPORTED, "build_backward: view %d has compact maps (the gradients are full maps)", v);
    for (int v = 0; v < n_views; ++v) {
        const tsplat_src_grads &gr = grads[v];
        if (!gr.depth || !gr.scale || !gr.opacity || !gr.feat)
            return fail(TSPLAT_ERR_INVALID_ARG, "build_backward: view %d: NULL gradient map", v);
        if (gr.quat && ((uintptr_t)gr.quat & 15)) return fail(TSPLAT_ERR_INVALID_ARG, "build_backward: view %d: quat gradient not 16-byte aligned", v);
        a.g[v].depth = gr.depth;
        a.g[v].scale = gr.scale;
        a.g[v].quat = views[v].quat ? gr.quat : nullptr;
        a.g[v].opacity = gr.opacity;
        a.g[v].feat = gr.feat;
    }
    a.d_mean = d_mean3d;
    a.d_cov = d_cov3d;
    a.d_opac = d_opac;
    a.d_feat = d_feat;
    launch_build_backward(a, s);
    return check_launch("build_backward");
}

tsplat_status tsplat_zbuffer(const tsplat_gaussians *g, const tsplat_camera *cam, float *out_depth, int32_t *out_id,
                             tsplat_ctx *ctx, void *stream) {
    if (!g || !cam || !out_depth || !ctx) return fail(TSPLAT_ERR_INVALID_ARG, "zbuffer: NULL argument");
    if (cam->width <= 0 || cam->height <= 0 || cam->width > 16383 || cam->height > 16383)
        return fail(TSPLAT_ERR_INVALID_ARG, "zbuffer: image %dx%d", cam->width, cam->height);
    cudaStream_t s = S(stream);
    TRY(grow(ctx->zkeys, (size_t)cam->width * cam->height * 8, s));
    launch_zbuffer(g->xyzo.as<float4>(), g->n_dev.as<uint32_t>(), g->cap, *cam, ctx->zkeys.as<unsigned long long>(),
                   out_depth, out_id, s);
    return check_launch("zbuffer");
}

tsplat_status tsplat_rasterize(int64_t n, const float *mean2d, const float *conic, const float *opac,
                               const float *depth, const int32_t *radius, const void *feat, int32_t C,
                               int32_t feat_dtype, int32_t width, int32_t height,
                               const tsplat_render_params *params, float *out_feat, float *out_alpha,
                               tsplat_ctx *ctx, void *stream) {
    TRY(check_common(ctx, width, height, C, feat_dtype, params, out_feat));
    if (n < 0 || n >= (int64_t)1 << 31) return fail(TSPLAT_ERR_INVALID_ARG, "rasterize: n = %lld", (long long)n);
    if (n > 0 && (!mean2d || !conic || !opac || !depth || !radius || !feat)) return fail(TSPLAT_ERR_INVALID_ARG, "rasterize: NULL array");
    if ((C * (int)feat_size(feat_dtype)) % 16 == 0 && ((uintptr_t)feat & 15))
        return fail(TSPLAT_ERR_INVALID_ARG, "rasterize: feat not 16-byte aligned");
    cudaStream_t s = S(stream);
    const int tiles_x = (width + TILE - 1) / TILE, tiles_y = (height + TILE - 1) / TILE;
    const bool async_mode = (params->flags & TSPLAT_RENDER_ASYNC) != 0;
    const bool split = feat_dtype == TSPLAT_F32;
    const size_t split_bytes = (size_t)std::max<int64_t>(n, 1) * 4 * padded_channels(C);
    if (async_mode) {
        if (ctx->hdr.bytes < (size_t)std::max<int64_t>(n, 1) * sizeof(Header) || !tiles_fit(ctx, (int64_t)tiles_x * tiles_y) ||
            (split && ctx->fsplit.bytes < split_bytes))
            return fail(TSPLAT_ERR_CAPACITY, "rasterize: TSPLAT_RENDER_ASYNC needs tsplat_ctx_reserve for these sizes");
    } else {
        TRY(ensure_n(ctx, n, s));
        TRY(ensure_pix(ctx, width, height, tiles_x * tiles_y, (params->flags & TSPLAT_RENDER_SAVE) != 0, s));
        if (split) TRY(grow(ctx->fsplit, split_bytes, s));
    }
    init_small(ctx, s);
    launch_fill_u32(small_ptr(ctx, SM_N), (uint32_t)n, 1, s);
    if (split) launch_feat_split((const float *)feat, small_ptr(ctx, SM_N), n, C, ctx->fsplit.p, s);
    TRY(mark(ctx, (params->flags & TSPLAT_RENDER_PROFILE) != 0, 0, s));
    const bool save = (params->flags & TSPLAT_RENDER_SAVE) != 0;
    tsplat_camera cam;
    memset(&cam, 0, sizeof(cam));
    cam.width = width;
    cam.height = height;
    ViewBatch vb;
    memset(&vb, 0, sizeof(vb));
    vb.n_views = 1;
    vb.n_tiles_total = (uint32_t)(tiles_x * tiles_y);
    vb.v[0] = make_view(cam, 0, out_feat, out_alpha, save ? ctx->tfinal.as<float>() : nullptr,
                        save ? ctx->last.as<uint32_t>() : nullptr);
    ProjectOut o = project_out(ctx);
    launch_prepare_2d(n, mean2d, conic, opac, depth, radius, *params, vb, ctx->views.as<RenderView>(), o, s);
    TRY(check_launch("rasterize: prepare"));
    ctx->has_cam = false;
    return render_tail(ctx, n, small_ptr(ctx, SM_N), vb, feat, split ? ctx->fsplit.p : nullptr, C, feat_dtype,
                       *params, s);
}

tsplat_status tsplat_backward(tsplat_ctx *c, const float *dL_dfeat, const float *dL_dalpha, float *d_mean2d,
                              float *d_conic, float *d_opac, float *d_feat, void *stream) {
    if (!c || !dL_dfeat) return fail(TSPLAT_ERR_INVALID_ARG, "backward: NULL argument");
    if (!c->saved) return fail(TSPLAT_ERR_INVALID_ARG, "backward: the last render on this context did not use TSPLAT_RENDER_SAVE");
    if (c->dtype == TSPLAT_F32 && !c->feat_split)
        return fail(TSPLAT_ERR_INVALID_ARG, "backward: the last render's FP32 features have no split rows");
    cudaStream_t s = S(stream);
    launch_zero_f32_n(d_mean2d, c->n_dev, 2, c->n_cap, s);
    launch_zero_f32_n(d_conic, c->n_dev, 3, c->n_cap, s);
    launch_zero_f32_n(d_opac, c->n_dev, 1, c->n_cap, s);
    launch_zero_f32_n(d_feat, c->n_dev, c->C, c->n_cap, s);
    BackwardArgs b;
    memset(&b, 0, sizeof(b));
    b.ranges = c->ranges.as<uint2>();
    b.ids = c->pairs;
    b.hdr = c->hdr.as<Header>();
    b.feat = c->feat;
    b.fsplit = c->feat_split;
    b.C = c->C;
    b.feat_dtype = c->dtype;
    b.W = c->W; b.H = c->H; b.tiles_x = c->tiles_x; b.tiles_y = c->tiles_y;
    b.alpha_max = c->alpha_max;
    b.alpha_min = c->alpha_min;
    b.log2_alpha_min = (float)log2((double)c->alpha_min);
    b.T_final = c->tfinal.as<float>();
    b.last = c->last.as<uint32_t>();
    b.dF = dL_dfeat;
    b.dA = dL_dalpha;
    b.d_mean2d = d_mean2d;
    b.d_conic = d_conic;
    b.d_opac = d_opac;
    b.d_feat = d_feat;
    b.unit_counter = small_ptr(c, SM_BWDCTR);
    b.tile_order = c->torder.as<uint32_t>();
    TRY_CUDA(cudaMemsetAsync(b.unit_counter, 0, sizeof(uint32_t), s));
    launch_backward(b, s);
    return check_launch("backward");
}

tsplat_status tsplat_ctx_timings(tsplat_ctx *c, float *ms, int32_t capacity, int32_t *n_out) {
    if (!c || !ms) return fail(TSPLAT_ERR_INVALID_ARG, "ctx_timings: NULL argument");
    if (c->n_prof == 0) return fail(TSPLAT_ERR_INVALID_ARG, "ctx_timings: no render with TSPLAT_RENDER_PROFILE since the last call");
    const int n = std::min<int>(capacity, tsplat_ctx::N_EV - 1);
    const int64_t k0 = std::max<int64_t>(0, c->n_prof - tsplat_ctx::RING);
    TRY_CUDA(cudaEventSynchronize(c->ev[(c->n_prof - 1) % tsplat_ctx::RING][tsplat_ctx::N_EV - 1]));
    for (int i = 0; i < n; ++i) ms[i] = 0.0f;
    for (int64_t k = k0; k < c->n_prof; ++k) {
        cudaEvent_t *row = c->ev[k % tsplat_ctx::RING];
        for (int i = 0; i < n; ++i) {
            float t = 0.0f;
            TRY_CUDA(cudaEventElapsedTime(&t, row[i], row[i + 1]));
            ms[i] += t;
        }
    }
    for (int i = 0; i < n; ++i) ms[i] /= (float)(c->n_prof - k0);
    c->n_prof = 0;
    if (n_out) *n_out = n;
    return TSPLAT_OK;
}

uint64_t tsplat_launch_count(void) { return g_launches.load(std::memory_order_relaxed); }

tsplat_status tsplat_ctx_status(tsplat_ctx *c) {
    if (!c) return fail(TSPLAT_ERR_INVALID_ARG, "ctx_status: ctx is NULL");
    TRY_CUDA(cudaStreamSynchronize(c->stream));
    uint32_t st = 0;
    TRY_CUDA(cudaMemcpy(&st, small_ptr(c, SM_STATUS), 4, cudaMemcpyDeviceToHost));
    if (st) return fail((tsplat_status)st, "device status %u (pair capacity %lld)", st, (long long)c->p_cap);
    return TSPLAT_OK;
}

tsplat_status tsplat_ctx_stats_get(tsplat_ctx *c, tsplat_ctx_stats *out) {
    if (!c || !out) return fail(TSPLAT_ERR_INVALID_ARG, "ctx_stats: NULL argument");
    TRY_CUDA(cudaStreamSynchronize(c->stream));
    uint32_t w[SM_WORDS];
    TRY_CUDA(cudaMemcpy(w, c->small.p, sizeof(w), cudaMemcpyDeviceToHost));
    uint32_t n = 0;
    if (c->n_dev) TRY_CUDA(cudaMemcpy(&n, c->n_dev, 4, cudaMemcpyDeviceToHost));
    out->n_gaussians = n;
    out->n_visible = w[SM_NVIS];
    out->n_pairs = w[SM_P];
    out->pair_capacity = c->p_cap;
    out->tiles_x = c->tiles_x;
    out->tiles_y = c->tiles_y;
    out->width = c->W;
    out->height = c->H;
    out->C = c->C;
    out->device_status = (int32_t)w[SM_STATUS];
    return TSPLAT_OK;
}

tsplat_status tsplat_ctx_export(tsplat_ctx *c, int32_t what, void *dst, size_t bytes, void *stream) {
    if (!c || !dst) return fail(TSPLAT_ERR_INVALID_ARG, "ctx_export: NULL argument");
    cudaStream_t s = S(stream);
    TRY_CUDA(cudaStreamSynchronize(c->stream));
    uint32_t n = 0, P = 0;
    if (c->n_dev) TRY_CUDA(cudaMemcpy(&n, c->n_dev, 4, cudaMemcpyDeviceToHost));
    TRY_CUDA(cudaMemcpy(&P, small_ptr(c, SM_PEFF), 4, cudaMemcpyDeviceToHost));
    const size_t HW = (size_t)c->W * c->H;
    size_t need = 0;
    switch (what) {
        case TSPLAT_EXPORT_RECT: need = (size_t)n * 16; break;
        case TSPLAT_EXPORT_DEPTHKEY: need = (size_t)n * 4; break;
        case TSPLAT_EXPORT_MEAN2D: need = (size_t)n * 8; break;
        case TSPLAT_EXPORT_CONIC: need = (size_t)n * 12; break;
        case TSPLAT_EXPORT_RADIUS: need = (size_t)n * 4; break;
        case TSPLAT_EXPORT_PAIRS: need = (size_t)P * 4; break;
        case TSPLAT_EXPORT_RANGES: need = (size_t)c->tiles_x * c->tiles_y * 8; break;
        case TSPLAT_EXPORT_TILE_ORDER: need = (size_t)c->n_slots * 4; break;
        case TSPLAT_EXPORT_TFINAL:
        case TSPLAT_EXPORT_LAST:
            if (!c->saved) return fail(TSPLAT_ERR_INVALID_ARG, "ctx_export: render without TSPLAT_RENDER_SAVE");
            need = HW * 4;
            break;
        default: return fail(TSPLAT_ERR_INVALID_ARG, "ctx_export: unknown item %d", what);
    }
    if (bytes < need) return fail(TSPLAT_ERR_CAPACITY, "ctx_export: need %zu bytes, got %zu", need, bytes);
    switch (what) {
        case TSPLAT_EXPORT_RECT: launch_export_rect(c->rect.as<uint2>(), c->n_dev, c->n_cap, (int32_t *)dst, s); break;
        case TSPLAT_EXPORT_DEPTHKEY: TRY_CUDA(cudaMemcpyAsync(dst, c->dkey.p, need, cudaMemcpyDeviceToDevice, s)); break;
        case TSPLAT_EXPORT_MEAN2D:
        case TSPLAT_EXPORT_CONIC: launch_export_header(c->hdr.as<Header>(), c->n_dev, c->n_cap, what, dst, s); break;
        case TSPLAT_EXPORT_RADIUS: TRY_CUDA(cudaMemcpyAsync(dst, c->radius.p, need, cudaMemcpyDeviceToDevice, s)); break;
        case TSPLAT_EXPORT_PAIRS: if (need) TRY_CUDA(cudaMemcpyAsync(dst, c->pairs, need, cudaMemcpyDeviceToDevice, s)); break;
        case TSPLAT_EXPORT_RANGES: TRY_CUDA(cudaMemcpyAsync(dst, c->ranges.p, need, cudaMemcpyDeviceToDevice, s)); break;
        case TSPLAT_EXPORT_TFINAL: TRY_CUDA(cudaMemcpyAsync(dst, c->tfinal.p, need, cudaMemcpyDeviceToDevice, s)); break;
        case TSPLAT_EXPORT_LAST: TRY_CUDA(cudaMemcpyAsync(dst, c->last.p, need, cudaMemcpyDeviceToDevice, s)); break;
        case TSPLAT_EXPORT_TILE_ORDER:
            if (need) TRY_CUDA(cudaMemcpyAsync(dst, c->torder.p, need, cudaMemcpyDeviceToDevice, s));
            break;
    }
    return check_launch("ctx_export");
}

}  // extern "C"

namespace tsp {
tsplat_status ctx_reserve_batch(tsplat_ctx *c, int64_t instances, int64_t pairs, int64_t tiles) {
    TRY(ensure_n(c, instances, nullptr));
    TRY(ensure_p(c, pairs, nullptr));
    TRY(ensure_tiles(c, tiles, nullptr));
    TRY_CUDA(cudaStreamSynchronize(nullptr));
    return TSPLAT_OK;
}
RenderView *ctx_view_table(tsplat_ctx *c) { return c->views.as<RenderView>(); }
int64_t ctx_pair_capacity(const tsplat_ctx *c) { return c->p_cap; }
uint32_t *ctx_status_word(tsplat_ctx *c) { return small_ptr(c, SM_STATUS); }
uint32_t *ctx_pairs_word(tsplat_ctx *c) { return small_ptr(c, SM_P); }
}  // namespace tsp
