// A9: serving -- continuous batching of target-view requests over the
// resident Gaussians of the current frame (Tele-Aloha renders the viewer's
// left and right eye views every frame, Sec. 4.2, and runs the whole
// pipeline as CUDA graphs, Sec. 5.3).
//
// A worker thread owns `lanes`: each lane is a render context reserved for a
// batch of up to 8 views plus a stream, and at most one batch per lane is on
// the device at a time, so up to n_lanes batches overlap.  The number of
// lanes follows from the memory budget.  Whenever a lane is free and
// requests are pending, the worker admits them in arrival order while the
// batch's estimated (Gaussian, tile) pairs fit the lane's pair buffer (the
// configured per-view estimate, scaled by the running ratio of measured to
// estimated pairs of the batches already retired), and
// launches the batch as one replay of a CUDA graph captured per (frame
// Gaussians, number of views); only the view table (cameras, output
// buffers, tile offsets) of the graph's projection launch is rewritten
// before each replay.  A batch whose pairs overflow is re-run one view at a
// time.  Latency = completion seen by the worker - submission.  With
// TSPLAT_SERVER_NO_GRAPH the batch is issued as plain launches instead; with
// one view per batch and one lane that is one-launch-sequence-per-view
// rendering behind the same queue.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <tuple>
#include <unordered_map>
#include <vector>

#include "common.cuh"
#include "internal.h"

using namespace tsp;

namespace {

double now_ms() {
    using namespace std::chrono;
    return duration<double, std::milli>(steady_clock::now().time_since_epoch()).count();
}

enum { REQ_PENDING = 0, REQ_RUNNING = 1, REQ_DONE = 2, REQ_FAILED = 3 };

struct Request {
    tsplat_camera cam;
    float *out_feat;
    float *out_alpha;
    double t_submit;
    double latency_ms;
    int64_t est_pairs;
    int state;
    bool solo;  // re-run alone after an overflow
    tsplat_status fail_status;
    char fail_msg[200];
};

void fail_request(Request &r, tsplat_status st, const char *msg) {
    r.state = REQ_FAILED;
    r.fail_status = st;
    snprintf(r.fail_msg, sizeof(r.fail_msg), "%s", msg);
}

// A captured graph holds the frame's buffers and capacity: (features,
// count word, capacity, number of views)
using GraphKey = std::tuple<const void *, const void *, int64_t, int>;

struct Lane {
    tsplat_ctx *ctx = nullptr;
    cudaStream_t stream = nullptr;
    cudaEvent_t done = nullptr;
    bool busy = false;
    std::vector<uint64_t> reqs;
    std::map<GraphKey, cudaGraphExec_t> graphs;
    std::deque<GraphKey> stores;      // frame stores with graphs, most recent last (at most 2)
    const tsplat_gaussians *frame = nullptr;  // frame of the batch in flight (under the server mutex)
    size_t prepared = 0;                       // prepare requests this lane has carried out
    float *dummy = nullptr;          // output of the warm-up run (16 x 16 views)
    uint32_t *status_host = nullptr; // pinned copy of the batch's device status word
    uint32_t *pairs_host = nullptr;  // pinned copy of the batch's pair count
    int64_t est = 0;                 // the batch's estimated pairs (configured estimate, unscaled)
    RenderView *table_host = nullptr; // pinned staging of the batch's view table
};

}  // namespace

struct tsplat_server {
    tsplat_server_config cfg;
    std::vector<Lane> lanes;
    std::thread worker;
    std::mutex mu;
    std::condition_variable cv;
    std::deque<uint64_t> pending;
    std::unordered_map<uint64_t, Request> reqs;
    uint64_t next_id = 1;
    const tsplat_gaussians *frame = nullptr;
    cudaEvent_t frame_ready = nullptr;  // recorded on the frame's last writer stream
    int64_t lane_bytes = 0;
    std::vector<const tsplat_gaussians *> prepare;  // stores whose graphs are captured ahead of use
    tsplat_status prepare_status = TSPLAT_OK;
    bool stop = false;
    tsplat_status error = TSPLAT_OK;
    // statistics
    std::vector<double> latencies;
    uint64_t batches = 0, views = 0, retries = 0;
    // admission: measured / estimated pairs of retired batches, a running
    // average (0 until the first batch retires, then the estimates scale by it)
    double pair_scale = 0.0;
    double t_first = 0, t_last = 0;
    int device = 0;
};

namespace {

int64_t est_pairs(const tsplat_server &S, int64_t cap, int width, int height) {
    return (int64_t)ceil(S.cfg.pairs_per_gaussian * (double)cap + S.cfg.pairs_per_pixel * (double)width * (double)height);
}

// Capture (once) the batched render of K views of `g` on this lane.  The
// graph's projection reads the view table from the context's device table,
// which launch_batch fills before each replay.
tsplat_status lane_graph(tsplat_server &S, Lane &L, const tsplat_gaussians *g, int K, cudaGraphExec_t *out) {
    GaussianStore gs;
    gaussians_peek(g, gs, nullptr);
    const GraphKey key(gs.feat, gs.n_dev, gs.cap, K);
    auto it = L.graphs.find(key);
    if (it != L.graphs.end()) {
        *out = it->second;
        return TSPLAT_OK;
    }
    // graphs are kept for the two most recent frame stores (double-buffered
    // frames); older stores' graphs are dropped
    const GraphKey store(gs.feat, gs.n_dev, gs.cap, 0);
    auto sit = std::find(L.stores.begin(), L.stores.end(), store);
    if (sit != L.stores.end()) L.stores.erase(sit);
    L.stores.push_back(store);
    while (L.stores.size() > 2) {
        const GraphKey old = L.stores.front();
        L.stores.pop_front();
        for (auto jt = L.graphs.begin(); jt != L.graphs.end();) {
            if (std::get<0>(jt->first) == std::get<0>(old) && std::get<1>(jt->first) == std::get<1>(old) &&
                std::get<2>(jt->first) == std::get<2>(old)) {
                cudaGraphExecDestroy(jt->second);
                jt = L.graphs.erase(jt);
            } else {
                ++jt;
            }
        }
    }
    // K views of the largest size: the captured grids and pass counts then
    // cover any mix of smaller views
    std::vector<tsplat_camera> cams(K);
    for (int v = 0; v < K; ++v) {
        memset(&cams[v], 0, sizeof(tsplat_camera));
        cams[v].width = S.cfg.max_width;
        cams[v].height = S.cfg.max_height;
        cams[v].fx = cams[v].fy = (float)S.cfg.max_width;
        cams[v].R[0] = cams[v].R[4] = cams[v].R[8] = 1.0f;
        cams[v].z_near = 0.2f;
        cams[v].z_far = 1e4f;
    }
    std::vector<float *> outs(K, L.dummy);
    tsplat_render_params p = S.cfg.params;
    p.flags = TSPLAT_RENDER_ASYNC;
    // a small plain run first, so that first-use set-up (kernel attributes,
    // occupancy) happens outside the capture; its K 16x16 views all write the
    // same dummy buffer
    std::vector<tsplat_camera> tiny = cams;
    for (auto &c : tiny) c.width = c.height = 16;
    tsplat_status st = render_batch_impl(g, tiny.data(), K, &p, outs.data(), nullptr, L.ctx, L.stream, false);
    if (st != TSPLAT_OK) return st;
    if (cudaStreamSynchronize(L.stream) != cudaSuccess) return record_error(TSPLAT_ERR_CUDA, "serve: warm-up failed");
    cudaGraph_t graph = nullptr;
    if (cudaStreamBeginCapture(L.stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
        return record_error(TSPLAT_ERR_CUDA, "serve: begin capture failed");
    st = render_batch_impl(g, cams.data(), K, &p, outs.data(), nullptr, L.ctx, L.stream, true);
    cudaError_t e = cudaStreamEndCapture(L.stream, &graph);
    if (st != TSPLAT_OK) {
        if (graph) cudaGraphDestroy(graph);
        return st;
    }
    if (e != cudaSuccess) {
        char msg[160];
        snprintf(msg, sizeof(msg), "serve: capture failed: %s", cudaGetErrorString(e));
        return record_error(TSPLAT_ERR_CUDA, msg);
    }
    cudaGraphExec_t exec = nullptr;
    e = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
        char msg[160];
        snprintf(msg, sizeof(msg), "serve: graph instantiation failed: %s", cudaGetErrorString(e));
        return record_error(TSPLAT_ERR_CUDA, msg);
    }
    L.graphs.emplace(key, exec);
    *out = exec;
    return TSPLAT_OK;
}

void batch_views(tsplat_server &S, const std::vector<uint64_t> &ids, std::vector<tsplat_camera> &cams,
                 std::vector<float *> &of, std::vector<float *> &oa) {
    const int K = (int)ids.size();
    cams.resize(K);
    of.resize(K);
    oa.resize(K);
    std::lock_guard<std::mutex> lock(S.mu);
    for (int v = 0; v < K; ++v) {
        const Request &r = S.reqs[ids[v]];
        cams[v] = r.cam;
        of[v] = r.out_feat;
        oa[v] = r.out_alpha;
    }
}

tsplat_status launch_batch(tsplat_server &S, Lane &L, const tsplat_gaussians *g, const std::vector<uint64_t> &ids) {
    const int K = (int)ids.size();
    std::vector<tsplat_camera> cams;
    std::vector<float *> of, oa;
    batch_views(S, ids, cams, of, oa);
    tsplat_render_params p = S.cfg.params;
    p.flags = TSPLAT_RENDER_ASYNC;
    if (S.cfg.flags & TSPLAT_SERVER_NO_GRAPH) {
        if (cudaStreamWaitEvent(L.stream, S.frame_ready, 0) != cudaSuccess)
            return record_error(TSPLAT_ERR_CUDA, "serve: stream wait failed");
        return render_batch_impl(g, cams.data(), K, &p, of.data(), oa.data(), L.ctx, L.stream, false);
    }
    cudaGraphExec_t exec = nullptr;
    tsplat_status st = lane_graph(S, L, g, K, &exec);
    if (st != TSPLAT_OK) return st;
    // the view table goes to the device ahead of the replay, on the lane's
    // stream (the previous batch of this lane has completed, so neither the
    // staging copy nor the device table is in use)
    ViewBatch vb;
    make_view_batch(cams.data(), K, of.data(), oa.data(), vb);
    memcpy(L.table_host, vb.v, sizeof(RenderView) * K);
    if (cudaMemcpyAsync(ctx_view_table(L.ctx), L.table_host, sizeof(RenderView) * K, cudaMemcpyHostToDevice,
                        L.stream) != cudaSuccess ||
        cudaStreamWaitEvent(L.stream, S.frame_ready, 0) != cudaSuccess || cudaGraphLaunch(exec, L.stream) != cudaSuccess)
        return record_error(TSPLAT_ERR_CUDA, "serve: graph launch failed");
    return TSPLAT_OK;
}

// Issue the batch on the lane and mark the lane busy (after the status copy
// and the completion event are queued behind the render)
tsplat_status issue_batch(tsplat_server &S, Lane &L, const tsplat_gaussians *g, const std::vector<uint64_t> &ids) {
    tsplat_status st = launch_batch(S, L, g, ids);
    if (st != TSPLAT_OK) return st;
    if (cudaMemcpyAsync(L.status_host, ctx_status_word(L.ctx), sizeof(uint32_t), cudaMemcpyDeviceToHost, L.stream) !=
            cudaSuccess ||
        cudaMemcpyAsync(L.pairs_host, ctx_pairs_word(L.ctx), sizeof(uint32_t), cudaMemcpyDeviceToHost, L.stream) !=
            cudaSuccess ||
        cudaEventRecord(L.done, L.stream) != cudaSuccess)
        return record_error(TSPLAT_ERR_CUDA, "serve: status copy or event record failed");
    std::lock_guard<std::mutex> lock(S.mu);
    L.est = 0;
    for (uint64_t id : ids) L.est += S.reqs[id].est_pairs;
    L.busy = true;
    L.frame = g;
    L.reqs = ids;
    S.batches += 1;
    S.views += ids.size();
    return TSPLAT_OK;
}

void worker_main(tsplat_server *Sp) {
    tsplat_server &S = *Sp;
    cudaSetDevice(S.device);
    for (;;) {
        bool progressed = false;
        // capture the graphs of every batch size for stores named by
        // tsplat_server_prepare, on idle lanes
        for (Lane &L : S.lanes) {
            const tsplat_gaussians *g = nullptr;
            {
                std::lock_guard<std::mutex> lock(S.mu);
                if (L.busy || L.prepared >= S.prepare.size()) continue;
                g = S.prepare[L.prepared];
            }
            tsplat_status st = TSPLAT_OK;
            if (!(S.cfg.flags & TSPLAT_SERVER_NO_GRAPH)) {
                cudaGraphExec_t exec = nullptr;
                for (int K = 1; K <= S.cfg.max_views_per_batch && st == TSPLAT_OK; ++K) st = lane_graph(S, L, g, K, &exec);
            }
            std::lock_guard<std::mutex> lock(S.mu);
            if (st != TSPLAT_OK) S.prepare_status = st;
            ++L.prepared;
            progressed = true;
            S.cv.notify_all();
        }
        // retire finished batches
        for (Lane &L : S.lanes) {
            if (!L.busy || cudaEventQuery(L.done) != cudaSuccess) continue;
            const tsplat_status dst = (tsplat_status)*reinterpret_cast<volatile uint32_t *>(L.status_host);
            const uint32_t pairs = *reinterpret_cast<volatile uint32_t *>(L.pairs_host);
            const double t = now_ms();
            std::lock_guard<std::mutex> lock(S.mu);
            if ((dst == TSPLAT_OK || dst == TSPLAT_ERR_CAPACITY) && L.est > 0) {  // the scan counts P either way
                const double r = (double)pairs / (double)L.est;
                S.pair_scale = S.pair_scale > 0.0 ? 0.8 * S.pair_scale + 0.2 * r : r;
            }
            if (dst == TSPLAT_ERR_CAPACITY && L.reqs.size() > 1) {
                // pairs overflowed the lane: run these views again one at a time
                for (auto it = L.reqs.rbegin(); it != L.reqs.rend(); ++it) {
                    Request &r = S.reqs[*it];
                    r.state = REQ_PENDING;
                    r.solo = true;
                    S.pending.push_front(*it);
                }
                S.retries += L.reqs.size();
            } else {
                char msg[96];
                snprintf(msg, sizeof(msg), "serve: the batch's device status was %d", (int)dst);
                for (uint64_t id : L.reqs) {
                    Request &r = S.reqs[id];
                    r.latency_ms = t - r.t_submit;
                    if (dst == TSPLAT_OK) {
                        r.state = REQ_DONE;
                        S.latencies.push_back(r.latency_ms);
                    } else {
                        fail_request(r, dst, msg);
                    }
                }
                S.t_last = t;
            }
            L.busy = false;
            L.frame = nullptr;
            L.reqs.clear();
            progressed = true;
            S.cv.notify_all();
        }
        // admit pending requests into free lanes
        for (Lane &L : S.lanes) {
            if (L.busy) continue;
            std::vector<uint64_t> batch;
            const tsplat_gaussians *frame = nullptr;
            {
                std::lock_guard<std::mutex> lock(S.mu);
                if (S.stop) break;
                if (!S.frame || S.pending.empty()) break;
                // views already on the device bound this batch (latency control)
                int room = S.cfg.max_views_per_batch;
                if (S.cfg.max_inflight_views > 0) {
                    int inflight = 0;
                    for (const Lane &O : S.lanes) inflight += O.busy ? (int)O.reqs.size() : 0;
                    room = std::min(room, S.cfg.max_inflight_views - inflight);
                    if (room <= 0) break;
                }
                frame = S.frame;
                const int64_t cap = (int64_t)(0.9 * (double)ctx_pair_capacity(L.ctx));
                const double scale = S.pair_scale > 0.0 ? 1.1 * S.pair_scale : 1.0;  // 10 % margin
                int64_t used = 0;
                while (!S.pending.empty() && (int)batch.size() < room) {
                    Request &r = S.reqs[S.pending.front()];
                    const int64_t need = (int64_t)ceil(scale * (double)r.est_pairs);
                    if (!batch.empty() && (r.solo || used + need > cap)) break;
                    batch.push_back(S.pending.front());
                    S.pending.pop_front();
                    r.state = REQ_RUNNING;
                    used += need;
                    if (r.solo) break;
                }
            }
            if (batch.empty()) break;
            tsplat_status st = issue_batch(S, L, frame, batch);
            if (st != TSPLAT_OK) {
                std::lock_guard<std::mutex> lock(S.mu);
                const char *why = tsplat_last_error();
                for (uint64_t id : batch) fail_request(S.reqs[id], st, why ? why : "serve: launch failed");
                S.error = st;
                S.cv.notify_all();
            }
            progressed = true;
        }
        std::unique_lock<std::mutex> lock(S.mu);
        if (S.stop) {
            bool any_busy = false;
            for (Lane &L : S.lanes) any_busy |= L.busy;
            if (!any_busy) break;
        }
        if (!progressed) S.cv.wait_for(lock, std::chrono::microseconds(20));
    }
}

}  // namespace

extern "C" {

void tsplat_server_config_default(tsplat_server_config *c) {
    if (!c) return;
    memset(c, 0, sizeof(*c));
    c->max_views_per_batch = 8;
    c->max_lanes = 3;
    c->max_width = 1024;
    c->max_height = 1024;
    c->max_gaussians = 1 << 22;
    c->C = 32;
    c->feat_dtype = TSPLAT_BF16;
    c->pairs_per_gaussian = 2.5f;
    c->pairs_per_pixel = 1.0f;
    c->flags = 0;
    c->budget_bytes = (int64_t)8 << 30;
    tsplat_render_params_default(&c->params);
}

tsplat_status tsplat_server_create(const tsplat_server_config *cfg, tsplat_server **out) {
    if (!cfg || !out) return record_error(TSPLAT_ERR_INVALID_ARG, "server_create: NULL argument");
    *out = nullptr;
    if (cfg->max_views_per_batch < 1 || cfg->max_views_per_batch > MAX_BATCH || cfg->max_lanes < 1 ||
        cfg->max_width < 1 || cfg->max_height < 1 || cfg->max_gaussians < 1 || cfg->max_inflight_views < 0 || !(cfg->pairs_per_pixel >= 0.f) || !(cfg->pairs_per_gaussian >= 0.f) ||
        cfg->pairs_per_pixel + cfg->pairs_per_gaussian <= 0.f)
        return record_error(TSPLAT_ERR_INVALID_ARG, "server_create: invalid configuration");
    tsplat_server *S = new tsplat_server();
    S->cfg = *cfg;
    cudaGetDevice(&S->device);
    if (cudaEventCreateWithFlags(&S->frame_ready, cudaEventDisableTiming) != cudaSuccess) {
        delete S;
        return record_error(TSPLAT_ERR_CUDA, "server_create: event creation failed");
    }
    // bytes of one lane: per instance 32 (record) + 8 (rect) + 16 (tile count, mask, depth key, radius),
    // per pair 16 (bucket keys and ids, scratch, sorted ids) with the 1/8 headroom of the pair buffers,
    // per tile 20 (range, order, count and cursor), plus the view table
    const int64_t K = cfg->max_views_per_batch;
    const int64_t inst = K * cfg->max_gaussians;
    const int64_t tiles = K * (int64_t)((cfg->max_width + TILE - 1) / TILE) * ((cfg->max_height + TILE - 1) / TILE);
    const int64_t pairs = K * est_pairs(*S, cfg->max_gaussians, cfg->max_width, cfg->max_height);
    const int64_t lane_bytes = inst * 56 + pairs * 18 + tiles * 20 + (int64_t)(1 << 20);
    const int64_t n_lanes = std::min<int64_t>(cfg->max_lanes, cfg->budget_bytes / std::max<int64_t>(lane_bytes, 1));
    S->lane_bytes = lane_bytes;
    if (n_lanes < 1) {
        cudaEventDestroy(S->frame_ready);
        delete S;
        return record_error(TSPLAT_ERR_OOM, "server_create: the memory budget does not hold one batch lane");
    }
    S->lanes.resize((size_t)n_lanes);
    for (Lane &L : S->lanes) {
        tsplat_status st = tsplat_ctx_create(&L.ctx);
        if (st == TSPLAT_OK) st = ctx_reserve_batch(L.ctx, inst, pairs, tiles);
        if (st == TSPLAT_OK && (cudaStreamCreateWithFlags(&L.stream, cudaStreamNonBlocking) != cudaSuccess ||
                                cudaEventCreateWithFlags(&L.done, cudaEventDisableTiming) != cudaSuccess ||
                                cudaMalloc(&L.dummy, sizeof(float) * 16 * 16 * (cfg->C + 1)) != cudaSuccess ||
                                cudaMallocHost(&L.status_host, sizeof(uint32_t)) != cudaSuccess ||
                                cudaMallocHost(&L.pairs_host, sizeof(uint32_t)) != cudaSuccess ||
                                cudaMallocHost(&L.table_host, sizeof(RenderView) * MAX_BATCH) != cudaSuccess))
            st = record_error(TSPLAT_ERR_CUDA, "server_create: stream/event allocation failed");
        if (st != TSPLAT_OK) {
            tsplat_server_destroy(S);
            return st;
        }
    }
    S->worker = std::thread(worker_main, S);
    *out = S;
    return TSPLAT_OK;
}

tsplat_status tsplat_server_destroy(tsplat_server *S) {
    if (!S) return TSPLAT_OK;
    {
        std::lock_guard<std::mutex> lock(S->mu);
        S->stop = true;
        S->pending.clear();
        S->cv.notify_all();
    }
    if (S->worker.joinable()) S->worker.join();
    for (Lane &L : S->lanes) {
        if (L.stream) cudaStreamSynchronize(L.stream);
        for (auto &kv : L.graphs)
            if (kv.second) cudaGraphExecDestroy(kv.second);
        if (L.done) cudaEventDestroy(L.done);
        if (L.stream) cudaStreamDestroy(L.stream);
        if (L.dummy) cudaFree(L.dummy);
        if (L.status_host) cudaFreeHost(L.status_host);
        if (L.pairs_host) cudaFreeHost(L.pairs_host);
        if (L.table_host) cudaFreeHost(L.table_host);
        if (L.ctx) tsplat_ctx_destroy(L.ctx);
    }
    if (S->frame_ready) cudaEventDestroy(S->frame_ready);
    delete S;
    return TSPLAT_OK;
}

tsplat_status tsplat_server_update_frame(tsplat_server *S, const tsplat_gaussians *g) {
    if (!S || !g) return record_error(TSPLAT_ERR_INVALID_ARG, "server_update_frame: NULL argument");
    int64_t cap = 0;
    int32_t C = 0, dt = 0;
    tsplat_gaussians_shape(g, &cap, &C, &dt);
    if (cap > S->cfg.max_gaussians || C != S->cfg.C || dt != S->cfg.feat_dtype)
        return record_error(TSPLAT_ERR_INVALID_ARG, "server_update_frame: Gaussians do not match the server configuration");
    GaussianStore gs;
    cudaStream_t writer = nullptr;
    gaussians_peek(g, gs, &writer);
    std::lock_guard<std::mutex> lock(S->mu);
    if (cudaEventRecord(S->frame_ready, writer) != cudaSuccess)
        return record_error(TSPLAT_ERR_CUDA, "server_update_frame: event record failed");
    S->frame = g;
    S->cv.notify_all();
    return TSPLAT_OK;
}

tsplat_status tsplat_server_prepare(tsplat_server *S, const tsplat_gaussians *g, double timeout_ms) {
    if (!S || !g) return record_error(TSPLAT_ERR_INVALID_ARG, "server_prepare: NULL argument");
    int64_t cap = 0;
    int32_t C = 0, dt = 0;
    tsplat_gaussians_shape(g, &cap, &C, &dt);
    if (cap > S->cfg.max_gaussians || C != S->cfg.C || dt != S->cfg.feat_dtype)
        return record_error(TSPLAT_ERR_INVALID_ARG, "server_prepare: Gaussians do not match the server configuration");
    std::unique_lock<std::mutex> lock(S->mu);
    S->prepare.push_back(g);
    const size_t want = S->prepare.size();
    S->cv.notify_all();
    const auto deadline = std::chrono::steady_clock::now() + std::chrono::microseconds((int64_t)(timeout_ms * 1000.0));
    for (;;) {
        bool all = true;
        for (const Lane &L : S->lanes) all &= L.prepared >= want;
        if (all) break;
        if (S->cv.wait_until(lock, deadline) == std::cv_status::timeout) return TSPLAT_ERR_TIMEOUT;
    }
    const tsplat_status st = S->prepare_status;
    S->prepare_status = TSPLAT_OK;
    return st == TSPLAT_OK ? TSPLAT_OK : record_error(st, "server_prepare: graph capture failed");
}

tsplat_status tsplat_server_release_frame(tsplat_server *S, const tsplat_gaussians *g, double timeout_ms) {
    if (!S || !g) return record_error(TSPLAT_ERR_INVALID_ARG, "server_release_frame: NULL argument");
    std::unique_lock<std::mutex> lock(S->mu);
    if (S->frame == g) return record_error(TSPLAT_ERR_INVALID_ARG, "server_release_frame: g is the current frame");
    const auto deadline = std::chrono::steady_clock::now() + std::chrono::microseconds((int64_t)(timeout_ms * 1000.0));
    for (;;) {
        bool used = false;
        for (const Lane &L : S->lanes) used |= L.busy && L.frame == g;
        if (!used) return TSPLAT_OK;
        if (S->cv.wait_until(lock, deadline) == std::cv_status::timeout) return TSPLAT_ERR_TIMEOUT;
    }
}

tsplat_status tsplat_server_submit(tsplat_server *S, const tsplat_camera *cam, float *out_feat, float *out_alpha,
                                   uint64_t *req_id) {
    if (!S || !cam || !out_feat || !req_id) return record_error(TSPLAT_ERR_INVALID_ARG, "server_submit: NULL argument");
    if (cam->width < 1 || cam->height < 1 || cam->width > S->cfg.max_width || cam->height > S->cfg.max_height)
        return record_error(TSPLAT_ERR_INVALID_ARG, "server_submit: view larger than the server's maximum");
    std::lock_guard<std::mutex> lock(S->mu);
    if (S->error != TSPLAT_OK) return record_error(S->error, "server_submit: the server failed earlier");
    Request r;
    r.cam = *cam;
    r.out_feat = out_feat;
    r.out_alpha = out_alpha;
    r.t_submit = now_ms();
    r.latency_ms = 0;
    r.est_pairs = est_pairs(*S, S->cfg.max_gaussians, cam->width, cam->height);
    r.state = REQ_PENDING;
    r.solo = false;
    r.fail_status = TSPLAT_OK;
    r.fail_msg[0] = 0;
    const uint64_t id = S->next_id++;
    S->reqs.emplace(id, r);
    S->pending.push_back(id);
    if (S->t_first == 0) S->t_first = r.t_submit;
    *req_id = id;
    S->cv.notify_all();
    return TSPLAT_OK;
}

tsplat_status tsplat_server_poll(tsplat_server *S, uint64_t req_id, double *latency_ms) {
    if (!S) return record_error(TSPLAT_ERR_INVALID_ARG, "server_poll: NULL argument");
    std::lock_guard<std::mutex> lock(S->mu);
    auto it = S->reqs.find(req_id);
    if (it == S->reqs.end()) return record_error(TSPLAT_ERR_INVALID_ARG, "server_poll: unknown request");
    if (it->second.state == REQ_FAILED) return record_error(it->second.fail_status, it->second.fail_msg);
    if (it->second.state != REQ_DONE) return TSPLAT_ERR_NOT_READY;
    if (latency_ms) *latency_ms = it->second.latency_ms;
    return TSPLAT_OK;
}

tsplat_status tsplat_server_wait(tsplat_server *S, uint64_t req_id, double timeout_ms, double *latency_ms) {
    if (!S) return record_error(TSPLAT_ERR_INVALID_ARG, "server_wait: NULL argument");
    std::unique_lock<std::mutex> lock(S->mu);
    const auto deadline = std::chrono::steady_clock::now() + std::chrono::microseconds((int64_t)(timeout_ms * 1000.0));
    for (;;) {
        auto it = S->reqs.find(req_id);
        if (it == S->reqs.end()) return record_error(TSPLAT_ERR_INVALID_ARG, "server_wait: unknown request");
        if (it->second.state == REQ_DONE) {
            if (latency_ms) *latency_ms = it->second.latency_ms;
            return TSPLAT_OK;
        }
        if (it->second.state == REQ_FAILED) return record_error(it->second.fail_status, it->second.fail_msg);
        if (S->cv.wait_until(lock, deadline) == std::cv_status::timeout) return TSPLAT_ERR_TIMEOUT;
    }
}

tsplat_status tsplat_server_get_stats(tsplat_server *S, tsplat_server_stats *out) {
    if (!S || !out) return record_error(TSPLAT_ERR_INVALID_ARG, "server_stats: NULL argument");
    std::lock_guard<std::mutex> lock(S->mu);
    memset(out, 0, sizeof(*out));
    std::vector<double> l = S->latencies;
    out->completed = (int64_t)l.size();
    out->batches = (int64_t)S->batches;
    out->views_launched = (int64_t)S->views;
    out->retried = (int64_t)S->retries;
    out->lanes = (int32_t)S->lanes.size();
    out->lane_bytes = S->lane_bytes;
    out->pending = (int64_t)S->pending.size();
    out->pair_scale = S->pair_scale;
    if (!l.empty()) {
        std::sort(l.begin(), l.end());
        auto pct = [&](double q) { return l[std::min(l.size() - 1, (size_t)floor(q * (double)(l.size() - 1) + 0.5))]; };
        out->p50_ms = pct(0.50);
        out->p99_ms = pct(0.99);
        out->max_ms = l.back();
        if (S->t_last > S->t_first) out->views_per_s = 1e3 * (double)l.size() / (S->t_last - S->t_first);
    }
    return TSPLAT_OK;
}

tsplat_status tsplat_server_reset_stats(tsplat_server *S) {
    if (!S) return record_error(TSPLAT_ERR_INVALID_ARG, "server_reset_stats: NULL argument");
    std::lock_guard<std::mutex> lock(S->mu);
    S->latencies.clear();
    S->batches = S->views = S->retries = 0;
    S->t_first = S->t_last = 0;
    for (auto it = S->reqs.begin(); it != S->reqs.end();)
        it = (it->second.state == REQ_DONE || it->second.state == REQ_FAILED) ? S->reqs.erase(it) : std::next(it);
    return TSPLAT_OK;
}

}  // extern "C"
