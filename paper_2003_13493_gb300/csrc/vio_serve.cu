// Serving loop behind vio_serve_* / vio_submit / vio_poll: frames from many
// camera streams arrive one by one; a scheduler thread batches whatever is
// pending into the next free "lane" (a CUDA stream with its own resident
// buffers and its own detector context), so work submitted while other
// batches are on the GPU is admitted as soon as a lane and device memory
// free up, and batches on different lanes overlap on the device.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <unordered_set>
#include <vector>

#include "../../include/vio.h"
#include "vio_ctx.h"

namespace {

using Clock = std::chrono::steady_clock;

uint64_t now_ns() {
    return (uint64_t)std::chrono::duration_cast<std::chrono::nanoseconds>(Clock::now().time_since_epoch()).count();
}

size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

struct Request {
    uint64_t ticket = 0;
    int stream_id = 0;
    const uint8_t* host = nullptr;
    vio_dims dims{};
    uint64_t t_submit = 0;
    size_t cost = 0;        // device bytes while in flight
    size_t ncell = 0;
};

struct Result {
    std::vector<vio_feature> cells;
    int32_t count = 0;
    uint64_t latency_ns = 0;
};

struct Lane {
    vio_ctx* ctx = nullptr;
    cudaStream_t stream = nullptr;
    cudaEvent_t done = nullptr;       // after the batch's last operation (timed)
    cudaEvent_t start = nullptr;      // before its first operation (timed)
    vio_feature* d_cells = nullptr;   // cells of all frames, then int32 counts
    size_t cells_cap = 0;
    uint8_t* h_cells = nullptr;       // pinned copy of d_cells
    size_t h_cap = 0;
    std::vector<Request> batch;       // in flight
    std::vector<size_t> cell_off;
    size_t bytes = 0;
    bool busy = false;
};

}  // namespace

struct vio_server_state {
    vio_serve_config cfg{};
    int device = 0;
    std::vector<Lane> lanes;
    std::mutex mu;
    std::condition_variable cv;
    std::deque<Request> pending;
    std::unordered_map<uint64_t, Result> done;
    std::unordered_set<uint64_t> live;   // submitted, not yet completed
    std::vector<uint64_t> latencies;  // completed requests, ns
    uint64_t next_ticket = 1;
    uint64_t submitted = 0, completed = 0, rejected = 0, batches = 0, batched_frames = 0;
    uint64_t max_batch_frames = 0, max_lanes_in_flight = 0, overlapped_batches = 0;
    // device-time intervals (ms after t0_ev) of the last retired batch of
    // each lane, for the overlap count
    cudaEvent_t t0_ev = nullptr;
    std::vector<float> last_begin, last_end;
    uint64_t t_first = 0, t_last = 0;
    size_t bytes_in_flight = 0;
    std::atomic<bool> stop{false};
    vio_status error = VIO_OK;
    std::thread worker;
};

// The context's serving state lives in a side table so that vio_ctx itself
// stays unaware of serving.
namespace {
std::mutex g_srv_mu;
std::unordered_map<const vio_ctx*, vio_server_state*> g_srv;

vio_server_state* server_of(const vio_ctx* ctx) {
    std::lock_guard<std::mutex> g(g_srv_mu);
    auto it = g_srv.find(ctx);
    return it == g_srv.end() ? nullptr : it->second;
}

size_t request_cost(const vio_dims& d, int levels, int cell) {
    size_t in = align_up((size_t)align_up(d.w, 16) * d.h, 256);
    size_t pyr = 0;
    for (int k = 1; k < levels; ++k) pyr += align_up(align_up(d.w >> k, 128) * (size_t)(d.h >> k), 256);
    const size_t nc = vio_num_cells(d.w, d.h, cell);
    return in + pyr + nc * (8 + 16);
}

vio_status grow_dev(void** p, size_t* cap, size_t need) {
    if (need <= *cap && *p) return VIO_OK;
    if (*p) cudaFree(*p);
    *p = nullptr;
    *cap = 0;
    size_t want = std::max(need, (size_t)1 << 20);
    if (cudaMalloc(p, want) != cudaSuccess) return VIO_ERR_OOM;
    *cap = want;
    return VIO_OK;
}

vio_status grow_host(uint8_t** p, size_t* cap, size_t need) {
    if (need <= *cap && *p) return VIO_OK;
    if (*p) cudaFreeHost(*p);
    *p = nullptr;
    *cap = 0;
    size_t want = std::max(need, (size_t)1 << 16);
    if (cudaHostAlloc((void**)p, want, cudaHostAllocDefault) != cudaSuccess) return VIO_ERR_OOM;
    *cap = want;
    return VIO_OK;
}

// Detects the batch on the lane's stream: pinned frames are read by the
// pyramid kernel through their device mapping, records are written straight
// into the lane's pinned result buffer, then the counts follow.
vio_status launch_lane(vio_server_state* S, Lane& L) {
    vio::NvtxRange nvtx("vio_serve_batch");
    const auto& c = S->cfg;
    const int n = (int)L.batch.size();
    size_t cell_need = 0;
    L.cell_off.assign(n, 0);
    for (int i = 0; i < n; ++i) {
        L.cell_off[i] = cell_need;
        cell_need += L.batch[i].ncell;
    }
    const size_t cell_bytes = cell_need * sizeof(vio_feature) + sizeof(int32_t) * n;
    vio_status st;
    if (cell_bytes > L.cells_cap || cell_bytes > L.h_cap) cudaStreamSynchronize(L.stream);
    if (cudaEventRecord(L.start, L.stream) != cudaSuccess) return VIO_ERR_CUDA;
    if ((st = grow_dev((void**)&L.d_cells, &L.cells_cap, cell_bytes)) != VIO_OK) return st;
    if ((st = grow_host(&L.h_cells, &L.h_cap, cell_bytes)) != VIO_OK) return st;
    std::vector<const uint8_t*> frames(n);
    std::vector<vio_dims> dims(n);
    std::vector<int4*> outs(n);
    bool all_direct = true;
    for (int i = 0; i < n; ++i) {
        frames[i] = L.batch[i].host;
        dims[i] = L.batch[i].dims;
        int4* mapped = static_cast<int4*>(
            const_cast<void*>(vio::host_device_alias(L.h_cells + L.cell_off[i] * sizeof(vio_feature))));
        const bool direct = mapped && ((uintptr_t)mapped & 15) == 0;
        all_direct &= direct;
        outs[i] = direct ? mapped : reinterpret_cast<int4*>(L.d_cells + L.cell_off[i]);
    }
    int32_t* d_counts = reinterpret_cast<int32_t*>(L.d_cells + cell_need);
    st = vio::detect_from_host(L.ctx, frames.data(), dims.data(), n, c.thresh, c.arc_len, c.cell_size, c.levels,
                               outs.data(), d_counts, L.stream);
    if (st != VIO_OK) return st;
    const size_t cbytes = cell_need * sizeof(vio_feature);
    const cudaError_t ce =
        all_direct ? cudaMemcpyAsync(L.h_cells + cbytes, d_counts, sizeof(int32_t) * n, cudaMemcpyDeviceToHost,
                                     L.stream)
                   : cudaMemcpyAsync(L.h_cells, L.d_cells, cell_bytes, cudaMemcpyDeviceToHost, L.stream);
    if (ce != cudaSuccess) return VIO_ERR_CUDA;
    if (cudaEventRecord(L.done, L.stream) != cudaSuccess) return VIO_ERR_CUDA;
    return VIO_OK;
}

void finish_lane(vio_server_state* S, Lane& L, int lane_index) {
    const int n = (int)L.batch.size();
    const uint64_t t = now_ns();
    // this batch's device-time interval against the other lanes' latest ones
    // (a lane's batches run one after another, so a batch of lane j that
    // overlaps this one is j's latest retired batch or one still running)
    float b = 0.f, e = 0.f;
    const bool timed = cudaEventElapsedTime(&b, S->t0_ev, L.start) == cudaSuccess &&
                       cudaEventElapsedTime(&e, S->t0_ev, L.done) == cudaSuccess;
    bool overlapped = false;
    if (timed) {
        for (int j = 0; j < (int)S->lanes.size(); ++j) {
            if (j == lane_index) continue;
            if (S->last_end[j] > S->last_begin[j] && S->last_begin[j] < e && b < S->last_end[j]) overlapped = true;
            const Lane& O = S->lanes[j];
            float ob = 0.f;
            // a batch still in flight on lane j that began before this one ended
            if (O.busy && cudaEventQuery(O.start) == cudaSuccess &&
                cudaEventElapsedTime(&ob, S->t0_ev, O.start) == cudaSuccess && ob < e)
                overlapped = true;
        }
        S->last_begin[lane_index] = b;
        S->last_end[lane_index] = e;
    } else {
        cudaGetLastError();
    }
    // the batch is complete; a device-side status of the lane stops serving
    const vio_status dst = vio_sync(L.ctx, reinterpret_cast<vio_stream>(L.stream));
    if (dst != VIO_OK) {
        std::lock_guard<std::mutex> g(S->mu);
        S->error = dst;
        S->stop = true;
    }
    size_t cell_total = 0;
    for (auto& r : L.batch) cell_total += r.ncell;
    const int32_t* counts = reinterpret_cast<const int32_t*>(L.h_cells + cell_total * sizeof(vio_feature));
    const vio_feature* cells = reinterpret_cast<const vio_feature*>(L.h_cells);
    std::lock_guard<std::mutex> g(S->mu);
    for (int i = 0; i < n; ++i) {
        const Request& r = L.batch[i];
        const uint64_t lat = t - r.t_submit;
        S->latencies.push_back(lat);
        S->live.erase(r.ticket);
        if (S->cfg.keep_results) {
            Result res;
            res.cells.assign(cells + L.cell_off[i], cells + L.cell_off[i] + r.ncell);
            res.count = counts[i];
            res.latency_ns = lat;
            S->done.emplace(r.ticket, std::move(res));
        }
    }
    S->completed += n;
    S->overlapped_batches += overlapped ? 1 : 0;
    S->t_last = t;
    S->bytes_in_flight -= L.bytes;
    L.bytes = 0;
    L.batch.clear();
    L.busy = false;
    S->cv.notify_all();
}

void worker_main(vio_server_state* S) {
    cudaSetDevice(S->device);
    const auto& c = S->cfg;
    uint64_t last_progress = now_ns();
    while (true) {
        bool progressed = false;
        // retire finished lanes
        for (int li = 0; li < (int)S->lanes.size(); ++li) {
            Lane& L = S->lanes[li];
            if (L.busy && cudaEventQuery(L.done) == cudaSuccess) {
                finish_lane(S, L, li);
                progressed = true;
            }
        }
        // admit pending frames into free lanes (continuous batching)
        for (auto& L : S->lanes) {
            if (L.busy) continue;
            {
                std::lock_guard<std::mutex> g(S->mu);
                if (S->pending.empty()) break;
                const uint64_t age = now_ns() - S->pending.front().t_submit;
                const bool full = (int)S->pending.size() >= c.max_batch;
                if (!full && age < (uint64_t)c.max_wait_us * 1000ull) break;
                while (!S->pending.empty() && (int)L.batch.size() < c.max_batch) {
                    const Request& r = S->pending.front();
                    // admit while the frames in flight fit the device budget
                    if (c.mem_budget_bytes && S->bytes_in_flight + r.cost > c.mem_budget_bytes &&
                        S->bytes_in_flight > 0)
                        break;
                    S->bytes_in_flight += r.cost;
                    L.bytes += r.cost;
                    L.batch.push_back(r);
                    S->pending.pop_front();
                }
                if (L.batch.empty()) break;
                S->batches += 1;
                S->batched_frames += L.batch.size();
                S->max_batch_frames = std::max<uint64_t>(S->max_batch_frames, L.batch.size());
                uint64_t in_flight = 1;
                for (const auto& O : S->lanes) in_flight += (&O != &L && O.busy) ? 1 : 0;
                S->max_lanes_in_flight = std::max(S->max_lanes_in_flight, in_flight);
            }
            L.busy = true;
            const vio_status st = launch_lane(S, L);
            if (st != VIO_OK) {
                std::lock_guard<std::mutex> g(S->mu);
                S->error = st;
                S->stop = true;
            }
            progressed = true;
        }
        if (S->stop.load()) {
            bool any_busy = false;
            for (auto& L : S->lanes) any_busy |= L.busy;
            std::lock_guard<std::mutex> g(S->mu);
            if (!any_busy && (S->pending.empty() || S->error != VIO_OK)) break;
        }
        if (progressed) {
            last_progress = now_ns();
        } else {
            // poll while batches are in flight or frames arrived recently;
            // block (submit notifies) after a quiet millisecond
            bool any_busy = false;
            for (auto& L : S->lanes) any_busy |= L.busy;
            if (any_busy || now_ns() - last_progress < 1000000ull) {
                std::this_thread::yield();
            } else {
                std::unique_lock<std::mutex> lk(S->mu);
                if (S->pending.empty() && !S->stop.load()) S->cv.wait_for(lk, std::chrono::milliseconds(1));
            }
        }
    }
}

void destroy_state(vio_server_state* S) {
    for (auto& L : S->lanes) {
        if (L.stream) cudaStreamSynchronize(L.stream);
        if (L.ctx) vio_destroy(L.ctx);
        if (L.stream) cudaStreamDestroy(L.stream);
        if (L.done) cudaEventDestroy(L.done);
        if (L.start) cudaEventDestroy(L.start);
        cudaFree(L.d_cells);
        if (L.h_cells) cudaFreeHost(L.h_cells);
    }
    if (S->t0_ev) cudaEventDestroy(S->t0_ev);
    delete S;
}

}  // namespace

extern "C" {

void vio_serve_config_default(vio_serve_config* c) {
    if (!c) return;
    std::memset(c, 0, sizeof(*c));
    c->thresh = 15;
    c->arc_len = 9;
    c->cell_size = 32;
    c->levels = 3;
    c->max_batch = 32;
    c->max_wait_us = 0;
    c->lanes = 3;
    c->mem_budget_bytes = (size_t)4 << 30;
    c->queue_capacity = 65536;
    c->keep_results = 1;
}

vio_status vio_serve_start(vio_ctx* ctx, const vio_serve_config* cfg) {
    if (!ctx || !cfg) return VIO_ERR_INVALID_ARG;
    if (server_of(ctx)) return VIO_ERR_BUSY;
    if (cfg->lanes < 1 || cfg->lanes > 8 || cfg->max_batch < 1 || cfg->max_batch > 1024 || cfg->max_wait_us < 0 ||
        cfg->queue_capacity < 1 || cfg->thresh < 0 || cfg->thresh > 255 || cfg->arc_len < 9 || cfg->arc_len > 16 ||
        cfg->cell_size < 32 || cfg->cell_size % 32 || cfg->levels < 1 || cfg->levels > VIO_MAX_LEVELS)
        return VIO_ERR_INVALID_ARG;
    // lanes score and suppress like the parent context
    vio_config base;
    if (vio_get_config(ctx, &base) != VIO_OK) return VIO_ERR_INVALID_ARG;
    base.mem_budget_bytes = 0;
    base.autotune = 0;
    base.profile = 0;
    const int dev = vio_device(ctx);
    if (dev < 0 || cudaSetDevice(dev) != cudaSuccess) return VIO_ERR_CUDA;
    auto* S = new vio_server_state();
    S->cfg = *cfg;
    S->device = dev;
    S->lanes.resize(cfg->lanes);
    for (auto& L : S->lanes) {
        vio_config lc = base;
        lc.device = dev;
        lc.max_frames = cfg->max_batch;
        vio_status st = vio_create(&L.ctx, &lc);
        if (st != VIO_OK) {
            destroy_state(S);
            return st;
        }
        if (cudaStreamCreateWithFlags(&L.stream, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreate(&L.done) != cudaSuccess || cudaEventCreate(&L.start) != cudaSuccess) {
            destroy_state(S);
            return VIO_ERR_CUDA;
        }
    }
    // the origin of the lanes' device-time intervals
    S->last_begin.assign(cfg->lanes, 0.f);
    S->last_end.assign(cfg->lanes, 0.f);
    if (cudaEventCreate(&S->t0_ev) != cudaSuccess || cudaEventRecord(S->t0_ev, S->lanes[0].stream) != cudaSuccess ||
        cudaEventSynchronize(S->t0_ev) != cudaSuccess) {
        destroy_state(S);
        return VIO_ERR_CUDA;
    }
    {
        std::lock_guard<std::mutex> g(g_srv_mu);
        g_srv[ctx] = S;
    }
    S->worker = std::thread(worker_main, S);
    return VIO_OK;
}

vio_status vio_submit(vio_ctx* ctx, int stream_id, const uint8_t* host_frame, vio_dims d, uint64_t* ticket) {
    vio_server_state* S = server_of(ctx);
    if (!S || !host_frame || !ticket) return VIO_ERR_INVALID_ARG;
    const int L = S->cfg.levels;
    if (d.w < 7 || d.h < 7 || d.w > 65535 || d.h > 65535 || (int64_t)d.w * d.h >= (1ll << 28) || d.pitch < d.w ||
        (d.w >> (L - 1)) < 7 || (d.h >> (L - 1)) < 7)
        return VIO_ERR_INVALID_ARG;
    Request r;
    r.stream_id = stream_id;
    r.host = host_frame;
    r.dims = d;
    r.t_submit = now_ns();
    r.cost = request_cost(d, L, S->cfg.cell_size);
    r.ncell = vio_num_cells(d.w, d.h, S->cfg.cell_size);
    std::lock_guard<std::mutex> g(S->mu);
    if (S->error != VIO_OK) return S->error;
    if ((int)S->pending.size() >= S->cfg.queue_capacity) {
        S->rejected += 1;
        return VIO_ERR_BUSY;
    }
    if (S->cfg.mem_budget_bytes && r.cost > S->cfg.mem_budget_bytes) return VIO_ERR_OOM;
    r.ticket = S->next_ticket++;
    *ticket = r.ticket;
    if (S->submitted == 0) S->t_first = r.t_submit;
    S->submitted += 1;
    S->live.insert(r.ticket);
    S->pending.push_back(r);
    S->cv.notify_all();
    return VIO_OK;
}

vio_status vio_poll(vio_ctx* ctx, uint64_t ticket, vio_feature* host_out, int32_t* count, int* done) {
    vio_server_state* S = server_of(ctx);
    if (!S || !done) return VIO_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> g(S->mu);
    if (S->error != VIO_OK) return S->error;
    auto it = S->done.find(ticket);
    if (it == S->done.end()) {
        *done = 0;
        // still queued or running; anything else was never issued or is taken
        return S->live.count(ticket) ? VIO_OK : VIO_ERR_NOT_FOUND;
    }
    if (host_out) std::memcpy(host_out, it->second.cells.data(), it->second.cells.size() * sizeof(vio_feature));
    if (count) *count = it->second.count;
    *done = 1;
    S->done.erase(it);
    return VIO_OK;
}

vio_status vio_serve_drain(vio_ctx* ctx, int timeout_ms) {
    vio_server_state* S = server_of(ctx);
    if (!S) return VIO_ERR_INVALID_ARG;
    std::unique_lock<std::mutex> lk(S->mu);
    const auto deadline = Clock::now() + std::chrono::milliseconds(timeout_ms);
    while (S->completed < S->submitted && S->error == VIO_OK) {
        if (S->cv.wait_until(lk, deadline) == std::cv_status::timeout && S->completed < S->submitted)
            return VIO_ERR_TIMEOUT;
    }
    return S->error;
}

vio_status vio_serve_stats(vio_ctx* ctx, vio_serve_stats_t* out) {
    vio_server_state* S = server_of(ctx);
    if (!S || !out) return VIO_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> g(S->mu);
    std::memset(out, 0, sizeof(*out));
    out->submitted = S->submitted;
    out->completed = S->completed;
    out->rejected = S->rejected;
    out->batches = S->batches;
    out->mean_batch = S->batches ? (double)S->batched_frames / (double)S->batches : 0.0;
    if (!S->latencies.empty()) {
        std::vector<uint64_t> v = S->latencies;
        auto pct = [&](double p) {
            size_t i = (size_t)(p * (double)(v.size() - 1) + 0.5);
            std::nth_element(v.begin(), v.begin() + i, v.end());
            return (double)v[i] * 1e-3;
        };
        out->p50_us = pct(0.50);
        out->p99_us = pct(0.99);
        out->max_us = (double)*std::max_element(v.begin(), v.end()) * 1e-3;
        double sum = 0;
        for (uint64_t x : v) sum += (double)x;
        out->mean_us = sum / (double)v.size() * 1e-3;
    }
    if (S->completed && S->t_last > S->t_first)
        out->frames_per_s = (double)S->completed / ((double)(S->t_last - S->t_first) * 1e-9);
    out->max_batch_frames = S->max_batch_frames;
    out->max_lanes_in_flight = S->max_lanes_in_flight;
    out->overlapped_batches = S->overlapped_batches;
    return VIO_OK;
}

vio_status vio_serve_stop(vio_ctx* ctx) {
    vio_server_state* S = server_of(ctx);
    if (!S) return VIO_ERR_INVALID_ARG;
    S->stop = true;
    S->cv.notify_all();
    if (S->worker.joinable()) S->worker.join();
    const vio_status err = S->error;
    {
        std::lock_guard<std::mutex> g(g_srv_mu);
        g_srv.erase(ctx);
    }
    destroy_state(S);
    return err;
}

}  // extern "C"
