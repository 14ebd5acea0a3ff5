// Host runtime behind include/vio.h: argument checks, resident buffers, the
// per-shape plan (work list, pyramid layout, tensor maps), CUDA-graph replay
// and the tile autotuner.
#include <cuda.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <unordered_map>
#include <vector>

#include "../../include/vio.h"
#include "vio_kernels.cuh"

using namespace vio;

namespace {

// ---------------------------------------------------------------------------
// Built variants of the fused kernel.
// ---------------------------------------------------------------------------
using DetectFn = void (*)(const CallHeader*, const FrameDesc*, const CUtensorMap*, const CUtensorMap*,
                          const WorkItem*, int32_t*, uint32_t*);
using PyrFn = void (*)(const CallHeader*, const FrameDesc*, const int32_t*);

struct Variant {
    int tw, th, smem;
    DetectFn fn[3];
};

template <int TW, int TH>
Variant make_variant() {
    return Variant{TW, TH, TileGeom<TW, TH>::SMEM,
                   {fast_nms_cell_kernel<TW, TH, 0>, fast_nms_cell_kernel<TW, TH, 1>,
                    fast_nms_cell_kernel<TW, TH, 2>}};
}

const std::vector<Variant>& variants() {
    static const std::vector<Variant> v = {make_variant<128, 32>(), make_variant<64, 32>(),
                                           make_variant<192, 32>(), make_variant<128, 64>(),
                                           make_variant<64, 64>()};
    return v;
}

PyrFn pyr_fn(int levels) {
    switch (levels) {
        case 2: return pyramid_kernel<2>;
        case 3: return pyramid_kernel<3>;
        case 4: return pyramid_kernel<4>;
        case 5: return pyramid_kernel<5>;
        default: return nullptr;
    }
}

size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

using EncodeTiledFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                   const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

// Layout of the per-call block uploaded before each launch.
struct CallLayout {
    size_t hdr = 0, fds = 0, maps0 = 0, bytes = 0;
    explicit CallLayout(int max_frames) {
        hdr = 0;
        fds = align_up(sizeof(CallHeader), 128);
        maps0 = align_up(fds + sizeof(FrameDesc) * max_frames, 128);
        bytes = align_up(maps0 + sizeof(CUtensorMap) * max_frames, 128);
    }
};

struct ShapeKey {
    std::vector<int32_t> v;
    bool operator==(const ShapeKey& o) const { return v == o.v; }
};
struct ShapeHash {
    size_t operator()(const ShapeKey& k) const {
        size_t h = 1469598103934665603ull;
        for (int32_t x : k.v) h = (h ^ (uint32_t)x) * 1099511628211ull;
        return h;
    }
};

struct MapKey {
    uintptr_t ptr;
    int32_t w, h, pitch, bw, bh;
    bool operator==(const MapKey& o) const {
        return ptr == o.ptr && w == o.w && h == o.h && pitch == o.pitch && bw == o.bw && bh == o.bh;
    }
};
struct MapHash {
    size_t operator()(const MapKey& k) const {
        return std::hash<uintptr_t>()(k.ptr) ^ ((size_t)k.w * 73856093u) ^ ((size_t)k.h * 19349663u) ^
               ((size_t)k.pitch * 83492791u) ^ ((size_t)k.bw << 40) ^ ((size_t)k.bh << 52);
    }
};

}  // namespace

// ---------------------------------------------------------------------------
// Context
// ---------------------------------------------------------------------------
struct Plan {
    ShapeKey key;
    int variant = 0;
    int levels = 1, cell = 32, n = 0, mode = 0;
    int n_items = 0, pyr_blocks = 0, grid = 0;
    std::vector<int> gw, gh, ncell;
    std::vector<size_t> key_off;                    // element offset into keys
    std::vector<std::vector<size_t>> lev_off;       // byte offset into pyramid arena
    std::vector<std::vector<int>> lev_pitch;
    size_t keys_total = 0, pyr_total = 0, cells_total = 0;
    // device data fixed for the plan's lifetime
    WorkItem* d_items = nullptr;
    CUtensorMap* d_mapsk = nullptr;     // [n][kMaxLevels-1], resident pyramid levels
    int32_t* d_block_start = nullptr;   // [n+1] pyramid blocks per frame, prefix sum
    cudaGraphExec_t graph = nullptr;
    void release() {
        if (graph) cudaGraphExecDestroy(graph);
        cudaFree(d_items);
        cudaFree(d_mapsk);
        cudaFree(d_block_start);
        graph = nullptr;
        d_items = nullptr;
        d_mapsk = nullptr;
        d_block_start = nullptr;
    }
};

struct vio_ctx {
    vio_config cfg{};
    int sm_count = 0;
    std::string err;
    EncodeTiledFn encode = nullptr;
    CallLayout layout{1};

    // resident device buffers
    uint8_t* d_call = nullptr;          // CallHeader | FrameDesc[] | maps0[]
    int32_t* d_counter = nullptr;
    uint64_t* d_keys = nullptr;
    size_t keys_cap = 0;
    uint8_t* d_pyr = nullptr;
    size_t pyr_cap = 0;
    uint8_t* d_in = nullptr;            // staged level-0 frames (host path / unaligned frames)
    size_t in_cap = 0;
    int4* d_cells = nullptr;            // host path: device-side output records + counts
    size_t cells_cap = 0;
    size_t bytes_in_use = 0;

    // host
    uint32_t* h_status = nullptr;       // pinned, device-mapped status word
    uint32_t* d_status = nullptr;
    uint8_t* h_stage = nullptr;         // pinned ring of call blocks
    int ring = 8, ring_pos = 0;
    std::vector<cudaEvent_t> ring_ev;
    uint8_t* h_out = nullptr;           // pinned host-path output staging
    size_t h_out_cap = 0;

    cudaEvent_t stage_ev[4] = {nullptr, nullptr, nullptr, nullptr};
    cudaStream_t capture_stream = nullptr;
    cudaEvent_t last_ev = nullptr;
    cudaStream_t last_stream = nullptr;
    bool have_last = false;

    std::unordered_map<ShapeKey, Plan, ShapeHash> plans;
    std::unordered_map<ShapeKey, int, ShapeHash> tuned;  // shape -> variant
    std::unordered_map<MapKey, CUtensorMap, MapHash> map_cache;
    int pinned_variant = -1;
    int last_variant = 0;
    void drop_plans() {
        for (auto& kv : plans) kv.second.release();
        plans.clear();
    }
};

namespace {

vio_status fail(vio_ctx* c, vio_status s, const std::string& msg) {
    if (c) c->err = msg;
    return s;
}

#define VIO_CK(call)                                                                          \
    do {                                                                                      \
        cudaError_t e_ = (call);                                                              \
        if (e_ != cudaSuccess) {                                                              \
            return fail(ctx, e_ == cudaErrorMemoryAllocation ? VIO_ERR_OOM : VIO_ERR_CUDA,    \
                        std::string(#call) + ": " + cudaGetErrorString(e_));                  \
        }                                                                                     \
    } while (0)

vio_status grow(vio_ctx* ctx, void** p, size_t* cap, size_t need, bool zero) {
    if (need <= *cap && *p) return VIO_OK;
    size_t want = std::max(need, *cap + *cap / 2);
    size_t budget = ctx->cfg.mem_budget_bytes;
    if (budget && ctx->bytes_in_use - *cap + want > budget) {
        want = need;
        if (ctx->bytes_in_use - *cap + want > budget)
            return fail(ctx, VIO_ERR_OOM, "context memory budget exceeded");
    }
    if (*p) {
        VIO_CK(cudaDeviceSynchronize());
        VIO_CK(cudaFree(*p));
        ctx->bytes_in_use -= *cap;
        *p = nullptr;
        *cap = 0;
    }
    VIO_CK(cudaMalloc(p, want));
    if (zero) VIO_CK(cudaMemset(*p, 0, want));
    *cap = want;
    ctx->bytes_in_use += want;
    return VIO_OK;
}

vio_status encode_map(vio_ctx* ctx, CUtensorMap* out, const void* ptr, int w, int h, int pitch, int bw, int bh) {
    MapKey key{(uintptr_t)ptr, w, h, pitch, bw, bh};
    auto it = ctx->map_cache.find(key);
    if (it != ctx->map_cache.end()) {
        *out = it->second;
        return VIO_OK;
    }
    cuuint64_t gdim[2] = {(cuuint64_t)w, (cuuint64_t)h};
    cuuint64_t gstride[1] = {(cuuint64_t)pitch};
    cuuint32_t box[2] = {(cuuint32_t)bw, (cuuint32_t)bh};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = ctx->encode(out, CU_TENSOR_MAP_DATA_TYPE_UINT8, 2, const_cast<void*>(ptr), gdim, gstride, box,
                             estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                             CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return fail(ctx, VIO_ERR_CUDA, "cuTensorMapEncodeTiled failed: " + std::to_string((int)r));
    if (ctx->map_cache.size() > 8192) ctx->map_cache.clear();
    ctx->map_cache.emplace(key, *out);
    return VIO_OK;
}

vio_status check_args(vio_ctx* ctx, const void* frames, const vio_dims* dims, int n, int thresh, int arc,
                      int cell, int levels, const void* outs) {
    if (!ctx) return VIO_ERR_INVALID_ARG;
    if (!frames || !dims || !outs) return fail(ctx, VIO_ERR_INVALID_ARG, "NULL frames, dims or outputs");
    if (n < 1 || n > ctx->cfg.max_frames)
        return fail(ctx, VIO_ERR_INVALID_ARG, "n_frames must be in 1..max_frames");
    if (thresh < 0 || thresh > 255) return fail(ctx, VIO_ERR_INVALID_ARG, "thresh must be in 0..255");
    if (ctx->cfg.score == VIO_SCORE_MT && thresh < 1)
        return fail(ctx, VIO_ERR_INVALID_ARG, "the MT score needs thresh >= 1");
    if (arc < 9 || arc > 16) return fail(ctx, VIO_ERR_INVALID_ARG, "arc_len must be in 9..16");
    if (cell < 32 || cell % 32 != 0) return fail(ctx, VIO_ERR_INVALID_ARG, "cell_size must be a positive multiple of 32");
    if (levels < 1 || levels > VIO_MAX_LEVELS) return fail(ctx, VIO_ERR_INVALID_ARG, "levels must be in 1..5");
    for (int i = 0; i < n; ++i) {
        const vio_dims& d = dims[i];
        if (d.w < 7 || d.h < 7 || d.w > 65535 || d.h > 65535 || (int64_t)d.w * d.h >= (1ll << 28))
            return fail(ctx, VIO_ERR_INVALID_ARG, "frame " + std::to_string(i) + ": size out of range");
        if (d.pitch < d.w) return fail(ctx, VIO_ERR_INVALID_ARG, "frame " + std::to_string(i) + ": pitch < w");
        if ((d.w >> (levels - 1)) < 7 || (d.h >> (levels - 1)) < 7)
            return fail(ctx, VIO_ERR_INVALID_ARG, "frame " + std::to_string(i) + ": smallest level below 7x7");
    }
    return VIO_OK;
}

ShapeKey shape_key(const vio_dims* dims, int n, int cell, int levels, int mode, int variant) {
    ShapeKey k;
    k.v.reserve(3 * n + 5);
    k.v.push_back(n);
    k.v.push_back(cell);
    k.v.push_back(levels);
    k.v.push_back(mode);
    k.v.push_back(variant);
    for (int i = 0; i < n; ++i) {
        k.v.push_back(dims[i].w);
        k.v.push_back(dims[i].h);
    }
    return k;
}

// Enqueues pyramid -> fused detect -> decode on `s` for plan p.
vio_status enqueue_kernels(vio_ctx* ctx, const Plan& p, cudaStream_t s) {
    const Variant& v = variants()[p.variant];
    auto* hdr = reinterpret_cast<const CallHeader*>(ctx->d_call + ctx->layout.hdr);
    auto* fds = reinterpret_cast<const FrameDesc*>(ctx->d_call + ctx->layout.fds);
    auto* maps0 = reinterpret_cast<const CUtensorMap*>(ctx->d_call + ctx->layout.maps0);
    const bool prof = ctx->cfg.profile != 0;
    // inside stream capture only an external record becomes a graph node
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (prof) VIO_CK(cudaStreamIsCapturing(s, &cap));
    const unsigned rec_flags = cap == cudaStreamCaptureStatusActive ? cudaEventRecordExternal : 0u;
    if (prof) VIO_CK(cudaEventRecordWithFlags(ctx->stage_ev[0], s, rec_flags));
    if (p.levels > 1) {
        pyr_fn(p.levels)<<<p.pyr_blocks, 256, 0, s>>>(hdr, fds, p.d_block_start);
        VIO_CK(cudaGetLastError());
    }
    if (prof) VIO_CK(cudaEventRecordWithFlags(ctx->stage_ev[1], s, rec_flags));
    v.fn[p.mode]<<<p.grid, 256, v.smem, s>>>(hdr, fds, maps0, p.d_mapsk, p.d_items, ctx->d_counter,
                                             ctx->d_status);
    VIO_CK(cudaGetLastError());
    if (prof) VIO_CK(cudaEventRecordWithFlags(ctx->stage_ev[2], s, rec_flags));
    decode_kernel<<<p.n, 256, 0, s>>>(hdr, fds, ctx->d_counter);
    VIO_CK(cudaGetLastError());
    if (prof) VIO_CK(cudaEventRecordWithFlags(ctx->stage_ev[3], s, rec_flags));
    return VIO_OK;
}

// Builds (or finds) the plan for this batch shape and makes the resident
// buffers large enough for it.
vio_status get_plan(vio_ctx* ctx, const vio_dims* dims, int n, int cell, int levels, int variant, Plan** out) {
    const int mode = ctx->cfg.score;
    ShapeKey key = shape_key(dims, n, cell, levels, mode, variant);
    auto it = ctx->plans.find(key);
    Plan* p = nullptr;
    if (it != ctx->plans.end()) {
        p = &it->second;
    } else {
        Plan np;
        np.key = key;
        np.variant = variant;
        np.levels = levels;
        np.cell = cell;
        np.n = n;
        np.mode = mode;
        const Variant& v = variants()[variant];
        std::vector<WorkItem> items;
        std::vector<int32_t> bstart(n + 1, 0);
        size_t koff = 0, poff = 0, coff = 0;
        np.lev_off.resize(n);
        np.lev_pitch.resize(n);
        for (int i = 0; i < n; ++i) {
            const int w = dims[i].w, h = dims[i].h;
            const int gw = (w + cell - 1) / cell, gh = (h + cell - 1) / cell;
            np.gw.push_back(gw);
            np.gh.push_back(gh);
            np.ncell.push_back(gw * gh);
            np.key_off.push_back(koff);
            koff += align_up((size_t)gw * gh, 16);
            coff += (size_t)gw * gh;
            np.lev_off[i].assign(kMaxLevels, 0);
            np.lev_pitch[i].assign(kMaxLevels, 0);
            for (int k = 1; k < levels; ++k) {
                const int wk = w >> k, hk = h >> k;
                const int pk = (int)align_up(wk, 128);
                np.lev_off[i][k] = poff;
                np.lev_pitch[i][k] = pk;
                poff += align_up((size_t)pk * hk, 256);
            }
            const int B = 1 << (levels - 1);
            const int bx = ((w + B - 1) / B + 31) / 32, by = ((h + B - 1) / B + 7) / 8;
            bstart[i + 1] = bstart[i] + (levels > 1 ? bx * by : 0);
        }
        // work list: level-major, then frame, then tile rows
        for (int k = 0; k < levels; ++k)
            for (int i = 0; i < n; ++i) {
                const int wk = dims[i].w >> k, hk = dims[i].h >> k;
                const int ntx = (wk + v.tw - 1) / v.tw, nty = (hk + v.th - 1) / v.th;
                for (int ty = 0; ty < nty; ++ty)
                    for (int tx = 0; tx < ntx; ++tx)
                        items.push_back(WorkItem{(uint16_t)i, (uint8_t)k, 0, (uint16_t)tx, (uint16_t)ty});
            }
        np.n_items = (int)items.size();
        np.pyr_blocks = bstart[n];
        np.keys_total = koff;
        np.pyr_total = poff;
        np.cells_total = coff;

        // resident buffers (keys are zero when allocated and cleared by decode);
        // growing them moves the arenas, which invalidates every other plan
        vio_status st;
        const void* keys0 = ctx->d_keys;
        const void* pyr0 = ctx->d_pyr;
        if ((st = grow(ctx, (void**)&ctx->d_keys, &ctx->keys_cap, np.keys_total * 8, true)) != VIO_OK) return st;
        if ((st = grow(ctx, (void**)&ctx->d_pyr, &ctx->pyr_cap, std::max<size_t>(np.pyr_total, 256), false)) != VIO_OK)
            return st;
        if (keys0 != ctx->d_keys || pyr0 != ctx->d_pyr || ctx->plans.size() >= 64) {
            VIO_CK(cudaDeviceSynchronize());
            ctx->drop_plans();
        }
        int occ = 0;
        VIO_CK(cudaFuncSetAttribute(v.fn[mode], cudaFuncAttributeMaxDynamicSharedMemorySize, v.smem));
        VIO_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, v.fn[mode], 256, v.smem));
        np.grid = std::max(1, std::min(occ, 8)) * ctx->sm_count;
        np.grid = std::min(np.grid, std::max(1, np.n_items));
        // tensor maps for levels >= 1 (resident pyramid, fixed per plan)
        std::vector<CUtensorMap> mapsk((size_t)n * (kMaxLevels - 1));
        for (int i = 0; i < n; ++i)
            for (int k = 1; k < levels; ++k) {
                if ((st = encode_map(ctx, &mapsk[(size_t)i * (kMaxLevels - 1) + k - 1], ctx->d_pyr + np.lev_off[i][k],
                                     dims[i].w >> k, dims[i].h >> k, np.lev_pitch[i][k], v.tw + 32, v.th + 8)) !=
                    VIO_OK)
                    return st;
            }
        auto upload = [&](void** dst, const void* src, size_t bytes) -> vio_status {
            VIO_CK(cudaMalloc(dst, std::max<size_t>(bytes, 16)));
            VIO_CK(cudaMemcpy(*dst, src, bytes, cudaMemcpyHostToDevice));
            return VIO_OK;
        };
        if ((st = upload((void**)&np.d_items, items.data(), items.size() * sizeof(WorkItem))) != VIO_OK ||
            (st = upload((void**)&np.d_mapsk, mapsk.data(), mapsk.size() * sizeof(CUtensorMap))) != VIO_OK ||
            (st = upload((void**)&np.d_block_start, bstart.data(), bstart.size() * sizeof(int32_t))) != VIO_OK) {
            np.release();
            return st;
        }
        p = &ctx->plans.emplace(key, std::move(np)).first->second;
        if (ctx->cfg.use_graphs) {
            cudaGraph_t g = nullptr;
            VIO_CK(cudaStreamBeginCapture(ctx->capture_stream, cudaStreamCaptureModeThreadLocal));
            vio_status es = enqueue_kernels(ctx, *p, ctx->capture_stream);
            cudaError_t ce = cudaStreamEndCapture(ctx->capture_stream, &g);
            if (es != VIO_OK) return es;
            VIO_CK(ce);
            VIO_CK(cudaGraphInstantiate(&p->graph, g, 0));
            cudaGraphDestroy(g);
        }
    }
    *out = p;
    return VIO_OK;
}

// Fills and uploads the call block, then launches the plan on `s`.
vio_status launch(vio_ctx* ctx, Plan& p, const uint8_t* const* lev0, const int* pitch0, const vio_dims* dims,
                  int thresh, int arc, int4* const* outs, int32_t* counts, cudaStream_t s) {
    const Variant& v = variants()[p.variant];
    const int n = p.n;
    // order against work of this context on another stream
    if (ctx->have_last && ctx->last_stream != s) VIO_CK(cudaStreamWaitEvent(s, ctx->last_ev, 0));
    // next staging slot
    const int slot = ctx->ring_pos;
    ctx->ring_pos = (ctx->ring_pos + 1) % ctx->ring;
    VIO_CK(cudaEventSynchronize(ctx->ring_ev[slot]));
    uint8_t* st = ctx->h_stage + (size_t)slot * ctx->layout.bytes;
    CallHeader* hdr = reinterpret_cast<CallHeader*>(st + ctx->layout.hdr);
    FrameDesc* fds = reinterpret_cast<FrameDesc*>(st + ctx->layout.fds);
    CUtensorMap* maps0 = reinterpret_cast<CUtensorMap*>(st + ctx->layout.maps0);
    std::memset(hdr, 0, sizeof(CallHeader));
    hdr->thresh = thresh;
    hdr->arc = arc;
    hdr->n_frames = n;
    hdr->n_items = p.n_items;
    hdr->mode = p.mode;
    hdr->cell = p.cell;
    hdr->levels = p.levels;
    hdr->counts = counts;
    for (int i = 0; i < n; ++i) {
        FrameDesc& f = fds[i];
        std::memset(&f, 0, sizeof(FrameDesc));
        f.w = dims[i].w;
        f.h = dims[i].h;
        f.gw = p.gw[i];
        f.gh = p.gh[i];
        const int B = 1 << (p.levels - 1);
        f.pyr_bx = ((f.w + B - 1) / B + 31) / 32;
        f.keys = ctx->d_keys + p.key_off[i];
        f.out = outs[i];
        f.lev[0] = const_cast<uint8_t*>(lev0[i]);
        f.pitch[0] = pitch0[i];
        for (int k = 1; k < p.levels; ++k) {
            f.lev[k] = ctx->d_pyr + p.lev_off[i][k];
            f.pitch[k] = p.lev_pitch[i][k];
        }
        vio_status es = encode_map(ctx, &maps0[i], lev0[i], f.w, f.h, pitch0[i], v.tw + 32, v.th + 8);
        if (es != VIO_OK) return es;
    }
    const size_t bytes = ctx->layout.maps0 + sizeof(CUtensorMap) * n;
    VIO_CK(cudaMemcpyAsync(ctx->d_call, st, bytes, cudaMemcpyHostToDevice, s));
    VIO_CK(cudaEventRecord(ctx->ring_ev[slot], s));
    if (p.graph) {
        VIO_CK(cudaGraphLaunch(p.graph, s));
    } else {
        vio_status es = enqueue_kernels(ctx, p, s);
        if (es != VIO_OK) return es;
    }
    VIO_CK(cudaEventRecord(ctx->last_ev, s));
    ctx->last_stream = s;
    ctx->have_last = true;
    return VIO_OK;
}

int pick_variant(vio_ctx* ctx, const vio_dims* dims, int n, int cell, int levels) {
    if (ctx->pinned_variant >= 0) return ctx->pinned_variant;
    ShapeKey k = shape_key(dims, n, cell, levels, ctx->cfg.score, -1);
    auto it = ctx->tuned.find(k);
    return it == ctx->tuned.end() ? 0 : it->second;
}

vio_status autotune(vio_ctx* ctx, const uint8_t* const* lev0, const int* pitch0, const vio_dims* dims, int n,
                    int thresh, int arc, int cell, int levels, int4* const* outs, int32_t* counts, cudaStream_t s) {
    ShapeKey k = shape_key(dims, n, cell, levels, ctx->cfg.score, -1);
    if (ctx->tuned.count(k)) return VIO_OK;
    cudaEvent_t e0, e1;
    VIO_CK(cudaEventCreate(&e0));
    VIO_CK(cudaEventCreate(&e1));
    float best = 1e30f;
    int best_v = 0;
    for (int vi = 0; vi < (int)variants().size(); ++vi) {
        Plan* p = nullptr;
        vio_status st = get_plan(ctx, dims, n, cell, levels, vi, &p);
        if (st != VIO_OK) return st;
        for (int r = 0; r < 2; ++r)
            if ((st = launch(ctx, *p, lev0, pitch0, dims, thresh, arc, outs, counts, s)) != VIO_OK) return st;
        VIO_CK(cudaEventRecord(e0, s));
        const int reps = 5;
        for (int r = 0; r < reps; ++r)
            if ((st = launch(ctx, *p, lev0, pitch0, dims, thresh, arc, outs, counts, s)) != VIO_OK) return st;
        VIO_CK(cudaEventRecord(e1, s));
        VIO_CK(cudaEventSynchronize(e1));
        float ms = 0;
        VIO_CK(cudaEventElapsedTime(&ms, e0, e1));
        if (ms < best) {
            best = ms;
            best_v = vi;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    ctx->tuned[k] = best_v;
    return VIO_OK;
}

vio_status detect_impl(vio_ctx* ctx, const uint8_t* const* lev0, const int* pitch0, const vio_dims* dims, int n,
                       int thresh, int arc, int cell, int levels, int4* const* outs, int32_t* counts,
                       cudaStream_t s) {
    if (ctx->cfg.autotune && ctx->pinned_variant < 0) {
        vio_status st = autotune(ctx, lev0, pitch0, dims, n, thresh, arc, cell, levels, outs, counts, s);
        if (st != VIO_OK) return st;
    }
    const int vi = pick_variant(ctx, dims, n, cell, levels);
    Plan* p = nullptr;
    vio_status st = get_plan(ctx, dims, n, cell, levels, vi, &p);
    if (st != VIO_OK) return st;
    ctx->last_variant = vi;
    return launch(ctx, *p, lev0, pitch0, dims, thresh, arc, outs, counts, s);
}

}  // namespace

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------
extern "C" {

void vio_config_default(vio_config* cfg) {
    if (!cfg) return;
    std::memset(cfg, 0, sizeof(*cfg));
    cfg->device = 0;
    cfg->mem_budget_bytes = 0;
    cfg->max_frames = 64;
    cfg->score = VIO_SCORE_SAD_B;
    cfg->autotune = 0;
    cfg->use_graphs = 1;
    cfg->profile = 0;
}

const char* vio_status_str(vio_status s) {
    switch (s) {
        case VIO_OK: return "ok";
        case VIO_ERR_INVALID_ARG: return "invalid argument";
        case VIO_ERR_OOM: return "out of device memory or over the context budget";
        case VIO_ERR_CUDA: return "CUDA error";
        case VIO_ERR_TIMEOUT: return "a bounded device-side wait timed out";
        case VIO_ERR_BUSY: return "queue full";
        case VIO_ERR_UNSUPPORTED: return "device is not an sm_103 GPU";
        case VIO_ERR_NOT_FOUND: return "unknown ticket";
    }
    return "unknown status";
}

const char* vio_last_error(const vio_ctx* ctx) { return ctx ? ctx->err.c_str() : "NULL context"; }

size_t vio_num_cells(int w, int h, int cell) {
    if (w < 1 || h < 1 || cell < 1) return 0;
    return (size_t)((w + cell - 1) / cell) * (size_t)((h + cell - 1) / cell);
}

int vio_num_variants(void) { return (int)variants().size(); }

vio_status vio_variant(int i, vio_tuning* out) {
    if (!out || i < 0 || i >= (int)variants().size()) return VIO_ERR_INVALID_ARG;
    out->tile_w = variants()[i].tw;
    out->tile_h = variants()[i].th;
    out->cta_per_sm = 0;
    out->variant = i;
    return VIO_OK;
}

vio_status vio_create(vio_ctx** out, const vio_config* cfg_in) {
    if (!out) return VIO_ERR_INVALID_ARG;
    *out = nullptr;
    vio_config cfg;
    if (cfg_in) cfg = *cfg_in; else vio_config_default(&cfg);
    if (cfg.max_frames < 1 || cfg.max_frames > 1024 || cfg.score < 0 || cfg.score > 2 || cfg.device < 0)
        return VIO_ERR_INVALID_ARG;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || cfg.device >= ndev) return VIO_ERR_CUDA;
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, cfg.device) != cudaSuccess) return VIO_ERR_CUDA;
    if (prop.major != 10 || prop.minor != 3) return VIO_ERR_UNSUPPORTED;
    if (cudaSetDevice(cfg.device) != cudaSuccess) return VIO_ERR_CUDA;

    vio_ctx* ctx = new vio_ctx();
    ctx->cfg = cfg;
    ctx->sm_count = prop.multiProcessorCount;
    ctx->layout = CallLayout(cfg.max_frames);
    cudaDriverEntryPointQueryResult q;
    void* fnp = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fnp, 12000, cudaEnableDefault, &q) !=
            cudaSuccess || !fnp) {
        delete ctx;
        return VIO_ERR_CUDA;
    }
    ctx->encode = reinterpret_cast<EncodeTiledFn>(fnp);
    auto cleanup = [&](vio_status s) {
        vio_destroy(ctx);
        return s;
    };
    if (cudaMalloc(&ctx->d_call, ctx->layout.bytes) != cudaSuccess) return cleanup(VIO_ERR_OOM);
    if (cudaMalloc(&ctx->d_counter, sizeof(int32_t) * 4) != cudaSuccess) return cleanup(VIO_ERR_OOM);
    if (cudaMemset(ctx->d_counter, 0, sizeof(int32_t) * 4) != cudaSuccess) return cleanup(VIO_ERR_CUDA);
    if (cudaHostAlloc(&ctx->h_status, 64, cudaHostAllocMapped) != cudaSuccess) return cleanup(VIO_ERR_OOM);
    *ctx->h_status = 0;
    if (cudaHostGetDevicePointer((void**)&ctx->d_status, ctx->h_status, 0) != cudaSuccess)
        return cleanup(VIO_ERR_CUDA);
    if (cudaHostAlloc(&ctx->h_stage, ctx->layout.bytes * ctx->ring, cudaHostAllocDefault) != cudaSuccess)
        return cleanup(VIO_ERR_OOM);
    ctx->ring_ev.resize(ctx->ring);
    for (auto& e : ctx->ring_ev) {
        if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) return cleanup(VIO_ERR_CUDA);
    }
    if (cudaEventCreateWithFlags(&ctx->last_ev, cudaEventDisableTiming) != cudaSuccess) return cleanup(VIO_ERR_CUDA);
    for (auto& e : ctx->stage_ev)
        if (cudaEventCreate(&e) != cudaSuccess) return cleanup(VIO_ERR_CUDA);
    if (cudaStreamCreateWithFlags(&ctx->capture_stream, cudaStreamNonBlocking) != cudaSuccess)
        return cleanup(VIO_ERR_CUDA);
    ctx->bytes_in_use = ctx->layout.bytes;
    *out = ctx;
    return VIO_OK;
}

vio_status vio_destroy(vio_ctx* ctx) {
    if (!ctx) return VIO_OK;
    cudaSetDevice(ctx->cfg.device);
    cudaDeviceSynchronize();
    ctx->drop_plans();
    cudaFree(ctx->d_call);
    cudaFree(ctx->d_counter);
    cudaFree(ctx->d_keys);
    cudaFree(ctx->d_pyr);
    cudaFree(ctx->d_in);
    cudaFree(ctx->d_cells);
    if (ctx->h_status) cudaFreeHost(ctx->h_status);
    if (ctx->h_stage) cudaFreeHost(ctx->h_stage);
    if (ctx->h_out) cudaFreeHost(ctx->h_out);
    for (auto& e : ctx->ring_ev)
        if (e) cudaEventDestroy(e);
    if (ctx->last_ev) cudaEventDestroy(ctx->last_ev);
    for (auto& e : ctx->stage_ev)
        if (e) cudaEventDestroy(e);
    if (ctx->capture_stream) cudaStreamDestroy(ctx->capture_stream);
    delete ctx;
    return VIO_OK;
}

vio_status vio_detect(vio_ctx* ctx, const uint8_t* const* frames, const vio_dims* dims, int n, int thresh,
                      int arc, int cell, int levels, vio_feature* const* out_cells, int32_t* out_counts,
                      vio_stream stream) {
    vio_status st = check_args(ctx, frames, dims, n, thresh, arc, cell, levels, out_cells);
    if (st != VIO_OK) return st;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    VIO_CK(cudaSetDevice(ctx->cfg.device));
    for (int i = 0; i < n; ++i)
        if (!frames[i] || !out_cells[i]) return fail(ctx, VIO_ERR_INVALID_ARG, "NULL frame or output pointer");
    // frames that TMA cannot address directly are staged into aligned slots
    std::vector<const uint8_t*> lev0(frames, frames + n);
    std::vector<int> pitch0(n);
    size_t need = 0;
    std::vector<size_t> off(n, (size_t)-1);
    for (int i = 0; i < n; ++i) {
        pitch0[i] = dims[i].pitch;
        if (((uintptr_t)frames[i] & 15) || (dims[i].pitch & 15)) {
            off[i] = need;
            need += align_up((size_t)align_up(dims[i].w, 16) * dims[i].h, 256);
        }
    }
    if (need) {
        if ((st = grow(ctx, (void**)&ctx->d_in, &ctx->in_cap, need, false)) != VIO_OK) return st;
        for (int i = 0; i < n; ++i)
            if (off[i] != (size_t)-1) {
                const int p = (int)align_up(dims[i].w, 16);
                VIO_CK(cudaMemcpy2DAsync(ctx->d_in + off[i], p, frames[i], dims[i].pitch, dims[i].w, dims[i].h,
                                         cudaMemcpyDeviceToDevice, s));
                lev0[i] = ctx->d_in + off[i];
                pitch0[i] = p;
            }
    }
    std::vector<int4*> outs(n);
    for (int i = 0; i < n; ++i) outs[i] = reinterpret_cast<int4*>(out_cells[i]);
    return detect_impl(ctx, lev0.data(), pitch0.data(), dims, n, thresh, arc, cell, levels, outs.data(), out_counts,
                       s);
}

vio_status vio_detect_host(vio_ctx* ctx, const uint8_t* const* host_frames, const vio_dims* dims, int n, int thresh,
                           int arc, int cell, int levels, vio_feature* const* host_cells, int32_t* host_counts,
                           vio_stream stream) {
    vio_status st = check_args(ctx, host_frames, dims, n, thresh, arc, cell, levels, host_cells);
    if (st != VIO_OK) return st;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    VIO_CK(cudaSetDevice(ctx->cfg.device));
    for (int i = 0; i < n; ++i)
        if (!host_frames[i] || !host_cells[i]) return fail(ctx, VIO_ERR_INVALID_ARG, "NULL frame or output pointer");
    std::vector<size_t> off(n);
    std::vector<int> pitch0(n);
    size_t need = 0, ncell_total = 0;
    std::vector<size_t> coff(n);
    for (int i = 0; i < n; ++i) {
        pitch0[i] = (int)align_up(dims[i].w, 16);
        off[i] = need;
        need += align_up((size_t)pitch0[i] * dims[i].h, 256);
        coff[i] = ncell_total;
        ncell_total += vio_num_cells(dims[i].w, dims[i].h, cell);
    }
    const size_t cell_bytes = ncell_total * sizeof(int4) + align_up(sizeof(int32_t) * n, 16);
    if ((st = grow(ctx, (void**)&ctx->d_in, &ctx->in_cap, need, false)) != VIO_OK) return st;
    if ((st = grow(ctx, (void**)&ctx->d_cells, &ctx->cells_cap, cell_bytes, false)) != VIO_OK) return st;
    if (ctx->h_out_cap < cell_bytes) {
        if (ctx->h_out) cudaFreeHost(ctx->h_out);
        ctx->h_out = nullptr;
        ctx->h_out_cap = 0;
        VIO_CK(cudaHostAlloc(&ctx->h_out, cell_bytes, cudaHostAllocDefault));
        ctx->h_out_cap = cell_bytes;
    }
    std::vector<const uint8_t*> lev0(n);
    std::vector<int4*> outs(n);
    for (int i = 0; i < n; ++i) {
        VIO_CK(cudaMemcpy2DAsync(ctx->d_in + off[i], pitch0[i], host_frames[i], dims[i].pitch, dims[i].w, dims[i].h,
                                 cudaMemcpyHostToDevice, s));
        lev0[i] = ctx->d_in + off[i];
        outs[i] = ctx->d_cells + coff[i];
    }
    int32_t* d_counts = reinterpret_cast<int32_t*>(ctx->d_cells + ncell_total);
    if ((st = detect_impl(ctx, lev0.data(), pitch0.data(), dims, n, thresh, arc, cell, levels, outs.data(),
                          d_counts, s)) != VIO_OK)
        return st;
    VIO_CK(cudaMemcpyAsync(ctx->h_out, ctx->d_cells, cell_bytes, cudaMemcpyDeviceToHost, s));
    VIO_CK(cudaStreamSynchronize(s));
    if (*ctx->h_status) {
        *ctx->h_status = 0;
        return fail(ctx, VIO_ERR_TIMEOUT, "a bounded device-side wait timed out");
    }
    const int4* rec = reinterpret_cast<const int4*>(ctx->h_out);
    for (int i = 0; i < n; ++i)
        std::memcpy(host_cells[i], rec + coff[i], vio_num_cells(dims[i].w, dims[i].h, cell) * sizeof(int4));
    if (host_counts)
        std::memcpy(host_counts, ctx->h_out + ncell_total * sizeof(int4), sizeof(int32_t) * n);
    return VIO_OK;
}

vio_status vio_sync(vio_ctx* ctx, vio_stream stream) {
    if (!ctx) return VIO_ERR_INVALID_ARG;
    VIO_CK(cudaSetDevice(ctx->cfg.device));
    VIO_CK(cudaStreamSynchronize(reinterpret_cast<cudaStream_t>(stream)));
    if (*ctx->h_status) {
        *ctx->h_status = 0;
        return fail(ctx, VIO_ERR_TIMEOUT, "a bounded device-side wait timed out");
    }
    return VIO_OK;
}

vio_status vio_stage_ms(vio_ctx* ctx, float* ms3) {
    if (!ctx || !ms3) return VIO_ERR_INVALID_ARG;
    if (!ctx->cfg.profile) return fail(ctx, VIO_ERR_INVALID_ARG, "context was created without profile = 1");
    if (!ctx->have_last) return fail(ctx, VIO_ERR_INVALID_ARG, "no call recorded yet");
    VIO_CK(cudaSetDevice(ctx->cfg.device));
    VIO_CK(cudaEventSynchronize(ctx->stage_ev[3]));
    for (int i = 0; i < 3; ++i) VIO_CK(cudaEventElapsedTime(&ms3[i], ctx->stage_ev[i], ctx->stage_ev[i + 1]));
    return VIO_OK;
}

vio_status vio_get_tuning(const vio_ctx* ctx, vio_tuning* out) {
    if (!ctx || !out) return VIO_ERR_INVALID_ARG;
    const int vi = ctx->pinned_variant >= 0 ? ctx->pinned_variant : ctx->last_variant;
    vio_variant(vi, out);
    return VIO_OK;
}

vio_status vio_set_tuning(vio_ctx* ctx, const vio_tuning* t) {
    if (!ctx) return VIO_ERR_INVALID_ARG;
    if (!t) {
        ctx->pinned_variant = -1;
        return VIO_OK;
    }
    if (t->variant < 0 || t->variant >= (int)variants().size())
        return fail(ctx, VIO_ERR_INVALID_ARG, "unknown variant");
    ctx->pinned_variant = t->variant;
    return VIO_OK;
}

}  // extern "C"
