// Internal: the context object behind include/vio.h and the host helpers the
// runtime's translation units share (resident buffers, error recording).
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <algorithm>
#include <array>
#include <string>
#include <unordered_map>
#include <vector>

#include "../../include/vio.h"
#include "vio_kernels.cuh"

namespace vio {

inline size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

constexpr int kMaxCtasPerSm = 4;  // the detect kernels' launch bounds

using EncodeTiledFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                   const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

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


// A named range on the profiler's timeline for the duration of a scope (NVTX;
// free when no profiler is attached).
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};

// One input slot of vio_detect_host_async: frames of one call in flight.
struct HostSlot {
    uint8_t* d_in = nullptr;
    size_t in_cap = 0;
    int32_t* d_counts = nullptr;
    size_t counts_cap = 0;
    cudaEvent_t done = nullptr;  // after the kernels that read the slot
    bool used = false;
};
constexpr int kHostSlots = 3;

// Resident state of the feature tracker (vio_track).
struct TrackState {
    uint8_t* d_call = nullptr;   // the current call block
    size_t call_cap = 0;
    uint8_t* h_stage = nullptr;  // pinned staging of the call block
    size_t stage_cap = 0;
    cudaEvent_t stage_ev = nullptr;
    uint8_t* d_pyr = nullptr;    // levels 1..L-1 of both frames of every pair
    size_t pyr_cap = 0;
    uint8_t* d_in = nullptr;     // level-0 copies of frames that are not 16-byte aligned
    size_t in_cap = 0;
    cudaEvent_t done_ev = nullptr;  // after the last call's kernels: the next call's stream waits on it
    bool have_done = false;
};

}  // namespace vio

// ---------------------------------------------------------------------------
// Context
// ---------------------------------------------------------------------------
struct vio_ctx {
    using EncodeTiledFn = vio::EncodeTiledFn;
    using ShapeKey = vio::ShapeKey;
    using ShapeHash = vio::ShapeHash;
    using MapKey = vio::MapKey;
    using MapHash = vio::MapHash;
    vio_config cfg{};
    int sm_count = 0;
    std::string err;
    EncodeTiledFn encode = nullptr;
    size_t call_cap = 0;

    // resident device buffers
    uint8_t* d_call = nullptr;          // the current call block
    int32_t* d_counter = nullptr;       // work-item counter of the fused kernel
    uint64_t* d_keys = nullptr;         // packed cell keys, zero when idle
    size_t keys_cap = 0;
    uint8_t* d_pyr = nullptr;           // pyramid levels 1..L-1 of every frame
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

    // one graph per (variant, levels, launch shape, CTAs per SM): every batch
    // shape replays it; shape 1 is the small-call shape (one CTA per SM at
    // most); CTAs per SM 0 = as many as fit
    cudaGraphExec_t graphs[8][vio::kMaxLevels + 1][2][vio::kMaxCtasPerSm + 1] = {};
    int occ_fused[8] = {};                 // CTAs per SM that fit, per variant
    int grid_sweep = 0;
    struct TuneChoice {
        int variant, ctas, cell;
    };
    std::unordered_map<ShapeKey, TuneChoice, ShapeHash> tuned;  // batch shape -> choice
    std::vector<vio_tuning> tune_log;      // the alternatives the last tuning run timed
    std::vector<float> tune_log_ms;
    std::unordered_map<MapKey, CUtensorMap, MapHash> map_cache;
    int pinned_variant = -1;
    int pinned_ctas = 0;
    int last_variant = 0;
    int last_ctas = 0;                     // CTAs per SM of the last launch (resolved)
    int last_cell = 0;                     // cell size of the last detection
    // levels of the most recent detection call, for vio_copy_level
    std::vector<std::array<const uint8_t*, vio::kMaxLevels>> last_lev;
    std::vector<std::array<int, vio::kMaxLevels>> last_pitch;
    std::vector<vio_dims> last_dims;
    int last_levels = 0;
    vio::TrackState track;
    vio::HostSlot hslots[vio::kHostSlots];
    int hslot_pos = 0;

    void drop_graphs() {
        for (auto& row : graphs)
            for (auto& pair : row)
                for (auto& shape : pair)
                    for (auto& g : shape)
                        if (g) {
                            cudaGraphExecDestroy(g);
                            g = nullptr;
                        }
    }
};

namespace vio {

inline vio_status fail(vio_ctx* c, vio_status s, const std::string& msg) {
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

// Grows a resident buffer to `need` bytes.  Growing waits for the device
// (the old buffer may still be in use), so buffers grow geometrically.
inline vio_status grow(vio_ctx* ctx, void** p, size_t* cap, size_t need, bool zero) {
    if (need <= *cap && *p) return VIO_OK;
    size_t want = std::max(need, *cap + *cap / 2);
    const size_t budget = ctx->cfg.mem_budget_bytes;
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

}  // namespace vio

namespace vio {
// Frees the tracker's resident buffers (vio_destroy).
void track_release(vio_ctx* ctx);
}  // namespace vio

namespace vio {
// Detects frames that live in host memory, asynchronously on s: pinned frames
// are uploaded by the pyramid kernel through their device mapping, others by
// the copy engines into the context's staging.  outs[i] may be device memory
// or the device mapping of pinned host memory; d_counts is device memory or
// nullptr.  Arguments are checked by the caller.
vio_status detect_from_host(vio_ctx* ctx, const uint8_t* const* host_frames, const vio_dims* dims, int n, int thresh,
                            int arc, int cell, int levels, int4* const* outs, int32_t* d_counts, cudaStream_t s);
// Device address of pinned host memory, else nullptr.
const void* host_device_alias(const void* host);
}  // namespace vio
