// Host runtime behind include/vio.h: argument checks, resident buffers, the
// per-call block (frame descriptors, tensor maps, tile table), CUDA-graph replay
// and the tile autotuner.
#include <cuda.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <array>
#include <chrono>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <unordered_map>
#include <vector>

#include "../../include/vio.h"
#include "vio_ctx.h"
#include "vio_kernels.cuh"
#include "vio_sweep.cuh"

using namespace vio;

namespace {

// ---------------------------------------------------------------------------
// Built variants of the fused kernel.
// ---------------------------------------------------------------------------
using DetectFn = void (*)(const uint8_t*, int32_t*, uint32_t*);
using PyrFn = void (*)(const uint8_t*);

struct Variant {
    int tw, th, radius, smem;
    DetectFn fn[3];
};

template <int TH, int R>
Variant make_variant() {
    return Variant{TileGeom<TH, R>::TW, TH, R, TileGeom<TH, R>::SMEM,
                   {fast_nms_cell_kernel<TH, 0, R>, fast_nms_cell_kernel<TH, 1, R>, fast_nms_cell_kernel<TH, 2, R>}};
}

// 3x3 NMS in three tile heights; the wider windows of radius R keep the
// score region at 64 rows.
const std::vector<Variant>& variants() {
    static const std::vector<Variant> v = {make_variant<62, 1>(), make_variant<30, 1>(), make_variant<126, 1>(),
                                           make_variant<60, 2>(), make_variant<58, 3>(), make_variant<56, 4>()};
    return v;
}

// first variant built for NMS radius r (the default tile shape of that radius)
int first_variant(int r) {
    for (int i = 0; i < (int)variants().size(); ++i)
        if (variants()[i].radius == r) return i;
    return -1;
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

constexpr int kBoxW = 144;  // TMA box width of every variant (height: th + 2 radius + 6)

// Bytes of the largest call block a context can send.
size_t call_block_cap(int max_frames) {
    size_t b = align_up(sizeof(CallHeader), 128);
    b += align_up(sizeof(FrameDesc) * max_frames, 128);
    b += align_up(sizeof(CUtensorMap) * max_frames, 128);
    b += align_up(sizeof(CUtensorMap) * max_frames * (kMaxLevels - 1), 128);
    b += align_up(sizeof(int32_t) * (max_frames * kMaxLevels + 1), 128);
    b += align_up(sizeof(int32_t) * (max_frames + 1), 128);
    b += align_up(sizeof(int32_t) * (max_frames + 1), 128);
    // sweep section and its output table
    b += align_up(sizeof(SweepInfo), 128);
    b += align_up(sizeof(int4*) * kMaxSweep * max_frames, 128);
    return b;
}

}  // namespace

namespace {

// Device address of pinned (page-locked, device-mapped) host memory, else
// nullptr (pageable memory, device memory, or an unknown pointer).
const void* device_alias(const void* host) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, host) != cudaSuccess) {
        cudaGetLastError();  // clear the error: an unknown pointer is not a failure here
        return nullptr;
    }
    return a.type == cudaMemoryTypeHost ? a.devicePointer : nullptr;
}

// Reads and clears the device status word after a synchronisation.
vio_status take_status(vio_ctx* ctx) {
    const uint32_t bits = *ctx->h_status;
    if (!bits) return VIO_OK;
    *ctx->h_status = 0;
    if (bits & kStatusTimeout) return fail(ctx, VIO_ERR_TIMEOUT, "a bounded device-side wait timed out");
    if (bits & kStatusBounds) return fail(ctx, VIO_ERR_CUDA, "a device-side index check failed (checked build)");
    return fail(ctx, VIO_ERR_CUDA, "a decoded feature lies outside its cell (corrupted cell keys)");
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
    if (ctx->map_cache.size() > 16384) ctx->map_cache.clear();
    ctx->map_cache.emplace(key, *out);
    return VIO_OK;
}

vio_status check_args(vio_ctx* ctx, const void* frames, const vio_dims* dims, int n, int thresh, int arc,
                      int cell, int levels, const void* outs, bool auto_cell = false) {
    if (!ctx) return VIO_ERR_INVALID_ARG;
    if (!frames || !dims || !outs) return fail(ctx, VIO_ERR_INVALID_ARG, "NULL frames, dims or outputs");
    if (n < 1 || n > ctx->cfg.max_frames)
        return fail(ctx, VIO_ERR_INVALID_ARG, "n_frames must be in 1..max_frames");
    if (thresh < 0 || thresh > 255) return fail(ctx, VIO_ERR_INVALID_ARG, "thresh must be in 0..255");
    if (ctx->cfg.score == VIO_SCORE_MT && thresh < 1)
        return fail(ctx, VIO_ERR_INVALID_ARG, "the MT score needs thresh >= 1");
    if (arc < 9 || arc > 16) return fail(ctx, VIO_ERR_INVALID_ARG, "arc_len must be in 9..16");
    if (!(auto_cell && cell == 0) && (cell < 32 || cell % 32 != 0))
        return fail(ctx, VIO_ERR_INVALID_ARG, "cell_size must be a positive multiple of 32");
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

ShapeKey shape_key(const vio_dims* dims, int n, int cell, int levels) {
    ShapeKey k;
    k.v.reserve(2 * n + 3);
    k.v.push_back(n);
    k.v.push_back(cell);
    k.v.push_back(levels);
    for (int i = 0; i < n; ++i) {
        k.v.push_back(dims[i].w);
        k.v.push_back(dims[i].h);
    }
    return k;
}

constexpr int kSmallDecodeCtas = 8;  // decode grid of a small call

#define VIO_CK_STATUS(call)                \
    do {                                   \
        const vio_status s_ = (call);      \
        if (s_ != VIO_OK) return s_;       \
    } while (0)

// CTAs of a fused-kernel variant that fit on one SM (sets the variant's
// dynamic shared-memory attribute the first time).
vio_status fused_occupancy(vio_ctx* ctx, int variant, int* occ) {
    if (!ctx->occ_fused[variant]) {
        const Variant& v = variants()[variant];
        int o = 0;
        VIO_CK(cudaFuncSetAttribute(v.fn[ctx->cfg.score], cudaFuncAttributeMaxDynamicSharedMemorySize, v.smem));
        VIO_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, v.fn[ctx->cfg.score], kThreads, v.smem));
        ctx->occ_fused[variant] = std::max(1, std::min(o, kMaxCtasPerSm));
    }
    *occ = ctx->occ_fused[variant];
    return VIO_OK;
}

// Enqueues pyramid -> fused detect -> decode on `s`; launch shapes depend only
// on the context and on `small` (the kernels read the batch from the call
// block and stride over whatever grid they get).  A small call (a few frames
// of VGA size: at most one detect item, two pyramid blocks per SM) launches
// one CTA per SM instead of filling every SM, which saves the start-up of CTAs
// that would find no work.
vio_status enqueue_kernels(vio_ctx* ctx, int variant, int levels, cudaStream_t s, bool pyramid = true,
                           bool small = false, int ctas = 0) {
    const Variant& v = variants()[variant];
    const int mode = ctx->cfg.score;
    const bool prof = ctx->cfg.profile != 0;
    // inside stream capture only an external record becomes a graph node
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (prof) VIO_CK(cudaStreamIsCapturing(s, &cap));
    const unsigned rec_flags = cap == cudaStreamCaptureStatusActive ? cudaEventRecordExternal : 0u;
    if (prof) VIO_CK(cudaEventRecordWithFlags(ctx->stage_ev[0], s, rec_flags));
    if (levels > 1 && pyramid) {
        pyr_fn(levels)<<<ctx->sm_count * (small ? 1 : 8), 256, 0, s>>>(ctx->d_call);
        VIO_CK(cudaGetLastError());
    }
    if (prof) VIO_CK(cudaEventRecordWithFlags(ctx->stage_ev[1], s, rec_flags));
    int occ = 0;
    VIO_CK_STATUS(fused_occupancy(ctx, variant, &occ));
    const int per_sm = ctas > 0 ? std::min(ctas, occ) : occ;
    const int grid = small ? ctx->sm_count : per_sm * ctx->sm_count;
    // the detect kernel and the decode are programmatic dependents of the
    // kernel before them: they launch while it drains and wait for it on
    // the device (griddep_wait) before reading what it wrote
    cudaLaunchAttribute pdl[1];
    pdl[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    pdl[0].val.programmaticStreamSerializationAllowed = 1;
    cudaLaunchConfig_t lc = {};
    lc.gridDim = dim3(grid);
    lc.blockDim = dim3(kThreads);
    lc.dynamicSmemBytes = v.smem;
    lc.stream = s;
    lc.attrs = pdl;
    lc.numAttrs = 1;
    VIO_CK(cudaLaunchKernelEx(&lc, v.fn[mode], (const uint8_t*)ctx->d_call, ctx->d_counter, ctx->d_status));
    if (prof) VIO_CK(cudaEventRecordWithFlags(ctx->stage_ev[2], s, rec_flags));
    cudaLaunchConfig_t ld = lc;
    ld.gridDim = dim3(small ? kSmallDecodeCtas : ctx->sm_count * 4);
    ld.blockDim = dim3(256);
    ld.dynamicSmemBytes = 0;
    VIO_CK(cudaLaunchKernelEx(&ld, decode_kernel, (const uint8_t*)ctx->d_call, ctx->d_counter));
    if (prof) VIO_CK(cudaEventRecordWithFlags(ctx->stage_ev[3], s, rec_flags));
    return VIO_OK;
}

// Graph slot `levels` holds pyramid -> detect -> decode; slot 0 holds
// detect -> decode alone (the pyramid is already in place).
vio_status get_graph(vio_ctx* ctx, int variant, int levels, bool pyramid, bool small, int ctas,
                     cudaGraphExec_t* out) {
    cudaGraphExec_t& g = ctx->graphs[variant][pyramid ? levels : 0][small ? 1 : 0][ctas];
    if (!g) {
        // the launch attributes and the occupancy are set up outside the capture
        int occ = 0;
        VIO_CK_STATUS(fused_occupancy(ctx, variant, &occ));
        (void)occ;
        cudaGraph_t graph = nullptr;
        VIO_CK(cudaStreamBeginCapture(ctx->capture_stream, cudaStreamCaptureModeThreadLocal));
        vio_status es = enqueue_kernels(ctx, variant, levels, ctx->capture_stream, pyramid, small, ctas);
        cudaError_t ce = cudaStreamEndCapture(ctx->capture_stream, &graph);
        if (es != VIO_OK) return es;
        VIO_CK(ce);
        VIO_CK(cudaGraphInstantiate(&g, graph, 0));
        cudaGraphDestroy(graph);
    }
    *out = g;
    return VIO_OK;
}

// Lays the batch out in the resident arenas, fills the call block, uploads
// it and launches the three kernels on `s`.
// Frames that the pyramid kernel uploads itself: src[i] non-null is the
// device mapping of frame i in host memory (row pitch pitch[i]); lev0[i] is
// then the device copy that kernel writes.
struct Upload {
    const uint8_t* const* src = nullptr;
    const int* pitch = nullptr;
};

// Up to kMaxSweep settings detected by one fused sweep launch (ordered by
// arc length); outs[s * n + i] receives frame i of setting s.
struct SweepSpec {
    int n_set = 0;
    int thresh[kMaxSweep] = {};
    int arc[kMaxSweep] = {};
    int4* const* outs = nullptr;
    int32_t* counts[kMaxSweep] = {};
};

constexpr int kSweepTH = 62;  // the sweep kernel's tile height (variant 0's geometry)

// Upload of host frames.  Frames that lie one after another in host memory
// (16-byte aligned start and pitch, rows padded by at most kSpanPad bytes,
// at most kSpanGap bytes between frames) form a span that one
// cudaMemcpyAsync copies, and keep their host pitch on the device: each copy
// costs about 2 us of copy-engine time on top of its bytes, a third of the
// upload time of 64 frames of 0.3 to 2 Mpixel copied one by one.  Other
// frames are copied alone (2-D, rows padded to 16 bytes).
struct UploadPlan {
    struct Copy {
        size_t dst;              // offset in the device buffer
        const uint8_t* src;
        size_t bytes;            // a 1-D copy of a span when w == 0
        int w, h, spitch, dpitch;  // a 2-D copy otherwise
    };
    std::vector<size_t> off;     // per frame: device offset of its first pixel
    std::vector<int> pitch;      // per frame: device row pitch
    std::vector<int> span_len;   // per frame: frames in its span
    std::vector<Copy> copies;
    size_t bytes = 0;            // device bytes the plan needs
};
constexpr size_t kSpanGap = 4096;
constexpr int kSpanPad = 256;

UploadPlan plan_upload(const uint8_t* const* host, const vio_dims* dims, int n) {
    UploadPlan p;
    p.off.resize(n);
    p.pitch.resize(n);
    p.span_len.resize(n);
    const auto spannable = [&](int j) {
        return ((uintptr_t)host[j] & 15) == 0 && (dims[j].pitch & 15) == 0 &&
               dims[j].pitch <= (int)align_up(dims[j].w, 16) + kSpanPad;
    };
    const auto end_of = [&](int j) { return host[j] + (size_t)dims[j].pitch * (dims[j].h - 1) + dims[j].w; };
    for (int i = 0; i < n;) {
        if (spannable(i)) {
            const uint8_t* end = end_of(i);
            int j = i + 1;
            while (j < n && spannable(j) && host[j] >= end && (size_t)(host[j] - end) <= kSpanGap) {
                end = end_of(j);
                ++j;
            }
            for (int k = i; k < j; ++k) {
                p.off[k] = p.bytes + (size_t)(host[k] - host[i]);
                p.pitch[k] = dims[k].pitch;
                p.span_len[k] = j - i;
            }
            p.copies.push_back({p.bytes, host[i], (size_t)(end - host[i]), 0, 0, 0, 0});
            p.bytes = align_up(p.bytes + (size_t)(end - host[i]), 256);
            i = j;
        } else {
            const int pitch = (int)align_up(dims[i].w, 16);
            p.off[i] = p.bytes;
            p.pitch[i] = pitch;
            p.span_len[i] = 1;
            p.copies.push_back({p.bytes, host[i], 0, dims[i].w, dims[i].h, dims[i].pitch, pitch});
            p.bytes = align_up(p.bytes + (size_t)pitch * dims[i].h, 256);
            ++i;
        }
    }
    return p;
}

// Enqueues the copies of a plan into the device buffer dst, leaving out copy
// c where (*skip)[c].
vio_status enqueue_upload(vio_ctx* ctx, const UploadPlan& p, uint8_t* dst, cudaStream_t s,
                          const std::vector<bool>* skip = nullptr) {
    for (size_t c = 0; c < p.copies.size(); ++c) {
        const UploadPlan::Copy& cp = p.copies[c];
        if (skip && (*skip)[c]) continue;
        if (cp.w == 0)
            VIO_CK(cudaMemcpyAsync(dst + cp.dst, cp.src, cp.bytes, cudaMemcpyHostToDevice, s));
        else
            VIO_CK(cudaMemcpy2DAsync(dst + cp.dst, cp.dpitch, cp.src, cp.spitch, cp.w, cp.h, cudaMemcpyHostToDevice,
                                     s));
    }
    return VIO_OK;
}

constexpr int kZeroCopyMin = 4;  // lone pinned frames per call read through their device mapping

// Pyramid (when asked), fused sweep and sweep decode, launched directly.
vio_status enqueue_sweep(vio_ctx* ctx, int levels, cudaStream_t s, bool pyramid, const SweepInfo* d_sw) {
    const bool prof = ctx->cfg.profile != 0;
    if (prof) VIO_CK(cudaEventRecord(ctx->stage_ev[0], s));
    if (levels > 1 && pyramid) {
        pyr_fn(levels)<<<ctx->sm_count * 8, 256, 0, s>>>(ctx->d_call);
        VIO_CK(cudaGetLastError());
    }
    if (prof) VIO_CK(cudaEventRecord(ctx->stage_ev[1], s));
    const int smem = SweepGeom<kSweepTH>::SMEM;
    if (!ctx->grid_sweep) {
        int occ = 0;
        VIO_CK(cudaFuncSetAttribute(fast_sweep_kernel<kSweepTH>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
        VIO_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fast_sweep_kernel<kSweepTH>, kThreads, smem));
        ctx->grid_sweep = std::max(1, occ) * ctx->sm_count;
    }
    fast_sweep_kernel<kSweepTH><<<ctx->grid_sweep, kThreads, smem, s>>>(ctx->d_call, d_sw, ctx->d_counter,
                                                                      ctx->d_status);
    VIO_CK(cudaGetLastError());
    if (prof) VIO_CK(cudaEventRecord(ctx->stage_ev[2], s));
    sweep_decode_kernel<<<ctx->sm_count * 4, 256, 0, s>>>(ctx->d_call, d_sw, ctx->d_counter);
    VIO_CK(cudaGetLastError());
    if (prof) VIO_CK(cudaEventRecord(ctx->stage_ev[3], s));
    return VIO_OK;
}

vio_status launch(vio_ctx* ctx, int variant, const uint8_t* const* lev0, const int* pitch0, const vio_dims* dims,
                  int n, int thresh, int arc, int cell, int levels, int4* const* outs, int32_t* counts,
                  cudaStream_t s, bool pyramid = true, Upload up = {}, const SweepSpec* sweep = nullptr,
                  int ctas = 0) {
    const Variant& v = variants()[variant];
    // arena layout
    size_t koff = 0, poff = 0;
    std::vector<size_t> key_off(n);
    std::vector<std::array<size_t, kMaxLevels>> lev_off(n);
    std::vector<std::array<int, kMaxLevels>> lev_pitch(n);
    for (int i = 0; i < n; ++i) {
        key_off[i] = koff;
        koff += align_up(vio_num_cells(dims[i].w, dims[i].h, cell), 16);
        for (int k = 1; k < levels; ++k) {
            const int wk = dims[i].w >> k, hk = dims[i].h >> k;
            lev_pitch[i][k] = (int)align_up(wk, 128);
            lev_off[i][k] = poff;
            poff += align_up((size_t)lev_pitch[i][k] * hk, 256);
        }
    }
    vio_status st;
    const void* keys0 = ctx->d_keys;
    const void* pyr0 = ctx->d_pyr;
    const int n_set = sweep ? sweep->n_set : 1;
    if ((st = grow(ctx, (void**)&ctx->d_keys, &ctx->keys_cap, koff * 8 * n_set, true)) != VIO_OK) return st;
    if ((st = grow(ctx, (void**)&ctx->d_pyr, &ctx->pyr_cap, std::max<size_t>(poff, 256), false)) != VIO_OK) return st;
    if (keys0 != ctx->d_keys || pyr0 != ctx->d_pyr) ctx->map_cache.clear();

    // order against work of this context on another stream
    if (ctx->have_last && ctx->last_stream != s) VIO_CK(cudaStreamWaitEvent(s, ctx->last_ev, 0));
    const int slot = ctx->ring_pos;
    ctx->ring_pos = (ctx->ring_pos + 1) % ctx->ring;
    VIO_CK(cudaEventSynchronize(ctx->ring_ev[slot]));
    uint8_t* st_base = ctx->h_stage + (size_t)slot * ctx->call_cap;

    // call block sections
    size_t off = align_up(sizeof(CallHeader), 128);
    const size_t off_fds = off;
    off += align_up(sizeof(FrameDesc) * n, 128);
    const size_t off_maps0 = off;
    off += align_up(sizeof(CUtensorMap) * n, 128);
    const size_t off_mapsk = off;
    off += align_up(sizeof(CUtensorMap) * n * (kMaxLevels - 1), 128);
    const size_t off_tiles = off;
    off += align_up(sizeof(int32_t) * (n * levels + 1), 128);
    const size_t off_blocks = off;
    off += align_up(sizeof(int32_t) * (n + 1), 128);
    const size_t off_cells = off;
    off += align_up(sizeof(int32_t) * (n + 1), 128);
    const size_t off_sweep = off;
    const size_t off_souts = off + align_up(sizeof(SweepInfo), 128);
    if (sweep) off = off_souts + align_up(sizeof(int4*) * n_set * n, 128);
    const size_t bytes = off;

    CallHeader* hdr = reinterpret_cast<CallHeader*>(st_base);
    FrameDesc* fds = reinterpret_cast<FrameDesc*>(st_base + off_fds);
    CUtensorMap* maps0 = reinterpret_cast<CUtensorMap*>(st_base + off_maps0);
    CUtensorMap* mapsk = reinterpret_cast<CUtensorMap*>(st_base + off_mapsk);
    int32_t* tiles = reinterpret_cast<int32_t*>(st_base + off_tiles);
    int32_t* blocks = reinterpret_cast<int32_t*>(st_base + off_blocks);
    int32_t* cells = reinterpret_cast<int32_t*>(st_base + off_cells);
    std::memset(hdr, 0, sizeof(CallHeader));
    hdr->thresh = thresh;
    hdr->arc = arc;
    hdr->n_frames = n;
    hdr->levels = levels;
    hdr->cell = cell;
    hdr->tile_h = v.th;
    hdr->counts = counts;
    hdr->off_fds = (uint32_t)off_fds;
    hdr->off_maps0 = (uint32_t)off_maps0;
    hdr->off_mapsk = (uint32_t)off_mapsk;
    hdr->off_tiles = (uint32_t)off_tiles;
    hdr->off_blocks = (uint32_t)off_blocks;
    hdr->off_cells = (uint32_t)off_cells;
    hdr->status = ctx->d_status;
    for (int k = 0; k < levels; ++k) {
        const uint64_t d = (uint64_t)(cell >> k);  // >= 2: cell is a multiple of 32, k <= 4
        hdr->cell_magic[k] = (uint32_t)(((1ull << 32) + d - 1) / d);
    }
    const int B = 1 << (levels - 1);
    blocks[0] = 0;
    cells[0] = 0;
    for (int i = 0; i < n; ++i) {
        FrameDesc& f = fds[i];
        std::memset(&f, 0, sizeof(FrameDesc));
        f.w = dims[i].w;
        f.h = dims[i].h;
        f.gw = (f.w + cell - 1) / cell;
        f.gh = (f.h + cell - 1) / cell;
        // pyramid CTAs cover 512 columns x 8B rows of level 0
        f.pyr_bx = (f.w + 511) / 512;
        f.pyr_magic = (uint32_t)(((1ull << 31) + f.pyr_bx - 1) / f.pyr_bx);
        const int pyr_by = (f.h + 8 * B - 1) / (8 * B);
        blocks[i + 1] = blocks[i] + (levels > 1 ? f.pyr_bx * pyr_by : 0);
        cells[i + 1] = cells[i] + f.gw * f.gh;
        f.keys = ctx->d_keys + key_off[i];
        f.out = outs[i];
        f.lev[0] = const_cast<uint8_t*>(lev0[i]);
        f.pitch[0] = pitch0[i];
        if (up.src && up.src[i]) {
            f.src0 = up.src[i];
            f.src0_pitch = up.pitch[i];
        }
        if ((st = encode_map(ctx, &maps0[i], lev0[i], f.w, f.h, pitch0[i], kBoxW, v.th + 2 * v.radius + 6)) != VIO_OK)
            return st;
        for (int k = 1; k < levels; ++k) {
            f.lev[k] = ctx->d_pyr + lev_off[i][k];
            f.pitch[k] = lev_pitch[i][k];
            if ((st = encode_map(ctx, &mapsk[(size_t)i * (kMaxLevels - 1) + k - 1], f.lev[k], f.w >> k, f.h >> k,
                                 f.pitch[k], kBoxW, v.th + 2 * v.radius + 6)) != VIO_OK)
                return st;
        }
    }
    ctx->last_levels = levels;
    ctx->last_dims.assign(dims, dims + n);
    ctx->last_lev.assign(n, {});
    ctx->last_pitch.assign(n, {});
    for (int i = 0; i < n; ++i)
        for (int k = 0; k < levels; ++k) {
            ctx->last_lev[i][k] = fds[i].lev[k];
            ctx->last_pitch[i][k] = fds[i].pitch[k];
        }
    // tiles: coarsest level first, entry (L-1-k)*n + f
    int acc = 0;
    for (int kk = 0; kk < levels; ++kk) {
        const int k = levels - 1 - kk;
        for (int i = 0; i < n; ++i) {
            tiles[kk * n + i] = acc;
            const int wk = dims[i].w >> k, hk = dims[i].h >> k;
            acc += ((wk + v.tw - 1) / v.tw) * ((hk + v.th - 1) / v.th);
        }
    }
    tiles[n * levels] = acc;
    hdr->n_items = acc;
    hdr->n_pyr_blocks = blocks[n];
    hdr->n_cells = cells[n];
    if (sweep) {
        SweepInfo* si = reinterpret_cast<SweepInfo*>(st_base + off_sweep);
        int4** so = reinterpret_cast<int4**>(st_base + off_souts);
        std::memset(si, 0, sizeof(SweepInfo));
        si->n_set = n_set;
        for (int j = 0; j < n_set; ++j) {
            si->thresh[j] = sweep->thresh[j];
            si->arc[j] = sweep->arc[j];
            si->counts[j] = sweep->counts[j];
        }
        si->set_stride = (int64_t)koff;
        si->outs = reinterpret_cast<int4* const*>(ctx->d_call + off_souts);
        for (int j = 0; j < n_set * n; ++j) so[j] = sweep->outs[j];
    }

    const bool small = acc <= ctx->sm_count && blocks[n] <= 2 * ctx->sm_count &&
                       cells[n] <= kSmallDecodeCtas * 256 * 4;

    VIO_CK(cudaMemcpyAsync(ctx->d_call, st_base, bytes, cudaMemcpyHostToDevice, s));
    VIO_CK(cudaEventRecord(ctx->ring_ev[slot], s));
    if (sweep) {
        if ((st = enqueue_sweep(ctx, levels, s, pyramid,
                                reinterpret_cast<const SweepInfo*>(ctx->d_call + off_sweep))) != VIO_OK)
            return st;
    } else if (ctx->cfg.use_graphs) {
        cudaGraphExec_t g = nullptr;
        if ((st = get_graph(ctx, variant, levels, pyramid, small, ctas, &g)) != VIO_OK) return st;
        VIO_CK(cudaGraphLaunch(g, s));
    } else if ((st = enqueue_kernels(ctx, variant, levels, s, pyramid, small, ctas)) != VIO_OK) {
        return st;
    }
    VIO_CK(cudaEventRecord(ctx->last_ev, s));
    ctx->last_stream = s;
    ctx->have_last = true;
    int occ = 1;
    if (!sweep) VIO_CK_STATUS(fused_occupancy(ctx, variant, &occ));
    // a sweep's launch shape is fixed: the CTAs per SM its registers and
    // shared memory allow
    ctx->last_ctas = sweep ? ctx->grid_sweep / ctx->sm_count : small ? 1 : (ctas > 0 ? std::min(ctas, occ) : occ);
    ctx->last_cell = cell;
    return VIO_OK;
}

// Times every combination of the context radius's tile variants, 2 to 4
// CTAs per SM (as far as they fit) and the candidate cell sizes (32 and 64
// when the call gave cell 0, else the call's) on the call's own batch: two
// untimed launches, then 5 timed by CUDA events on the call's stream.  The
// fastest is kept for the batch shape; every alternative and its time go to
// the tuning log.
vio_status autotune(vio_ctx* ctx, const ShapeKey& key, const uint8_t* const* lev0, const int* pitch0,
                    const vio_dims* dims, int n, int thresh, int arc, int cell, int levels, int4* const* outs,
                    int32_t* counts, cudaStream_t s, Upload up = {}) {
    cudaEvent_t e0, e1;
    VIO_CK(cudaEventCreate(&e0));
    VIO_CK(cudaEventCreate(&e1));
    float best = 1e30f;
    vio_ctx::TuneChoice choice{first_variant(ctx->cfg.nms_radius), 0, cell ? cell : 32};
    ctx->tune_log.clear();
    ctx->tune_log_ms.clear();
    vio_status st = VIO_OK;
    const int cells[2] = {cell ? cell : 32, 64};
    const int n_cells = cell ? 1 : 2;
    for (int vi = 0; vi < (int)variants().size() && st == VIO_OK; ++vi) {
        if (variants()[vi].radius != ctx->cfg.nms_radius) continue;
        int occ = 1;
        if ((st = fused_occupancy(ctx, vi, &occ)) != VIO_OK) break;
        for (int ctas = std::min(2, occ); ctas <= occ && st == VIO_OK; ++ctas) {
            for (int ci = 0; ci < n_cells && st == VIO_OK; ++ci) {
                const int c = cells[ci];
                for (int r = 0; r < 2 && st == VIO_OK; ++r)
                    st = launch(ctx, vi, lev0, pitch0, dims, n, thresh, arc, c, levels, outs, counts, s, true, up,
                                nullptr, ctas);
                if (st != VIO_OK) break;
                VIO_CK(cudaEventRecord(e0, s));
                const int reps = 5;
                for (int r = 0; r < reps && st == VIO_OK; ++r)
                    st = launch(ctx, vi, lev0, pitch0, dims, n, thresh, arc, c, levels, outs, counts, s, true, up,
                                nullptr, ctas);
                VIO_CK(cudaEventRecord(e1, s));
                VIO_CK(cudaEventSynchronize(e1));
                float ms = 0;
                VIO_CK(cudaEventElapsedTime(&ms, e0, e1));
                ms /= reps;
                vio_tuning t{variants()[vi].tw, variants()[vi].th, ctas, vi, variants()[vi].radius, c};
                ctx->tune_log.push_back(t);
                ctx->tune_log_ms.push_back(ms);
                if (ms < best) {
                    best = ms;
                    choice = {vi, ctas, c};
                }
            }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st == VIO_OK) ctx->tuned[key] = choice;
    return st;
}

// Resolves the launch configuration (pinned, tuned or default) and the cell
// size (cell 0: tuned, else 32) and launches.
vio_status detect_impl(vio_ctx* ctx, const uint8_t* const* lev0, const int* pitch0, const vio_dims* dims, int n,
                       int thresh, int arc, int cell, int levels, int4* const* outs, int32_t* counts,
                       cudaStream_t s, Upload up = {}) {
    int vi = ctx->pinned_variant;
    int ctas = ctx->pinned_ctas;
    int c = cell ? cell : 32;
    if (vi < 0) {
        vi = first_variant(ctx->cfg.nms_radius);
        if (ctx->cfg.autotune) {
            const ShapeKey key = shape_key(dims, n, cell, levels);
            auto it = ctx->tuned.find(key);
            if (it == ctx->tuned.end()) {
                vio_status st = autotune(ctx, key, lev0, pitch0, dims, n, thresh, arc, cell, levels, outs, counts, s, up);
                if (st != VIO_OK) return st;
                it = ctx->tuned.find(key);
            }
            vi = it->second.variant;
            ctas = it->second.ctas;
            c = it->second.cell;
        }
    }
    ctx->last_variant = vi;
    return launch(ctx, vi, lev0, pitch0, dims, n, thresh, arc, c, levels, outs, counts, s, true, up, nullptr, ctas);
}

// One warp waits on a barrier that nothing completes; the bounded wait gives
// up after limit_ns and records the timeout (vio_selftest_timeout).
__global__ void selftest_wait_kernel(uint32_t* status, uint64_t limit_ns) {
    __shared__ uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        fence_barrier_init();
    }
    __syncwarp();
    if (threadIdx.x == 0 && !mbar_wait_bounded(&bar, 0, limit_ns)) atomicOr(status, kStatusTimeout);
}

}  // namespace

namespace vio {

vio_status detect_from_host(vio_ctx* ctx, const uint8_t* const* host_frames, const vio_dims* dims, int n, int thresh,
                            int arc, int cell, int levels, int4* const* outs, int32_t* d_counts, cudaStream_t s) {
    // Frames alone in pinned host memory, when a call has at least
    // kZeroCopyMin of them, are read by the pyramid kernel through their
    // device mapping (it writes the device copy of level 0 as it goes): their
    // upload overlaps the pyramid and costs no copy each.  A call with fewer
    // copies them (the copy engine's latency is lower for a frame or two).
    // Spans of frames that lie one after another take one copy-engine copy
    // each; so does anything else.
    const UploadPlan plan = plan_upload(host_frames, dims, n);
    vio_status st;
    if ((st = grow(ctx, (void**)&ctx->d_in, &ctx->in_cap, std::max<size_t>(plan.bytes, 256), false)) != VIO_OK)
        return st;
    std::vector<const uint8_t*> lev0(n), src0(n, nullptr);
    std::vector<int> src_pitch(n, 0);
    std::vector<bool> skip(plan.copies.size(), false);
    int n_mapped = 0;
    for (int i = 0, c = 0; i < n; c++) {
        const int len = plan.span_len[i];
        const uint8_t* mapped = len == 1 ? static_cast<const uint8_t*>(device_alias(host_frames[i])) : nullptr;
        if (levels > 1 && mapped && ((uintptr_t)mapped & 15) == 0 && (dims[i].pitch & 15) == 0) {
            src0[i] = mapped;
            src_pitch[i] = dims[i].pitch;
            skip[c] = true;
            ++n_mapped;
        }
        i += len;
    }
    const bool any_up = n_mapped >= kZeroCopyMin;
    if (!any_up) std::fill(skip.begin(), skip.end(), false);
    for (int i = 0; i < n; ++i) lev0[i] = ctx->d_in + plan.off[i];
    if ((st = enqueue_upload(ctx, plan, ctx->d_in, s, &skip)) != VIO_OK) return st;
    Upload up;
    if (any_up) {
        up.src = src0.data();
        up.pitch = src_pitch.data();
    }
    return detect_impl(ctx, lev0.data(), plan.pitch.data(), dims, n, thresh, arc, cell, levels, outs, d_counts, s, up);
}

const void* host_device_alias(const void* host) { return device_alias(host); }

}  // namespace vio

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
    cfg->nms_radius = 1;
}

vio_status vio_get_config(const vio_ctx* ctx, vio_config* out) {
    if (!ctx || !out) return VIO_ERR_INVALID_ARG;
    *out = ctx->cfg;
    return VIO_OK;
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

vio_status vio_copy_level(vio_ctx* ctx, int frame, int level, uint8_t* dst, int dst_pitch, vio_stream stream) {
    if (!ctx) return VIO_ERR_INVALID_ARG;
    if (ctx->last_levels < 1 || frame < 0 || frame >= (int)ctx->last_dims.size() || level < 0 ||
        level >= ctx->last_levels || !dst)
        return fail(ctx, VIO_ERR_INVALID_ARG, "no such level of the most recent detection");
    const vio_dims& d = ctx->last_dims[frame];
    const int w = d.w >> level, h = d.h >> level;
    if (dst_pitch < w) return fail(ctx, VIO_ERR_INVALID_ARG, "dst_pitch < level width");
    VIO_CK(cudaSetDevice(ctx->cfg.device));
    VIO_CK(cudaMemcpy2DAsync(dst, (size_t)dst_pitch, ctx->last_lev[frame][level], (size_t)ctx->last_pitch[frame][level],
                             (size_t)w, (size_t)h, cudaMemcpyDefault, reinterpret_cast<cudaStream_t>(stream)));
    return VIO_OK;
}

int vio_num_variants(void) { return (int)variants().size(); }

vio_status vio_variant(int i, vio_tuning* out) {
    if (!out || i < 0 || i >= (int)variants().size()) return VIO_ERR_INVALID_ARG;
    out->tile_w = variants()[i].tw;
    out->tile_h = variants()[i].th;
    out->cta_per_sm = 0;
    out->variant = i;
    out->nms_radius = variants()[i].radius;
    out->cell_size = 0;
    return VIO_OK;
}

int vio_autotune_log(const vio_ctx* ctx, vio_tuning* configs, float* ms, int cap) {
    if (!ctx) return -1;
    const int n = (int)ctx->tune_log.size();
    for (int i = 0; i < n && i < cap; ++i) {
        if (configs) configs[i] = ctx->tune_log[i];
        if (ms) ms[i] = ctx->tune_log_ms[i];
    }
    return n;
}

vio_status vio_create(vio_ctx** out, const vio_config* cfg_in) {
    if (!out) return VIO_ERR_INVALID_ARG;
    *out = nullptr;
    vio_config cfg;
    if (cfg_in) cfg = *cfg_in; else vio_config_default(&cfg);
    if (cfg.max_frames < 1 || cfg.max_frames > 1024 || cfg.score < 0 || cfg.score > 2 || cfg.device < 0 ||
        first_variant(cfg.nms_radius) < 0)
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
    ctx->call_cap = call_block_cap(cfg.max_frames);
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
    if (cudaMalloc(&ctx->d_call, ctx->call_cap) != cudaSuccess) return cleanup(VIO_ERR_OOM);
    if (cudaMalloc(&ctx->d_counter, sizeof(int32_t) * 4) != cudaSuccess) return cleanup(VIO_ERR_OOM);
    if (cudaMemset(ctx->d_counter, 0, sizeof(int32_t) * 4) != cudaSuccess) return cleanup(VIO_ERR_CUDA);
    if (cudaHostAlloc(&ctx->h_status, 64, cudaHostAllocMapped) != cudaSuccess) return cleanup(VIO_ERR_OOM);
    *ctx->h_status = 0;
    if (cudaHostGetDevicePointer((void**)&ctx->d_status, ctx->h_status, 0) != cudaSuccess)
        return cleanup(VIO_ERR_CUDA);
    if (cudaHostAlloc(&ctx->h_stage, ctx->call_cap * ctx->ring, cudaHostAllocDefault) != cudaSuccess)
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
    ctx->bytes_in_use = ctx->call_cap;
    *out = ctx;
    return VIO_OK;
}

int vio_device(const vio_ctx* ctx) { return ctx ? ctx->cfg.device : -1; }

vio_status vio_destroy(vio_ctx* ctx) {
    if (!ctx) return VIO_OK;
    vio_serve_stop(ctx);  // no-op unless serving
    cudaSetDevice(ctx->cfg.device);
    cudaDeviceSynchronize();
    ctx->drop_graphs();
    track_release(ctx);
    for (auto& hs : ctx->hslots) {
        cudaFree(hs.d_in);
        cudaFree(hs.d_counts);
        if (hs.done) cudaEventDestroy(hs.done);
    }
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
    NvtxRange nvtx("vio_detect");
    vio_status st = check_args(ctx, frames, dims, n, thresh, arc, cell, levels, out_cells, true);
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

vio_status vio_detect_sweep(vio_ctx* ctx, const uint8_t* const* frames, const vio_dims* dims, int n,
                            const int* thresholds, const int* arc_lens, int n_params, int cell, int levels,
                            vio_feature* const* out_cells, int32_t* out_counts, vio_stream stream) {
    NvtxRange nvtx("vio_detect_sweep");
    if (!ctx) return VIO_ERR_INVALID_ARG;
    if (!thresholds || !arc_lens || n_params < 1 || n_params > 64)
        return fail(ctx, VIO_ERR_INVALID_ARG, "n_params must be in 1..64 with thresholds and arc lengths");
    vio_status st;
    for (int p = 0; p < n_params; ++p)
        if ((st = check_args(ctx, frames, dims, n, thresholds[p], arc_lens[p], cell, levels, out_cells)) != VIO_OK)
            return st;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    VIO_CK(cudaSetDevice(ctx->cfg.device));
    for (int i = 0; i < n_params * n; ++i)
        if (!out_cells[i]) return fail(ctx, VIO_ERR_INVALID_ARG, "NULL output pointer");
    for (int i = 0; i < n; ++i)
        if (!frames[i]) return fail(ctx, VIO_ERR_INVALID_ARG, "NULL frame pointer");
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
    int vi = ctx->pinned_variant >= 0 ? ctx->pinned_variant : first_variant(ctx->cfg.nms_radius);
    if (ctx->pinned_variant < 0 && ctx->cfg.autotune) {
        const ShapeKey key = shape_key(dims, n, cell, levels);
        if (!ctx->tuned.count(key)) {
            std::vector<int4*> outs0(n);
            for (int i = 0; i < n; ++i) outs0[i] = reinterpret_cast<int4*>(out_cells[i]);
            if ((st = autotune(ctx, key, lev0.data(), pitch0.data(), dims, n, thresholds[0], arc_lens[0], cell,
                               levels, outs0.data(), out_counts, s)) != VIO_OK)
                return st;
        }
        vi = ctx->tuned[key].variant;
    }
    ctx->last_variant = vi;
    if (ctx->cfg.score == VIO_SCORE_SAD_B && ctx->cfg.nms_radius == 1 && n_params > 1) {
        // fused sweep: settings grouped by threshold, up to kMaxSweep per
        // launch (the coarse test runs at a group's lowest threshold), each
        // group ordered by arc length so that settings of one arc length
        // share the kernel's window minima; the pyramid is built by the first
        // launch
        std::vector<int> order(n_params);
        for (int p = 0; p < n_params; ++p) order[p] = p;
        std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return thresholds[a] < thresholds[b]; });
        for (int g0 = 0; g0 < n_params; g0 += kMaxSweep)
            std::stable_sort(order.begin() + g0, order.begin() + std::min(n_params, g0 + kMaxSweep),
                             [&](int a, int b) { return arc_lens[a] < arc_lens[b]; });
        std::vector<int4*> outs((size_t)kMaxSweep * n);
        // the tile table and tensor-map boxes of the sweep kernel's geometry
        int v0 = first_variant(1);
        for (int i = 0; i < (int)variants().size(); ++i)
            if (variants()[i].radius == 1 && variants()[i].th == kSweepTH) v0 = i;
        for (int g0 = 0; g0 < n_params; g0 += kMaxSweep) {
            SweepSpec sp;
            sp.n_set = std::min(kMaxSweep, n_params - g0);
            for (int j = 0; j < sp.n_set; ++j) {
                const int p = order[g0 + j];
                sp.thresh[j] = thresholds[p];
                sp.arc[j] = arc_lens[p];
                sp.counts[j] = out_counts ? out_counts + (size_t)p * n : nullptr;
                for (int i = 0; i < n; ++i) outs[(size_t)j * n + i] = reinterpret_cast<int4*>(out_cells[(size_t)p * n + i]);
            }
            sp.outs = outs.data();
            if ((st = launch(ctx, v0, lev0.data(), pitch0.data(), dims, n, sp.thresh[0], sp.arc[0], cell, levels,
                             outs.data(), nullptr, s, g0 == 0, {}, &sp)) != VIO_OK)
                return st;
        }
        return VIO_OK;
    }
    // the pyramid is built by the first detection and read by all of them
    std::vector<int4*> outs(n);
    for (int p = 0; p < n_params; ++p) {
        for (int i = 0; i < n; ++i) outs[i] = reinterpret_cast<int4*>(out_cells[(size_t)p * n + i]);
        if ((st = launch(ctx, vi, lev0.data(), pitch0.data(), dims, n, thresholds[p], arc_lens[p], cell, levels,
                         outs.data(), out_counts ? out_counts + (size_t)p * n : nullptr, s, p == 0)) != VIO_OK)
            return st;
    }
    return VIO_OK;
}

vio_status vio_detect_host(vio_ctx* ctx, const uint8_t* const* host_frames, const vio_dims* dims, int n, int thresh,
                           int arc, int cell, int levels, vio_feature* const* host_cells, int32_t* host_counts,
                           vio_stream stream) {
    NvtxRange nvtx("vio_detect_host");
    vio_status st = check_args(ctx, host_frames, dims, n, thresh, arc, cell, levels, host_cells);
    if (st != VIO_OK) return st;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    VIO_CK(cudaSetDevice(ctx->cfg.device));
    for (int i = 0; i < n; ++i)
        if (!host_frames[i] || !host_cells[i]) return fail(ctx, VIO_ERR_INVALID_ARG, "NULL frame or output pointer");
    size_t ncell_total = 0;
    std::vector<size_t> coff(n);
    for (int i = 0; i < n; ++i) {
        coff[i] = ncell_total;
        ncell_total += vio_num_cells(dims[i].w, dims[i].h, cell);
    }
    const size_t cell_bytes = ncell_total * sizeof(int4) + align_up(sizeof(int32_t) * n, 16);
    if ((st = grow(ctx, (void**)&ctx->d_cells, &ctx->cells_cap, cell_bytes, false)) != VIO_OK) return st;
    if (ctx->h_out_cap < cell_bytes) {
        if (ctx->h_out) cudaFreeHost(ctx->h_out);
        ctx->h_out = nullptr;
        ctx->h_out_cap = 0;
        VIO_CK(cudaHostAlloc(&ctx->h_out, cell_bytes, cudaHostAllocDefault));
        ctx->h_out_cap = cell_bytes;
    }
    // records go straight into pinned output buffers; others come back
    // through the context's staging
    std::vector<int4*> outs(n);
    std::vector<bool> direct_out(n, false);
    bool all_direct = true;
    for (int i = 0; i < n; ++i) {
        int4* out_mapped = static_cast<int4*>(const_cast<void*>(device_alias(host_cells[i])));
        direct_out[i] = out_mapped && ((uintptr_t)out_mapped & 15) == 0;
        all_direct &= direct_out[i];
        outs[i] = direct_out[i] ? out_mapped : ctx->d_cells + coff[i];
    }
    int32_t* d_counts = reinterpret_cast<int32_t*>(ctx->d_cells + ncell_total);
    if ((st = vio::detect_from_host(ctx, host_frames, dims, n, thresh, arc, cell, levels, outs.data(), d_counts, s)) !=
        VIO_OK)
        return st;
    if (all_direct)
        VIO_CK(cudaMemcpyAsync(ctx->h_out + ncell_total * sizeof(int4), d_counts, sizeof(int32_t) * n,
                               cudaMemcpyDeviceToHost, s));
    else
        VIO_CK(cudaMemcpyAsync(ctx->h_out, ctx->d_cells, cell_bytes, cudaMemcpyDeviceToHost, s));
    VIO_CK(cudaStreamSynchronize(s));
    if ((st = take_status(ctx)) != VIO_OK) return st;
    const int4* rec = reinterpret_cast<const int4*>(ctx->h_out);
    for (int i = 0; i < n; ++i)
        if (!direct_out[i])
            std::memcpy(host_cells[i], rec + coff[i], vio_num_cells(dims[i].w, dims[i].h, cell) * sizeof(int4));
    if (host_counts)
        std::memcpy(host_counts, ctx->h_out + ncell_total * sizeof(int4), sizeof(int32_t) * n);
    return VIO_OK;
}

vio_status vio_detect_host_async(vio_ctx* ctx, const uint8_t* const* host_frames, const vio_dims* dims, int n,
                                 int thresh, int arc, int cell, int levels, vio_feature* const* host_cells,
                                 int32_t* host_counts, vio_stream stream) {
    NvtxRange nvtx("vio_detect_host_async");
    vio_status st = check_args(ctx, host_frames, dims, n, thresh, arc, cell, levels, host_cells);
    if (st != VIO_OK) return st;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    VIO_CK(cudaSetDevice(ctx->cfg.device));
    std::vector<int4*> outs(n);
    for (int i = 0; i < n; ++i) {
        if (!host_frames[i] || !host_cells[i]) return fail(ctx, VIO_ERR_INVALID_ARG, "NULL frame or output pointer");
        int4* mapped = static_cast<int4*>(const_cast<void*>(device_alias(host_cells[i])));
        if (!mapped || ((uintptr_t)mapped & 15))
            return fail(ctx, VIO_ERR_INVALID_ARG, "host_cells must be pinned, 16-byte aligned host memory");
        outs[i] = mapped;
    }
    if (host_counts && !device_alias(host_counts))
        return fail(ctx, VIO_ERR_INVALID_ARG, "host_counts must be pinned host memory");
    HostSlot& slot = ctx->hslots[ctx->hslot_pos];
    ctx->hslot_pos = (ctx->hslot_pos + 1) % kHostSlots;
    if (!slot.done) VIO_CK(cudaEventCreateWithFlags(&slot.done, cudaEventDisableTiming));
    // the kernels of the slot's previous call have read its frames
    if (slot.used) VIO_CK(cudaStreamWaitEvent(s, slot.done, 0));
    const UploadPlan plan = plan_upload(host_frames, dims, n);
    if ((st = grow(ctx, (void**)&slot.d_in, &slot.in_cap, std::max<size_t>(plan.bytes, 256), false)) != VIO_OK)
        return st;
    if ((st = grow(ctx, (void**)&slot.d_counts, &slot.counts_cap, sizeof(int32_t) * n, false)) != VIO_OK) return st;
    std::vector<const uint8_t*> lev0(n);
    for (int i = 0; i < n; ++i) lev0[i] = slot.d_in + plan.off[i];
    if ((st = enqueue_upload(ctx, plan, slot.d_in, s)) != VIO_OK) return st;
    // the detection waits for the context's previous call (another stream's
    // included), so the copies above overlap that call's kernels
    if ((st = detect_impl(ctx, lev0.data(), plan.pitch.data(), dims, n, thresh, arc, cell, levels, outs.data(),
                          slot.d_counts, s)) != VIO_OK)
        return st;
    if (host_counts)
        VIO_CK(cudaMemcpyAsync(host_counts, slot.d_counts, sizeof(int32_t) * n, cudaMemcpyDeviceToHost, s));
    VIO_CK(cudaEventRecord(slot.done, s));
    slot.used = true;
    return VIO_OK;
}

vio_status vio_sync(vio_ctx* ctx, vio_stream stream) {
    if (!ctx) return VIO_ERR_INVALID_ARG;
    VIO_CK(cudaSetDevice(ctx->cfg.device));
    VIO_CK(cudaStreamSynchronize(reinterpret_cast<cudaStream_t>(stream)));
    return take_status(ctx);
}

vio_status vio_selftest_timeout(vio_ctx* ctx, uint32_t limit_us) {
    if (!ctx || limit_us < 1 || limit_us > 1000000) return VIO_ERR_INVALID_ARG;
    VIO_CK(cudaSetDevice(ctx->cfg.device));
    cudaStream_t s = nullptr;
    VIO_CK(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
    selftest_wait_kernel<<<1, 32, 0, s>>>(ctx->d_status, (uint64_t)limit_us * 1000ull);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaStreamDestroy(s);
    if (e != cudaSuccess) return fail(ctx, VIO_ERR_CUDA, std::string("selftest: ") + cudaGetErrorString(e));
    const vio_status st = take_status(ctx);
    if (st != VIO_OK) return st;
    return fail(ctx, VIO_ERR_CUDA, "selftest: the bounded wait did not report its timeout");
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
    out->cta_per_sm = ctx->last_ctas;
    out->cell_size = ctx->last_cell;
    return VIO_OK;
}

vio_status vio_set_tuning(vio_ctx* ctx, const vio_tuning* t) {
    if (!ctx) return VIO_ERR_INVALID_ARG;
    if (!t) {
        ctx->pinned_variant = -1;
        ctx->pinned_ctas = 0;
        return VIO_OK;
    }
    if (t->variant < 0 || t->variant >= (int)variants().size())
        return fail(ctx, VIO_ERR_INVALID_ARG, "unknown variant");
    if (variants()[t->variant].radius != ctx->cfg.nms_radius)
        return fail(ctx, VIO_ERR_INVALID_ARG, "variant was built for another NMS radius");
    if (t->cta_per_sm < 0 || t->cta_per_sm > kMaxCtasPerSm)
        return fail(ctx, VIO_ERR_INVALID_ARG, "cta_per_sm must be in 0..4");
    ctx->pinned_variant = t->variant;
    ctx->pinned_ctas = t->cta_per_sm;
    return VIO_OK;
}

}  // extern "C"
