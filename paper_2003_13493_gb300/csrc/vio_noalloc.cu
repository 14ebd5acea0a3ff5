// vio_detect_noalloc: detection of one frame without allocating anything.
//
// Some callers cannot allocate device memory at the moment they need a
// detection: code running inside a memory pool's accounting, a real-time
// loop where cudaMalloc's implicit device synchronisation and unbounded
// latency are not allowed, or a plug-in whose host process owns all
// allocations.  This entry point needs no context: the working memory the
// kernels use besides the caller's frame and outputs (the per-call block,
// the work counter and status word, the cell keys and the pyramid levels)
// lives in one file-scope device array of fixed size that the library
// holds on every device that loads it, until the process exits.
#include <cuda.h>
#include <cuda_runtime.h>

#include <cstring>
#include <mutex>

#include "../../include/vio.h"
// This translation unit compiles the kernels of vio_kernels.cuh a second
// time.  decode_kernel is static, so each unit launches its own copy; the
// template kernels' host stubs, however, are merged by the linker, so a
// launch from here may run the copy registered by another unit (and the
// other way round).  That is only correct while vio_kernels.cuh keeps no
// file-scope __device__ or __constant__ state: its kernels must read
// everything from their arguments.
#include "vio_kernels.cuh"

using namespace vio;

namespace {

// The shared working memory.  Zero when the module loads; every call
// re-clears what must start at zero.  Calls that overlap on the GPU share it
// and race.
static __device__ __align__(256) uint8_t g_noalloc_scratch[VIO_NOALLOC_SCRATCH_BYTES];

constexpr int kTH = 62;          // tile rows of the fused kernel variant used here
constexpr int kBoxW = 144;       // its TMA box width
constexpr size_t kCallOff = 0;   // call block
constexpr size_t kCallCap = 2048;
constexpr size_t kCountOff = 2048;  // work counter, then status word
constexpr size_t kKeysOff = 4096;   // cell keys, then the pyramid levels

// Largest call block for one frame: header, one frame descriptor, one
// level-0 map, kMaxLevels - 1 level maps, three small prefix tables.  The
// sections start at multiples of 128 bytes and hold pointers and tensor maps
// (aligned like CUtensorMap), so the block itself is aligned like a tensor map.
struct alignas(alignof(CUtensorMap)) NoallocBlock {
    uint8_t bytes[kCallCap];
};
static_assert(alignof(NoallocBlock) >= alignof(CUtensorMap), "tensor maps inside the block stay aligned");

__global__ void noalloc_load_call(const __grid_constant__ NoallocBlock blk, uint8_t* __restrict__ dst, int n) {
    for (int i = threadIdx.x; i < n; i += blockDim.x) dst[i] = blk.bytes[i];
}

using EncodeTiledFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                   const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

// Per-device set-up, done by the first call on each device.
struct DeviceSetup {
    bool ready = false;
    uint8_t* scratch = nullptr;  // device address of g_noalloc_scratch on this device
    int sm_count = 0;
    int grid_fused[3] = {0, 0, 0};
};
constexpr int kMaxDevices = 64;
std::mutex g_setup_mu;
DeviceSetup g_setup[kMaxDevices];
EncodeTiledFn g_encode = nullptr;

using FusedFn = void (*)(const uint8_t*, int32_t*, uint32_t*);
FusedFn fused_fn(int score) {
    switch (score) {
        case 0: return fast_nms_cell_kernel<kTH, 0>;
        case 1: return fast_nms_cell_kernel<kTH, 1>;
        default: return fast_nms_cell_kernel<kTH, 2>;
    }
}

using PyrFn = void (*)(const uint8_t*);
PyrFn pyr_fn(int levels) {
    switch (levels) {
        case 2: return pyramid_kernel<2>;
        case 3: return pyramid_kernel<3>;
        case 4: return pyramid_kernel<4>;
        default: return pyramid_kernel<5>;
    }
}

size_t round_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

vio_status setup_device(int dev, DeviceSetup** out) {
    if (dev < 0 || dev >= kMaxDevices) return VIO_ERR_UNSUPPORTED;
    std::lock_guard<std::mutex> g(g_setup_mu);
    DeviceSetup& s = g_setup[dev];
    if (!s.ready) {
        // the array's name is only a host-side handle: ask for its address on
        // this device (the caller made `dev` current)
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return VIO_ERR_CUDA;
        int major = 0, minor = 0;
        if (cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&s.sm_count, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
            return VIO_ERR_CUDA;
        if (major != 10 || minor != 3) return VIO_ERR_UNSUPPORTED;
        if (!g_encode) {
            cudaDriverEntryPointQueryResult q;
            void* fn = nullptr;
            if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) !=
                    cudaSuccess || !fn)
                return VIO_ERR_CUDA;
            g_encode = reinterpret_cast<EncodeTiledFn>(fn);
        }
        for (int m = 0; m < 3; ++m) {
            const FusedFn fn = fused_fn(m);
            int occ = 0;
            if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, TileGeom<kTH>::SMEM) !=
                    cudaSuccess ||
                cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, kThreads, TileGeom<kTH>::SMEM) != cudaSuccess)
                return VIO_ERR_CUDA;
            s.grid_fused[m] = (occ > 0 ? occ : 1) * s.sm_count;
        }
        s.scratch = static_cast<uint8_t*>(p);
        s.ready = true;
    }
    *out = &s;
    return VIO_OK;
}

bool encode(CUtensorMap* m, const void* ptr, int w, int h, int pitch) {
    cuuint64_t gdim[2] = {(cuuint64_t)w, (cuuint64_t)h};
    cuuint64_t gstride[1] = {(cuuint64_t)pitch};
    cuuint32_t box[2] = {(cuuint32_t)kBoxW, (cuuint32_t)(kTH + 8)};
    cuuint32_t estr[2] = {1, 1};
    return g_encode(m, CU_TENSOR_MAP_DATA_TYPE_UINT8, 2, const_cast<void*>(ptr), gdim, gstride, box, estr,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace

extern "C" vio_status vio_detect_noalloc(const uint8_t* frame, vio_dims d, int thresh, int arc_len, int cell,
                                         int levels, int score, vio_feature* out_cells, int32_t* out_count,
                                         vio_stream stream) {
    // arguments (the same ranges as vio_detect, plus TMA-ready framing)
    if (!frame || !out_cells) return VIO_ERR_INVALID_ARG;
    if (score < 0 || score > 2 || thresh < 0 || thresh > 255 || (score == VIO_SCORE_MT && thresh < 1) ||
        arc_len < 9 || arc_len > 16 || cell < 32 || cell % 32 != 0 || levels < 1 || levels > VIO_MAX_LEVELS)
        return VIO_ERR_INVALID_ARG;
    if (d.w < 7 || d.h < 7 || d.w > 65535 || d.h > 65535 || (int64_t)d.w * d.h >= (1ll << 28) || d.pitch < d.w ||
        (d.w >> (levels - 1)) < 7 || (d.h >> (levels - 1)) < 7)
        return VIO_ERR_INVALID_ARG;
    if (((uintptr_t)frame & 15) || (d.pitch & 15)) return VIO_ERR_INVALID_ARG;

    // scratch needed: keys, then each pyramid level with a 128-byte pitch
    const int gw = (d.w + cell - 1) / cell, gh = (d.h + cell - 1) / cell;
    size_t need = kKeysOff + round_up((size_t)gw * gh * 8, 256);
    size_t lev_off[kMaxLevels] = {0, 0, 0, 0, 0};
    int lev_pitch[kMaxLevels] = {0, 0, 0, 0, 0};
    for (int k = 1; k < levels; ++k) {
        lev_pitch[k] = (int)round_up((size_t)(d.w >> k), 128);
        lev_off[k] = need;
        need += round_up((size_t)lev_pitch[k] * (size_t)(d.h >> k), 256);
    }
    if (need > VIO_NOALLOC_SCRATCH_BYTES) return VIO_ERR_INVALID_ARG;

    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return VIO_ERR_CUDA;
    DeviceSetup* S = nullptr;
    vio_status st = setup_device(dev, &S);
    if (st != VIO_OK) return st;
    uint8_t* base = S->scratch;
    int32_t* counter = reinterpret_cast<int32_t*>(base + kCountOff);
    uint32_t* status = reinterpret_cast<uint32_t*>(base + kCountOff + 4);
    uint64_t* keys = reinterpret_cast<uint64_t*>(base + kKeysOff);

    // the call block, built on the stack: header, frame, maps, tables
    NoallocBlock blk;
    std::memset(&blk, 0, sizeof(blk));
    size_t off = round_up(sizeof(CallHeader), 128);
    const size_t off_fds = off;
    off += round_up(sizeof(FrameDesc), 128);
    const size_t off_maps0 = off;
    off += round_up(sizeof(CUtensorMap), 128);
    const size_t off_mapsk = off;
    off += round_up(sizeof(CUtensorMap) * (kMaxLevels - 1), 128);
    const size_t off_tiles = off;
    off += round_up(sizeof(int32_t) * (levels + 1), 128);
    const size_t off_blocks = off;
    off += round_up(sizeof(int32_t) * 2, 128);
    const size_t off_cells = off;
    off += round_up(sizeof(int32_t) * 2, 128);
    const size_t bytes = off;
    static_assert(sizeof(CallHeader) <= 128 && sizeof(FrameDesc) <= 128, "call block layout");
    if (bytes > kCallCap) return VIO_ERR_INVALID_ARG;

    CallHeader* hdr = reinterpret_cast<CallHeader*>(blk.bytes);
    FrameDesc* fd = reinterpret_cast<FrameDesc*>(blk.bytes + off_fds);
    CUtensorMap* map0 = reinterpret_cast<CUtensorMap*>(blk.bytes + off_maps0);
    CUtensorMap* mapk = reinterpret_cast<CUtensorMap*>(blk.bytes + off_mapsk);
    int32_t* tiles = reinterpret_cast<int32_t*>(blk.bytes + off_tiles);
    int32_t* blocks = reinterpret_cast<int32_t*>(blk.bytes + off_blocks);
    int32_t* cells = reinterpret_cast<int32_t*>(blk.bytes + off_cells);
    hdr->thresh = thresh;
    hdr->arc = arc_len;
    hdr->n_frames = 1;
    hdr->levels = levels;
    hdr->cell = cell;
    hdr->tile_h = kTH;
    hdr->counts = out_count;
    // the decode's cell-key check reports into the scratch status word too
    // (cleared below with the counter); this entry point does not read it back
    hdr->status = status;
    hdr->off_fds = (uint32_t)off_fds;
    hdr->off_maps0 = (uint32_t)off_maps0;
    hdr->off_mapsk = (uint32_t)off_mapsk;
    hdr->off_tiles = (uint32_t)off_tiles;
    hdr->off_blocks = (uint32_t)off_blocks;
    hdr->off_cells = (uint32_t)off_cells;
    for (int k = 0; k < levels; ++k) {
        const uint64_t dv = (uint64_t)(cell >> k);
        hdr->cell_magic[k] = (uint32_t)(((1ull << 32) + dv - 1) / dv);
    }
    const int B = 1 << (levels - 1);
    fd->w = d.w;
    fd->h = d.h;
    fd->gw = gw;
    fd->gh = gh;
    fd->pyr_bx = (d.w + 511) / 512;
    fd->pyr_magic = (uint32_t)(((1ull << 31) + fd->pyr_bx - 1) / fd->pyr_bx);
    fd->keys = keys;
    fd->out = reinterpret_cast<int4*>(out_cells);
    fd->lev[0] = const_cast<uint8_t*>(frame);
    fd->pitch[0] = d.pitch;
    if (!encode(map0, frame, d.w, d.h, d.pitch)) return VIO_ERR_CUDA;
    for (int k = 1; k < levels; ++k) {
        fd->lev[k] = base + lev_off[k];
        fd->pitch[k] = lev_pitch[k];
        if (!encode(&mapk[k - 1], fd->lev[k], d.w >> k, d.h >> k, lev_pitch[k])) return VIO_ERR_CUDA;
    }
    blocks[0] = 0;
    blocks[1] = levels > 1 ? fd->pyr_bx * ((d.h + 8 * B - 1) / (8 * B)) : 0;
    cells[0] = 0;
    cells[1] = gw * gh;
    int acc = 0;
    for (int kk = 0; kk < levels; ++kk) {
        const int k = levels - 1 - kk;
        tiles[kk] = acc;
        acc += (((d.w >> k) + TileGeom<kTH>::TW - 1) / TileGeom<kTH>::TW) * (((d.h >> k) + kTH - 1) / kTH);
    }
    tiles[levels] = acc;
    hdr->n_items = acc;
    hdr->n_pyr_blocks = blocks[1];
    hdr->n_cells = cells[1];

    // clear what must start at zero, load the call block, run the kernels
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    if (cudaMemsetAsync(base + kCountOff, 0, 8, s) != cudaSuccess) return VIO_ERR_CUDA;
    if (cudaMemsetAsync(keys, 0, (size_t)gw * gh * 8, s) != cudaSuccess) return VIO_ERR_CUDA;
    noalloc_load_call<<<1, 256, 0, s>>>(blk, base + kCallOff, (int)bytes);
    if (levels > 1) pyr_fn(levels)<<<S->sm_count * 8, 256, 0, s>>>(base + kCallOff);
    fused_fn(score)<<<S->grid_fused[score], kThreads, TileGeom<kTH>::SMEM, s>>>(base + kCallOff, counter, status);
    decode_kernel<<<S->sm_count * 4, 256, 0, s>>>(base + kCallOff, counter);
    return cudaGetLastError() == cudaSuccess ? VIO_OK : VIO_ERR_CUDA;
}
