// Host side of the feature tracker behind vio_track (Section II-E): argument
// checks, the resident pyramid of both frames of every pair (built by the
// detector's pyramid kernel), the per-call block and the launches.
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <vector>

#include "../../include/vio.h"
#include "vio_ctx.h"
#include "vio_track.cuh"

using namespace vio;

namespace {

using PyrFn = void (*)(const uint8_t*);

PyrFn track_pyr_fn(int levels) {
    switch (levels) {
        case 2: return pyramid_kernel<2>;
        case 3: return pyramid_kernel<3>;
        case 4: return pyramid_kernel<4>;
        case 5: return pyramid_kernel<5>;
        default: return nullptr;
    }
}

bool valid_params(const vio_track_params& p) {
    return p.levels >= 1 && p.levels <= kMaxLevels && (p.patch_fine == 8 || p.patch_fine == 16) &&
           (p.patch_coarse == 8 || p.patch_coarse == 16) && p.max_iters >= 1 && p.max_iters <= 100 &&
           std::isfinite(p.min_update) && p.min_update >= 0.f && p.model >= 0 && p.model <= 3;
}

// Grows a pinned host buffer; the previous contents are not kept.
vio_status grow_pinned(vio_ctx* ctx, uint8_t** p, size_t* cap, size_t need) {
    if (need <= *cap && *p) return VIO_OK;
    if (*p) {
        VIO_CK(cudaFreeHost(*p));
        *p = nullptr;
        *cap = 0;
    }
    const size_t want = std::max(need, (size_t)4096);
    VIO_CK(cudaHostAlloc((void**)p, want, cudaHostAllocDefault));
    *cap = want;
    return VIO_OK;
}

}  // namespace

namespace vio {

void track_release(vio_ctx* ctx) {
    TrackState& t = ctx->track;
    if (t.stage_ev) cudaEventSynchronize(t.stage_ev);
    if (t.d_call) cudaFree(t.d_call);
    if (t.d_pyr) cudaFree(t.d_pyr);
    if (t.d_in) cudaFree(t.d_in);
    if (t.h_stage) cudaFreeHost(t.h_stage);
    if (t.stage_ev) cudaEventDestroy(t.stage_ev);
    if (t.done_ev) cudaEventDestroy(t.done_ev);
    ctx->bytes_in_use -= t.call_cap + t.pyr_cap + t.in_cap;
    t = TrackState{};
}

}  // namespace vio

extern "C" {

void vio_track_params_default(vio_track_params* p) {
    if (!p) return;
    std::memset(p, 0, sizeof(*p));
    p->levels = 3;
    p->patch_fine = 16;
    p->patch_coarse = 8;
    p->max_iters = 30;
    p->min_update = 0.01f;
    p->model = VIO_TRACK_GAIN | VIO_TRACK_OFFSET;
}

namespace {

vio_status track_impl(vio_ctx* ctx, const uint8_t* const* prev, const uint8_t* const* next, const vio_dims* dims,
                      int n_pairs, const void* const* pts_in, const int* n_pts, const vio_track_params* params,
                      vio_track_result* const* out, vio_stream stream, bool cells_in) {
    const float* const* pts = reinterpret_cast<const float* const*>(pts_in);
    if (!ctx) return VIO_ERR_INVALID_ARG;
    vio_track_params p;
    if (params) p = *params; else vio_track_params_default(&p);
    if (!valid_params(p)) return fail(ctx, VIO_ERR_INVALID_ARG, "tracker parameters out of range");
    if (n_pairs < 0 || n_pairs > ctx->cfg.max_frames)
        return fail(ctx, VIO_ERR_INVALID_ARG, "n_pairs must be in 0..max_frames");
    if (n_pairs == 0) return VIO_OK;
    if (!prev || !next || !dims || !pts || !n_pts || !out)
        return fail(ctx, VIO_ERR_INVALID_ARG, "NULL argument");
    const int L = p.levels;
    long long total = 0;
    for (int i = 0; i < n_pairs; ++i) {
        const vio_dims& d = dims[i];
        if (d.w < 7 || d.h < 7 || (d.w >> (L - 1)) < 7 || (d.h >> (L - 1)) < 7 || d.pitch < d.w ||
            (long long)d.w * d.h >= (1ll << 28))
            return fail(ctx, VIO_ERR_INVALID_ARG, "frame size out of range for the pyramid");
        if (!prev[i] || !next[i]) return fail(ctx, VIO_ERR_INVALID_ARG, "NULL frame");
        if (n_pts[i] < 0) return fail(ctx, VIO_ERR_INVALID_ARG, "negative feature count");
        if (n_pts[i] > 0 && (!pts[i] || !out[i])) return fail(ctx, VIO_ERR_INVALID_ARG, "NULL feature array");
        total += n_pts[i];
    }
    if (total == 0) return VIO_OK;
    if (total > (1ll << 24)) return fail(ctx, VIO_ERR_INVALID_ARG, "more than 2^24 features in one call");
    VIO_CK(cudaSetDevice(ctx->cfg.device));
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    TrackState& T = ctx->track;
    const int nf = 2 * n_pairs;

    // resident layout: staged level-0 copies and levels 1..L-1 of every frame
    std::vector<size_t> in_off(nf, (size_t)-1), lev_off(nf * kMaxLevels, 0);
    std::vector<int> lev_pitch(nf * kMaxLevels, 0);
    size_t ioff = 0, poff = 0;
    for (int f = 0; f < nf; ++f) {
        const vio_dims& d = dims[f >> 1];
        const uint8_t* src = (f & 1) ? next[f >> 1] : prev[f >> 1];
        if (((uintptr_t)src & 15) || (d.pitch & 15)) {
            in_off[f] = ioff;
            ioff += align_up(align_up(d.w, 16) * (size_t)d.h, 256);
        }
        for (int k = 1; k < L; ++k) {
            lev_pitch[f * kMaxLevels + k] = (int)align_up(d.w >> k, 128);
            lev_off[f * kMaxLevels + k] = poff;
            poff += align_up((size_t)lev_pitch[f * kMaxLevels + k] * (d.h >> k), 256);
        }
    }
    // call block sections
    size_t off = align_up(sizeof(CallHeader), 128);
    const size_t off_fds = off;
    off += align_up(sizeof(FrameDesc) * nf, 128);
    const size_t off_blocks = off;
    off += align_up(sizeof(int32_t) * (nf + 1), 128);
    const size_t off_track = off;
    off += align_up(sizeof(TrackHeader), 128);
    const size_t off_pairs = off;
    off += align_up(sizeof(TrackPair) * n_pairs, 128);
    const size_t off_prefix = off;
    off += align_up(sizeof(int32_t) * (n_pairs + 1), 128);
    const size_t bytes = off;

    vio_status st;
    if (!T.stage_ev) VIO_CK(cudaEventCreateWithFlags(&T.stage_ev, cudaEventDisableTiming));
    if (!T.done_ev) VIO_CK(cudaEventCreateWithFlags(&T.done_ev, cudaEventDisableTiming));
    VIO_CK(cudaEventSynchronize(T.stage_ev));  // the previous call's upload has left the staging buffer
    // the previous call's kernels read the device buffers this call rewrites
    if (T.have_done) VIO_CK(cudaStreamWaitEvent(s, T.done_ev, 0));
    if ((st = grow(ctx, (void**)&T.d_in, &T.in_cap, std::max<size_t>(ioff, 256), false)) != VIO_OK) return st;
    if ((st = grow(ctx, (void**)&T.d_pyr, &T.pyr_cap, std::max<size_t>(poff, 256), false)) != VIO_OK) return st;
    if ((st = grow(ctx, (void**)&T.d_call, &T.call_cap, bytes, false)) != VIO_OK) return st;
    if ((st = grow_pinned(ctx, &T.h_stage, &T.stage_cap, bytes)) != VIO_OK) return st;

    uint8_t* hb = T.h_stage;
    std::memset(hb, 0, bytes);
    CallHeader* hdr = reinterpret_cast<CallHeader*>(hb);
    FrameDesc* fds = reinterpret_cast<FrameDesc*>(hb + off_fds);
    int32_t* blocks = reinterpret_cast<int32_t*>(hb + off_blocks);
    TrackHeader* th = reinterpret_cast<TrackHeader*>(hb + off_track);
    TrackPair* tps = reinterpret_cast<TrackPair*>(hb + off_pairs);
    int32_t* prefix = reinterpret_cast<int32_t*>(hb + off_prefix);
    hdr->n_frames = nf;
    hdr->levels = L;
    // the pyramid kernel reads only the frame descriptors and block prefix;
    // the detector's other sections are empty here
    hdr->off_fds = (uint32_t)off_fds;
    hdr->off_blocks = (uint32_t)off_blocks;
    hdr->off_maps0 = hdr->off_mapsk = hdr->off_tiles = hdr->off_cells = (uint32_t)off_blocks;
    const int B = 1 << (L - 1);
    blocks[0] = 0;
    for (int f = 0; f < nf; ++f) {
        const vio_dims& d = dims[f >> 1];
        const uint8_t* src = (f & 1) ? next[f >> 1] : prev[f >> 1];
        FrameDesc& fd = fds[f];
        fd.w = d.w;
        fd.h = d.h;
        fd.pyr_bx = (d.w + 511) / 512;
        fd.pyr_magic = (uint32_t)(((1ull << 31) + fd.pyr_bx - 1) / fd.pyr_bx);
        const int pyr_by = (d.h + 8 * B - 1) / (8 * B);
        blocks[f + 1] = blocks[f] + (L > 1 ? fd.pyr_bx * pyr_by : 0);
        if (in_off[f] != (size_t)-1) {
            const int pp = (int)align_up(d.w, 16);
            VIO_CK(cudaMemcpy2DAsync(T.d_in + in_off[f], pp, src, d.pitch, d.w, d.h, cudaMemcpyDeviceToDevice, s));
            fd.lev[0] = T.d_in + in_off[f];
            fd.pitch[0] = pp;
        } else {
            fd.lev[0] = const_cast<uint8_t*>(src);
            fd.pitch[0] = d.pitch;
        }
        for (int k = 1; k < L; ++k) {
            fd.lev[k] = T.d_pyr + lev_off[f * kMaxLevels + k];
            fd.pitch[k] = lev_pitch[f * kMaxLevels + k];
        }
    }
    hdr->n_pyr_blocks = blocks[nf];
    th->levels = L;
    th->patch_fine = p.patch_fine;
    th->patch_coarse = p.patch_coarse;
    th->max_iters = p.max_iters;
    th->min_update = p.min_update;
    th->model = p.model;
    th->n_pairs = n_pairs;
    th->n_features = (int)total;
    th->off_pairs = (uint32_t)off_pairs;
    th->off_prefix = (uint32_t)off_prefix;
    th->cells_in = cells_in ? 1 : 0;
    prefix[0] = 0;
    for (int i = 0; i < n_pairs; ++i) {
        tps[i].pts = pts[i];
        tps[i].out = reinterpret_cast<float*>(out[i]);
        prefix[i + 1] = prefix[i] + n_pts[i];
    }

    VIO_CK(cudaMemcpyAsync(T.d_call, hb, bytes, cudaMemcpyHostToDevice, s));
    VIO_CK(cudaEventRecord(T.stage_ev, s));
    // the kernel strides over its grid: a few frames' blocks need no more than one CTA per SM
    const int pyr_grid = blocks[nf] <= 2 * ctx->sm_count ? ctx->sm_count : ctx->sm_count * 8;
    if (L > 1) track_pyr_fn(L)<<<pyr_grid, 256, 0, s>>>(T.d_call);
    VIO_CK(cudaGetLastError());
    const int grid = (int)((total + kTrackWarps - 1) / kTrackWarps);
    track_kernel<<<grid, kTrackWarps * 32, 0, s>>>(T.d_call, (uint32_t)off_track);
    VIO_CK(cudaGetLastError());
    VIO_CK(cudaEventRecord(T.done_ev, s));
    T.have_done = true;
    return VIO_OK;
}

}  // namespace

vio_status vio_track(vio_ctx* ctx, const uint8_t* const* prev, const uint8_t* const* next, const vio_dims* dims,
                     int n_pairs, const float* const* pts, const int* n_pts, const vio_track_params* params,
                     vio_track_result* const* out, vio_stream stream) {
    NvtxRange nvtx("vio_track");
    return track_impl(ctx, prev, next, dims, n_pairs, reinterpret_cast<const void* const*>(pts), n_pts, params, out,
                      stream, false);
}

vio_status vio_track_cells(vio_ctx* ctx, const uint8_t* const* prev, const uint8_t* const* next,
                           const vio_dims* dims, int n_pairs, const vio_feature* const* cells, const int* n_cells,
                           const vio_track_params* params, vio_track_result* const* out, vio_stream stream) {
    NvtxRange nvtx("vio_track_cells");
    return track_impl(ctx, prev, next, dims, n_pairs, reinterpret_cast<const void* const*>(cells), n_cells, params,
                      out, stream, true);
}

}  // extern "C"
