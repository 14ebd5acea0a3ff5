// Device code of the feature tracker (Section II-E, Eqs. 2-6): one warp per
// feature, patch sums reduced with an xor butterfly of warp shuffles, fp32.
#pragma once
#include <stdint.h>

#include "vio_kernels.cuh"

namespace vio {

// Tracker call block, after the pyramid's CallHeader / FrameDesc[2n] /
// blocks[2n+1] sections (frame 2i is pair i's previous frame, 2i+1 its next
// frame):
//   TrackHeader
//   TrackPair pairs[n]
//   int32 prefix[n + 1]      prefix sums of the features per pair
struct TrackHeader {
    int32_t levels, patch_fine, patch_coarse, max_iters;
    float min_update;
    int32_t model, n_pairs, n_features;
    uint32_t off_pairs, off_prefix;
    int32_t cells_in;      // 1: the inputs are detector records (x, y, level, score)
    int32_t pad;
};

struct TrackPair {
    const float* pts;   // 2 floats per feature, or 4 int32 per detector record (cells_in)
    float* out;         // 8 words per feature (vio_track_result)
};

constexpr int kTrackWarps = 8;  // features per CTA
constexpr int kTrackMaxGrid = 18 * 18;

// Bilinear sample of an 8-bit image at (x, y), 0 <= x <= W-2, 0 <= y <= H-2.
__device__ __forceinline__ float bilinear(const uint8_t* __restrict__ img, int pitch, float x, float y) {
    const float fx = floorf(x), fy = floorf(y);
    const float ax = x - fx, ay = y - fy;
    const uint8_t* p = img + (size_t)(int)fy * pitch + (int)fx;
    const float a = __ldg(p), b = __ldg(p + 1), c = __ldg(p + pitch), d = __ldg(p + pitch + 1);
    const float top = fmaf(ax, b - a, a), bot = fmaf(ax, d - c, c);
    return fmaf(ay, bot - top, top);
}

__device__ __forceinline__ bool inside(float x, float y, int w, int h) {
    return x >= 0.f && y >= 0.f && x <= (float)(w - 2) && y <= (float)(h - 2);
}

// Sum over the warp; every lane ends with the same bits (each butterfly
// stage adds the same two values on both partners).
__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int m = 16; m > 0; m >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, m);
    return v;
}

// In-place Cholesky factor of the symmetric 4x4 A (lower triangle used);
// false when a pivot is not positive.
__device__ __forceinline__ bool cholesky4(float (&A)[4][4]) {
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        float d = A[j][j];
#pragma unroll
        for (int k = 0; k < j; ++k) d -= A[j][k] * A[j][k];
        if (!(d > 0.f)) return false;
        const float l = sqrtf(d);
        A[j][j] = l;
#pragma unroll
        for (int i = j + 1; i < 4; ++i) {
            float s = A[i][j];
#pragma unroll
            for (int k = 0; k < j; ++k) s -= A[i][k] * A[j][k];
            A[i][j] = s / l;
        }
    }
    return true;
}

// Solves L L^T x = b with the factor from cholesky4 and the reciprocals of
// its diagonal (computed once per level: the iterations then multiply).
__device__ __forceinline__ void chol_solve4(const float (&L)[4][4], const float (&inv)[4], const float (&b)[4],
                                            float (&x)[4]) {
    float y[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        float s = b[i];
#pragma unroll
        for (int k = 0; k < i; ++k) s -= L[i][k] * y[k];
        y[i] = s * inv[i];
    }
#pragma unroll
    for (int i = 3; i >= 0; --i) {
        float s = y[i];
#pragma unroll
        for (int k = i + 1; k < 4; ++k) s -= L[k][i] * x[k];
        x[i] = s * inv[i];
    }
}

struct TrackLevel {
    const uint8_t* prev;
    const uint8_t* next;
    int pitch_prev, pitch_next, w, h;
};

// One pyramid level of one feature with a P x P patch.  State (t, alpha,
// beta, iters, residual) is kept identical on all lanes.  Returns false when
// the track is lost.
template <int P>
__device__ bool track_level(const TrackLevel& lv, float cx, float cy, float* tg, int lane, int model, int max_iters,
                            float min_update, float& tx, float& ty, float& alpha, float& beta, int& iters,
                            float& residual) {
    constexpr int G = P + 2;       // template grid with a one-sample border
    constexpr int NPX = P * P / 32;  // patch pixels per lane
    const float o0 = cx - 0.5f * (P - 1), o1 = cy - 0.5f * (P - 1);
    // template grid: sample (i, j) at (o0 - 1 + i, o1 - 1 + j)
    bool ok = true;
    for (int idx = lane; idx < G * G; idx += 32) {
        const int j = idx / G, i = idx - j * G;
        const float gx = o0 - 1.f + (float)i, gy = o1 - 1.f + (float)j;
        if (inside(gx, gy, lv.w, lv.h))
            tg[idx] = bilinear(lv.prev, lv.pitch_prev, gx, gy);
        else
            ok = false;
    }
    if (!__all_sync(0xFFFFFFFFu, ok)) return false;
    __syncwarp();

    // Each lane owns a strip of NPX consecutive patch rows in one column:
    // column i = lane % P, rows j = (lane / P) * NPX + m.  The samples of a
    // strip share their column, so each iteration reads NPX + 1 pairs of
    // pixels and blends each pair once (the bilinear weights are the same for
    // every sample of the patch: all sit at integer offsets from one point).
    const int col = lane % P, row0 = (lane / P) * NPX;
    // U (Eq. 4) of this lane's pixels, with the appearance at the start of the level
    const float g = 1.f + alpha;
    float T[NPX], Ux[NPX], Uy[NPX];
    float h00 = 0, h01 = 0, h02 = 0, h03 = 0, h11 = 0, h12 = 0, h13 = 0, h22 = 0, h23 = 0, h33 = 0;
#pragma unroll
    for (int m = 0; m < NPX; ++m) {
        const float* c = tg + (row0 + m + 1) * G + (col + 1);
        T[m] = c[0];
        Ux[m] = g * (0.5f * (c[1] - c[-1]));
        Uy[m] = g * (0.5f * (c[G] - c[-G]));
        h00 = fmaf(Ux[m], Ux[m], h00);
        h01 = fmaf(Ux[m], Uy[m], h01);
        h02 = fmaf(Ux[m], T[m], h02);
        h03 += Ux[m];
        h11 = fmaf(Uy[m], Uy[m], h11);
        h12 = fmaf(Uy[m], T[m], h12);
        h13 += Uy[m];
        h22 = fmaf(T[m], T[m], h22);
        h23 += T[m];
        h33 += 1.f;
    }
    const bool use_gain = model & 1, use_off = model & 2;
    float L[4][4];
    L[0][0] = warp_sum(h00);
    L[1][0] = warp_sum(h01);
    L[1][1] = warp_sum(h11);
    // parameters the model does not estimate get an identity row: their update is 0
    L[2][0] = use_gain ? warp_sum(h02) : 0.f;
    L[2][1] = use_gain ? warp_sum(h12) : 0.f;
    L[2][2] = use_gain ? warp_sum(h22) : 1.f;
    L[3][0] = use_off ? warp_sum(h03) : 0.f;
    L[3][1] = use_off ? warp_sum(h13) : 0.f;
    L[3][2] = use_off && use_gain ? warp_sum(h23) : 0.f;
    L[3][3] = use_off ? warp_sum(h33) : 1.f;
    L[0][1] = L[0][2] = L[0][3] = L[1][2] = L[1][3] = L[2][3] = 0.f;
    if (!cholesky4(L)) return false;
    const float inv[4] = {1.f / L[0][0], 1.f / L[1][1], 1.f / L[2][2], 1.f / L[3][3]};
    const float min2 = min_update * min_update;
    float rr_last = -1.f;  // squared residual sum of the latest iteration

    for (int it = 0; it < max_iters; ++it) {
        // this lane's samples: column xs, rows ys .. ys + NPX - 1 of the next image
        const float xs = o0 + (float)col + tx, ys = o1 + (float)row0 + ty;
        ok = inside(xs, ys, lv.w, lv.h) && inside(xs, ys + (float)(NPX - 1), lv.w, lv.h);
        if (!__all_sync(0xFFFFFFFFu, ok)) {
            if (rr_last >= 0.f) residual = sqrtf(rr_last * (1.f / (P * P)));
            return false;
        }
        const float fx = floorf(xs), fy = floorf(ys);
        const float ax = xs - fx, ay = ys - fy;
        const uint8_t* q = lv.next + (size_t)(int)fy * lv.pitch_next + (int)fx;
        float top = fmaf(ax, (float)__ldg(q + 1) - (float)__ldg(q), (float)__ldg(q));
        float b0 = 0, b1 = 0, b2 = 0, b3 = 0, rr = 0;
#pragma unroll
        for (int m = 0; m < NPX; ++m) {
            q += lv.pitch_next;
            const float bot = fmaf(ax, (float)__ldg(q + 1) - (float)__ldg(q), (float)__ldg(q));
            const float r = fmaf(ay, bot - top, top) - fmaf(1.f + alpha, T[m], beta);
            top = bot;
            b0 = fmaf(Ux[m], r, b0);
            b1 = fmaf(Uy[m], r, b1);
            b2 = fmaf(T[m], r, b2);
            b3 += r;
            rr = fmaf(r, r, rr);
        }
        const float b[4] = {warp_sum(b0), warp_sum(b1), use_gain ? warp_sum(b2) : 0.f, use_off ? warp_sum(b3) : 0.f};
        rr_last = warp_sum(rr);
        float dq[4];
        chol_solve4(L, inv, b, dq);
        tx -= dq[0];
        ty -= dq[1];
        alpha += dq[2];
        beta += dq[3];
        ++iters;
        if (dq[0] * dq[0] + dq[1] * dq[1] < min2) {
            residual = sqrtf(rr_last * (1.f / (P * P)));
            return true;
        }
    }
    if (rr_last >= 0.f) residual = sqrtf(rr_last * (1.f / (P * P)));
    return true;
}

__global__ void __launch_bounds__(kTrackWarps * 32, 3) track_kernel(const uint8_t* __restrict__ call,
                                                                uint32_t off_track) {
    __shared__ float grid_sh[kTrackWarps][kTrackMaxGrid];
    const CallView cv(call);
    const TrackHeader* th = reinterpret_cast<const TrackHeader*>(call + off_track);
    const TrackPair* pairs = reinterpret_cast<const TrackPair*>(call + th->off_pairs);
    const int32_t* prefix = reinterpret_cast<const int32_t*>(call + th->off_prefix);
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int f = blockIdx.x * kTrackWarps + wib;
    if (f >= th->n_features) return;
    const int pr = upper_index(prefix, th->n_pairs, f);
    const int j = f - prefix[pr];
    const TrackPair tp = pairs[pr];
    const FrameDesc& fp = cv.fds[2 * pr];
    const FrameDesc& fn = cv.fds[2 * pr + 1];
    float x, y;
    if (th->cells_in) {
        // a detector record: an empty cell (level < 0) gives an empty result
        const int4 rec = reinterpret_cast<const int4*>(tp.pts)[j];
        if (rec.z < 0) {
            if (lane == 0) {
                float4* o = reinterpret_cast<float4*>(tp.out + 8 * j);
                o[0] = make_float4(-1.f, -1.f, 0.f, 0.f);
                o[1] = make_float4(__int_as_float(0), __int_as_float(0), 0.f, 0.f);
            }
            return;
        }
        x = (float)rec.x;
        y = (float)rec.y;
    } else {
        x = tp.pts[2 * j];
        y = tp.pts[2 * j + 1];
    }
    float tx = 0.f, ty = 0.f, alpha = 0.f, beta = 0.f, residual = 0.f;
    int iters = 0;
    bool ok = true;
    const int L = th->levels;
    int k = L - 1;
    for (; k >= 0; --k) {
        const TrackLevel lv{fp.lev[k], fn.lev[k], fp.pitch[k], fn.pitch[k], fp.w >> k, fp.h >> k};
        const float s = 1.f / (float)(1 << k);
        const float cx = (x + 0.5f) * s - 0.5f, cy = (y + 0.5f) * s - 0.5f;
        const int P = k == 0 ? th->patch_fine : th->patch_coarse;
        ok = P == 16 ? track_level<16>(lv, cx, cy, grid_sh[wib], lane, th->model, th->max_iters, th->min_update, tx,
                                       ty, alpha, beta, iters, residual)
                     : track_level<8>(lv, cx, cy, grid_sh[wib], lane, th->model, th->max_iters, th->min_update, tx,
                                      ty, alpha, beta, iters, residual);
        if (!ok) break;
        if (k > 0) {
            tx *= 2.f;
            ty *= 2.f;
        }
        __syncwarp();  // the template grid is rewritten by the next level
    }
    if (lane == 0) {
        // a lost track reports its estimate so far in level-0 pixels
        const float sc = ok ? 1.f : (float)(1 << k);
        float4* o = reinterpret_cast<float4*>(tp.out + 8 * j);
        o[0] = make_float4(x + tx * sc, y + ty * sc, alpha, beta);
        o[1] = make_float4(__int_as_float(ok ? 1 : 0), __int_as_float(iters), residual, 0.f);
    }
}

}  // namespace vio
