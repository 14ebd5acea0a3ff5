// Device code: pyramid half-sampling, the fused FAST + 3x3 NMS + cell-max
// kernel, and the cell decode.  All arithmetic is integer.
#pragma once
#include <cuda.h>
#include <stdint.h>

#include "ptx.cuh"

namespace vio {

constexpr int kMaxLevels = 5;
constexpr uint32_t kStatusTimeout = 1u;
constexpr uint64_t kWaitLimitNs = 1000000000ull;  // 1 s per bounded wait

// Per-frame descriptor, rewritten by the host for every call.
struct FrameDesc {
    int32_t w, h;          // level-0 size
    int32_t gw, gh;        // cell grid
    int32_t pyr_bx;        // pyramid thread blocks along x
    int32_t pad0;
    uint64_t* keys;        // gw * gh packed cell keys (0 = empty)
    int4* out;             // gw * gh output records
    uint8_t* lev[kMaxLevels];   // level 0 is the caller's frame (read only)
    int32_t pitch[kMaxLevels];
    int32_t pad1[3];
};

// Call-wide scalars, rewritten by the host for every call.
struct CallHeader {
    int32_t thresh, arc, n_frames, n_items;
    int32_t mode, cell, levels, pad0;
    int32_t* counts;       // device int32[n_frames] or nullptr
    uint64_t pad1[3];
};

struct WorkItem {
    uint16_t frame;
    uint8_t level;
    uint8_t pad;
    uint16_t tx, ty;
};

// ---------------------------------------------------------------------------
// Pyramid: one thread owns a B x B block of level 0 (B = 2^(L-1)) and writes
// every level-k pixel that block produces, k = 1..L-1.  Level k+1 is the 2x2
// mean of level k rounded half up, taken from the rounded level-k values.
// ---------------------------------------------------------------------------
template <int L>
__global__ void __launch_bounds__(256) pyramid_kernel(const CallHeader* __restrict__ hdr,
                                                      const FrameDesc* __restrict__ fds,
                                                      const int32_t* __restrict__ block_start) {
    constexpr int B = 1 << (L - 1);
    const int nf = hdr->n_frames;
    // frame owning this block: block_start is the prefix sum of blocks per frame
    int lo = 0, hi = nf - 1;
    const int b = blockIdx.x;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (block_start[mid] <= b) lo = mid; else hi = mid - 1;
    }
    const FrameDesc& fd = fds[lo];
    const int lb = b - block_start[lo];
    const int tx = (lb % fd.pyr_bx) * 32 + (threadIdx.x & 31);
    const int ty = (lb / fd.pyr_bx) * 8 + (threadIdx.x >> 5);

    // level-1 values of this block, computed from level 0
    constexpr int B1 = B / 2;
    uint32_t v[B1][B1];
    const int W = fd.w, H = fd.h;
    const int W1 = W >> 1, H1 = H >> 1;
    const uint8_t* src = fd.lev[0];
    const int sp = fd.pitch[0];
#pragma unroll
    for (int j = 0; j < B1; ++j) {
        const int y1 = ty * B1 + j;
#pragma unroll
        for (int i = 0; i < B1; ++i) {
            const int x1 = tx * B1 + i;
            uint32_t s = 0;
            if (x1 < W1 && y1 < H1) {
                const uint8_t* p = src + (size_t)(2 * y1) * sp + 2 * x1;
                s = (p[0] + p[1] + p[sp] + p[sp + 1] + 2u) >> 2;
                fd.lev[1][(size_t)y1 * fd.pitch[1] + x1] = (uint8_t)s;
            }
            v[j][i] = s;
        }
    }
    // higher levels from the registers
    int Wk = W1, Hk = H1;
#pragma unroll
    for (int k = 2; k < L; ++k) {
        const int n = B >> k;       // pixels of level k per thread per axis
        Wk >>= 1;
        Hk >>= 1;
        uint8_t* dst = fd.lev[k];
        const int dp = fd.pitch[k];
#pragma unroll
        for (int j = 0; j < B1; ++j) {
#pragma unroll
            for (int i = 0; i < B1; ++i) {
                if (j < n && i < n) {
                    const uint32_t s = (v[2 * j][2 * i] + v[2 * j][2 * i + 1] + v[2 * j + 1][2 * i] +
                                        v[2 * j + 1][2 * i + 1] + 2u) >> 2;
                    const int xk = tx * n + i, yk = ty * n + j;
                    if (xk < Wk && yk < Hk) dst[(size_t)yk * dp + xk] = (uint8_t)s;
                    v[j][i] = s;
                }
            }
        }
    }
}

// ---------------------------------------------------------------------------
// FAST segment test and scores on a shared-memory tile.
// ---------------------------------------------------------------------------

// Radius-3 Bresenham circle, clockwise from the top (Section II-D).
__device__ __forceinline__ int circ_dx(int i) {
    constexpr int8_t d[16] = {0, 1, 2, 3, 3, 3, 2, 1, 0, -1, -2, -3, -3, -3, -2, -1};
    return d[i];
}
__device__ __forceinline__ int circ_dy(int i) {
    constexpr int8_t d[16] = {-3, -3, -2, -1, 0, 1, 2, 3, 3, 3, 2, 1, 0, -1, -2, -3};
    return d[i];
}

// Start positions s (bits 0..15) of cyclic runs of >= n ones in the 16-bit
// mask m: the mask is doubled to 32 bits (a rotation without wrap-around),
// runs of 8 come from three AND-shift doublings and the run of n from two
// overlapping runs of 8 that are n-8 apart.
__device__ __forceinline__ uint32_t arc_starts(uint32_t m, int n) {
    uint32_t r = m | (m << 16);
    r &= r >> 1;
    r &= r >> 2;
    r &= r >> 4;
    r &= r >> (n - 8);
    return r & 0xFFFFu;
}

// 16-bit rotate left of the low 16 bits.
__device__ __forceinline__ uint32_t rotl16(uint32_t m, int s) {
    return ((m << s) | (m >> (16 - s))) & 0xFFFFu;
}

// Score of the pixel at smem pointer p (row pitch P); 0 if not a corner.
template <int MODE>
__device__ __forceinline__ uint32_t fast_score(const uint8_t* __restrict__ p, int P, int t, int n) {
    const int c = p[0];
    const int hi = c + t, lo = c - t;
    // coarse test (CCRF of Algorithm 1): an arc of >= 9 contains two
    // cyclically adjacent compass points (0,4), (4,8), (8,12) or (12,0).
    {
        const int v0 = p[-3 * P], v4 = p[3], v8 = p[3 * P], v12 = p[-3];
        const bool b0 = v0 > hi, b4 = v4 > hi, b8 = v8 > hi, b12 = v12 > hi;
        const bool d0 = v0 < lo, d4 = v4 < lo, d8 = v8 < lo, d12 = v12 < lo;
        const bool pass = ((b0 | b8) & (b4 | b12)) | ((d0 | d8) & (d4 | d12));
        if (!pass) return 0;
    }
    int v[16];
    uint32_t bm = 0, dm = 0;
#pragma unroll
    for (int i = 0; i < 16; ++i) {
        v[i] = p[circ_dy(i) * P + circ_dx(i)];
        bm |= (uint32_t)(v[i] > hi) << i;
        dm |= (uint32_t)(v[i] < lo) << i;
    }
    // at most one polarity can hold n >= 9 points
    const bool bright = __popc(bm) >= n;
    const uint32_t m = bright ? bm : dm;
    const uint32_t starts = arc_starts(m, n);
    if (starts == 0) return 0;
    if (MODE == 0) {  // SAD-B
        uint32_t s = 0;
#pragma unroll
        for (int i = 0; i < 16; ++i) s += (uint32_t)abs(v[i] - c);
        return s;
    } else if (MODE == 1) {  // SAD-A: the run is the union of all passing windows
        uint32_t r = starts;
        uint32_t d = r;
        d |= rotl16(d, 1);
        d |= rotl16(d, 2);
        d |= rotl16(d, 4);  // windows of 8 starting at each start
        const uint32_t run = d | rotl16(d, n - 8);
        uint32_t s = 0;
#pragma unroll
        for (int i = 0; i < 16; ++i) s += ((run >> i) & 1u) ? (uint32_t)abs(v[i] - c) : 0u;
        return s;
    } else {  // MT: largest window minimum of the arc's polarity, minus 1
        // Raising the threshold only removes points from the masks, so only
        // windows that pass at `t` can pass above it; their minimum
        // difference d (strictly above the threshold) gives MT = d - 1.
        int dp[16];
#pragma unroll
        for (int i = 0; i < 16; ++i) dp[i] = bright ? v[i] - c : c - v[i];
        int best = 0;
#pragma unroll
        for (int s0 = 0; s0 < 16; ++s0) {
            if ((starts >> s0) & 1u) {
                int mn = 255;
#pragma unroll
                for (int j = 0; j < 16; ++j)
                    if (j < n) mn = min(mn, dp[(s0 + j) & 15]);
                best = max(best, mn);
            }
        }
        return (uint32_t)(best - 1);
    }
}

// ---------------------------------------------------------------------------
// Fused detect: persistent CTAs pull (frame, level, tile) items from a
// counter.  Per item: TMA-load the tile plus a 4-pixel halo (3 for the
// circle, 1 for NMS), score the tile plus a 1-pixel ring into shared
// memory, then apply 3x3 NMS and fold survivors into the cell keys.
// ---------------------------------------------------------------------------
template <int TW, int TH>
struct TileGeom {
    static constexpr int BW = TW + 32;  // box width: x from x0-16, 16-byte aligned
    static constexpr int BH = TH + 8;   // box height: y from y0-4
    static constexpr int BOX = BW * BH;
    static constexpr int SW = TW + 2;   // score tile with a 1-pixel ring
    static constexpr int SH = TH + 2;
    static constexpr int IMG_OFF = 0;
    static constexpr int SC_OFF = (BOX + 127) / 128 * 128;
    static constexpr int SMEM = SC_OFF + SW * SH * 2 + 128;  // +128: base alignment slack
    static_assert(TW % 16 == 0 && BW <= 256 && BH <= 256, "TMA box limits");
};

template <int TW, int TH, int MODE>
__global__ void __launch_bounds__(256) fast_nms_cell_kernel(
    const CallHeader* __restrict__ hdr, const FrameDesc* __restrict__ fds,
    const CUtensorMap* __restrict__ maps0, const CUtensorMap* __restrict__ mapsk,
    const WorkItem* __restrict__ items, int32_t* __restrict__ counter, uint32_t* __restrict__ status) {
    using G = TileGeom<TW, TH>;
    extern __shared__ __align__(128) uint8_t smem_raw[];
    __shared__ uint64_t bar;
    __shared__ int32_t item_sh;
    // TMA destinations must be 128-byte aligned
    uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~uintptr_t(127));
    uint8_t* img = smem + G::IMG_OFF;
    uint16_t* sc = reinterpret_cast<uint16_t*>(smem + G::SC_OFF);

    const int tid = threadIdx.x;
    if (tid == 0) {
        mbar_init(&bar, 1);
        fence_barrier_init();
    }
    __syncthreads();
    const int n_items = hdr->n_items;
    const int thresh = hdr->thresh, n_arc = hdr->arc, cell = hdr->cell;
    uint32_t phase = 0;

    for (;;) {
        if (tid == 0) item_sh = atomicAdd(counter, 1);
        __syncthreads();
        const int it = item_sh;
        if (it >= n_items) break;
        const WorkItem wi = items[it];
        const FrameDesc& fd = fds[wi.frame];
        const int k = wi.level;
        const int Wk = fd.w >> k, Hk = fd.h >> k;
        const int x0 = wi.tx * TW, y0 = wi.ty * TH;
        if (tid == 0) {
            const CUtensorMap* map = k == 0 ? &maps0[wi.frame] : &mapsk[wi.frame * (kMaxLevels - 1) + k - 1];
            fence_tensormap_acquire(map);
            mbar_arrive_expect_tx(&bar, G::BOX);
            tma_load_2d(img, map, &bar, x0 - 16, y0 - 4);
        }
        const bool ok = mbar_wait_bounded(&bar, phase, kWaitLimitNs);
        phase ^= 1u;
        if (!__syncthreads_and(ok)) {
            if (tid == 0) atomicOr(status, kStatusTimeout);
            return;
        }
        // scores of the tile plus a 1-pixel ring
        for (int i = tid; i < G::SW * G::SH; i += blockDim.x) {
            const int sy = i / G::SW, sx = i - sy * G::SW;
            const int x = x0 - 1 + sx, y = y0 - 1 + sy;
            uint32_t s = 0;
            if (x >= 3 && y >= 3 && x < Wk - 3 && y < Hk - 3)
                s = fast_score<MODE>(img + (sy + 3) * G::BW + (sx + 15), G::BW, thresh, n_arc);
            sc[i] = (uint16_t)s;
        }
        __syncthreads();
        // 3x3 NMS and cell maximum
        for (int i = tid; i < TW * TH; i += blockDim.x) {
            const int oy = i / TW, ox = i - oy * TW;
            const uint16_t* q = sc + (oy + 1) * G::SW + (ox + 1);
            const uint32_t s = q[0];
            if (s == 0) continue;
            const bool keep = s >= q[-G::SW - 1] && s >= q[-G::SW] && s >= q[-G::SW + 1] && s >= q[-1] &&
                              s >= q[1] && s >= q[G::SW - 1] && s >= q[G::SW] && s >= q[G::SW + 1];
            if (!keep) continue;
            const int x = x0 + ox, y = y0 + oy;
            const uint32_t lin = ((uint32_t)k << 28) | (uint32_t)(y * Wk + x);
            const uint64_t key = ((uint64_t)s << 32) | (uint64_t)(0xFFFFFFFFu - lin);
            const int cx = (x << k) / cell, cy = (y << k) / cell;
            atomicMax(reinterpret_cast<unsigned long long*>(&fd.keys[cy * fd.gw + cx]),
                      (unsigned long long)key);
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// Decode: one CTA per frame turns keys into records, counts non-empty cells
// and clears the keys (and the work counter) for the next call.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) decode_kernel(const CallHeader* __restrict__ hdr,
                                                     const FrameDesc* __restrict__ fds,
                                                     int32_t* __restrict__ counter) {
    const FrameDesc& fd = fds[blockIdx.x];
    const int ncell = fd.gw * fd.gh;
    int cnt = 0;
    for (int i = threadIdx.x; i < ncell; i += blockDim.x) {
        const uint64_t key = fd.keys[i];
        int4 rec = make_int4(-1, -1, -1, 0);
        if (key != 0) {
            const uint32_t lin = 0xFFFFFFFFu - (uint32_t)key;
            const int k = (int)(lin >> 28);
            const uint32_t idx = lin & 0x0FFFFFFFu;
            const uint32_t wk = (uint32_t)(fd.w >> k);
            const int y = (int)(idx / wk), x = (int)(idx - (uint32_t)y * wk);
            rec = make_int4(x << k, y << k, k, (int)(key >> 32));
            fd.keys[i] = 0;
            ++cnt;
        }
        fd.out[i] = rec;
    }
    cnt = __reduce_add_sync(0xFFFFFFFFu, cnt);
    __shared__ int part[8];
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = cnt;
    __syncthreads();
    if (threadIdx.x == 0) {
        int t = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += part[w];
        if (hdr->counts) hdr->counts[blockIdx.x] = t;
        if (blockIdx.x == 0) *counter = 0;
    }
}

}  // namespace vio
