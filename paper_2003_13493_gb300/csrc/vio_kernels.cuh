// Device code: pyramid half-sampling, the fused FAST + NMS + cell-max kernel
// (3x3 to 9x9 NMS windows, scores SAD-B / SAD-A / MT), and the cell decode.
// All arithmetic is integer.
#pragma once
#include <cuda.h>
#include <stdint.h>

#include "ptx.cuh"

namespace vio {

constexpr int kMaxLevels = 5;
constexpr int kPrefixCache = 1025;  // prefix-table entries a kernel copies to shared memory (1024 frames)
constexpr uint32_t kStatusTimeout = 1u;  // a bounded wait gave up
constexpr uint32_t kStatusBadKey = 2u;   // a decoded cell key lies outside its cell
constexpr uint32_t kStatusBounds = 4u;   // checked build: an index left its buffer

// Index checks of the checked build (compiled with -DVIO_CHECKED): a failed
// check records kStatusBounds and the access is skipped.  In the normal
// build every check is `true` and compiles away.
__device__ __forceinline__ bool vio_guard(bool in_bounds, uint32_t* status) {
#ifdef VIO_CHECKED
    if (!in_bounds && status) atomicOr(status, kStatusBounds);
    return in_bounds;
#else
    (void)in_bounds;
    (void)status;
    return true;
#endif
}
constexpr uint64_t kWaitLimitNs = 1000000000ull;  // 1 s per bounded wait

// Per-frame descriptor, rewritten by the host for every call.
struct FrameDesc {
    int32_t w, h;          // level-0 size
    int32_t gw, gh;        // cell grid
    int32_t pyr_bx;        // pyramid thread blocks along x
    int32_t src0_pitch;    // row pitch of src0
    uint64_t* keys;        // gw * gh packed cell keys (0 = empty)
    int4* out;             // gw * gh output records (device or device-mapped host memory)
    const uint8_t* src0;   // non-null: level 0 is read from here (device-mapped host
                           // memory) by the pyramid kernel, which also writes it to lev[0]
    uint8_t* lev[kMaxLevels];   // level 0 is the caller's frame (read only)
    int32_t pitch[kMaxLevels];
    uint32_t pyr_magic;    // ceil(2^31 / pyr_bx): block row = umulhi(2 * block, pyr_magic), exact below 2^16
    int32_t pad1[2];
};

// Everything one call needs is uploaded as one contiguous block; this header
// sits at its start and holds the byte offsets of the other sections:
//   FrameDesc fds[n]
//   CUtensorMap maps0[n]                    level 0 (the caller's frames)
//   CUtensorMap mapsk[n][kMaxLevels - 1]    levels 1.. (resident pyramid)
//   int32 tiles[n * levels + 1]             prefix sums of tiles, coarsest
//                                           level first: entry (L-1-k)*n + f
//   int32 blocks[n + 1]                     prefix sums of pyramid blocks
//   int32 cells[n + 1]                      prefix sums of cells per frame
struct CallHeader {
    int32_t thresh, arc, n_frames, levels;
    int32_t cell, n_items, n_pyr_blocks, tile_h;
    int32_t* counts;       // device int32[n_frames] or nullptr
    uint32_t off_fds, off_maps0, off_mapsk, off_tiles, off_blocks, off_cells;
    // cell_magic[k] = ceil(2^32 / (cell >> k)): for level coordinates
    // x < 2^16, umulhi(x, magic) == x / (cell >> k) == (x << k) / cell exactly
    uint32_t cell_magic[kMaxLevels];
    int32_t n_cells;       // cells of all frames
    uint32_t* status;      // device-visible status word for the decode's checks, or nullptr
};

struct CallView {
    const CallHeader* h;
    const FrameDesc* fds;
    const CUtensorMap* maps0;
    const CUtensorMap* mapsk;
    const int32_t* tiles;
    const int32_t* blocks;
    const int32_t* cells;
    __device__ __forceinline__ explicit CallView(const uint8_t* call)
        : h(reinterpret_cast<const CallHeader*>(call)),
          fds(reinterpret_cast<const FrameDesc*>(call + h->off_fds)),
          maps0(reinterpret_cast<const CUtensorMap*>(call + h->off_maps0)),
          mapsk(reinterpret_cast<const CUtensorMap*>(call + h->off_mapsk)),
          tiles(reinterpret_cast<const int32_t*>(call + h->off_tiles)),
          blocks(reinterpret_cast<const int32_t*>(call + h->off_blocks)),
          cells(reinterpret_cast<const int32_t*>(call + h->off_cells)) {}
};

// Largest i in [0, n) with a[i] <= v, for a non-decreasing a with a[0] <= v.
__device__ __forceinline__ int upper_index(const int32_t* a, int n, int v) {
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (a[mid] <= v) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// ---------------------------------------------------------------------------
// Pyramid: one thread owns 16 columns x B rows of level 0 (B = 2^(L-1)) and
// writes every pixel of levels 1..L-1 that block produces.  Level k+1 is the
// 2x2 mean of level k rounded half up, (a+b+c+d+2)>>2, taken from the
// rounded level-k values.  Level 0 is read with 16-byte loads; level 1 is
// computed two pixels per 32-bit word (16-bit lanes) and stored 8 bytes at a
// time; level 2 adds those words of two rows lane-wise and is stored 4 bytes
// at a time; levels 3 and 4, a sixteenth of the work and less, are scalar.
// A CTA covers 512 columns x 8B rows; the grid strides over all CTAs of all
// frames (blocks[] is the per-frame prefix sum).
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t pair_sums(uint32_t w) {  // [w0+w1, w2+w3] in 16-bit lanes
    return (w & 0x00FF00FFu) + __byte_perm(w, 0u, 0x4341);   // bytes 1 and 3 into the low halves
}

template <int L>
__global__ void __launch_bounds__(256) pyramid_kernel(const uint8_t* __restrict__ call) {
    constexpr int B = 1 << (L - 1);
    constexpr int B1 = B / 2;
    griddep_launch_dependents();
    const CallView cv(call);
    const int nf = cv.h->n_frames, nb = cv.h->n_pyr_blocks;
    // the block prefix sums, searched once per block by every thread: in
    // shared memory when they fit (a search of the global table is a chain of
    // dependent loads)
    __shared__ int32_t blocks_sh[kPrefixCache];
    const int32_t* blocks = nf < kPrefixCache ? blocks_sh : cv.blocks;
    if (nf < kPrefixCache)
        for (int i = threadIdx.x; i <= nf; i += blockDim.x) blocks_sh[i] = cv.blocks[i];
    __syncthreads();
    for (int b = blockIdx.x; b < nb; b += gridDim.x) {
        const int f = upper_index(blocks, nf, b);
        const FrameDesc& fd = cv.fds[f];
        const int lb = b - blocks[f];
        const int brow = (int)__umulhi(2u * (uint32_t)lb, fd.pyr_magic);
        const int tx = (lb - brow * fd.pyr_bx) * 32 + (threadIdx.x & 31);
        const int ty = brow * 8 + (threadIdx.x >> 5);
        const int W = fd.w, H = fd.h;
        const int x0 = tx * 16, y0 = ty * B;
        if (x0 >= W || y0 >= H) continue;
        const int W1 = W >> 1, H1 = H >> 1;
        // level 0 comes from the frame itself or, when the frame sits in
        // host memory, from its device mapping; then this kernel is also the
        // upload and writes the rows it reads to the device copy of level 0
        const bool upload = fd.src0 != nullptr;
        const uint8_t* src = upload ? fd.src0 : fd.lev[0];
        const int sp = upload ? fd.src0_pitch : fd.pitch[0];
        // level 0 rows; the last partial chunk of a row is read byte by byte
        uint4 r[B];
#pragma unroll
        for (int j = 0; j < B; ++j) {
            const int y = y0 + j;
            r[j] = make_uint4(0, 0, 0, 0);
            if (y < H) {
                const uint8_t* p = src + (size_t)y * sp + x0;
                uint8_t* d = fd.lev[0] + (size_t)y * fd.pitch[0] + x0;
                if (x0 + 16 <= W) {
                    r[j] = *reinterpret_cast<const uint4*>(p);
                    if (upload) *reinterpret_cast<uint4*>(d) = r[j];
                } else {
                    uint32_t wv[4] = {0, 0, 0, 0};
                    for (int i = 0; i < W - x0; ++i) {
                        const uint8_t b = p[i];
                        wv[i >> 2] |= (uint32_t)b << (8 * (i & 3));
                        if (upload) d[i] = b;
                    }
                    r[j] = make_uint4(wv[0], wv[1], wv[2], wv[3]);
                }
            }
        }
        // level 1: 8 pixels per row as 4 words of two 16-bit lanes
        uint32_t q[B1][4];
#pragma unroll
        for (int j = 0; j < B1; ++j) {
            const uint32_t t[4] = {r[2 * j].x, r[2 * j].y, r[2 * j].z, r[2 * j].w};
            const uint32_t u[4] = {r[2 * j + 1].x, r[2 * j + 1].y, r[2 * j + 1].z, r[2 * j + 1].w};
#pragma unroll
            for (int w = 0; w < 4; ++w)
                q[j][w] = ((pair_sums(t[w]) + pair_sums(u[w]) + 0x00020002u) >> 2) & 0x00FF00FFu;
            const int y1 = ty * B1 + j, x1 = tx * 8;
            if (y1 < H1 && x1 < W1) {
                // pixels past W1 land in the row padding of the resident level (pitch >= W1 rounded to 128)
                const uint2 v = make_uint2(__byte_perm(q[j][0], q[j][1], 0x6420), __byte_perm(q[j][2], q[j][3], 0x6420));
                *reinterpret_cast<uint2*>(fd.lev[1] + (size_t)y1 * fd.pitch[1] + x1) = v;
            }
        }
        if constexpr (L > 2) {
            // level 2, 4 pixels per thread and row: the two level-1 rows of a
            // pair added lane-wise, then the two lanes of each word
            constexpr int B2 = B1 / 2;
            uint32_t p2[B2][4];
#pragma unroll
            for (int j = 0; j < B2; ++j) {
#pragma unroll
                for (int w = 0; w < 4; ++w) {
                    const uint32_t sum = q[2 * j][w] + q[2 * j + 1][w];
                    p2[j][w] = ((sum & 0xFFFFu) + (sum >> 16) + 2u) >> 2;
                }
                const int y2 = ty * B2 + j, x2 = tx * 4;
                // pixels past W2 land in the row padding (pitch >= W2 rounded to 128)
                if (y2 < (H >> 2) && x2 < (W >> 2))
                    *reinterpret_cast<uint32_t*>(fd.lev[2] + (size_t)y2 * fd.pitch[2] + x2) =
                        p2[j][0] | (p2[j][1] << 8) | (p2[j][2] << 16) | (p2[j][3] << 24);
            }
            if constexpr (L > 3) {
                // levels 3.. as scalars from the rounded level-2 values
                constexpr int N2 = 4;
                uint32_t v[B2][N2];
#pragma unroll
                for (int j = 0; j < B2; ++j)
#pragma unroll
                    for (int i = 0; i < N2; ++i) v[j][i] = p2[j][i];
                int Wk = W >> 2, Hk = H >> 2, rows = B2, cols = N2;
#pragma unroll
                for (int k = 3; k < L; ++k) {
                    rows >>= 1;
                    cols >>= 1;
                    Wk >>= 1;
                    Hk >>= 1;
                    uint8_t* dst = fd.lev[k];
                    const int dp = fd.pitch[k];
#pragma unroll
                    for (int j = 0; j < B2; ++j)
#pragma unroll
                        for (int i = 0; i < N2; ++i)
                            if (j < rows && i < cols) {
                                const uint32_t sum = v[2 * j][2 * i] + v[2 * j][2 * i + 1] + v[2 * j + 1][2 * i] +
                                                     v[2 * j + 1][2 * i + 1] + 2u;
                                v[j][i] = sum >> 2;
                                const int xk = tx * cols + i, yk = ty * rows + j;
                                if (xk < Wk && yk < Hk) dst[(size_t)yk * dp + xk] = (uint8_t)v[j][i];
                            }
                }
            }
        }
    }
}

// ---------------------------------------------------------------------------
// FAST segment test and scores on a shared-memory tile.
// ---------------------------------------------------------------------------

// Radius-3 Bresenham circle, clockwise from the top (Section II-D).
__host__ __device__ constexpr int circ_dx(int i) {
    return i == 0 ? 0 : i == 1 ? 1 : i == 2 ? 2 : i <= 5 ? 3 : i == 6 ? 2 : i == 7 ? 1 : i == 8 ? 0
         : i == 9 ? -1 : i == 10 ? -2 : i <= 13 ? -3 : i == 14 ? -2 : -1;
}
__host__ __device__ constexpr int circ_dy(int i) {
    return i <= 1 ? -3 : i == 2 ? -2 : i == 3 ? -1 : i == 4 ? 0 : i == 5 ? 1 : i == 6 ? 2 : i <= 9 ? 3
         : i == 10 ? 2 : i == 11 ? 1 : i == 12 ? 0 : i == 13 ? -1 : i == 14 ? -2 : -3;
}

// Start positions s (bits 0..15) of cyclic runs of >= n ones in the 16-bit
// mask m: the mask is doubled to 32 bits (a rotation without wrap-around),
// runs of 8 come from three AND-shift doublings and the run of n from two
// overlapping runs of 8 that are n-8 apart.
__device__ __forceinline__ uint32_t arc_starts(uint32_t m, int n) {
    uint32_t r = m * 0x10001u;
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

// [sign(a byte 1), sign(a byte 3), sign(b byte 1), sign(b byte 3)]: each result
// byte is 0xFF when the bit 15 / bit 31 it is taken from is set, else 0x00
// (the PTX byte permute with the sign-replicate bit set in every selector).
__device__ __forceinline__ uint32_t prmt_sign_flags(uint32_t a, uint32_t b) {
    uint32_t d;
    asm("prmt.b32 %0, %1, %2, 0xFDB9;" : "=r"(d) : "r"(a), "r"(b));
    return d;
}

// Four bytes packed into one word, byte 0 first.
__device__ __forceinline__ uint32_t pack4(uint32_t a, uint32_t b, uint32_t c, uint32_t d) {
    return __byte_perm(__byte_perm(a, b, 0x0040), __byte_perm(c, d, 0x0040), 0x5410);
}

// 16-bit-lane minimum and maximum on the DPX unit.
__device__ __forceinline__ uint32_t min16x2(uint32_t a, uint32_t b) { return __vimin3_u16x2(a, b, b); }

// Window minima of the circle's signed differences (the sweep's full test,
// the MT score).  D[i] holds point i's biased
// differences, v - c + 256 in the low 16-bit lane (brighter) and c - v + 256
// in the high lane (darker), both in 1..511 so no lane borrows; W8[i] is the
// lane-wise minimum over points i .. i+7 (cyclic), from minima of three.
__device__ __forceinline__ void window_minima8_of(const uint32_t (&v)[16], uint32_t c, uint32_t (&W8)[16]) {
    const uint32_t K = (256u - c) | ((256u + c) << 16);
    uint32_t D[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) D[i] = K + v[i] * 0xFFFF0001u;
    uint32_t W3[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) W3[i] = __vimin3_u16x2(D[i], D[(i + 1) & 15], D[(i + 2) & 15]);
#pragma unroll
    for (int i = 0; i < 16; ++i) W8[i] = __vimin3_u16x2(W3[i], W3[(i + 3) & 15], W3[(i + 5) & 15]);
}

// p: the candidate in a tile of row pitch PITCH bytes.
template <int PITCH>
__device__ __forceinline__ void window_minima8(const uint8_t* __restrict__ p, uint32_t (&W8)[16]) {
    uint32_t v[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = p[circ_dy(i) * PITCH + circ_dx(i)];
    window_minima8_of(v, p[0], W8);
}

// Largest minimum over the 16 windows of 8 + R points (both polarities),
// still biased by 256: the candidate is a corner at threshold t for arc
// length 8 + R exactly when the result is >= t + 257.  A window of 8 + R
// points is two overlapping windows of 8, R apart.
template <int R>
__device__ __forceinline__ uint32_t best_window_min(const uint32_t (&W8)[16]) {
    uint32_t m[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) m[i] = min16x2(W8[i], W8[(i + R) & 15]);
    uint32_t b = __vimax3_u16x2(m[0], m[1], m[2]);
    b = __vimax3_u16x2(b, m[3], m[4]);
    b = __vimax3_u16x2(b, m[5], m[6]);
    b = __vimax3_u16x2(b, m[7], m[8]);
    b = __vimax3_u16x2(b, m[9], m[10]);
    b = __vimax3_u16x2(b, m[11], m[12]);
    b = __vimax3_u16x2(b, m[13], m[14]);
    b = __vimax3_u16x2(b, m[15], m[15]);
    return max(b & 0xFFFFu, b >> 16);
}

__device__ __forceinline__ uint32_t best_window_min_for_arc(const uint32_t (&W8)[16], int n) {
    switch (n) {  // uniform over the launch
        case 9: return best_window_min<1>(W8);
        case 10: return best_window_min<2>(W8);
        case 11: return best_window_min<3>(W8);
        case 12: return best_window_min<4>(W8);
        case 13: return best_window_min<5>(W8);
        case 14: return best_window_min<6>(W8);
        case 15: return best_window_min<7>(W8);
        default: return best_window_min<8>(W8);
    }
}

// Full segment test and score of the pixel at shared-memory pointer p in a
// tile of row pitch P (compile time).  Returns 0 when it is not a corner.
//
// Eq. 1 labels come from one IMAD per circle point: with
//   W = ((0x7FFF - c - t) | (0x7FFF + c - t) << 16) + v * (1 - 2^16)
// the low 16-bit lane is v + 0x7FFF - (c + t), whose bit 15 is set exactly
// when v > c + t (brighter), and the high lane is 0x7FFF + (c - t) - v,
// whose bit 31 is set exactly when v < c - t (darker).  Neither lane leaves
// its 16 bits, so the two compares are exact for all v, c in 0..255 and
// t in 0..255.  The flags become masks in two steps: a byte permute with
// sign replication turns the flag bits (bits 15 and 31 are the sign bits of
// bytes 1 and 3) of points i and i + 8 into four 0x00 / 0xFF bytes
// [bright_i, dark_i, bright_i+8, dark_i+8]; keeping bit i of each byte and
// OR-ing the eight words gives bright 0..7, dark 0..7, bright 8..15 and
// dark 8..15 in bytes 0..3; a last permute orders them as the 16-bit bright
// mask in bits 0..15 and the dark mask in bits 16..31, bit i = point i.
template <int MODE, int P, bool SCORE = true>
__device__ __forceinline__ uint32_t eval_corner(const uint8_t* __restrict__ p, int t, int n) {
    const uint32_t c = p[0];
    uint32_t v[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = p[circ_dy(i) * P + circ_dx(i)];
    const uint32_t K = ((0x7FFFu - c - (uint32_t)t) & 0xFFFFu) | ((0x7FFFu + c - (uint32_t)t) << 16);
    uint32_t w[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) w[i] = K + v[i] * 0xFFFF0001u;
    uint32_t bytes = 0;
#pragma unroll
    for (int i = 0; i < 8; ++i) bytes |= prmt_sign_flags(w[i], w[i + 8]) & (0x01010101u << i);
    const uint32_t acc = __byte_perm(bytes, 0u, 0x3120);
    const uint32_t bm = acc & 0xFFFFu, dm = acc >> 16;
    // at most one polarity can hold n >= 9 points
    const bool bright = __popc(bm) >= n;
    const uint32_t starts = arc_starts(bright ? bm : dm, n);
    if (starts == 0) return 0;
    if (!SCORE) return 1;
    if (MODE == 0) {  // SAD-B: sum of |I_x - I_c| over the circle
        const uint32_t c4 = c * 0x01010101u;
        uint32_t s = __vsadu4(pack4(v[0], v[1], v[2], v[3]), c4);
        s += __vsadu4(pack4(v[4], v[5], v[6], v[7]), c4);
        s += __vsadu4(pack4(v[8], v[9], v[10], v[11]), c4);
        s += __vsadu4(pack4(v[12], v[13], v[14], v[15]), c4);
        return s;
    } else if (MODE == 1) {  // SAD-A: the run is the union of all passing windows
        uint32_t d = starts;
        d |= rotl16(d, 1);
        d |= rotl16(d, 2);
        d |= rotl16(d, 4);  // windows of 8 starting at each start
        const uint32_t run = d | rotl16(d, n - 8);
        // SAD over the run: each nibble of the run mask spreads to a byte
        // mask of its four circle points (bit i -> bit 8i by one multiply;
        // the shifted copies occupy disjoint bits, so nothing carries)
        const uint32_t c4 = c * 0x01010101u;
        uint32_t s = 0;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const uint32_t m = (((run >> (4 * q)) & 0xFu) * 0x00204081u & 0x01010101u) * 0xFFu;
            s += __vsadu4(pack4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]) & m, c4 & m);
        }
        return s;
    } else {  // MT: the largest t at which the pixel is still a corner
        // = the largest minimum over all windows of n points of the signed
        // differences, minus 1 (both polarities at once: the one that is not
        // the corner's has no window above 0, as no pixel holds arcs of 9 of
        // both polarities); biased by 256
        uint32_t W8[16];
        window_minima8_of(v, c, W8);
        return best_window_min_for_arc(W8, n) - 257u;
    }
}

// MT score of a pixel already known to be a corner for arc length n: the
// largest minimum over the windows of n signed differences, minus 1 (biased
// by 256 as in eval_corner).
template <int P>
__device__ __forceinline__ uint32_t mt_of_corner(const uint8_t* __restrict__ p, int n) {
    uint32_t W8[16];
    window_minima8<P>(p, W8);
    return best_window_min_for_arc(W8, n) - 257u;
}

// SAD-B of the pixel at p (row pitch P): sum of |I_x - I_c| over the circle.
template <int P>
__device__ __forceinline__ uint32_t sad_b(const uint8_t* __restrict__ p) {
    const uint32_t c4 = p[0] * 0x01010101u;
    uint32_t v[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = p[circ_dy(i) * P + circ_dx(i)];
    uint32_t s = __vsadu4(pack4(v[0], v[1], v[2], v[3]), c4);
    s += __vsadu4(pack4(v[4], v[5], v[6], v[7]), c4);
    s += __vsadu4(pack4(v[8], v[9], v[10], v[11]), c4);
    s += __vsadu4(pack4(v[12], v[13], v[14], v[15]), c4);
    return s;
}

// Byte-wise |a - b| > t for the 4 pixels of a word, without carries between
// bytes: with k7 = 127 - t (t < 128), (d & 0x7F) + k7 carries into bit 7 iff
// (d & 0x7F) > t, and a set bit 7 of d alone means d >= 128 > t; with
// k7 = 255 - t (t >= 128) the carry means (d & 0x7F) > t - 128, which counts
// only together with bit 7 of d.  The flags are bit 7 of each byte; the
// other bits are left over and cleared by the caller.
template <bool HIGH_T>
__device__ __forceinline__ uint32_t gt_flags(uint32_t a, uint32_t b, uint32_t k7) {
    const uint32_t d = __vabsdiffu4(a, b);
    const uint32_t f = (d & 0x7F7F7F7Fu) + k7;
    return HIGH_T ? (f & d) : (f | d);
}

// ---------------------------------------------------------------------------
// Fused detect: persistent CTAs pull (frame, level, tile) items from a
// counter.  A tile is 120 x TH level pixels; its "score region" adds a ring
// (4 px left and right, R rows up and down for an NMS radius R) so that it is
// exactly 128 pixels wide: lane l owns the 4-pixel word of columns 4l..4l+3
// of every row, and each of the 8 consumer warps owns a band of consecutive
// rows.
// Per item:
//   1. The producer (one thread) claims the item, computes its constants
//      and TMA loads the region plus the 3-pixel circle halo (box 144 x
//      TH+2R+6) into one of two image buffers; the other buffer is loading
//      the next item meanwhile.
//   2. Coarse test on every score-region pixel of the warp's band, 4 pixels
//      per lane (the 8-point rule for arcs n <= 11 and R <= 2, else the
//      compass rule), pixels outside the testable area masked off; one warp
//      scan places each lane's kept pixels in the warp's queue, written by a
//      two-ended bit walk as raw codes (coarse_and_compact).
//   3. Each warp runs the full segment test on its queue and compacts the
//      corners in place, then scores the corners and writes the scores into
//      the score tile.
//   4. Once its two neighbouring warps have written their scores (the NMS
//      reads up to R rows of theirs; per-warp mbarriers, see neighbours_wait),
//      (2R+1)x(2R+1) NMS on the corner list (for R > 1 the nearest ring
//      first, the outer rings on its survivors); each survivor folds its
//      packed key into the global cell key with a 64-bit max reduction.
// ---------------------------------------------------------------------------
constexpr int kTileW = 120;  // output pixels per tile row, every variant

template <int TH, int R = 1>
struct TileGeom {
    static constexpr int TW = kTileW;      // output pixels per tile row
    static constexpr int SW = 128;         // score-region width (x0-4 .. x0+124)
    static constexpr int SR = TH + 2 * R;  // score-region rows (y0-R .. y0+TH+R): NMS radius R
    static constexpr int BW = 144;         // TMA box width (16-byte multiple)
    static constexpr int BH = SR + 6;      // box rows y0-R-3 .. y0+TH+R+3
    static constexpr int BOX = BW * BH;
    static constexpr int BOXA = (BOX + 127) / 128 * 128;
    static constexpr int WARPS = 8;
    static constexpr int PPW = SR / 2 / WARPS;  // row pairs per warp
    static constexpr int QCAP = PPW * 2 * SW;   // per-warp queue capacity (every pixel)
    static constexpr int NBUF = 2;              // image buffers in the TMA ring
    static constexpr int IMG_OFF = 0;
    static constexpr int SC_OFF = NBUF * BOXA;
    static constexpr int Q_OFF = SC_OFF + SR * SW * 2;
    static constexpr int SMEM = Q_OFF + WARPS * QCAP * 2 + 128;  // +128: base alignment slack
    static_assert(SR % (2 * WARPS) == 0, "row pairs must split evenly over the warps");
    static_assert(BH <= 256, "TMA box limit");
    static_assert(R >= 1 && R <= 4, "the 4-pixel column ring holds NMS radii up to 4");
};

constexpr int kConsumers = 256;             // 8 warps that detect
constexpr int kThreads = kConsumers + 32;   // + 1 producer warp (items, TMA)

// A work item decoded from its index: item i of the call's tile table.
struct Item {
    int frame, level, tx, ty;
};

// What the consumers need of an item, written by the producer next to the
// image buffer it fills.
struct ItemInfo {
    int32_t id;            // item index; >= n_items ends the consumers' loop
    int32_t level, x0, y0;
    int32_t wk, hk, gw, gh;
    uint32_t magic;                    // cell magic of the level
    int32_t xoff;                      // box column of score column 0
    int32_t row_lo, row_hi, xlo, xhi;  // testable score rows, kept score columns
    uint64_t* keys;
};

// Item i of the call's tile table: entry j = (L-1-k)*n + f (coarsest level first).
__device__ __forceinline__ Item decode_item(const CallView& cv, const int32_t* tiles, int it) {
    const int n = cv.h->n_frames, L = cv.h->levels;
    const int j = upper_index(tiles, n * L, it);
    Item r;
    r.frame = j % n;
    r.level = L - 1 - j / n;
    const int t = it - tiles[j];
    const int wk = cv.fds[r.frame].w >> r.level;
    const int ntx = (wk + kTileW - 1) / kTileW;
    r.ty = t / ntx;
    r.tx = t - r.ty * ntx;
    return r;
}

// Score-region index of a raw walk code (w << 10 | lane << 5 | bit b) of the
// warp whose rows start at r0: row r0 + 8w + (b & 7), column 4 lane + (b >> 3);
// (code >> 3) & 0x7F is that column, (code >> 7) & ~7 is 8w.
__device__ __forceinline__ int walk_code_index(uint32_t code, int r0) {
    return (int)(((uint32_t)r0 + (code & 7u) + ((code >> 7) & ~7u)) << 7) + (int)((code >> 3) & 0x7Fu);
}

// bits 7, 15, 23, 31 -> bits 28..31: the product's other terms stay below bit 28
__device__ __forceinline__ uint32_t nibble(uint32_t keep) { return (keep * 0x00204081u) >> 28; }

// Coarse test (the CCRF of Algorithm 1) over this warp's score rows,
// appending the kept pixels (score-region index row * 128 + column) to the
// warp's queue; returns the queue length.
//
// Warp w owns the 2*PPW score rows starting at r0 = 2*PPW*w; lane l owns the
// 4-pixel word of score columns 4l .. 4l+3 in every one of them, so a row is
// one conflict-free 128-byte read per warp.  The rule: an arc of n >= 9
// contiguous points contains floor(n/4) >= 2 cyclically consecutive compass
// points (0, 4, 8, 12), all darker or all brighter and so all with
// |I_x - I_c| > t; a pixel is kept when two adjacent compass points (n <= 11)
// or three of the four (n >= 12) differ from the centre by more than t.  With
// EIGHT (n <= 11, NMS radius <= 2) the stronger rule on the eight even
// circle points (compass points and the (+-2, +-2) diagonals) applies: an arc
// of n >= 9 holds floor(n/2) >= 4 cyclically consecutive even points, so a
// pixel is kept when four consecutive of the eight differ by more than t.
// Neither rule drops a corner.
//
// Each comparison is made once and serves two pixels: rows y and y+3 of a
// column give the S flag of row y and the N flag of row y+3; columns x and
// x+3 of a row give the E flag of x and the W flag of x+3 (the W flags of a
// word come from the E flags of the word to its left, a lane shuffle away);
// likewise (x, y)-(x+2, y+2) is SE of the first and NW of the second, and
// (x, y)-(x-2, y+2) is SW of the first and NE of the second.  The shuffles
// leave the outermost columns of lanes 0 and 31 without the left or right
// neighbour word; those columns are outside the NMS region for radius 1
// (lane 0's W flags of columns 0..2) and radius <= 2 (the diagonal flags of
// columns 0, 1, 126, 127), so a radius of 2 reads the left word for its W
// flags and radii >= 3 use the compass rule on every level.
//
// The kept-pixel bits of a lane gather in 32-bit words, eight rows per
// word (bit 8j + i of word w = row r0 + 8w + i, column 4l + j: each row's
// flags, bit 7 of each byte, enter at the top and move down one bit per
// row); one warp scan of the popcounts places each lane's run in the queue,
// and each lane writes its pixels by walking its set bits, from both ends
// at once, as raw codes.  (Spreading the
// bits over the warp first, by a skewed bit transpose, balances the walk but
// scatters the queue, and the full test's circle reads then conflict in
// shared memory: slower.)
// vm: bit 7 of byte j set when column 4l + j is inside the columns NMS reads.
template <bool HIGH_T, bool THREE, int TH, int R, bool EIGHT = false>
__device__ __forceinline__ int coarse_and_compact(const uint8_t* img, uint16_t* queue, int xw, uint32_t k7,
                                                  int warp, int lane, int row_lo, int row_hi, uint32_t vm,
                                                  uint32_t* status = nullptr) {
    using G = TileGeom<TH, R>;
    constexpr int RW = G::BW / 4;      // words per box row
    constexpr int RPW = 2 * G::PPW;    // score rows per warp
    constexpr int NW = (4 * RPW + 31) / 32;  // mask words per lane
    static_assert(!EIGHT || R <= 2, "the diagonal flags of the edge lanes cover NMS radii <= 2");
    constexpr uint32_t kFull = 0xFFFFFFFFu;
    const int r0 = RPW * warp;
    // this lane's word in box row r0 (score row r is box row r + 3)
    const uint32_t* col = reinterpret_cast<const uint32_t*>(img) + r0 * RW + xw + lane;
    uint32_t m[NW];
#pragma unroll
    for (int w = 0; w < NW; ++w) m[w] = 0u;
    // One pass down the rows: step jj reads box row r0 + jj (C[jj]), forms
    // the comparisons that row completes, and emits score row i = jj - 6,
    // whose flags are then all known:
    //   Dv[j]: box rows j and j + 3 (S flags of box row j, N flags of j + 3);
    //   D1[j] / D2[j]: box row j against the pixels 2 right / 2 left of row
    //   j + 2 (SE / SW flags of row j, NW / NE flags of row j + 2).
    uint32_t C[RPW + 6], Dv[RPW + 3], D1[RPW + 3], D2[RPW + 3];
#pragma unroll
    for (int jj = 0; jj < RPW + 6; ++jj) {
        C[jj] = col[jj * RW];
        if (jj >= 3) Dv[jj - 3] = gt_flags<HIGH_T>(C[jj - 3], C[jj], k7);
        if (EIGHT && jj >= 3 && jj - 2 < RPW + 3) {
            const int j = jj - 2;
            const uint32_t r2 = col[jj * RW + 1];
            const uint32_t l2 = __shfl_up_sync(kFull, C[jj], 1);
            D1[j] = gt_flags<HIGH_T>(C[j], __byte_perm(C[jj], r2, 0x5432), k7);
            D2[j] = gt_flags<HIGH_T>(C[j], __byte_perm(l2, C[jj], 0x5432), k7);
        }
        if (jj < 6) continue;
        const int i = jj - 6;  // score row r0 + i is box row r0 + j
        const int j = i + 3;
        const uint32_t c = C[j];
        const uint32_t rw = col[j * RW + 1];
        // E flags of this word; W flags from the E flags of the word to the left
        const uint32_t fe = gt_flags<HIGH_T>(c, __byte_perm(c, rw, 0x6543), k7);
        uint32_t el;
        if (R == 1) {
            el = __shfl_up_sync(kFull, fe, 1);
        } else {
            const uint32_t lw = col[j * RW - 1];
            el = gt_flags<HIGH_T>(lw, __byte_perm(lw, c, 0x6543), k7);
        }
        const uint32_t fw = __byte_perm(el, fe, 0x4321);
        const uint32_t fn = Dv[i], fs = Dv[j];
        uint32_t keep;
        if (EIGHT) {
            const uint32_t fse = D1[j], fsw = D2[j];
            const uint32_t fnw = __byte_perm(__shfl_up_sync(kFull, D1[j - 2], 1), D1[j - 2], 0x5432);
            const uint32_t fne = __byte_perm(D2[j - 2], __shfl_down_sync(kFull, D2[j - 2], 1), 0x5432);
            // the 8 runs of four on the cycle N NE E SE S SW W NW, grouped by
            // their middle three around a diagonal
            const uint32_t xne = fn & fne & fe, xse = fe & fse & fs, xsw = fs & fsw & fw, xnw = fw & fnw & fn;
            keep = ((xne | xsw) & (fse | fnw)) | ((xse | xnw) & (fne | fsw));
        } else if (THREE) {  // at least 3 of 4 (any 3 of 4 cyclic positions are consecutive)
            keep = (fn & fe & (fs | fw)) | (fs & fw & (fn | fe));
        } else {             // two adjacent: (N|S) & (E|W)
            keep = (fn | fs) & (fe | fw);
        }
        // row i of word i / 8 lands in bit i % 8 of each byte after the
        // remaining shifts of that word: bit 8j + (i % 8) = row, column 4l + j
        m[i / 8] = (m[i / 8] >> 1) | (keep & 0x80808080u);
    }
    // a last word of fewer than 8 rows: its first row down to bit 0
    if (RPW % 8) m[NW - 1] >>= 8 - RPW % 8;
    // rows outside the testable area and columns outside the NMS region
    const uint32_t cols = ((vm >> 7) & 0x01010101u) * 0xFFu;
#pragma unroll
    for (int w = 0; w < NW; ++w) {
        const int lo = min(max(row_lo - r0 - 8 * w, 0), 8), hi = min(max(row_hi - r0 - 8 * w, 0), 8);
        const uint32_t rows = ((0xFFu << lo) & ~(0xFFu << hi) & 0xFFu) * 0x01010101u;
        m[w] &= rows & cols;
    }
    int cnt = 0;
#pragma unroll
    for (int w = 0; w < NW; ++w) cnt += __popc(m[w]);
    int incl = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(kFull, incl, o);
        if (lane >= o) incl += y;
    }
    int pos = incl - cnt;
    // bit b of word w stands for row r0 + 8w + (b & 7), column 4l + (b >> 3)
#pragma unroll
    for (int w = 0; w < NW; ++w) {
        uint32_t mw = m[w];
        // the highest and the lowest set bit per step: half the steps, and
        // two chains that do not depend on each other.  The queue takes the
        // raw code w << 10 | lane << 5 | bit, which the full test turns into
        // the pixel (walk_code_index): the walk is as slow as its busiest
        // lane, the full test is balanced.
        const int cbase = (w << 10) | (lane << 5);
        while (mw) {
            const int bh = 31 - __clz(mw);
            const uint32_t lowbit = mw & (0u - mw);
            const int bl = 31 - __clz(lowbit);
            const uint32_t hb = 1u << bh;
            mw &= (mw - 1u) & ~hb;
            if (vio_guard(pos < G::QCAP, status)) queue[pos] = (uint16_t)(cbase | bh);
            const bool two = lowbit != hb;
            if (two && vio_guard(pos + 1 < G::QCAP, status)) queue[pos + 1] = (uint16_t)(cbase | bl);
            pos += two ? 2 : 1;
        }
    }
    return __shfl_sync(kFull, incl, 31);
}

// Consumer warps synchronise with their neighbours only.  Warp w owns score
// rows [2*PPW*w, 2*PPW*(w+1)) and its NMS reads R <= 2*PPW rows beyond them,
// so only warps w-1 and w+1 read its rows.  Per tile t each warp arrives on
// sc_bar[w] once its scores are written and on nms_bar[w] once its NMS is
// done (one arrival per phase, phase t for tile t).  Before its NMS a warp
// waits for phase t of its neighbours' sc_bar; before writing the scores of
// tile t (its own rows only) it waits for phase t-1 of its neighbours'
// nms_bar and zeroes its rows.  A warp can thus run at most one phase ahead
// of a neighbour, which keeps the parity waits exact.  Returns false on a
// timed-out wait (status set).
__device__ __forceinline__ bool neighbours_wait(uint64_t* bars, int warp, int n_warps, uint32_t parity, int lane,
                                                uint32_t* status) {
    const bool ok = (warp == 0 || mbar_wait_bounded(&bars[warp - 1], parity, kWaitLimitNs)) &&
                    (warp == n_warps - 1 || mbar_wait_bounded(&bars[warp + 1], parity, kWaitLimitNs));
    if (!ok && lane == 0) atomicOr(status, kStatusTimeout);
    return ok;
}

// Start of a tile's score writes (see neighbours_wait).  T: the tile's
// element type (rows of G::SW elements).
template <int TH, int R, typename T>
__device__ __forceinline__ bool own_rows_reset(uint64_t* nms_bars, int t, T* tile, int warp, int lane,
                                               uint32_t* status) {
    using G = TileGeom<TH, R>;
    static_assert(2 * G::PPW * G::WARPS == G::SR, "warps own all score rows");
    static_assert(R <= 2 * G::PPW, "the NMS reads the rows of adjacent warps only");
    constexpr int N16 = 2 * G::PPW * G::SW * (int)sizeof(T) / 16;  // 16-byte words per warp
    static_assert(N16 % 32 == 0, "whole 16-byte stores per lane");
    if (t == 0) return true;  // zeroed at kernel start
    if (!neighbours_wait(nms_bars, warp, G::WARPS, (t - 1) & 1, lane, status)) return false;
    uint4* own = reinterpret_cast<uint4*>(tile + 2 * G::PPW * warp * G::SW);
#pragma unroll
    for (int j = 0; j < N16 / 32; ++j) own[lane + 32 * j] = make_uint4(0u, 0u, 0u, 0u);
    __syncwarp();
    return true;
}

// Producer of the detect kernels (one thread): claims work items from the
// counter one ahead of their use, decodes each into the tile it covers and
// issues the TMA load of the tile and its halo into the next buffer of the
// ring once the consumer warps have released it.  An item index >= n_items
// tells the consumers to stop.
template <int TH, int R>
__device__ __forceinline__ void produce_tiles(const CallView& cv, const int32_t* tiles, int32_t* counter,
                                              uint32_t* status, ItemInfo* info, uint64_t* full_bar,
                                              uint64_t* empty_bar, uint8_t* smem) {
    using G = TileGeom<TH, R>;
    constexpr int NB = G::NBUF;
    const int n_items = cv.h->n_items;
    int claimed = atomicAdd(counter, 1);
    for (int t = 0;; ++t) {
        const int b = t % NB;
        const int it = claimed;
        if (it < n_items) claimed = atomicAdd(counter, 1);
        if (t >= NB && !mbar_wait_bounded(&empty_bar[b], ((t / NB) - 1) & 1, kWaitLimitNs)) {
            atomicOr(status, kStatusTimeout);
            return;
        }
        ItemInfo& in = info[b];
        in.id = it;
        if (it >= n_items) {
            mbar_arrive(&full_bar[b]);
            return;
        }
        const Item wi = decode_item(cv, tiles, it);
        const FrameDesc& fd = cv.fds[wi.frame];
        in.level = wi.level;
        in.x0 = wi.tx * G::TW;
        in.y0 = wi.ty * TH;
        in.wk = fd.w >> wi.level;
        in.hk = fd.h >> wi.level;
        in.gw = fd.gw;
        in.gh = fd.gh;
        in.keys = fd.keys;
        // per-item constants, computed once here instead of by every
        // consumer warp: score column 0 is level x = x0 - 4 and box column
        // 0 is (x0 - 8) & ~15; score row r is level y = y0 - R + r; testable
        // pixels are 3 <= x < Wk - 3, 3 <= y < Hk - 3; the NMS reads score
        // columns 4 - R .. 123 + R only
        in.magic = cv.h->cell_magic[wi.level];
        in.xoff = in.x0 - 4 - ((in.x0 - 8) & ~15);
        in.row_lo = max(0, 3 - in.y0 + R);
        in.row_hi = min(G::SR, in.hk - 3 - in.y0 + R);
        in.xlo = max(4 - R, 7 - in.x0);
        in.xhi = min(124 + R, in.wk + 1 - in.x0);
        const CUtensorMap* map =
            wi.level == 0 ? &cv.maps0[wi.frame] : &cv.mapsk[wi.frame * (kMaxLevels - 1) + wi.level - 1];
        fence_tensormap_acquire(map);
        mbar_arrive_expect_tx(&full_bar[b], G::BOX);
        tma_load_2d(smem + G::IMG_OFF + b * G::BOXA, map, &full_bar[b], (in.x0 - 8) & ~15, in.y0 - R - 3);
    }
}

// NMS ring K around the score at q (row pitch SW): true when s is >= the
// 8K scores at Chebyshev distance K.
template <int K, int SW>
__device__ __forceinline__ bool ring_max(const uint16_t* q, uint32_t s) {
    bool ok = true;
#pragma unroll
    for (int dx = -K; dx <= K; ++dx) ok &= (s >= q[-K * SW + dx]) & (s >= q[K * SW + dx]);
#pragma unroll
    for (int dy = -K + 1; dy <= K - 1; ++dy) ok &= (s >= q[dy * SW - K]) & (s >= q[dy * SW + K]);
    return ok;
}

// One NMS pass of a wide window: keeps the corners of queue[0, n) that pass
// ring K, compacted in place; returns how many.
template <int K, int SW>
__device__ __forceinline__ int nms_ring_pass(uint16_t* queue, int n, const uint16_t* sc, int lane, uint32_t lt_mask) {
    int np = 0;
    for (int e0 = 0; e0 < n; e0 += 32) {
        const int e = e0 + lane;
        int idx = 0;
        bool ok = false;
        if (e < n) {
            idx = queue[e];
            ok = ring_max<K, SW>(sc + idx, sc[idx]);
        }
        const uint32_t bm = __ballot_sync(0xFFFFFFFFu, ok);
        if (ok) queue[np + __popc(bm & lt_mask)] = (uint16_t)idx;
        np += __popc(bm);
    }
    return np;
}

template <int TH, int MODE, int R = 1>
__global__ void __launch_bounds__(kThreads, 4) fast_nms_cell_kernel(const uint8_t* __restrict__ call,
                                                                 int32_t* __restrict__ counter,
                                                                 uint32_t* __restrict__ status) {
    using G = TileGeom<TH, R>;
    constexpr int NB = G::NBUF;
    extern __shared__ __align__(128) uint8_t smem_raw[];
    __shared__ uint64_t full_bar[NB], empty_bar[NB], sc_bar[G::WARPS], nms_bar[G::WARPS];
    __shared__ ItemInfo info[NB];
    // the tile table, copied once so that the producer's search stays on chip
    constexpr int kTileCache = 512;
    __shared__ int32_t tiles_sh[kTileCache];
    // TMA destinations must be 128-byte aligned
    uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~uintptr_t(127));
    uint16_t* sc = reinterpret_cast<uint16_t*>(smem + G::SC_OFF);

    const CallView cv(call);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int n_items = cv.h->n_items;

    if (tid == 0) {
        for (int b = 0; b < NB; ++b) {
            mbar_init(&full_bar[b], 1);
            mbar_init(&empty_bar[b], kConsumers / 32);  // one arrival per consumer warp
        }
        for (int w = 0; w < G::WARPS; ++w) {
            mbar_init(&sc_bar[w], 1);
            mbar_init(&nms_bar[w], 1);
        }
        fence_barrier_init();
    }
    // the score tile starts zero; only corners are written, and each warp
    // zeroes its rows before the next tile's writes
    for (int i = tid; i < G::SR * G::SW / 8; i += kThreads) reinterpret_cast<uint4*>(sc)[i] = make_uint4(0, 0, 0, 0);
    // the decode kernel adds up the per-frame counts from zero
    if (blockIdx.x == 0 && cv.h->counts)
        for (int f = tid; f < cv.h->n_frames; f += kThreads) cv.h->counts[f] = 0;
    const int n_tiles = cv.h->n_frames * cv.h->levels + 1;
    const bool cached = n_tiles <= kTileCache;
    if (cached)
        for (int i = tid; i < n_tiles; i += kThreads) tiles_sh[i] = cv.tiles[i];
    __syncthreads();

    griddep_launch_dependents();
    if (warp == kConsumers / 32) {
        // the pyramid levels the tiles read are written by the kernel before
        // this one, which may still be running (programmatic dependent launch)
        if (lane == 0) {
            griddep_wait();
            produce_tiles<TH, R>(cv, cached ? tiles_sh : cv.tiles, counter, status, info, full_bar, empty_bar, smem);
        }
        return;
    }

    // ---- consumer warps ----
    uint16_t* queue = reinterpret_cast<uint16_t*>(smem + G::Q_OFF) + warp * G::QCAP;
    const uint32_t lt_mask = (1u << lane) - 1u;
    const int thresh = cv.h->thresh, n_arc = cv.h->arc;
    const bool high_t = thresh >= 128;
    const bool three = n_arc >= 12;
    const uint32_t k7 = (uint32_t)((high_t ? 255 : 127) - thresh) * 0x01010101u;

    for (int t = 0;; ++t) {
        const int b = t % NB;
        if (!mbar_wait_bounded(&full_bar[b], (t / NB) & 1, kWaitLimitNs)) {
            if (lane == 0) atomicOr(status, kStatusTimeout);
            return;
        }
        const ItemInfo in = info[b];
        if (in.id >= n_items) break;
        const uint8_t* img = smem + G::IMG_OFF + b * G::BOXA;
        const int k = in.level, Wk = in.wk, x0 = in.x0, y0 = in.y0;
        const uint32_t magic = in.magic;
        const int xoff = in.xoff;

        // 2. coarse test + compaction.  Testable pixels: 3 <= x < Wk-3, 3 <= y < Hk-3.
        int total;
        {
            // score row r is level y = y0 - R + r; score column c is level x = x0 - 4 + c
            const int row_lo = in.row_lo, row_hi = in.row_hi;
            // vm: bit 7 of byte j set when xlo <= 4 lane + j < xhi; byte j of
            // cols4 + (128 - x) reaches bit 7 exactly when 4 lane + j >= x
            // (all values below 256: no carries between bytes)
            const uint32_t cols4 = (uint32_t)(4 * lane) * 0x01010101u + 0x03020100u;
            const uint32_t vm = (cols4 + (uint32_t)(0x80 - in.xlo) * 0x01010101u) &
                                ~(cols4 + (uint32_t)(0x80 - in.xhi) * 0x01010101u) & 0x80808080u;
            const int xw = xoff / 4;
            // the 8-point test (n <= 11 and NMS radius <= 2; n >= 12 keeps 3 of 4)
            constexpr bool kEight = R <= 2;
            if (!three) {
                total = high_t ? coarse_and_compact<true, false, TH, R, kEight>(img, queue, xw, k7, warp, lane, row_lo, row_hi, vm, status)
                               : coarse_and_compact<false, false, TH, R, kEight>(img, queue, xw, k7, warp, lane, row_lo, row_hi, vm, status);
            } else {
                total = high_t ? coarse_and_compact<true, true, TH, R>(img, queue, xw, k7, warp, lane, row_lo, row_hi, vm, status)
                               : coarse_and_compact<false, true, TH, R>(img, queue, xw, k7, warp, lane, row_lo, row_hi, vm, status);
            }
        }
        __syncwarp();

        // 3. full test on this warp's queue; corners are compacted in place
        int ncorner = 0;
        const uint8_t* img_base = img + 3 * G::BW + xoff;
        for (int e0 = 0; e0 < total; e0 += 32) {
            const int e = e0 + lane;
            uint32_t s = 0;
            int idx = 0;
            if (e < total && vio_guard(e < G::QCAP, status)) {
                idx = walk_code_index(queue[e], 2 * G::PPW * warp);
                // box offset of score-region pixel (idx >> 7, idx & 127); the
                // score is taken below, on the compacted corners only
                if (vio_guard(idx < G::SR * G::SW, status))
                    s = eval_corner<MODE, G::BW, false>(img_base + idx + 16 * (idx >> 7), thresh, n_arc);
            }
            const uint32_t cm = __ballot_sync(0xFFFFFFFFu, s != 0);
            if (s) queue[ncorner + __popc(cm & lt_mask)] = (uint16_t)idx;
            ncorner += __popc(cm);
        }
        if (!own_rows_reset<TH, R>(nms_bar, t, sc, warp, lane, status)) return;
        for (int e = lane; e < ncorner; e += 32) {
            const int idx = queue[e];
            const uint8_t* p = img_base + idx + 16 * (idx >> 7);
            // MT of a known corner needs no segment test: the largest window
            // minimum alone (see eval_corner)
            sc[idx] = (uint16_t)(MODE == 0   ? sad_b<G::BW>(p)
                                 : MODE == 2 ? mt_of_corner<G::BW>(p, n_arc)
                                             : eval_corner<MODE, G::BW, true>(p, thresh, n_arc));
        }
        // this warp is done with the image buffer, and its scores are written
        __syncwarp();
        if (lane == 0) {
            mbar_arrive(&empty_bar[b]);
            mbar_arrive(&sc_bar[warp]);
        }
        // the neighbours' scores of this tile are written
        if (!neighbours_wait(sc_bar, warp, G::WARPS, t & 1, lane, status)) return;

        // 4. NMS on the corners, cell maximum by a 64-bit max reduction per
        // survivor.  A window wider than 3x3 is tested ring by ring: the 8
        // nearest neighbours of every corner first, which suppress most
        // corners, then each further ring on the corners that passed the
        // rings inside it (compacted to the front of the queue).
        int nnms = ncorner;
        if constexpr (R > 1) {
            int npass = 0;
            for (int e0 = 0; e0 < ncorner; e0 += 32) {
                const int e = e0 + lane;
                int idx = 0;
                bool ok = false;
                if (e < ncorner) {
                    idx = queue[e];
                    const int sr = idx >> 7, scx = idx & 127;
                    if (scx >= 4 && scx < 4 + G::TW && sr >= R && sr < R + TH) {
                        const uint16_t* q = sc + idx;
                        const uint32_t s = q[0];
                        ok = true;
#pragma unroll
                        for (int dy = -1; dy <= 1; ++dy)
#pragma unroll
                            for (int dx = -1; dx <= 1; ++dx)
                                if (dy != 0 || dx != 0) ok &= s >= q[dy * G::SW + dx];
                    }
                }
                const uint32_t bm = __ballot_sync(0xFFFFFFFFu, ok);
                if (ok) queue[npass + __popc(bm & lt_mask)] = (uint16_t)idx;
                npass += __popc(bm);
            }
            nnms = npass;
            if constexpr (R > 2) nnms = nms_ring_pass<2, G::SW>(queue, nnms, sc, lane, lt_mask);
            if constexpr (R > 3) nnms = nms_ring_pass<3, G::SW>(queue, nnms, sc, lane, lt_mask);
        }
        for (int e0 = 0; e0 < nnms; e0 += 32) {
            const int e = e0 + lane;
            uint32_t cell_id = 0xFFFFFFFFu;
            uint32_t hi = 0, lo = 0;
            if (e < nnms) {
                const int idx = queue[e];
                const int sr = idx >> 7, scx = idx & 127;
                // (with R > 1 the first pass kept corners inside the tile only)
                const bool inside = R > 1 || (scx >= 4 && scx < 4 + G::TW && sr >= R && sr < R + TH);
                if (inside) {
                    // (2R+1) x (2R+1) neighbourhood: keep when >= every neighbour
                    // (for R > 1 the outermost ring; the passes above did the rest)
                    const uint16_t* q = sc + idx;
                    const uint32_t s = q[0];
                    bool keep = true;
                    if constexpr (R == 1) {
                        // (this loop form, not ring_max<1>: the MT kernel is
                        // 5 % slower with the latter)
#pragma unroll
                        for (int dy = -1; dy <= 1; ++dy)
#pragma unroll
                            for (int dx = -1; dx <= 1; ++dx)
                                if (dy != 0 || dx != 0) keep &= s >= q[dy * G::SW + dx];
                    } else {
                        keep = ring_max<R, G::SW>(q, s);
                    }
                    if (keep) {
                        const uint32_t x = (uint32_t)(x0 - 4 + scx), y = (uint32_t)(y0 - R + sr);
                        const uint32_t cx = __umulhi(x, magic), cy = __umulhi(y, magic);
                        if (vio_guard(cx < (uint32_t)in.gw && cy < (uint32_t)in.gh, status)) {
                            cell_id = cy * (uint32_t)in.gw + cx;
                            hi = s;
                            lo = 0xFFFFFFFFu - (((uint32_t)k << 28) | (y * (uint32_t)Wk + x));
                        }
                    }
                }
            }
            // each survivor folds its key into the cell's (a warp-wide max
            // for survivors sharing a cell first was 2.6 % slower: its votes,
            // shuffle and reductions form one long dependent chain)
            if (hi != 0) red_max_u64(reinterpret_cast<unsigned long long*>(&in.keys[cell_id]),
                                     ((unsigned long long)hi << 32) | lo);
        }
        // this warp's NMS reads of the score tile are done
        __syncwarp();
        if (lane == 0) mbar_arrive(&nms_bar[warp]);
    }
}

// ---------------------------------------------------------------------------
// Decode: one thread per cell of all frames turns its key into a record,
// clears the key for the next call and counts non-empty cells per frame
// (warp-aggregated; the fused kernel zeroed the counts).
// ---------------------------------------------------------------------------
static __global__ void __launch_bounds__(256) decode_kernel(const uint8_t* __restrict__ call, int32_t* __restrict__ counter) {
    // the cell keys are final once the detect kernel before this one has
    // completed (it may still be running: programmatic dependent launch)
    griddep_wait();
    const CallView cv(call);
    const int nf = cv.h->n_frames, total = cv.h->n_cells;
    int32_t* counts = cv.h->counts;
    const int lane = threadIdx.x & 31;
    // the cell prefix sums in shared memory when they fit (see pyramid_kernel)
    __shared__ int32_t cells_sh[kPrefixCache];
    const int32_t* cells = nf < kPrefixCache ? cells_sh : cv.cells;
    if (nf < kPrefixCache)
        for (int j = threadIdx.x; j <= nf; j += blockDim.x) cells_sh[j] = cv.cells[j];
    __syncthreads();
    for (int base = blockIdx.x * blockDim.x; base < total; base += gridDim.x * blockDim.x) {
        const int i = base + threadIdx.x;
        int f = -1;
        bool hit = false;
        if (i < total) {
            f = upper_index(cells, nf, i);
            const FrameDesc& fd = cv.fds[f];
            const int c = i - cells[f];
            const uint64_t key = fd.keys[c];
            int4 rec = make_int4(-1, -1, -1, 0);
            if (key != 0) {
                const uint32_t lin = 0xFFFFFFFFu - (uint32_t)key;
                const int k = (int)(lin >> 28);
                const uint32_t idx = lin & 0x0FFFFFFFu;
                const uint32_t wk = (uint32_t)(fd.w >> k);
                const int y = (int)(idx / wk), x = (int)(idx - (uint32_t)y * wk);
                rec = make_int4(x << k, y << k, k, (int)(key >> 32));
                fd.keys[c] = 0;
                hit = true;
                // consistency of the packed key with the cell it was folded into
                const uint32_t magic = cv.h->cell_magic[0];
                if (cv.h->status && (k >= cv.h->levels || rec.x >= fd.w || rec.y >= fd.h ||
                                     __umulhi((uint32_t)rec.y, magic) * (uint32_t)fd.gw +
                                             __umulhi((uint32_t)rec.x, magic) != (uint32_t)c))
                    atomicOr(cv.h->status, kStatusBadKey);
            }
            fd.out[c] = rec;
        }
        if (counts) {
            // lanes of one frame add their hits with one atomic
            uint32_t pend = __ballot_sync(0xFFFFFFFFu, f >= 0);
            while (pend) {
                const int leader = __ffs(pend) - 1;
                const int fl = __shfl_sync(0xFFFFFFFFu, f, leader);
                const uint32_t grp = __ballot_sync(0xFFFFFFFFu, f == fl);
                const uint32_t hits = __popc(__ballot_sync(0xFFFFFFFFu, f == fl && hit));
                if (lane == leader && hits) atomicAdd(&counts[fl], (int)hits);
                pend &= ~grp;
            }
        }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) *counter = 0;
}

}  // namespace vio
