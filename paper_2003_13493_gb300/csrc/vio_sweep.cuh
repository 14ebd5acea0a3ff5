// Fused threshold / arc-length sweep: up to 8 detector settings (threshold,
// arc length) over the same frames in one pass.  Each tile is loaded once,
// the coarse test runs once at the lowest threshold (its candidates are a
// superset of every setting's), and so does the plain segment test, at the
// lowest threshold and the shortest arc length (its corners are a superset
// of every setting's).  Instead of forming Eq. 1's labels per threshold, the
// survivors' second test finds, once per distinct arc length n, the largest
// threshold at which the candidate is a corner: the segment test holds at t
// exactly when some n
// cyclically consecutive signed differences (v - c for a brighter arc, c - v
// for a darker one) all exceed t, i.e. when the largest minimum over all
// windows of n points exceeds t.  A setting (t, n) then costs one compare.
// NMS and the cell maximum run per setting on a per-pixel bit mask of the
// settings in which the pixel is a corner.  SAD-B is the score: it does not
// depend on the setting, so one 16-bit score tile serves all of them.
#pragma once
#include <stdint.h>

#include "vio_kernels.cuh"

namespace vio {

constexpr int kMaxSweep = 8;

// Sweep section of a call block (the detector sections come first).
struct SweepInfo {
    int32_t n_set;                 // settings in this launch, 1..kMaxSweep
    int32_t thresh[kMaxSweep];
    int32_t arc[kMaxSweep];        // non-decreasing: settings of one arc length are adjacent
    int32_t pad;
    int64_t set_stride;            // keys of setting s: FrameDesc::keys + s * set_stride
    int4* const* outs;             // [n_set * n_frames] output records, setting-major
    int32_t* counts[kMaxSweep];    // per setting: [n_frames] non-empty cells, or nullptr
};

// SAD-B of circle values v around centre value c: sum of |I_x - I_c|.
__device__ __forceinline__ uint32_t sad_b_of(const uint32_t (&v)[16], uint32_t c) {
    const uint32_t c4 = c * 0x01010101u;
    uint32_t s = __vsadu4(pack4(v[0], v[1], v[2], v[3]), c4);
    s += __vsadu4(pack4(v[4], v[5], v[6], v[7]), c4);
    s += __vsadu4(pack4(v[8], v[9], v[10], v[11]), c4);
    s += __vsadu4(pack4(v[12], v[13], v[14], v[15]), c4);
    return s;
}

template <int TH>
struct SweepGeom : TileGeom<TH, 1> {
    using B = TileGeom<TH, 1>;
    static constexpr int MK_OFF = B::Q_OFF + B::WARPS * B::QCAP * 2;  // uint8 setting mask per score pixel
    static constexpr int SMEM = MK_OFF + B::SR * B::SW + 128;
};

template <int TH>
__global__ void __launch_bounds__(kThreads, 3) fast_sweep_kernel(const uint8_t* __restrict__ call,
                                                                const SweepInfo* __restrict__ sw,
                                                                int32_t* __restrict__ counter,
                                                                uint32_t* __restrict__ status) {
    using G = SweepGeom<TH>;
    constexpr int NB = G::NBUF;
    extern __shared__ __align__(128) uint8_t smem_raw[];
    __shared__ uint64_t full_bar[NB], empty_bar[NB], sc_bar[G::WARPS], nms_bar[G::WARPS];
    __shared__ ItemInfo info[NB];
    constexpr int kTileCache = 512;
    __shared__ int32_t tiles_sh[kTileCache];
    __shared__ int32_t set_t[kMaxSweep], set_n[kMaxSweep];
    uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~uintptr_t(127));
    uint16_t* sc = reinterpret_cast<uint16_t*>(smem + G::SC_OFF);
    uint8_t* mk = smem + G::MK_OFF;

    const CallView cv(call);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int n_items = cv.h->n_items;
    const int n_set = sw->n_set;

    if (tid == 0) {
        for (int b = 0; b < NB; ++b) {
            mbar_init(&full_bar[b], 1);
            mbar_init(&empty_bar[b], kConsumers / 32);
        }
        for (int w = 0; w < G::WARPS; ++w) {
            mbar_init(&sc_bar[w], 1);
            mbar_init(&nms_bar[w], 1);
        }
        fence_barrier_init();
    }
    if (tid < kMaxSweep) {
        set_t[tid] = tid < n_set ? sw->thresh[tid] : 0;
        set_n[tid] = tid < n_set ? sw->arc[tid] : 16;
    }
    // score and setting-mask tiles start zero; only corners are written, and
    // each warp zeroes its rows before the next tile's writes
    for (int i = tid; i < G::SR * G::SW / 8; i += kThreads) reinterpret_cast<uint4*>(sc)[i] = make_uint4(0, 0, 0, 0);
    for (int i = tid; i < G::SR * G::SW / 16; i += kThreads) reinterpret_cast<uint4*>(mk)[i] = make_uint4(0, 0, 0, 0);
    if (blockIdx.x == 0)
        for (int f = tid; f < n_set * cv.h->n_frames; f += kThreads) {
            int32_t* cs = sw->counts[f / cv.h->n_frames];
            if (cs) cs[f % cv.h->n_frames] = 0;
        }
    const int n_tiles = cv.h->n_frames * cv.h->levels + 1;
    const bool cached = n_tiles <= kTileCache;
    if (cached)
        for (int i = tid; i < n_tiles; i += kThreads) tiles_sh[i] = cv.tiles[i];
    __syncthreads();

    if (warp == kConsumers / 32) {
        if (lane == 0) produce_tiles<TH, 1>(cv, cached ? tiles_sh : cv.tiles, counter, status, info, full_bar, empty_bar,
                                            smem);
        return;
    }

    // ---- consumer warps ----
    uint16_t* queue = reinterpret_cast<uint16_t*>(smem + G::Q_OFF) + warp * G::QCAP;
    const uint32_t lt_mask = (1u << lane) - 1u;
    // the coarse test at the lowest threshold with the two-adjacent rule
    // keeps every pixel any setting can accept
    int tmin = set_t[0], arc_min = set_n[0];
    for (int s = 1; s < n_set; ++s) {
        tmin = min(tmin, set_t[s]);
        arc_min = min(arc_min, set_n[s]);
    }
    const bool high_t = tmin >= 128;
    const uint32_t k7 = (uint32_t)((high_t ? 255 : 127) - tmin) * 0x01010101u;
    const int64_t stride = sw->set_stride;
    // the usual launch has at most two arc lengths (settings ordered by arc
    // length): then each candidate's largest window minimum is found once per
    // arc length and the settings are 8 unrolled compares against thresholds
    // held in registers; more arc lengths take the general loop
    const int arc_a = set_n[0];
    int arc_b = arc_a, n_arcs = 1;
    for (int s = 1; s < n_set; ++s)
        if (set_n[s] != set_n[s - 1]) {
            ++n_arcs;
            arc_b = set_n[s];
        }
    const bool two_arcs = n_arcs <= 2;
    // settings 2j and 2j+1 in the two 16-bit lanes of tpair[j]: threshold +
    // 257 (an unused setting gets 0x7FFF, which no window minimum reaches),
    // and in nibble pairs of selp a byte-permute selector that takes each
    // lane's window minimum from best_a (bytes 0-1) or best_b (bytes 2-3)
    uint32_t tpair[kMaxSweep / 2], selp[kMaxSweep / 4] = {0u, 0u};
#pragma unroll
    for (int j = 0; j < kMaxSweep / 2; ++j) {
        uint32_t pr = 0, sl = 0;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int s = 2 * j + h;
            const bool use_b = s < n_set && set_n[s] == arc_b && arc_b != arc_a;
            pr |= (s < n_set ? (uint32_t)set_t[s] + 257u : 0x7FFFu) << (16 * h);
            sl |= (use_b ? 0x32u : 0x10u) << (8 * h);
        }
        tpair[j] = pr;
        selp[j / 2] |= sl << (16 * (j & 1));
    }

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

        int total;
        {
            // the producer's per-item rows and columns (NMS radius 1)
            const int row_lo = in.row_lo, row_hi = in.row_hi;
            const uint32_t cols4 = (uint32_t)(4 * lane) * 0x01010101u + 0x03020100u;
            const uint32_t vm = (cols4 + (uint32_t)(0x80 - in.xlo) * 0x01010101u) &
                                ~(cols4 + (uint32_t)(0x80 - in.xhi) * 0x01010101u) & 0x80808080u;
            const int xw = xoff / 4;
            // levels >= 1: the 8-point test, also a necessary condition for every arc length
            if (k > 0)
                total = high_t ? coarse_and_compact<true, false, TH, 1, true>(img, queue, xw, k7, warp, lane, row_lo,
                                                                              row_hi, vm, status)
                               : coarse_and_compact<false, false, TH, 1, true>(img, queue, xw, k7, warp, lane, row_lo,
                                                                               row_hi, vm, status);
            else
                total = high_t ? coarse_and_compact<true, false, TH, 1>(img, queue, xw, k7, warp, lane, row_lo,
                                                                         row_hi, vm, status)
                               : coarse_and_compact<false, false, TH, 1>(img, queue, xw, k7, warp, lane, row_lo,
                                                                          row_hi, vm, status);
        }
        __syncwarp();

        // full test, pass 1: the single-setting segment test at the lowest
        // threshold and the shortest arc length, whose corners include every
        // setting's (n consecutive differences beyond t >= tmin hold n_min
        // consecutive ones beyond tmin); survivors compacted in place
        int nsurv = 0;
        const uint8_t* img_base = img + 3 * G::BW + xoff;
        for (int e0 = 0; e0 < total; e0 += 32) {
            const int e = e0 + lane;
            uint32_t s = 0;
            int idx = 0;
            if (e < total && vio_guard(e < G::QCAP, status)) {
                idx = walk_code_index(queue[e], 2 * G::PPW * warp);
                if (vio_guard(idx < G::SR * G::SW, status))
                    s = eval_corner<0, G::BW, false>(img_base + idx + 16 * (idx >> 7), tmin, arc_min);
            }
            const uint32_t cm = __ballot_sync(0xFFFFFFFFu, s != 0);
            if (s) queue[nsurv + __popc(cm & lt_mask)] = (uint16_t)idx;
            nsurv += __popc(cm);
        }

        // the score and mask rows of this warp are free once its neighbours'
        // NMS of the previous tile is done
        if (!own_rows_reset<TH, 1>(nms_bar, t, sc, warp, lane, status) ||
            !own_rows_reset<TH, 1>(nms_bar, t, mk, warp, lane, status))
            return;
        // pass 2, on the survivors: the settings in which each is a corner
        // (window minima), its SAD-B score, compacted in place again
        int ncorner = 0;
        for (int e0 = 0; e0 < nsurv; e0 += 32) {
            const int e = e0 + lane;
            uint32_t cmask = 0, score = 0;
            int idx = 0;
            if (e < nsurv) {
                idx = queue[e];
                const uint8_t* p = img_base + idx + 16 * (idx >> 7);
                uint32_t v[16];
#pragma unroll
                for (int i = 0; i < 16; ++i) v[i] = p[circ_dy(i) * G::BW + circ_dx(i)];
                const uint32_t c = p[0];
                // the score first, so that the circle values die as the
                // window minima are formed
                score = sad_b_of(v, c);
                uint32_t W8[16];
                window_minima8_of(v, c, W8);
                if (two_arcs) {  // uniform
                    const uint32_t best_a = best_window_min_for_arc(W8, arc_a);
                    const uint32_t best_b = arc_b != arc_a ? best_window_min_for_arc(W8, arc_b) : best_a;
                    // per pair: lane value 0x8000 + best - (t + 257) stays
                    // in 1 .. 0x81FF (no carry or borrow between the lanes)
                    // and has bit 15 set exactly when best >= t + 257
                    const uint32_t bb = best_a | (best_b << 16);
                    uint32_t z = 0;
#pragma unroll
                    for (int j = 0; j < kMaxSweep / 2; ++j) {
                        const uint32_t x = __byte_perm(bb, 0u, selp[j / 2] >> (16 * (j & 1))) + 0x80008000u - tpair[j];
                        z |= (x & 0x80008000u) >> (15 - 2 * j);  // bits 2j and 16 + 2j
                    }
                    cmask = (z | (z >> 15)) & 0xFFu;
                } else {
                    int prev_n = 0;
                    uint32_t best = 0;
                    for (int s = 0; s < n_set; ++s) {  // uniform; settings of one arc length are adjacent
                        const int ns = set_n[s];
                        if (ns != prev_n) {
                            best = best_window_min_for_arc(W8, ns);
                            prev_n = ns;
                        }
                        if (best >= (uint32_t)set_t[s] + 257u) cmask |= 1u << s;
                    }
                }
            }
            const uint32_t cm = __ballot_sync(0xFFFFFFFFu, cmask != 0);
            if (cmask) {
                queue[ncorner + __popc(cm & lt_mask)] = (uint16_t)idx;
                mk[idx] = (uint8_t)cmask;
                sc[idx] = (uint16_t)score;
            }
            ncorner += __popc(cm);
        }
        // this warp is done with the image buffer, and its scores and masks are written
        __syncwarp();
        if (lane == 0) {
            mbar_arrive(&empty_bar[b]);
            mbar_arrive(&sc_bar[warp]);
        }
        // the neighbours' scores and masks of this tile are written
        if (!neighbours_wait(sc_bar, warp, G::WARPS, t & 1, lane, status)) return;

        // 3x3 NMS of every setting at once: a neighbour suppresses the pixel
        // in the settings where it is a corner with a higher score
        for (int e0 = 0; e0 < ncorner; e0 += 32) {
            const int e = e0 + lane;
            uint32_t keep = 0, cell_id = 0xFFFFFFFFu, hi = 0, lo = 0;
            if (e < ncorner) {
                const int idx = queue[e];
                const int sr = idx >> 7, scx = idx & 127;
                if (scx >= 4 && scx < 4 + G::TW && sr >= 1 && sr < 1 + TH) {
                    const uint16_t* q = sc + idx;
                    const uint8_t* qm = mk + idx;
                    const uint32_t s = q[0];
                    uint32_t allowed = 0xFFu;
#pragma unroll
                    for (int dy = -1; dy <= 1; ++dy)
#pragma unroll
                        for (int dx = -1; dx <= 1; ++dx)
                            if (dy != 0 || dx != 0) {
                                const int o = dy * G::SW + dx;
                                allowed &= s >= q[o] ? 0xFFu : ~(uint32_t)qm[o];
                            }
                    keep = qm[0] & allowed;
                    if (keep) {
                        const uint32_t x = (uint32_t)(x0 - 4 + scx), y = (uint32_t)(y0 - 1 + sr);
                        const uint32_t cx = __umulhi(x, magic), cy = __umulhi(y, magic);
                        if (vio_guard(cx < (uint32_t)in.gw && cy < (uint32_t)in.gh, status)) {
                            cell_id = cy * (uint32_t)in.gw + cx;
                            hi = s;
                            lo = 0xFFFFFFFFu - (((uint32_t)k << 28) | (y * (uint32_t)Wk + x));
                        } else {
                            keep = 0;
                        }
                    }
                }
            }
            // each survivor folds its key into the cell of every setting it
            // survives in (warp-wide maxima per setting first, with a vote per
            // setting, made the kernel 12 % slower)
            for (uint32_t kk = keep; kk; kk &= kk - 1u) {
                const int s = __ffs(kk) - 1;
                red_max_u64(reinterpret_cast<unsigned long long*>(in.keys + s * stride) + cell_id,
                            ((unsigned long long)hi << 32) | lo);
            }
        }
        // this warp's NMS reads of the score and mask tiles are done
        __syncwarp();
        if (lane == 0) mbar_arrive(&nms_bar[warp]);
    }
}

// Decode of a sweep: one thread per (setting, cell) of all frames.
static __global__ void __launch_bounds__(256) sweep_decode_kernel(const uint8_t* __restrict__ call,
                                                                 const SweepInfo* __restrict__ sw,
                                                                 int32_t* __restrict__ counter) {
    const CallView cv(call);
    const int nf = cv.h->n_frames, cells = cv.h->n_cells;
    const int total = sw->n_set * cells;
    const int lane = threadIdx.x & 31;
    // the cell prefix sums in shared memory when they fit (see pyramid_kernel)
    __shared__ int32_t cells_sh[kPrefixCache];
    const int32_t* cell_pre = nf < kPrefixCache ? cells_sh : cv.cells;
    if (nf < kPrefixCache)
        for (int j = threadIdx.x; j <= nf; j += blockDim.x) cells_sh[j] = cv.cells[j];
    __syncthreads();
    for (int base = blockIdx.x * blockDim.x; base < total; base += gridDim.x * blockDim.x) {
        const int i = base + threadIdx.x;
        int g = -1;  // (setting, frame) group of this thread
        bool hit = false;
        if (i < total) {
            const int s = i / cells, ci = i - s * cells;
            const int f = upper_index(cell_pre, nf, ci);
            const FrameDesc& fd = cv.fds[f];
            const int c = ci - cell_pre[f];
            uint64_t* kp = fd.keys + s * sw->set_stride + c;
            const uint64_t key = *kp;
            int4 rec = make_int4(-1, -1, -1, 0);
            if (key != 0) {
                const uint32_t lin = 0xFFFFFFFFu - (uint32_t)key;
                const int k = (int)(lin >> 28);
                const uint32_t idx = lin & 0x0FFFFFFFu;
                const uint32_t wk = (uint32_t)(fd.w >> k);
                const int y = (int)(idx / wk), x = (int)(idx - (uint32_t)y * wk);
                rec = make_int4(x << k, y << k, k, (int)(key >> 32));
                *kp = 0;
                hit = true;
                const uint32_t magic = cv.h->cell_magic[0];
                if (cv.h->status && (k >= cv.h->levels || rec.x >= fd.w || rec.y >= fd.h ||
                                     __umulhi((uint32_t)rec.y, magic) * (uint32_t)fd.gw +
                                             __umulhi((uint32_t)rec.x, magic) != (uint32_t)c))
                    atomicOr(cv.h->status, kStatusBadKey);
            }
            sw->outs[s * nf + f][c] = rec;
            g = s * nf + f;
        }
        // lanes of one (setting, frame) add their hits with one atomic
        uint32_t pend = __ballot_sync(0xFFFFFFFFu, g >= 0);
        while (pend) {
            const int leader = __ffs(pend) - 1;
            const int gl = __shfl_sync(0xFFFFFFFFu, g, leader);
            const uint32_t grp = __ballot_sync(0xFFFFFFFFu, g == gl);
            const uint32_t hits = __popc(__ballot_sync(0xFFFFFFFFu, g == gl && hit));
            int32_t* cs = sw->counts[gl / nf];
            if (lane == leader && hits && cs) atomicAdd(&cs[gl % nf], (int)hits);
            pend &= ~grp;
        }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) *counter = 0;
}

}  // namespace vio
