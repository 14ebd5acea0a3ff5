/*
 * Plain CPU oracle for pyramidal FAST detection with 3x3 non-maxima
 * suppression and one-feature-per-cell selection (NMS-C).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, obviously-correct
 * statement of what the GPU path must compute.  Only the test-suite, the
 * smoke check and the benchmark's CPU-baseline leg load it; the library
 * never does.  It shares no code, header or table with the CUDA path.
 *
 * Every function follows the paper ("Faster than FAST: GPU-Accelerated
 * Frontend for High-Speed VIO", Nagy, Foehn, Scaramuzza, IROS 2020):
 *
 *   pyramid          Section II-B (subsampled pyramid), Section III-C
 *                    (every level half the size of the one above); 2x2 mean,
 *                    rounded half up: (a+b+c+d+2)>>2.
 *   circle / labels  Section II-D, Eq. 1 (radius-3 Bresenham circle of 16
 *                    points; darker / similar / brighter with strict
 *                    inequalities against the threshold).
 *   segment test     Section II-D: a contiguous arc of at least N points,
 *                    all darker or all brighter; a 3-pixel border skipped.
 *   scores           Section II-D: SAD-B, SAD-A, MT; 0 when the test fails.
 *   NMS              Algorithm 1 (on every scale); Section I-B (Moore
 *                    neighbourhood of side 2n+1: n = 1 gives 3x3, n = 2..4
 *                    the 5x5..9x9 windows of Table III).
 *   NMS-C            Algorithm 1 (after all scales), Section II-B (one
 *                    feature per cell, the highest score) and Section II-C
 *                    (one grid for all levels, level-k positions scaled
 *                    up by 2^k).
 *
 * Readings where the paper is silent:
 *   - circle order: clockwise from the top point (0,-3);
 *   - SAD-B sums |I_x - I_center| over all 16 points, SAD-A over the
 *     maximal homogeneous run that makes the point a corner;
 *   - MT is the largest t in [eps, 255] at which the point is a corner;
 *   - NMS keeps a pixel when its score is > 0 and >= each of its
 *     (2n+1)^2 - 1 neighbours, n = 1 (3x3) unless asked otherwise (pixels
 *     outside the level count as 0);
 *   - cell winner: highest score, then lower level, then lower y, then
 *     lower x (all in level coordinates); position reported as
 *     (x << k, y << k); an empty cell is (-1, -1, -1, 0);
 *   - partial right/bottom cells are kept: ceil(W/C) x ceil(H/C) cells.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORACLE_SAD_B 0
#define ORACLE_SAD_A 1
#define ORACLE_MT 2

/* Radius-3 Bresenham circle, 16 points, clockwise from the top (Sec. II-D). */
static const int CIRCLE_DX[16] = {0, 1, 2, 3, 3, 3, 2, 1, 0, -1, -2, -3, -3, -3, -2, -1};
static const int CIRCLE_DY[16] = {-3, -3, -2, -1, 0, 1, 2, 3, 3, 3, 2, 1, 0, -1, -2, -3};

int oracle_abi_version(void) { return 1; }

void oracle_circle(int* dx, int* dy) {
    for (int i = 0; i < 16; ++i) {
        dx[i] = CIRCLE_DX[i];
        dy[i] = CIRCLE_DY[i];
    }
}

/* One half-sampling step: dst is (w>>1) x (h>>1). */
void oracle_halfsample(const uint8_t* src, int w, int h, int pitch, uint8_t* dst, int dpitch) {
    int w2 = w >> 1, h2 = h >> 1;
    for (int y = 0; y < h2; ++y) {
        for (int x = 0; x < w2; ++x) {
            int a = src[(2 * y) * pitch + 2 * x];
            int b = src[(2 * y) * pitch + 2 * x + 1];
            int c = src[(2 * y + 1) * pitch + 2 * x];
            int d = src[(2 * y + 1) * pitch + 2 * x + 1];
            dst[y * dpitch + x] = (uint8_t)((a + b + c + d + 2) >> 2);
        }
    }
}

/* Label of circle point value v against centre c (Eq. 1): +1 brighter, -1 darker, 0 similar. */
static int label_of(int v, int c, int t) {
    if (v > c + t) return 1;
    if (v < c - t) return -1;
    return 0;
}

/* Segment test on a label vector: is there a start s with labels
 * s, s+1, ..., s+N-1 (cyclically) all equal to `pol` (+1 or -1)? */
static int has_arc(const int* lab, int pol, int n_arc) {
    for (int s = 0; s < 16; ++s) {
        int ok = 1;
        for (int j = 0; j < n_arc; ++j) {
            if (lab[(s + j) % 16] != pol) {
                ok = 0;
                break;
            }
        }
        if (ok) return 1;
    }
    return 0;
}

/* The segment test stated on two 16-bit masks (bit i = label of point i);
 * used to pin the mask formulation against the label formulation. */
int oracle_arc_from_masks(uint32_t bright, uint32_t dark, int n_arc) {
    int lb[16], ld[16];
    for (int i = 0; i < 16; ++i) {
        lb[i] = (bright >> i) & 1u;
        ld[i] = (dark >> i) & 1u;
    }
    return has_arc(lb, 1, n_arc) || has_arc(ld, 1, n_arc);
}

static void circle_values(const uint8_t* img, int pitch, int x, int y, int* v) {
    for (int i = 0; i < 16; ++i) v[i] = img[(y + CIRCLE_DY[i]) * pitch + (x + CIRCLE_DX[i])];
}

/* Segment test at threshold t for the pixel (x, y); caller guarantees the
 * circle is inside the image. */
int oracle_is_corner(const uint8_t* img, int pitch, int x, int y, int t, int n_arc) {
    int v[16], lab[16];
    int c = img[y * pitch + x];
    circle_values(img, pitch, x, y, v);
    for (int i = 0; i < 16; ++i) lab[i] = label_of(v[i], c, t);
    return has_arc(lab, 1, n_arc) || has_arc(lab, -1, n_arc);
}

/* Score of one pixel (Sec. II-D); 0 when outside the 3-pixel border or
 * when the segment test fails at threshold `thresh`. */
int oracle_score_pixel(const uint8_t* img, int w, int h, int pitch, int x, int y, int thresh,
                       int n_arc, int mode) {
    if (x < 3 || y < 3 || x >= w - 3 || y >= h - 3) return 0;
    if (!oracle_is_corner(img, pitch, x, y, thresh, n_arc)) return 0;
    int v[16], lab[16];
    int c = img[y * pitch + x];
    circle_values(img, pitch, x, y, v);
    for (int i = 0; i < 16; ++i) lab[i] = label_of(v[i], c, thresh);

    if (mode == ORACLE_SAD_B) {
        int s = 0;
        for (int i = 0; i < 16; ++i) s += abs(v[i] - c);
        return s;
    }
    if (mode == ORACLE_SAD_A) {
        /* the polarity that has the arc */
        int pol = has_arc(lab, 1, n_arc) ? 1 : -1;
        int all = 1;
        for (int i = 0; i < 16; ++i)
            if (lab[i] != pol) all = 0;
        if (all) {
            int s = 0;
            for (int i = 0; i < 16; ++i) s += abs(v[i] - c);
            return s;
        }
        /* maximal runs of `pol`: start where the previous point is not `pol` */
        int best = 0;
        for (int s0 = 0; s0 < 16; ++s0) {
            if (lab[s0] != pol || lab[(s0 + 15) % 16] == pol) continue;
            int len = 0, sum = 0;
            while (len < 16 && lab[(s0 + len) % 16] == pol) {
                sum += abs(v[(s0 + len) % 16] - c);
                ++len;
            }
            if (len >= n_arc && sum > best) best = sum;
        }
        return best;
    }
    /* MT: the largest threshold at which the point is still a corner. */
    for (int t = 255; t >= thresh; --t)
        if (oracle_is_corner(img, pitch, x, y, t, n_arc)) return t;
    return 0; /* unreachable: the test passed at `thresh` */
}

void oracle_score_map(const uint8_t* img, int w, int h, int pitch, int thresh, int n_arc, int mode,
                      int32_t* out) {
    for (int y = 0; y < h; ++y)
        for (int x = 0; x < w; ++x)
            out[y * w + x] = oracle_score_pixel(img, w, h, pitch, x, y, thresh, n_arc, mode);
}

/* NMS over the (2n+1) x (2n+1) Moore neighbourhood (Section I-B; n = 1 is
 * the 3x3 case of Algorithm 1, n = 2..4 the larger windows of Table III) on
 * a dense w x h score map (row pitch w). */
void oracle_nms(const int32_t* s, int w, int h, int n, int32_t* out) {
    for (int y = 0; y < h; ++y) {
        for (int x = 0; x < w; ++x) {
            int v = s[y * w + x];
            int keep = v > 0;
            for (int dy = -n; dy <= n && keep; ++dy) {
                for (int dx = -n; dx <= n; ++dx) {
                    if (dx == 0 && dy == 0) continue;
                    int xx = x + dx, yy = y + dy;
                    int nv = (xx >= 0 && yy >= 0 && xx < w && yy < h) ? s[yy * w + xx] : 0;
                    if (v < nv) {
                        keep = 0;
                        break;
                    }
                }
            }
            out[y * w + x] = keep ? v : 0;
        }
    }
}

void oracle_nms3(const int32_t* s, int w, int h, int32_t* out) { oracle_nms(s, w, h, 1, out); }

/* Is candidate (s1, k1, y1, x1) a better cell winner than (s0, k0, y0, x0)? */
static int better(int s1, int k1, int y1, int x1, int s0, int k0, int y0, int x0) {
    if (s1 != s0) return s1 > s0;
    if (k1 != k0) return k1 < k0;
    if (y1 != y0) return y1 < y0;
    return x1 < x0;
}

int oracle_num_cells(int w, int h, int cell) {
    return ((w + cell - 1) / cell) * ((h + cell - 1) / cell);
}

/*
 * Full detection of one frame.  `out` receives 4 int32 per cell, row-major
 * over the ceil(w/cell) x ceil(h/cell) level-0 grid: x, y, level, score.
 * Returns the number of non-empty cells, or -1 on allocation failure.
 */
int oracle_detect_nms(const uint8_t* img, int w, int h, int pitch, int thresh, int n_arc, int cell,
                      int levels, int mode, int nms_radius, int32_t* out) {
    int gw = (w + cell - 1) / cell, gh = (h + cell - 1) / cell;
    int ncell = gw * gh;
    for (int i = 0; i < ncell; ++i) {
        out[4 * i + 0] = -1;
        out[4 * i + 1] = -1;
        out[4 * i + 2] = -1;
        out[4 * i + 3] = 0;
    }
    /* level k image, dense with pitch wk */
    int wk = w, hk = h;
    uint8_t* lev = (uint8_t*)malloc((size_t)w * h + 1);
    int32_t* sc = (int32_t*)malloc(sizeof(int32_t) * ((size_t)w * h + 1));
    int32_t* nm = (int32_t*)malloc(sizeof(int32_t) * ((size_t)w * h + 1));
    if (!lev || !sc || !nm) {
        free(lev);
        free(sc);
        free(nm);
        return -1;
    }
    for (int y = 0; y < h; ++y) memcpy(lev + (size_t)y * w, img + (size_t)y * pitch, w);

    for (int k = 0; k < levels; ++k) {
        if (k > 0) {
            uint8_t* nxt = (uint8_t*)malloc((size_t)(wk >> 1) * (hk >> 1) + 1);
            if (!nxt) {
                free(lev);
                free(sc);
                free(nm);
                return -1;
            }
            oracle_halfsample(lev, wk, hk, wk, nxt, wk >> 1);
            free(lev);
            lev = nxt;
            wk >>= 1;
            hk >>= 1;
        }
        oracle_score_map(lev, wk, hk, wk, thresh, n_arc, mode, sc);
        oracle_nms(sc, wk, hk, nms_radius, nm);
        for (int y = 0; y < hk; ++y) {
            for (int x = 0; x < wk; ++x) {
                int s = nm[y * wk + x];
                if (s <= 0) continue;
                int cx = (x << k) / cell, cy = (y << k) / cell;
                int32_t* o = out + 4 * (cy * gw + cx);
                int ok = o[2] < 0;
                if (!ok) {
                    int k0 = o[2];
                    ok = better(s, k, y, x, o[3], k0, o[1] >> k0, o[0] >> k0);
                }
                if (ok) {
                    o[0] = x << k;
                    o[1] = y << k;
                    o[2] = k;
                    o[3] = s;
                }
            }
        }
    }
    free(lev);
    free(sc);
    free(nm);
    int cnt = 0;
    for (int i = 0; i < ncell; ++i) cnt += out[4 * i + 2] >= 0;
    return cnt;
}

int oracle_detect(const uint8_t* img, int w, int h, int pitch, int thresh, int n_arc, int cell, int levels,
                  int mode, int32_t* out) {
    return oracle_detect_nms(img, w, h, pitch, thresh, n_arc, cell, levels, mode, 1, out);
}
