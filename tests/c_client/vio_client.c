/* A plain C client of include/vio.h: no Python, no PyTorch.  It draws a
 * deterministic test frame (bright squares on a ramp, the same formula as
 * tests/test_gpu_c_client.py), detects it through the device-buffer and the
 * host-buffer entry points, tracks a few positions into a shifted copy, and
 * prints the results as text for the test to compare with the oracle. */
#include <cuda_runtime.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include "vio.h"

#define W 640
#define H 480
#define CELL 32
#define LEVELS 3

static unsigned char pixel(int x, int y) {
    int v = 40 + (x + 2 * y) % 90;
    if ((x / 24 + y / 24) % 3 == 0 && x % 24 > 5 && y % 24 > 7) v = 200 + (x * 7 + y * 3) % 50;
    return (unsigned char)v;
}

static int fail(const char* what, vio_status s, vio_ctx* ctx) {
    fprintf(stderr, "%s: %s (%s)\n", what, vio_status_str(s), ctx ? vio_last_error(ctx) : "");
    return 1;
}

int main(void) {
    const int ncell = (int)vio_num_cells(W, H, CELL);
    unsigned char* frame = (unsigned char*)malloc((size_t)W * H);
    unsigned char* moved = (unsigned char*)malloc((size_t)W * H);
    vio_feature* host_cells = (vio_feature*)malloc(sizeof(vio_feature) * ncell);
    vio_feature* dev_copy = (vio_feature*)malloc(sizeof(vio_feature) * ncell);
    for (int y = 0; y < H; ++y)
        for (int x = 0; x < W; ++x) {
            frame[y * W + x] = pixel(x, y);
            moved[y * W + x] = pixel(x >= 3 ? x - 3 : 0, y >= 2 ? y - 2 : 0);  /* shifted by (3, 2) */
        }

    vio_config cfg;
    vio_config_default(&cfg);
    vio_ctx* ctx = NULL;
    vio_status s = vio_create(&ctx, &cfg);
    if (s != VIO_OK) return fail("vio_create", s, ctx);

    /* device buffers */
    unsigned char *d_frame = NULL, *d_moved = NULL;
    vio_feature* d_cells = NULL;
    int32_t* d_count = NULL;
    if (cudaMalloc((void**)&d_frame, (size_t)W * H) != cudaSuccess ||
        cudaMalloc((void**)&d_moved, (size_t)W * H) != cudaSuccess ||
        cudaMalloc((void**)&d_cells, sizeof(vio_feature) * ncell) != cudaSuccess ||
        cudaMalloc((void**)&d_count, sizeof(int32_t)) != cudaSuccess)
        return fail("cudaMalloc", VIO_ERR_OOM, NULL);
    cudaMemcpy(d_frame, frame, (size_t)W * H, cudaMemcpyHostToDevice);
    cudaMemcpy(d_moved, moved, (size_t)W * H, cudaMemcpyHostToDevice);

    const uint8_t* frames[1] = {d_frame};
    vio_dims dims[1] = {{W, H, W}};
    vio_feature* outs[1] = {d_cells};
    s = vio_detect(ctx, frames, dims, 1, 15, 9, CELL, LEVELS, outs, d_count, NULL);
    if (s == VIO_OK) s = vio_sync(ctx, NULL);
    if (s != VIO_OK) return fail("vio_detect", s, ctx);
    int32_t count = 0;
    cudaMemcpy(dev_copy, d_cells, sizeof(vio_feature) * ncell, cudaMemcpyDeviceToHost);
    cudaMemcpy(&count, d_count, sizeof(int32_t), cudaMemcpyDeviceToHost);

    /* host buffers: must give the same records */
    const uint8_t* hframes[1] = {frame};
    vio_feature* houts[1] = {host_cells};
    int32_t hcount = -1;
    s = vio_detect_host(ctx, hframes, dims, 1, 15, 9, CELL, LEVELS, houts, &hcount, NULL);
    if (s != VIO_OK) return fail("vio_detect_host", s, ctx);
    if (hcount != count || memcmp(host_cells, dev_copy, sizeof(vio_feature) * ncell) != 0) {
        fprintf(stderr, "host and device paths differ\n");
        return 1;
    }
    printf("count %d\n", count);
    for (int c = 0; c < ncell; ++c)
        printf("cell %d %d %d %d %d\n", c, dev_copy[c].x, dev_copy[c].y, dev_copy[c].level, dev_copy[c].score);

    /* track the first detected features into the shifted frame */
    float pts[2 * 8];
    int np = 0;
    for (int c = 0; c < ncell && np < 8; ++c) {
        const vio_feature f = dev_copy[c];
        if (f.level >= 0 && f.x >= 40 && f.x < W - 40 && f.y >= 40 && f.y < H - 40) {
            pts[2 * np] = (float)f.x;
            pts[2 * np + 1] = (float)f.y;
            ++np;
        }
    }
    float* d_pts = NULL;
    vio_track_result* d_res = NULL;
    vio_track_result res[8];
    cudaMalloc((void**)&d_pts, sizeof(pts));
    cudaMalloc((void**)&d_res, sizeof(res));
    cudaMemcpy(d_pts, pts, sizeof(pts), cudaMemcpyHostToDevice);
    vio_track_params tp;
    vio_track_params_default(&tp);
    tp.model = 0;
    tp.max_iters = 20;
    tp.min_update = 0.0f;
    const uint8_t* prev[1] = {d_frame};
    const uint8_t* next[1] = {d_moved};
    const float* pp[1] = {d_pts};
    vio_track_result* rr[1] = {d_res};
    s = vio_track(ctx, prev, next, dims, 1, pp, &np, &tp, rr, NULL);
    if (s == VIO_OK) s = vio_sync(ctx, NULL);
    if (s != VIO_OK) return fail("vio_track", s, ctx);
    cudaMemcpy(res, d_res, sizeof(vio_track_result) * np, cudaMemcpyDeviceToHost);
    for (int i = 0; i < np; ++i)
        printf("track %.1f %.1f %.4f %.4f %d\n", pts[2 * i], pts[2 * i + 1], res[i].x, res[i].y, res[i].status);

    cudaFree(d_frame);
    cudaFree(d_moved);
    cudaFree(d_cells);
    cudaFree(d_count);
    cudaFree(d_pts);
    cudaFree(d_res);
    vio_destroy(ctx);
    free(frame);
    free(moved);
    free(host_cells);
    free(dev_copy);
    return 0;
}
