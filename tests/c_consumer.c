/* A plain C caller of libseg: the call sequence of one segmentation job through the C-ABI of
 * include/seg.h, host buffers in and out. A bright 40 x 40 square on a dark 96 x 96 noiseless
 * image, started from a 24 x 24 square label; 30 piecewise-constant Sobolev iterations.
 * Prints "ok <particles> <accepted> <foreground pixels>" and exits 0, or prints the error and
 * exits 1. Built by the tests (gcc -std=c99) against libseg.so. */
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include "seg.h"

#define H 96
#define W 96

static int fail(const char* what, int code)
{
    printf("%s: %s (%d) %s\n", what, seg_strerror(code), code, seg_last_cuda_error());
    return 1;
}

int main(void)
{
    static float image[H * W];
    static int32_t labels[H * W];
    for (int y = 0; y < H; y++)
        for (int x = 0; x < W; x++) {
            image[y * W + x] = (y >= 28 && y < 68 && x >= 28 && x < 68) ? 1.0f : 0.0f;
            labels[y * W + x] = (y >= 36 && y < 60 && x >= 36 && x < 60) ? 1 : 0;
        }
    seg_params p;
    memset(&p, 0, sizeof p);          /* every option at its default, reserved fields zero */
    p.ndim = 2;
    p.dtype = SEG_F32;
    p.shape[0] = 1;
    p.shape[1] = H;
    p.shape[2] = W;
    p.model = SEG_PC;
    p.connectivity = 4;
    p.lambda = 0.04;
    p.cutoff = 3.0;
    p.gradient = SEG_SOBOLEV;
    p.validate = 1;

    size_t bytes = 0;
    int rc = seg_estimate_bytes(&p, 2, &bytes);
    if (rc != SEG_OK) return fail("seg_estimate_bytes", rc);
    seg_ctx* ctx = NULL;
    rc = seg_init(&p, image, labels, NULL, &ctx);
    if (rc != SEG_OK) return fail("seg_init", rc);
    seg_status st;
    memset(&st, 0, sizeof st);
    int64_t accepted = 0;
    for (int it = 0; it < 30; it++) {
        rc = seg_step(ctx, 1, &st);
        if (rc != SEG_OK) {
            seg_destroy(ctx);
            return fail("seg_step", rc);
        }
        accepted += st.n_accepted;
    }
    rc = seg_labels(ctx, labels, (size_t)(H * W));
    if (rc != SEG_OK) {
        seg_destroy(ctx);
        return fail("seg_labels", rc);
    }
    int64_t n[2];
    double S[2], Q[2];
    rc = seg_stats(ctx, n, S, Q, 2);
    seg_destroy(ctx);
    if (rc != SEG_OK) return fail("seg_stats", rc);
    int64_t fg = 0;
    for (int i = 0; i < H * W; i++) fg += labels[i] == 1;
    if (fg != n[1] || n[0] + n[1] != H * W) {
        printf("statistics disagree with the labels: %lld %lld %lld\n", (long long)fg, (long long)n[0], (long long)n[1]);
        return 1;
    }
    printf("ok %lld %lld %lld\n", (long long)st.particles_total, (long long)accepted, (long long)fg);
    return 0;
}
