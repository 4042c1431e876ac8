/* Drives the CPU oracle's entry points on small, ragged and degenerate cases so that a
 * build with AddressSanitizer and UndefinedBehaviorSanitizer (tests/test_oracle_sanitizers.py)
 * sees every indexing path: one and three scales, 4 and 8 paths, both merges, the
 * gradient table, top-level tiles, per-level windows, N = 3 and 5, the left-right check
 * with both maps, the per-level stage dump, and the road functions on the output.
 * Images come from a fixed linear congruential sequence (test data, not method
 * arithmetic).  Exit status 0 when every call reports success. */
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include "../oracle/mpv_oracle.h"

static uint32_t lcg_state = 12345u;
static uint8_t next_byte(void)
{
    lcg_state = lcg_state * 1664525u + 1013904223u;
    return (uint8_t)(lcg_state >> 24);
}

/* left: smoothed noise; right: left shifted by d (border bytes fresh) */
static void make_pair(int W, int H, int pitch, int d, uint8_t *L, uint8_t *R)
{
    for (int y = 0; y < H; ++y)
        for (int x = 0; x < pitch; ++x) L[y * pitch + x] = next_byte();
    for (int y = 0; y < H; ++y)
        for (int x = 0; x < W; ++x)
            R[y * pitch + x] = x + d < W ? L[y * pitch + x + d] : next_byte();
}

static ora_params base(int D, int S, int paths)
{
    ora_params p;
    memset(&p, 0, sizeof(p));
    p.max_disparity = D;
    p.num_scales = S;
    p.num_paths = paths;
    p.p1 = 10;
    p.trunc = 30;
    p.ssim_window = 5;
    p.lr_check = 1;
    p.lr_tol = 1;
    p.merge_mode = ORA_MERGE_SUM;
    return p;
}

static int run_case(const char *name, int W, int H, const ora_params *p)
{
    const int pitch = W + 3;   /* a pitch wider than the image */
    uint8_t *L = malloc((size_t)pitch * H), *R = malloc((size_t)pitch * H);
    uint16_t *dL = malloc(sizeof(uint16_t) * W * H), *dR = malloc(sizeof(uint16_t) * W * H);
    int bad = 0;
    make_pair(W, H, pitch, 3, L, R);
    if (ora_check_params(W, H, p) != 0) {
        fprintf(stderr, "%s: parameters rejected\n", name);
        bad = 1;
    } else if (ora_match(L, R, W, H, pitch, p, dL, dR) != 0) {
        fprintf(stderr, "%s: ora_match failed\n", name);
        bad = 1;
    }
    for (int l = 0; !bad && l < p->num_scales; ++l) {
        int Wl, Hl;
        ora_level_dims(W, H, p->num_scales, l, &Wl, &Hl);
        const int Dw = ora_level_window(p, l);
        int32_t *lo = malloc(sizeof(int32_t) * Wl * Hl);
        int32_t *C = malloc(sizeof(int32_t) * Wl * Hl * Dw);
        int64_t *S = malloc(sizeof(int64_t) * Wl * Hl * Dw);
        uint16_t *d = malloc(sizeof(uint16_t) * Wl * Hl);
        if (ora_view_stage(L, R, W, H, pitch, p, l, lo, C, S, d) != 0) {
            fprintf(stderr, "%s: ora_view_stage level %d failed\n", name, l);
            bad = 1;
        }
        free(lo);
        free(C);
        free(S);
        free(d);
    }
    if (!bad) {   /* road functions on the left map (0xFFFF pixels are skipped) */
        const int D = p->max_disparity;
        uint32_t *Hx = malloc(sizeof(uint32_t) * H * D), *Hy = malloc(sizeof(uint32_t) * W * D);
        int32_t *P = malloc(sizeof(int32_t) * D);
        ora_vdisparity(dL, W, H, W, D, Hx);
        ora_udisparity(dL, W, H, W, D, Hy);
        (void)ora_road_profile(Hx, H, D, 4, P);
        free(Hx);
        free(Hy);
        free(P);
    }
    free(L);
    free(R);
    free(dL);
    free(dR);
    printf("%s: %s\n", name, bad ? "FAILED" : "ok");
    return bad;
}

int main(void)
{
    int bad = 0;
    int32_t lut[256];
    for (int i = 0; i < 256; ++i) lut[i] = 10 - (i * 10) / 256;
    ora_params p;

    p = base(16, 1, 4);
    bad |= run_case("one scale, 4 paths, 37x23", 37, 23, &p);
    p = base(1, 1, 4);
    bad |= run_case("D = 1, 5x5", 5, 5, &p);
    p = base(32, 3, 8);
    bad |= run_case("three scales, 8 paths, 61x45", 61, 45, &p);
    p = base(32, 3, 8);
    p.ssim_window = 3;
    p.trunc = ORA_NO_TRUNC;
    bad |= run_case("N = 3, untruncated", 41, 29, &p);
    p = base(24, 2, 8);
    p.merge_mode = ORA_MERGE_PAPER;
    bad |= run_case("layered merge", 33, 21, &p);
    p = base(24, 2, 8);
    p.grad_lut = lut;
    bad |= run_case("gradient table", 35, 19, &p);
    p = base(24, 2, 8);
    p.grad_lut = lut;
    p.merge_mode = ORA_MERGE_PAPER;
    bad |= run_case("layered merge with the gradient table", 30, 18, &p);
    p = base(32, 3, 8);
    p.top_block = 4;
    bad |= run_case("top-level tiles", 48, 40, &p);
    p = base(64, 3, 8);
    p.windows[0] = 24;
    p.windows[1] = 10;
    bad |= run_case("per-level windows", 70, 30, &p);
    p = base(32, 3, 8);
    p.block[0] = 3;
    p.block[1] = 2;
    bad |= run_case("mode blocks 3, 2", 53, 37, &p);
    p = base(16, 1, 8);
    p.lr_check = 0;
    bad |= run_case("no left-right check", 20, 12, &p);
    return bad;
}
