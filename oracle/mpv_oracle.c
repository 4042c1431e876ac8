/*
 * mpv_oracle.c -- CPU oracle for the multi-scale fast MPV stereo matcher.
 *
 * TEST INFRASTRUCTURE ONLY: loaded by the test suite, the smoke check and the
 * benchmark's CPU-baseline leg, never by the CUDA library.  Plain, single-threaded,
 * int64, written for reading against the paper rather than for speed:
 *
 *   cost      Section 3.2, Eq. (components) and Eq. (ssim), in an exact integer form
 *   envelope  Eq. (e(p,u)) with full connectivity, and the two-sweep recursion of
 *             Section 3.3 (Eqs. 1-8) that replaces the O(m^2) minimum by O(2m)
 *   paths     Section 3.2, bi-directional Viterbi along 4 or 8 scan directions,
 *             summed (Eq. viterbi) and reduced by winner-take-all
 *   pyramid   Section 3.4: 2x2 down-sampling, full range at the top level only,
 *             block-mode seeding, per-pixel interpolation at the finest level,
 *             per-pixel search windows with virtual (absent) nodes outside them.
 *
 * Readings of the paper where it is silent or garbled are named R1..R16 below
 * and listed with their justification in the design notes of the repository.
 */
#include "mpv_oracle.h"

#include <stdlib.h>
#include <string.h>

#define ORA_INF (((int64_t)1) << 60)

static int clampi(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }
static int64_t min64(int64_t a, int64_t b) { return a < b ? a : b; }
static int64_t abs64(int64_t a) { return a < 0 ? -a : a; }

/* ------------------------------------------------------------------------------ */
/* Cost: Section 3.2                                                                */
/* ------------------------------------------------------------------------------ */

/* C1 = (K1 L)^2, C2 = (K2 L)^2 with K1 = 0.01, K2 = 0.03, L = 255 (R3: the paper only
 * says K << 1; these are the values of the SSIM paper it follows).  The sums below are
 * n^2 times the means/variances, so the constants are scaled by n^2 and rounded half
 * up (R4).  (K1 L)^2 n^2 = 65025 n^2 / 10^4 and (K2 L)^2 n^2 = 585225 n^2 / 10^4.     */
int64_t ora_c1(int N)
{
    int64_t n = (int64_t)N * N;
    return (65025 * n * n + 5000) / 10000;
}

int64_t ora_c2(int N)
{
    int64_t n = (int64_t)N * N;
    return (585225 * n * n + 5000) / 10000;
}

/* SSIM matching cost with alpha = beta = gamma = 1 and C3 = C2/2 (Eq. ssim).  With
 * those exponents l*c*s is the closed form
 *     (2 mu_x mu_y + C1)(2 sigma_xy + C2) / ((mu_x^2 + mu_y^2 + C1)(sigma_x^2 + sigma_y^2 + C2))
 * (R2: Eq. components prints the contrast denominator and the structure term garbled;
 * the standard definitions of the cited SSIM paper are used).  Multiplying every
 * mean by n and every second moment by n^2 gives integers:
 *     A1 = 2 Sx Sy + c1,   B1 = Sx^2 + Sy^2 + c1,
 *     A2 = 2 (n Sxy - Sx Sy) + c2,   B2 = n (Sxx + Syy) - Sx^2 - Sy^2 + c2,
 * SSIM = A1 A2 / (B1 B2), and cost = floor(L (1 - SSIM) / 2) = floor(255 (den-num) / (2 den)).
 * Patches are N x N, centred at (x,y) in I0 and (x-u,y) in I1, with coordinates
 * clamped to the image (R1: N unspecified, default 5).  A match that falls left of
 * I1 (x - u < 0) costs the maximum, 255 (R5).                                        */
int32_t ora_ssim_cost(const uint8_t *I0, const uint8_t *I1, int W, int H, int pitch,
                      int N, int x, int y, int u)
{
    if (x - u < 0) return 255;
    const int r = (N - 1) / 2;
    const int64_t n = (int64_t)N * N;
    int64_t Sx = 0, Sy = 0, Sxx = 0, Syy = 0, Sxy = 0;
    for (int dy = -r; dy <= r; ++dy) {
        const int yy = clampi(y + dy, 0, H - 1);
        for (int dx = -r; dx <= r; ++dx) {
            const int64_t a = I0[(int64_t)yy * pitch + clampi(x + dx, 0, W - 1)];
            const int64_t b = I1[(int64_t)yy * pitch + clampi(x - u + dx, 0, W - 1)];
            Sx += a;
            Sy += b;
            Sxx += a * a;
            Syy += b * b;
            Sxy += a * b;
        }
    }
    const int64_t c1 = ora_c1(N), c2 = ora_c2(N);
    const int64_t A1 = 2 * Sx * Sy + c1;
    const int64_t B1 = Sx * Sx + Sy * Sy + c1;
    const int64_t A2 = 2 * (n * Sxy - Sx * Sy) + c2;
    const int64_t B2 = n * (Sxx + Syy) - Sx * Sx - Sy * Sy + c2;
    const int64_t num = A1 * A2;
    const int64_t den = B1 * B2;
    return (int32_t)((255 * (den - num)) / (2 * den));
}

void ora_cost_volume(const uint8_t *I0, const uint8_t *I1, int W, int H, int pitch, int N,
                     const int32_t *lo, int Dw, int32_t *C)
{
    for (int y = 0; y < H; ++y)
        for (int x = 0; x < W; ++x) {
            const int base = lo ? lo[(int64_t)y * W + x] : 0;
            int32_t *c = C + ((int64_t)y * W + x) * Dw;
            for (int k = 0; k < Dw; ++k)
                c[k] = ora_ssim_cost(I0, I1, W, H, pitch, N, x, y, base + k);
        }
}

/* ------------------------------------------------------------------------------ */
/* Min-convolution with the jump penalty: Eq. (e(p,u)) and Section 3.3               */
/* ------------------------------------------------------------------------------ */

/* Jump penalty eps(u,v) = min(p1 |u - v|, T): the TV term lambda |u - u'| of Eq. (EU)
 * with constant weight (the gradient weighting e^{-|G|} is not part of the plain
 * path), truncated at T (R6; T = ORA_NO_TRUNC keeps the paper's literal form).      */
static int64_t eps(int64_t u, int64_t v, int64_t p1, int64_t T)
{
    const int64_t e = p1 * abs64(u - v);
    return (T >= ORA_NO_TRUNC) ? e : min64(e, T);
}

/* Full connectivity (L_u = all nodes of the previous pixel): O(Dw^2). */
void ora_envelope_naive(const int64_t *A, int lo_prev, int lo, int Dw, int64_t p1,
                        int64_t T, int64_t *M)
{
    for (int k = 0; k < Dw; ++k) {
        int64_t best = ORA_INF;
        for (int j = 0; j < Dw; ++j)
            best = min64(best, A[j] + eps(lo + k, lo_prev + j, p1, T));
        M[k] = best;
    }
}

/* Section 3.3: since eps(u,v) = p1 + eps(u-1,v) for u > v (Eq. 6 with unit step p1),
 * the minimum over all predecessors splits into one upward sweep over u (predecessors
 * v <= u) and one downward sweep (v >= u), each O(m):
 *     F(u) = min(A(u), F(u-1) + p1),     M(u) = min(F(u), M(u+1) + p1),
 * then the truncation M'(u) = min(M(u), min_v A(v) + T) (R7: Eqs. 2 and 8 are printed
 * with garbled indices and only the v <= u side).  Labels are absolute disparities, so
 * a pixel whose window differs from its predecessor's connects through the penalty;
 * labels outside the predecessor's window are virtual nodes with infinite energy (R8).
 */
void ora_envelope_fast(const int64_t *A, int lo_prev, int lo, int Dw, int64_t p1,
                       int64_t T, int64_t *M)
{
    const int ulo = lo < lo_prev ? lo : lo_prev;
    const int uhi = (lo > lo_prev ? lo : lo_prev) + Dw;  /* exclusive */
    const int n = uhi - ulo;
    int64_t *F = (int64_t *)malloc(sizeof(int64_t) * (size_t)n);
    int64_t amin = ORA_INF;
    for (int j = 0; j < Dw; ++j) amin = min64(amin, A[j]);
    /* upward sweep */
    int64_t run = ORA_INF;
    for (int i = 0; i < n; ++i) {
        const int u = ulo + i;
        const int64_t a = (u >= lo_prev && u < lo_prev + Dw) ? A[u - lo_prev] : ORA_INF;
        run = min64(a, run + p1);
        if (run > ORA_INF) run = ORA_INF;
        F[i] = run;
    }
    /* downward sweep */
    run = ORA_INF;
    for (int i = n - 1; i >= 0; --i) {
        run = min64(F[i], run + p1);
        if (run > ORA_INF) run = ORA_INF;
        F[i] = run;
    }
    for (int k = 0; k < Dw; ++k) {
        int64_t m = F[lo + k - ulo];
        if (T < ORA_NO_TRUNC) m = min64(m, amin + T);
        M[k] = m;
    }
    free(F);
}

/* ------------------------------------------------------------------------------ */
/* Directional Viterbi passes and their sum                                          */
/* ------------------------------------------------------------------------------ */

/* Viterbi recursion along direction r = (dx,dy): the first in-image pixel of a path
 * takes its own cost, every later pixel p adds its cost to the envelope of the
 * predecessor p - r (Eq. e(p,u)).  The bounded form subtracts min_v L(p-r, v), a
 * per-pixel constant that does not change any argmin of the sum.                   */
int ora_path(const int32_t *C, const int32_t *lo, int W, int H, int Dw, int dx, int dy,
             int64_t p1, int64_t T, int normalized, int use_naive, int check, int64_t *L)
{
    int status = 0;
    int64_t *M = (int64_t *)malloc(sizeof(int64_t) * (size_t)Dw);
    int64_t *M2 = (int64_t *)malloc(sizeof(int64_t) * (size_t)Dw);
    for (int yi = 0; yi < H; ++yi) {
        const int y = dy >= 0 ? yi : H - 1 - yi;
        for (int xi = 0; xi < W; ++xi) {
            const int x = dx >= 0 ? xi : W - 1 - xi;
            const int64_t idx = (int64_t)y * W + x;
            const int32_t *c = C + idx * Dw;
            int64_t *l = L + idx * Dw;
            const int px = x - dx, py = y - dy;
            if (px < 0 || px >= W || py < 0 || py >= H) {
                for (int k = 0; k < Dw; ++k) l[k] = c[k];
                continue;
            }
            const int64_t pidx = (int64_t)py * W + px;
            const int64_t *A = L + pidx * Dw;
            const int lo_p = lo ? lo[idx] : 0;
            const int lo_q = lo ? lo[pidx] : 0;
            if (use_naive)
                ora_envelope_naive(A, lo_q, lo_p, Dw, p1, T, M);
            else
                ora_envelope_fast(A, lo_q, lo_p, Dw, p1, T, M);
            if (check) {
                if (use_naive)
                    ora_envelope_fast(A, lo_q, lo_p, Dw, p1, T, M2);
                else
                    ora_envelope_naive(A, lo_q, lo_p, Dw, p1, T, M2);
                for (int k = 0; k < Dw; ++k)
                    if (M[k] != M2[k]) status = -1;
            }
            int64_t amin = ORA_INF;
            for (int j = 0; j < Dw; ++j) amin = min64(amin, A[j]);
            for (int k = 0; k < Dw; ++k)
                l[k] = (int64_t)c[k] + M[k] - (normalized ? amin : 0);
        }
    }
    free(M);
    free(M2);
    return status;
}

/* Scan directions: horizontal pair, vertical pair, then the two diagonal pairs
 * (Table alg, steps 1-4; Fig. search_path).                                          */
static const int ora_dirs[8][2] = {{1, 0}, {-1, 0}, {0, 1}, {0, -1},
                                   {1, 1}, {-1, -1}, {-1, 1}, {1, -1}};

int ora_aggregate(const int32_t *C, const int32_t *lo, int W, int H, int Dw, int num_paths,
                  int64_t p1, int64_t T, int normalized, int64_t *S)
{
    const int64_t n = (int64_t)W * H * Dw;
    int64_t *L = (int64_t *)malloc(sizeof(int64_t) * (size_t)n);
    if (!L) return -2;
    memset(S, 0, sizeof(int64_t) * (size_t)n);
    int status = 0;
    for (int r = 0; r < num_paths; ++r) {
        if (ora_path(C, lo, W, H, Dw, ora_dirs[r][0], ora_dirs[r][1], p1, T, normalized, 0, 0,
                     L))
            status = -1;
        for (int64_t i = 0; i < n; ++i) S[i] += L[i];
    }
    free(L);
    return status;
}

/* ------------------------------------------------------------------------------ */
/* Penalties per step: the gradient-weighted TV term and the paper's asymmetric     */
/* left-to-right pass; the hierarchical merge of Section 3.2                         */
/* ------------------------------------------------------------------------------ */

static int64_t eps_pen(int64_t u, int64_t v, const ora_penalty *e)
{
    if (u == v) return 0;
    const int64_t up = u > v;
    const int64_t d = up ? u - v : v - u;
    const int64_t slope = up ? e->p_up : e->p_dn;
    const int64_t T = up ? e->T_up : e->T_dn;
    const int64_t x = slope * d;
    return (T >= ORA_NO_TRUNC) ? x : min64(x, T);
}

/* Full connectivity with the step's penalty: O(Dw^2). */
void ora_envelope_naive_pen(const int64_t *A, int lo_prev, int lo, int Dw,
                            const ora_penalty *e, int64_t *M)
{
    for (int k = 0; k < Dw; ++k) {
        int64_t best = ORA_INF;
        for (int j = 0; j < Dw; ++j)
            best = min64(best, A[j] + eps_pen(lo + k, lo_prev + j, e));
        M[k] = best;
    }
}

/* Section 3.3 with two slopes: predecessors v <= u are reached by the upward sweep
 *     F(u) = min(A(u), F(u-1) + p_up),
 * predecessors v >= u by the downward sweep
 *     G(u) = min(A(u), G(u+1) + p_dn),
 * and the truncations by the running minima of A from each side:
 *     M'(u) = min(F(u), G(u), min_{v<=u} A(v) + T_up, min_{v>=u} A(v) + T_dn).
 * With p_up = p_dn and T_up = T_dn this is the symmetric envelope of ora_envelope_fast. */
void ora_envelope_fast_pen(const int64_t *A, int lo_prev, int lo, int Dw,
                           const ora_penalty *e, int64_t *M)
{
    const int ulo = lo < lo_prev ? lo : lo_prev;
    const int uhi = (lo > lo_prev ? lo : lo_prev) + Dw;  /* exclusive */
    const int n = uhi - ulo;
    int64_t *F = (int64_t *)malloc(sizeof(int64_t) * (size_t)n);
    int64_t *G = (int64_t *)malloc(sizeof(int64_t) * (size_t)n);
    int64_t *P = (int64_t *)malloc(sizeof(int64_t) * (size_t)n);
    int64_t *Sm = (int64_t *)malloc(sizeof(int64_t) * (size_t)n);
    int64_t run = ORA_INF, pm = ORA_INF;
    for (int i = 0; i < n; ++i) {
        const int u = ulo + i;
        const int64_t a = (u >= lo_prev && u < lo_prev + Dw) ? A[u - lo_prev] : ORA_INF;
        run = min64(a, run + e->p_up);
        if (run > ORA_INF) run = ORA_INF;
        pm = min64(pm, a);
        F[i] = run;
        P[i] = pm;
    }
    run = ORA_INF;
    pm = ORA_INF;
    for (int i = n - 1; i >= 0; --i) {
        const int u = ulo + i;
        const int64_t a = (u >= lo_prev && u < lo_prev + Dw) ? A[u - lo_prev] : ORA_INF;
        run = min64(a, run + e->p_dn);
        if (run > ORA_INF) run = ORA_INF;
        pm = min64(pm, a);
        G[i] = run;
        Sm[i] = pm;
    }
    for (int k = 0; k < Dw; ++k) {
        const int i = lo + k - ulo;
        int64_t m = min64(F[i], G[i]);
        if (e->T_up < ORA_NO_TRUNC) m = min64(m, P[i] + e->T_up);
        if (e->T_dn < ORA_NO_TRUNC) m = min64(m, Sm[i] + e->T_dn);
        M[k] = m;
    }
    free(F);
    free(G);
    free(P);
    free(Sm);
}

/* Slope of the step into pixel (x,y) from its predecessor (px,py): Eq. EU weights the
 * TV term by e^{-|G|}, G the intensity gradient of I0; here G is the intensity
 * difference between the two pixels the step connects, and the weight comes from a
 * caller-supplied table of 256 integer slopes (f2 reading: the table replaces
 * lambda e^{-|G|} and keeps the penalty an integer).                                  */
static int64_t step_slope(int64_t p1, const int32_t *lut, const uint8_t *I0, int pitch, int x,
                          int y, int px, int py)
{
    if (!lut) return p1;
    const int a = I0[(int64_t)y * pitch + x], b = I0[(int64_t)py * pitch + px];
    return lut[a > b ? a - b : b - a];
}

/* Section 3.4, read literally (f3): the top level split into block x block tiles, each
 * tile its own MPV problem - a step whose predecessor lies in another tile starts the
 * scan path anew.  block = 0: no split.                                               */
static int crosses_block(int x, int y, int px, int py, int block)
{
    return block > 0 && (x / block != px / block || y / block != py / block);
}

static int path_pen_impl(const int64_t *Q, const int32_t *lo, int W, int H, int Dw, int dx,
                         int dy, int64_t p1, int64_t T, const int32_t *lut, const uint8_t *I0,
                         int pitch, int double_up, int normalize_out, int use_naive, int check,
                         int block, int64_t *L);

int ora_path_pen(const int64_t *Q, const int32_t *lo, int W, int H, int Dw, int dx, int dy,
                 int64_t p1, int64_t T, const int32_t *lut, const uint8_t *I0, int pitch,
                 int double_up, int normalize_out, int use_naive, int check, int64_t *L)
{
    return path_pen_impl(Q, lo, W, H, Dw, dx, dy, p1, T, lut, I0, pitch, double_up,
                         normalize_out, use_naive, check, 0, L);
}

static int path_pen_impl(const int64_t *Q, const int32_t *lo, int W, int H, int Dw, int dx,
                         int dy, int64_t p1, int64_t T, const int32_t *lut, const uint8_t *I0,
                         int pitch, int double_up, int normalize_out, int use_naive, int check,
                         int block, int64_t *L)
{
    int status = 0;
    int64_t *M = (int64_t *)malloc(sizeof(int64_t) * (size_t)Dw);
    int64_t *M2 = (int64_t *)malloc(sizeof(int64_t) * (size_t)Dw);
    /* the bounded energies of the predecessor are kept apart from the output, which
     * may be normalised                                                              */
    int64_t *B = (int64_t *)malloc(sizeof(int64_t) * (size_t)W * H * Dw);
    for (int yi = 0; yi < H; ++yi) {
        const int y = dy >= 0 ? yi : H - 1 - yi;
        for (int xi = 0; xi < W; ++xi) {
            const int x = dx >= 0 ? xi : W - 1 - xi;
            const int64_t idx = (int64_t)y * W + x;
            const int64_t *q = Q + idx * Dw;
            int64_t *b = B + idx * Dw;
            const int px = x - dx, py = y - dy;
            if (px < 0 || px >= W || py < 0 || py >= H || crosses_block(x, y, px, py, block)) {
                for (int k = 0; k < Dw; ++k) b[k] = q[k];
            } else {
                const int64_t pidx = (int64_t)py * W + px;
                const int64_t *A = B + pidx * Dw;
                const int lo_p = lo ? lo[idx] : 0;
                const int lo_q = lo ? lo[pidx] : 0;
                const int64_t P = step_slope(p1, lut, I0, pitch, x, y, px, py);
                ora_penalty e;
                e.p_dn = P;
                e.T_dn = T;
                e.p_up = double_up ? 2 * P : P;
                e.T_up = (double_up && T < ORA_NO_TRUNC) ? 2 * T : T;
                if (use_naive)
                    ora_envelope_naive_pen(A, lo_q, lo_p, Dw, &e, M);
                else
                    ora_envelope_fast_pen(A, lo_q, lo_p, Dw, &e, M);
                if (check) {
                    if (use_naive)
                        ora_envelope_fast_pen(A, lo_q, lo_p, Dw, &e, M2);
                    else
                        ora_envelope_naive_pen(A, lo_q, lo_p, Dw, &e, M2);
                    for (int k = 0; k < Dw; ++k)
                        if (M[k] != M2[k]) status = -1;
                }
                int64_t amin = ORA_INF;
                for (int j = 0; j < Dw; ++j) amin = min64(amin, A[j]);
                for (int k = 0; k < Dw; ++k) b[k] = q[k] + M[k] - amin;
            }
            int64_t bmin = ORA_INF;
            for (int k = 0; k < Dw; ++k) bmin = min64(bmin, b[k]);
            int64_t *l = L + idx * Dw;
            for (int k = 0; k < Dw; ++k) l[k] = b[k] - (normalize_out ? bmin : 0);
        }
    }
    free(B);
    free(M);
    free(M2);
    return status;
}

static int aggregate_grad_impl(const int32_t *C, const int32_t *lo, int W, int H, int Dw,
                               int num_paths, int64_t p1, int64_t T, const int32_t *lut,
                               const uint8_t *I0, int pitch, int block, int64_t *S);

int ora_aggregate_grad(const int32_t *C, const int32_t *lo, int W, int H, int Dw,
                       int num_paths, int64_t p1, int64_t T, const int32_t *lut,
                       const uint8_t *I0, int pitch, int64_t *S)
{
    return aggregate_grad_impl(C, lo, W, H, Dw, num_paths, p1, T, lut, I0, pitch, 0, S);
}

static int aggregate_grad_impl(const int32_t *C, const int32_t *lo, int W, int H, int Dw,
                               int num_paths, int64_t p1, int64_t T, const int32_t *lut,
                               const uint8_t *I0, int pitch, int block, int64_t *S)
{
    const int64_t n = (int64_t)W * H * Dw;
    int64_t *Q = (int64_t *)malloc(sizeof(int64_t) * (size_t)n);
    int64_t *L = (int64_t *)malloc(sizeof(int64_t) * (size_t)n);
    if (!Q || !L) {
        free(Q);
        free(L);
        return -2;
    }
    for (int64_t i = 0; i < n; ++i) Q[i] = C[i];
    memset(S, 0, sizeof(int64_t) * (size_t)n);
    int status = 0;
    for (int r = 0; r < num_paths; ++r) {
        if (path_pen_impl(Q, lo, W, H, Dw, ora_dirs[r][0], ora_dirs[r][1], p1, T, lut, I0,
                          pitch, 0, 0, 0, 0, block, L))
            status = -1;
        for (int64_t i = 0; i < n; ++i) S[i] += L[i];
    }
    free(Q);
    free(L);
    return status;
}

/* Section 3.2, Fig. merging and Table alg: the passes run in layers - left/right,
 * up/down, then the two diagonal pairs - each layer a forward and a backward pass over
 * the previous layer's node energies (the cost for the first layer).  The two passes
 * of a layer are compared after per-pixel min-normalisation (reading: the paper gives
 * no scale for the energies it merges), and merged by the minimum for the horizontal
 * layer (sharper edges) and by the mean, rounded down, for the others (less noise).
 * The left-to-right pass charges a jump from a smaller to a larger disparity twice
 * (reading: "twice penalty" doubles both the slope and the truncation).  The last
 * layer's merged energies are the output.                                            */
static int aggregate_paper_impl(const int32_t *C, const int32_t *lo, int W, int H, int Dw,
                                int num_paths, int64_t p1, int64_t T, const int32_t *lut,
                                const uint8_t *I0, int pitch, int block, int64_t *S);

int ora_aggregate_paper(const int32_t *C, const int32_t *lo, int W, int H, int Dw,
                        int num_paths, int64_t p1, int64_t T, const int32_t *lut,
                        const uint8_t *I0, int pitch, int64_t *S)
{
    return aggregate_paper_impl(C, lo, W, H, Dw, num_paths, p1, T, lut, I0, pitch, 0, S);
}

int ora_aggregate_blocks(const int32_t *C, const int32_t *lo, int W, int H, int Dw,
                         int num_paths, int64_t p1, int64_t T, const int32_t *lut,
                         const uint8_t *I0, int pitch, int merge_mode, int block, int64_t *S)
{
    if (merge_mode == ORA_MERGE_PAPER)
        return aggregate_paper_impl(C, lo, W, H, Dw, num_paths, p1, T, lut, I0, pitch, block, S);
    return aggregate_grad_impl(C, lo, W, H, Dw, num_paths, p1, T, lut, I0, pitch, block, S);
}

static int aggregate_paper_impl(const int32_t *C, const int32_t *lo, int W, int H, int Dw,
                                int num_paths, int64_t p1, int64_t T, const int32_t *lut,
                                const uint8_t *I0, int pitch, int block, int64_t *S)
{
    const int64_t n = (int64_t)W * H * Dw;
    int64_t *Q = (int64_t *)malloc(sizeof(int64_t) * (size_t)n);
    int64_t *F = (int64_t *)malloc(sizeof(int64_t) * (size_t)n);
    int64_t *B = (int64_t *)malloc(sizeof(int64_t) * (size_t)n);
    if (!Q || !F || !B) {
        free(Q);
        free(F);
        free(B);
        return -2;
    }
    for (int64_t i = 0; i < n; ++i) Q[i] = C[i];
    int status = 0;
    const int layers = num_paths / 2;
    for (int layer = 0; layer < layers; ++layer) {
        const int *fw = ora_dirs[2 * layer], *bw = ora_dirs[2 * layer + 1];
        const int double_up = (fw[0] == 1 && fw[1] == 0);
        if (path_pen_impl(Q, lo, W, H, Dw, fw[0], fw[1], p1, T, lut, I0, pitch, double_up, 1,
                          0, 0, block, F))
            status = -1;
        if (path_pen_impl(Q, lo, W, H, Dw, bw[0], bw[1], p1, T, lut, I0, pitch, 0, 1, 0, 0,
                          block, B))
            status = -1;
        for (int64_t i = 0; i < n; ++i)
            Q[i] = layer == 0 ? min64(F[i], B[i]) : (F[i] + B[i]) / 2;
    }
    memcpy(S, Q, sizeof(int64_t) * (size_t)n);
    free(Q);
    free(F);
    free(B);
    return status;
}

/* Winner-take-all over each pixel's window, ties to the smallest disparity (R9). */
void ora_wta(const int64_t *S, const int32_t *lo, int W, int H, int Dw, uint16_t *d)
{
    for (int64_t i = 0; i < (int64_t)W * H; ++i) {
        const int64_t *s = S + i * Dw;
        int best = 0;
        for (int k = 1; k < Dw; ++k)
            if (s[k] < s[best]) best = k;
        d[i] = (uint16_t)((lo ? lo[i] : 0) + best);
    }
}

/* ------------------------------------------------------------------------------ */
/* Pyramid: Section 3.4                                                              */
/* ------------------------------------------------------------------------------ */

/* 2x2 box average, round half up, the last row/column replicated when odd (R12). */
void ora_downsample2(const uint8_t *in, int W, int H, int pitch, uint8_t *out, int out_pitch)
{
    const int W2 = (W + 1) / 2, H2 = (H + 1) / 2;
    for (int y = 0; y < H2; ++y)
        for (int x = 0; x < W2; ++x) {
            const int x0 = 2 * x, x1 = clampi(2 * x + 1, 0, W - 1);
            const int y0 = 2 * y, y1 = clampi(2 * y + 1, 0, H - 1);
            const int s = in[(int64_t)y0 * pitch + x0] + in[(int64_t)y0 * pitch + x1] +
                          in[(int64_t)y1 * pitch + x0] + in[(int64_t)y1 * pitch + x1];
            out[(int64_t)y * out_pitch + x] = (uint8_t)((s + 2) >> 2);
        }
}

void ora_level_dims(int W, int H, int S, int l, int *Wl, int *Hl)
{
    int w = W, h = H;
    for (int i = S - 1; i > l; --i) {
        w = (w + 1) / 2;
        h = (h + 1) / 2;
    }
    *Wl = w;
    *Hl = h;
}

/* Top level searches ceil(D / 2^(S-1)) labels: a quarter of the range for three
 * scales (Section 3.4).                                                            */
int ora_level_range(int D, int S, int l)
{
    const int sh = S - 1 - l;
    return (D + (1 << sh) - 1) >> sh;
}

/* The top level covers its full range; finer level l searches a window of Dw_l
 * labels: windows[l-1] when set, else `window`, else D/4 (R15, from Eqs. Ot1 and Ot2,
 * whose d/4 becomes a width per level in the variable form), clamped to the level's
 * range D_l.                                                                         */
int ora_level_window(const ora_params *p, int l)
{
    const int Dl = ora_level_range(p->max_disparity, p->num_scales, l);
    if (l == 0) return Dl;
    int Dw = p->windows[l - 1] > 0 ? p->windows[l - 1]
                                    : (p->window > 0 ? p->window : p->max_disparity / 4);
    if (Dw < 1) Dw = 1;
    return Dw < Dl ? Dw : Dl;
}

static int level_block(const ora_params *p, int l)
{
    const int b = p->block[l - 1];
    if (b > 0) return b;
    return (l == p->num_scales - 1) ? 1 : 2;
}

/* Seeding of a finer level from the coarser WTA map (Section 3.4): every coarse
 * disparity is doubled (the sampling rate).  With a block side b >= 2 the mode of the
 * doubled values over each b x b block of coarse pixels (ties to the smaller value)
 * seeds every child pixel of that block.  With b = 1 (the last level, where "each
 * pixel is a block") a child at even (x,y) takes its parent's doubled value and the
 * other children the rounded mean of their 2 or 4 nearest doubled parents (R14), the
 * neighbour index clamped at the border.  The window is [lo, lo+Dw) with
 * lo = clamp(c - Dw/2, 0, Dl - Dw).                                                   */
void ora_seed(const uint16_t *dprev, int Wp, int Hp, int W, int H, int block, int Dw,
              int Dl, int32_t *lo)
{
    int *vals = (int *)malloc(sizeof(int) * (size_t)(block * block + 1));
    for (int y = 0; y < H; ++y)
        for (int x = 0; x < W; ++x) {
            int c;
            if (block >= 2) {
                const int bx = (x / 2) / block, by = (y / 2) / block;
                int cnt = 0;
                for (int qy = by * block; qy < (by + 1) * block && qy < Hp; ++qy)
                    for (int qx = bx * block; qx < (bx + 1) * block && qx < Wp; ++qx)
                        vals[cnt++] = 2 * (int)dprev[(int64_t)qy * Wp + qx];
                int best = vals[0], best_n = 0;
                for (int i = 0; i < cnt; ++i) {
                    int m = 0;
                    for (int j = 0; j < cnt; ++j) m += (vals[j] == vals[i]);
                    if (m > best_n || (m == best_n && vals[i] < best)) {
                        best = vals[i];
                        best_n = m;
                    }
                }
                c = best;
            } else {
                int xs[2], ys[2], nx, ny;
                if (x % 2 == 0) {
                    xs[0] = x / 2;
                    nx = 1;
                } else {
                    xs[0] = (x - 1) / 2;
                    xs[1] = clampi((x + 1) / 2, 0, Wp - 1);
                    nx = 2;
                }
                if (y % 2 == 0) {
                    ys[0] = y / 2;
                    ny = 1;
                } else {
                    ys[0] = (y - 1) / 2;
                    ys[1] = clampi((y + 1) / 2, 0, Hp - 1);
                    ny = 2;
                }
                int sum = 0;
                for (int i = 0; i < ny; ++i)
                    for (int j = 0; j < nx; ++j)
                        sum += 2 * (int)dprev[(int64_t)ys[i] * Wp + xs[j]];
                const int k = nx * ny;
                c = (sum + k / 2) / k;
            }
            lo[(int64_t)y * W + x] = clampi(c - Dw / 2, 0, Dl - Dw);
        }
    free(vals);
}

int64_t ora_node_count(int W, int H, const ora_params *p)
{
    int64_t total = 0;
    for (int l = 0; l < p->num_scales; ++l) {
        int Wl, Hl;
        ora_level_dims(W, H, p->num_scales, l, &Wl, &Hl);
        total += (int64_t)Wl * Hl * ora_level_window(p, l);
    }
    return total;
}

int ora_check_params(int W, int H, const ora_params *p)
{
    const int N = p->ssim_window;
    if (N != 3 && N != 5) return -1;
    if (p->num_scales < 1 || p->num_scales > 4) return -1;
    if (p->num_paths != 4 && p->num_paths != 8) return -1;
    if (p->p1 < 0 || p->trunc < 0 || p->window < 0 || p->lr_tol < 0) return -1;
    if (W < N || H < N) return -1;
    if (p->max_disparity < 1 || p->max_disparity > W || p->max_disparity > 1024) return -1;
    int W0, H0;
    ora_level_dims(W, H, p->num_scales, 0, &W0, &H0);
    if (W0 < N || H0 < N) return -1;
    for (int l = 1; l < p->num_scales; ++l)
        if (p->block[l - 1] < 0 || p->block[l - 1] > 8 || p->windows[l - 1] < 0) return -1;
    if (p->merge_mode != ORA_MERGE_SUM && p->merge_mode != ORA_MERGE_PAPER) return -1;
    if (p->top_block < 0) return -1;
    if (p->grad_lut)
        for (int g = 0; g < 256; ++g)
            if (p->grad_lut[g] < 0 || p->grad_lut[g] > p->p1) return -1;
    const int64_t jump = (int64_t)p->p1 * (p->max_disparity - 1);
    const int64_t pen = p->trunc < jump ? p->trunc : jump;
    if ((int64_t)p->num_paths * (255 + pen) >= 65535) return -1;
    return 0;
}

/* ------------------------------------------------------------------------------ */
/* The matcher                                                                       */
/* ------------------------------------------------------------------------------ */

typedef struct {
    int W, H;
    uint8_t *I0, *I1;  /* pitch = W */
} ora_level_img;

static void build_pyramid(const uint8_t *I0, const uint8_t *I1, int W, int H, int pitch,
                          int S, ora_level_img *lv)
{
    for (int l = S - 1; l >= 0; --l) {
        int Wl, Hl;
        ora_level_dims(W, H, S, l, &Wl, &Hl);
        lv[l].W = Wl;
        lv[l].H = Hl;
        lv[l].I0 = (uint8_t *)malloc((size_t)Wl * Hl);
        lv[l].I1 = (uint8_t *)malloc((size_t)Wl * Hl);
        if (l == S - 1) {
            for (int y = 0; y < H; ++y) {
                memcpy(lv[l].I0 + (int64_t)y * W, I0 + (int64_t)y * pitch, (size_t)W);
                memcpy(lv[l].I1 + (int64_t)y * W, I1 + (int64_t)y * pitch, (size_t)W);
            }
        } else {
            ora_downsample2(lv[l + 1].I0, lv[l + 1].W, lv[l + 1].H, lv[l + 1].W, lv[l].I0, Wl);
            ora_downsample2(lv[l + 1].I1, lv[l + 1].W, lv[l + 1].H, lv[l + 1].W, lv[l].I1, Wl);
        }
    }
}

static void free_pyramid(ora_level_img *lv, int S)
{
    for (int l = 0; l < S; ++l) {
        free(lv[l].I0);
        free(lv[l].I1);
    }
}

/* Runs levels 0..last of one view; fills the stage buffers of level `last` when given. */
static int run_view(const uint8_t *I0, const uint8_t *I1, int W, int H, int pitch,
                    const ora_params *p, int last, int32_t *lo_out, int32_t *C_out,
                    int64_t *S_out, uint16_t *d_out)
{
    const int S = p->num_scales;
    ora_level_img lv[4];
    build_pyramid(I0, I1, W, H, pitch, S, lv);
    const int64_t T = p->trunc;
    uint16_t *dprev = NULL;
    int Wp = 0, Hp = 0, status = 0;
    for (int l = 0; l <= last; ++l) {
        const int Wl = lv[l].W, Hl = lv[l].H;
        const int Dl = ora_level_range(p->max_disparity, S, l);
        const int Dw = ora_level_window(p, l);
        const int64_t npx = (int64_t)Wl * Hl;
        int32_t *lo = (int32_t *)calloc((size_t)npx, sizeof(int32_t));
        int32_t *C = (int32_t *)malloc(sizeof(int32_t) * (size_t)(npx * Dw));
        int64_t *Sv = (int64_t *)malloc(sizeof(int64_t) * (size_t)(npx * Dw));
        uint16_t *d = (uint16_t *)malloc(sizeof(uint16_t) * (size_t)npx);
        if (!lo || !C || !Sv || !d) {
            free(lo); free(C); free(Sv); free(d); free(dprev);
            free_pyramid(lv, S);
            return -2;
        }
        if (l > 0) ora_seed(dprev, Wp, Hp, Wl, Hl, level_block(p, l), Dw, Dl, lo);
        ora_cost_volume(lv[l].I0, lv[l].I1, Wl, Hl, Wl, p->ssim_window, lo, Dw, C);
        int ag;
        if (l == 0 && p->top_block > 0)
            ag = ora_aggregate_blocks(C, lo, Wl, Hl, Dw, p->num_paths, p->p1, T, p->grad_lut,
                                      lv[l].I0, Wl, p->merge_mode, p->top_block, Sv);
        else if (p->merge_mode == ORA_MERGE_PAPER)
            ag = ora_aggregate_paper(C, lo, Wl, Hl, Dw, p->num_paths, p->p1, T, p->grad_lut,
                                     lv[l].I0, Wl, Sv);
        else if (p->grad_lut)
            ag = ora_aggregate_grad(C, lo, Wl, Hl, Dw, p->num_paths, p->p1, T, p->grad_lut,
                                    lv[l].I0, Wl, Sv);
        else
            ag = ora_aggregate(C, lo, Wl, Hl, Dw, p->num_paths, p->p1, T, 1, Sv);
        if (ag) status = -1;
        ora_wta(Sv, lo, Wl, Hl, Dw, d);
        if (l == last) {
            if (lo_out) memcpy(lo_out, lo, sizeof(int32_t) * (size_t)npx);
            if (C_out) memcpy(C_out, C, sizeof(int32_t) * (size_t)(npx * Dw));
            if (S_out) memcpy(S_out, Sv, sizeof(int64_t) * (size_t)(npx * Dw));
            if (d_out) memcpy(d_out, d, sizeof(uint16_t) * (size_t)npx);
        }
        free(lo);
        free(C);
        free(Sv);
        free(dprev);
        dprev = d;
        Wp = Wl;
        Hp = Hl;
    }
    free(dprev);
    free_pyramid(lv, S);
    return status;
}

int ora_match_view(const uint8_t *I0, const uint8_t *I1, int W, int H, int pitch,
                   const ora_params *p, uint16_t *d)
{
    if (ora_check_params(W, H, p)) return -3;
    return run_view(I0, I1, W, H, pitch, p, p->num_scales - 1, NULL, NULL, NULL, d);
}

int ora_view_stage(const uint8_t *I0, const uint8_t *I1, int W, int H, int pitch,
                   const ora_params *p, int level, int32_t *lo, int32_t *C, int64_t *S,
                   uint16_t *d)
{
    if (ora_check_params(W, H, p)) return -3;
    if (level < 0 || level >= p->num_scales) return -3;
    return run_view(I0, I1, W, H, pitch, p, level, lo, C, S, d);
}

/* Left-right check (not in the paper; R11): keep d_L(x) when the match x - d_L(x) is
 * inside the right image and the right view's disparity there agrees within tol.   */
void ora_lr_check(const uint16_t *dL, const uint16_t *dR, int W, int H, int tol,
                  uint16_t *out)
{
    for (int y = 0; y < H; ++y)
        for (int x = 0; x < W; ++x) {
            const int d = dL[(int64_t)y * W + x];
            uint16_t v = ORA_INVALID;
            if (x - d >= 0) {
                const int dr = dR[(int64_t)y * W + (x - d)];
                const int diff = d > dr ? d - dr : dr - d;
                if (diff <= tol) v = (uint16_t)d;
            }
            out[(int64_t)y * W + x] = v;
        }
}

static void mirror(const uint8_t *in, int W, int H, int pitch, uint8_t *out)
{
    for (int y = 0; y < H; ++y)
        for (int x = 0; x < W; ++x) out[(int64_t)y * W + x] = in[(int64_t)y * pitch + W - 1 - x];
}

/* The right view is the same matcher on the mirrored, swapped pair: matching right
 * pixel x' at disparity u against left pixel x' + u is matching mirrored-right pixel
 * W-1-x' against mirrored-left pixel W-1-x'-u.                                        */
int ora_match(const uint8_t *I0, const uint8_t *I1, int W, int H, int pitch,
              const ora_params *p, uint16_t *dL, uint16_t *dR)
{
    if (ora_check_params(W, H, p)) return -3;
    const int64_t npx = (int64_t)W * H;
    uint16_t *dl = (uint16_t *)malloc(sizeof(uint16_t) * (size_t)npx);
    int status = ora_match_view(I0, I1, W, H, pitch, p, dl);
    if (p->lr_check || dR) {
        uint8_t *m0 = (uint8_t *)malloc((size_t)npx), *m1 = (uint8_t *)malloc((size_t)npx);
        uint16_t *drm = (uint16_t *)malloc(sizeof(uint16_t) * (size_t)npx);
        uint16_t *dr = (uint16_t *)malloc(sizeof(uint16_t) * (size_t)npx);
        mirror(I1, W, H, pitch, m0);
        mirror(I0, W, H, pitch, m1);
        if (ora_match_view(m0, m1, W, H, W, p, drm)) status = -1;
        for (int y = 0; y < H; ++y)
            for (int x = 0; x < W; ++x) dr[(int64_t)y * W + x] = drm[(int64_t)y * W + W - 1 - x];
        if (dR) memcpy(dR, dr, sizeof(uint16_t) * (size_t)npx);
        if (p->lr_check)
            ora_lr_check(dl, dr, W, H, p->lr_tol, dL);
        else
            memcpy(dL, dl, sizeof(uint16_t) * (size_t)npx);
        free(m0); free(m1); free(drm); free(dr);
    } else {
        memcpy(dL, dl, sizeof(uint16_t) * (size_t)npx);
    }
    free(dl);
    return status;
}

/* ------------------------------------------------------------------------------ */
/* Road detection (Section 3.5)                                                      */
/* ------------------------------------------------------------------------------ */

/* Eq. disp_map: the histogram of each image row over the disparities. */
void ora_vdisparity(const uint16_t *U, int W, int H, int pitch, int D, uint32_t *Hx)
{
    memset(Hx, 0, sizeof(uint32_t) * (size_t)H * D);
    for (int y = 0; y < H; ++y)
        for (int x = 0; x < W; ++x) {
            const int u = U[(int64_t)y * pitch + x];
            if (u < D) Hx[(int64_t)y * D + u] += 1;
        }
}

/* Eq. hy: the histogram of each image column; the equation prints the column index in
 * the disparity's Kronecker delta, read as the disparity index (R21).                  */
void ora_udisparity(const uint16_t *U, int W, int H, int pitch, int D, uint32_t *Hy)
{
    memset(Hy, 0, sizeof(uint32_t) * (size_t)W * D);
    for (int y = 0; y < H; ++y)
        for (int x = 0; x < W; ++x) {
            const int u = U[(int64_t)y * pitch + x];
            if (u < D) Hy[(int64_t)x * D + u] += 1;
        }
}

/* Eqs. e and P_hat: e(i,j) = Hx(i,j) + max_{0 < j - j' < eta} e(i-1, j'), e(0,j) = Hx(0,j),
 * a node without an admissible predecessor is unreachable (R22); the path runs over all
 * D disparities and is read back from the best final row.                              */
int64_t ora_road_profile(const uint32_t *Hx, int H, int D, int eta, int32_t *P)
{
    const int64_t NEG = -1;
    int64_t *e = (int64_t *)malloc(sizeof(int64_t) * (size_t)H * D);
    int32_t *from = (int32_t *)malloc(sizeof(int32_t) * (size_t)H * D);
    for (int j = 0; j < H; ++j) {
        e[(int64_t)j * D + 0] = Hx[(int64_t)j * D + 0];
        from[(int64_t)j * D + 0] = -1;
    }
    for (int i = 1; i < D; ++i)
        for (int j = 0; j < H; ++j) {
            int64_t best = NEG;
            int arg = -1;
            for (int jp = j - eta + 1; jp <= j - 1; ++jp) {
                if (jp < 0) continue;
                const int64_t v = e[(int64_t)jp * D + i - 1];
                if (v > best) {
                    best = v;
                    arg = jp;
                }
            }
            e[(int64_t)j * D + i] = best == NEG ? NEG : best + Hx[(int64_t)j * D + i];
            from[(int64_t)j * D + i] = arg;
        }
    int64_t best = NEG;
    int arg = -1;
    for (int j = 0; j < H; ++j) {
        const int64_t v = e[(int64_t)j * D + D - 1];
        if (v > best) {
            best = v;
            arg = j;
        }
    }
    for (int i = D - 1; i >= 0; --i) {
        P[i] = arg;
        if (arg >= 0) arg = from[(int64_t)arg * D + i];
    }
    free(e);
    free(from);
    return best;
}
