/*
 * mpv_oracle.h -- CPU oracle for the multi-scale fast MPV stereo matcher.
 *
 * TEST INFRASTRUCTURE ONLY.  This is a plain, slow, single-threaded restatement of
 * what the matcher computes, written from the paper's definitions (Section 3.2,
 * Section 3.3 and Section 3.4 of "A Robust Real-Time Computing-based Environment
 * Sensing System for Intelligent Vehicle", arXiv 2001.09678).  Only the test suite,
 * the smoke check and the benchmark's CPU-baseline leg may load it.  It shares no
 * code, header, table or constant with the CUDA library, and the CUDA library never
 * loads it.
 *
 * All costs and energies are integers.  Energies are held in int64.
 */
#ifndef MPV_ORACLE_H
#define MPV_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define ORA_INVALID 0xFFFFu
#define ORA_NO_TRUNC 0x7FFFFFFF

#define ORA_MERGE_SUM 0    /* S = sum of the directional passes (Eq. viterbi)          */
#define ORA_MERGE_PAPER 1  /* hierarchical layers H, V, two diagonals (Section 3.2)   */

typedef struct {
    int32_t max_disparity;  /* D: labels 0..D-1 at full resolution              */
    int32_t num_scales;     /* S: pyramid levels, factor 2 (Section 3.4)          */
    int32_t num_paths;      /* 4 (horizontal + vertical) or 8 (+ two diagonals)   */
    int32_t p1;             /* lambda: penalty per pixel of disparity jump (Eq. EU) */
    int32_t trunc;          /* T: truncation of the jump penalty, ORA_NO_TRUNC = none */
    int32_t ssim_window;    /* N: SSIM patch side, 3 or 5                          */
    int32_t window;         /* Dw at the finer levels; 0 selects D/4              */
    int32_t block[4];       /* mode-block side per finer level (1 = interpolate)  */
    int32_t lr_check;       /* 1: left-right consistency check on the output      */
    int32_t lr_tol;         /* accepted |d_L - d_R| in pixels                      */
    int32_t merge_mode;     /* ORA_MERGE_SUM or ORA_MERGE_PAPER                    */
    const int32_t *grad_lut;/* NULL, or 256 jump slopes indexed by |I0(p) - I0(p-r)| */
    int32_t top_block;      /* > 0: top level split into independent tiles of this side */
    int32_t windows[4];     /* Dw of finer level l at index l-1; 0 takes `window`  */
} ora_params;

/* Integer SSIM constants: round(C1 * n^2), round(C2 * n^2), n = N*N. */
int64_t ora_c1(int N);
int64_t ora_c2(int N);

/* Matching cost of pixel (x,y) at absolute disparity u (Eq. components, Eq. ssim). */
int32_t ora_ssim_cost(const uint8_t *I0, const uint8_t *I1, int W, int H, int pitch,
                      int N, int x, int y, int u);

/* Cost volume C[y][x][k], k in [0,Dw), disparity u = lo[y*W+x] + k (lo may be NULL = 0). */
void ora_cost_volume(const uint8_t *I0, const uint8_t *I1, int W, int H, int pitch, int N,
                     const int32_t *lo, int Dw, int32_t *C);

/* Min-convolution of the previous pixel's energies with the jump penalty
 * (Eq. e(p,u)): M[k] = min_{v in [lo_prev, lo_prev+Dw)} A[v-lo_prev] + eps(lo+k, v),
 * eps(u,v) = min(p1*|u-v|, T).  The naive form scans every pair (O(Dw^2)); the fast
 * form is the two-sweep recursion of Section 3.3 (Eqs. 1-8).                        */
void ora_envelope_naive(const int64_t *A, int lo_prev, int lo, int Dw, int64_t p1,
                        int64_t T, int64_t *M);
void ora_envelope_fast(const int64_t *A, int lo_prev, int lo, int Dw, int64_t p1,
                       int64_t T, int64_t *M);

/* One directional Viterbi pass (dx,dy) over the volume: L[y][x][k].
 * normalized = 1: the bounded form L = C + M' - min_v L(prev, v);
 * normalized = 0: the literal recursion E = C + M'.
 * use_naive selects the O(Dw^2) envelope.  Returns 0, or -1 if the fast and naive
 * envelopes ever disagree when check = 1.                                           */
int ora_path(const int32_t *C, const int32_t *lo, int W, int H, int Dw, int dx, int dy,
             int64_t p1, int64_t T, int normalized, int use_naive, int check, int64_t *L);

/* Sum of the num_paths directional passes: S[y][x][k] (Eq. viterbi). */
int ora_aggregate(const int32_t *C, const int32_t *lo, int W, int H, int Dw, int num_paths,
                  int64_t p1, int64_t T, int normalized, int64_t *S);

/* Jump penalty of one step with separate slopes and truncations for upward jumps
 * (u > v: the disparity grows along the scan) and downward jumps (u < v):
 *     eps(u,v) = min(p_up (u-v), T_up)  for u > v,   min(p_dn (v-u), T_dn)  for u < v. */
typedef struct {
    int64_t p_up, p_dn;
    int64_t T_up, T_dn;     /* ORA_NO_TRUNC = no truncation */
} ora_penalty;

void ora_envelope_naive_pen(const int64_t *A, int lo_prev, int lo, int Dw,
                            const ora_penalty *e, int64_t *M);
void ora_envelope_fast_pen(const int64_t *A, int lo_prev, int lo, int Dw,
                           const ora_penalty *e, int64_t *M);

/* Directional pass over an int64 data term Q with a penalty per step: slope
 * P(p) = lut[|I0(p) - I0(p-r)|] when lut != NULL (Eq. EU's gradient weighting), else
 * p1; truncation T; with double_up = 1 upward jumps cost twice (slope 2P, truncation
 * 2T).  Output: the bounded form L = Q + M' - min_v L(p-r,v) (normalize_out = 0) or
 * the per-pixel min-normalised Lhat(p,u) = L(p,u) - min_v L(p,v) (normalize_out = 1).
 * Returns -1 if check = 1 and the fast and naive envelopes ever disagree.             */
int ora_path_pen(const int64_t *Q, const int32_t *lo, int W, int H, int Dw, int dx, int dy,
                 int64_t p1, int64_t T, const int32_t *lut, const uint8_t *I0, int pitch,
                 int double_up, int normalize_out, int use_naive, int check, int64_t *L);

/* Sum of the bounded passes with per-step (gradient) penalties; equal to
 * ora_aggregate when lut == NULL.                                                   */
int ora_aggregate_grad(const int32_t *C, const int32_t *lo, int W, int H, int Dw,
                       int num_paths, int64_t p1, int64_t T, const int32_t *lut,
                       const uint8_t *I0, int pitch, int64_t *S);

/* The paper's hierarchical merge: layers H, V (and the two diagonal pairs for 8
 * paths), each a forward and a backward pass over the previous layer's output; the
 * two normalised passes merge by min (H) or floor of the mean (other layers); the
 * left-to-right pass charges upward jumps twice.  S = the last layer's output.      */
int ora_aggregate_paper(const int32_t *C, const int32_t *lo, int W, int H, int Dw,
                        int num_paths, int64_t p1, int64_t T, const int32_t *lut,
                        const uint8_t *I0, int pitch, int64_t *S);

/* Aggregation (merge_mode SUM or PAPER) with the image split into independent
 * block x block tiles: a scan path restarts where it enters another tile (Section 3.4's
 * "MPV for each block" at the top level).                                            */
int ora_aggregate_blocks(const int32_t *C, const int32_t *lo, int W, int H, int Dw,
                         int num_paths, int64_t p1, int64_t T, const int32_t *lut,
                         const uint8_t *I0, int pitch, int merge_mode, int block, int64_t *S);

/* Winner-take-all: d = lo + argmin_k S, ties to the smallest k. */
void ora_wta(const int64_t *S, const int32_t *lo, int W, int H, int Dw, uint16_t *d);

/* 2x2 box down-sampling with round-half-up, odd edge replicated (Section 3.4). */
void ora_downsample2(const uint8_t *in, int W, int H, int pitch, uint8_t *out, int out_pitch);

/* Window lower bounds lo[y][x] of a finer level seeded from the coarser level's WTA
 * map dprev (Wp x Hp): block mode (block >= 2) or linear interpolation (block == 1),
 * then lo = clamp(c - Dw/2, 0, Dl - Dw).                                           */
void ora_seed(const uint16_t *dprev, int Wp, int Hp, int W, int H, int block, int Dw,
              int Dl, int32_t *lo);

/* Level geometry of the pyramid; level 0 is the coarsest (Section 3.4 numbering). */
void ora_level_dims(int W, int H, int S, int l, int *Wl, int *Hl);
int ora_level_range(int D, int S, int l);   /* D_l = ceil(D / 2^(S-1-l))     */
int ora_level_window(const ora_params *p, int l);  /* labels evaluated per pixel */

/* Number of evaluated (pixel, label) nodes of one view (the work model, Eqs. Ot-O). */
int64_t ora_node_count(int W, int H, const ora_params *p);

/* Validates parameters against image size; 0 when usable. */
int ora_check_params(int W, int H, const ora_params *p);

/* One view of the matcher: pre-check WTA map of the finest level. */
int ora_match_view(const uint8_t *I0, const uint8_t *I1, int W, int H, int pitch,
                   const ora_params *p, uint16_t *d);

/* Full matcher: left disparity with the left-right check (0xFFFF = rejected) and,
 * when dR != NULL, the right view's map in right-image coordinates.               */
int ora_match(const uint8_t *I0, const uint8_t *I1, int W, int H, int pitch,
              const ora_params *p, uint16_t *dL, uint16_t *dR);

/* Left-right check of two maps (right map in right-image coordinates). */
void ora_lr_check(const uint16_t *dL, const uint16_t *dR, int W, int H, int tol,
                  uint16_t *out);

/* Per-level stage dump of one view: lo, cost and summed volume of level l.
 * Buffers sized by ora_level_dims / ora_level_window.  Returns 0 on success.        */
int ora_view_stage(const uint8_t *I0, const uint8_t *I1, int W, int H, int pitch,
                   const ora_params *p, int level, int32_t *lo, int32_t *C, int64_t *S,
                   uint16_t *d);

/* ------------------------------------------------------------------------------ */
/* Road detection on the disparity map (Section 3.5: Eqs. disp_map, hy, e, P_hat)     */
/* ------------------------------------------------------------------------------ */

/* v-disparity: Hx[j*D + i] = number of pixels of row j whose disparity is i (i < D);
 * other values (0xFFFF = rejected) are not counted.  U: W x H, rows `pitch` apart.   */
void ora_vdisparity(const uint16_t *U, int W, int H, int pitch, int D, uint32_t *Hx);

/* u-disparity: Hy[j*D + i] = number of pixels of column j whose disparity is i.      */
void ora_udisparity(const uint16_t *U, int W, int H, int pitch, int D, uint32_t *Hy);

/* Road profile: the row path j = P(i) over the disparities i = 0..D-1 that maximises
 * sum_i Hx[P(i)][i] with 0 < P(i) - P(i-1) < eta.  Returns the maximum, or -1 (and P
 * all -1) when no such path fits in H rows.  Ties go to the smaller row, at the end
 * and at every predecessor.                                                          */
int64_t ora_road_profile(const uint32_t *Hx, int H, int D, int eta, int32_t *P);

#ifdef __cplusplus
}
#endif
#endif
