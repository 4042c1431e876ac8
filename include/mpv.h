/*
 * mpv.h -- C ABI of the GB300 multi-scale fast MPV (Multi-Path-Viterbi) stereo matcher.
 *
 * The method is the stereo matcher of Section 3.2-3.4 of "A Robust Real-Time
 * Computing-based Environment Sensing System for Intelligent Vehicle" (Xie, Long,
 * Zhang, Sun; arXiv 2001.09678):
 *   - an SSIM matching cost between N x N patches of the rectified left image I0 and
 *     right image I1 (Section 3.2, Eq. components and Eq. ssim), kept as integers;
 *   - bi-directional Viterbi passes along 4 or 8 scan directions with full
 *     connectivity between disparity nodes under an L1 (total-variation) jump penalty
 *     (Eq. EU, Eq. e(p,u)), evaluated by the O(2m) two-sweep recursion of Section 3.3;
 *   - the sum of the path energies and winner-take-all (Eq. viterbi);
 *   - the coarse-to-fine pyramid of Section 3.4: full range only at the top level,
 *     finer levels search a per-pixel window seeded by block mode and, at the finest
 *     level, interpolation (Eqs. Ot-O);
 *   - a left-right consistency check on the output.
 * Every cost and energy is an integer; results are bit-identical to the definition.
 *
 * Conventions shared by every entry point:
 *   - Image and disparity pointers passed to mpv_match / mpv_match_batch are DEVICE
 *     pointers owned by the caller; the library never frees them.  Images are uint8,
 *     row-major, rows `pitch` bytes apart.  Disparities are uint16, rows `disp_pitch`
 *     elements apart; MPV_INVALID marks a pixel rejected by the left-right check.
 *   - A context owns its device workspace (grown on demand with cudaMalloc) and is
 *     used by one host thread at a time.  There is no global state.
 *   - Calls are asynchronous on `cuda_stream` (a cudaStream_t; NULL = legacy default
 *     stream).  Device-side failures are latched in the context and returned by the
 *     next call or by mpv_sync.
 *   - Invalid arguments return MPV_ERR_INVALID_ARG and leave every output untouched.
 *     No entry point aborts, traps or throws.
 */
#ifndef MPV_H
#define MPV_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct mpv_ctx mpv_ctx;

typedef enum {
    MPV_OK = 0,
    MPV_ERR_INVALID_ARG = 1,  /* a parameter or size outside the documented range      */
    MPV_ERR_UNSUPPORTED = 2,  /* valid request the library does not implement          */
    MPV_ERR_OOM = 3,          /* workspace allocation failed or exceeds the byte budget */
    MPV_ERR_CUDA = 4,         /* a CUDA runtime call failed                              */
    MPV_ERR_TIMEOUT = 5,      /* a bounded device-side wait expired                      */
    MPV_ERR_INTERNAL = 6      /* a device-side consistency check failed                  */
} mpv_status;

#define MPV_INVALID 0xFFFFu
#define MPV_NO_TRUNC 0x7FFFFFFF

#define MPV_MERGE_SUM 0         /* S = sum of the directional energies (Eq. viterbi)     */
#define MPV_MERGE_PAPER 1       /* the paper's layered merge (Section 3.2, Table alg):     */
                                /* left/right, up/down, then the two diagonal pairs; each  */
                                /* layer's two passes run over the previous layer's merged */
                                /* energies and merge by min (horizontal) or floor of the  */
                                /* mean (others), after per-pixel min-normalisation; the   */
                                /* left-to-right pass charges upward jumps twice           */
#define MPV_PROPOSAL_PYRAMID 0  /* finer-level windows from the coarser level (Sec. 3.4) */
#define MPV_PROPOSAL_LEARNED 1  /* finest-level windows from the learned proposal        */
#define MPV_FALLBACK_NONE 0     /* learned proposal: keep its result whatever its windows */
#define MPV_FALLBACK_PYRAMID 1  /* ... re-match the frame with the pyramid (Sec. 3.4)     */
#define MPV_FALLBACK_FULL 2     /* ... re-match it at full range, one scale (exact MPV)   */

/* Matcher parameters.  Fill with mpv_default_params, then override. */
typedef struct {
    uint32_t struct_size;   /* = sizeof(mpv_params); guards ABI evolution                  */
    int32_t max_disparity;  /* D >= 1: labels 0..D-1 at full resolution (Eq. Ot's d)       */
    int32_t num_scales;     /* S in [1,4]: pyramid levels, factor 2 (Section 3.4: S = 3)  */
    int32_t num_paths;      /* 4 (left/right, up/down) or 8 (+ both diagonals; Table alg) */
    int32_t p1;             /* lambda >= 0: penalty per pixel of disparity jump (Eq. EU)  */
    int32_t trunc;          /* T >= 0: the jump penalty is min(p1*|du|, T); MPV_NO_TRUNC   */
                            /* keeps the paper's untruncated form                          */
    int32_t ssim_window;    /* N in {3,5}: SSIM patch side (Section 3.2, "N x N")          */
    int32_t window;         /* Dw > 0: labels searched per pixel below the top level;      */
                            /* 0 selects D/4 (Eqs. Ot1, Ot2)                               */
    int32_t block[4];       /* mode-block side (in coarse pixels) for levels 1..S-1;       */
                            /* 1 = per-pixel interpolation, 0 = default (2, 1 at finest)  */
    int32_t lr_check;       /* 1: left-right check on the output, 0: raw left WTA map     */
    int32_t lr_tol;         /* accepted |d_L - d_R| in pixels (default 1)                  */
    int32_t merge_mode;     /* MPV_MERGE_SUM or MPV_MERGE_PAPER                             */
    int32_t proposal;       /* MPV_PROPOSAL_PYRAMID or MPV_PROPOSAL_LEARNED                */
    int32_t top_block;      /* > 0: the top pyramid level is split into independent tiles  */
                            /* of top_block x top_block pixels, MPV per tile (Section 3.4, */
                            /* read literally); 0 (default): the whole top level           */
    int32_t windows[4];     /* per-level window Dw of levels 1..S-1 (index l-1), each >= 0; */
                            /* 0 (default) takes `window` (Eqs. Ot1, Ot2 with their d/4    */
                            /* replaced by a width of the caller's choice per level)       */
    int32_t fallback;       /* learned proposal only: MPV_FALLBACK_PYRAMID (default),      */
                            /* MPV_FALLBACK_FULL or MPV_FALLBACK_NONE                      */
    int32_t fallback_edge_bp; /* the frame is re-matched when more than this many of every */
                            /* 10000 matched pixels (both views) have their winning label  */
                            /* on an edge of the proposed window while the range goes on   */
                            /* past it; 0..10000, default 1500 (15 %)                      */
} mpv_params;

/* One stereo pair of a batch.  All pointers are device pointers. */
typedef struct {
    const uint8_t *left;    /* I0, width x height, rows `pitch` bytes apart            */
    const uint8_t *right;   /* I1, same geometry                                       */
    int32_t width, height;
    int32_t pitch;          /* bytes, >= width                                         */
    int32_t max_disparity;  /* 0 = the context's D                                     */
    uint16_t *disp;         /* output, rows disp_pitch elements apart                 */
    int32_t disp_pitch;     /* elements, >= width                                      */
    uint16_t *disp_right;   /* optional right-view map (right-image coordinates), NULL */
} mpv_pair;

/* Default parameters: D = 128, S = 3, 8 paths, p1 = 10, T = 30, N = 5, Dw = D/4,
 * blocks {2,1}, left-right check on with tolerance 1, summed merge, pyramid windows. */
mpv_status mpv_default_params(mpv_params *p);

/* Creates a context on CUDA device `device`.  *out receives the handle. */
mpv_status mpv_create(int device, mpv_ctx **out);

/* Copies and validates `p` (MPV_ERR_INVALID_ARG: out of range; the context keeps its
 * previous parameters).  Size-dependent checks are made by each match call.          */
mpv_status mpv_set_params(mpv_ctx *ctx, const mpv_params *p);
mpv_status mpv_get_params(const mpv_ctx *ctx, mpv_params *p);

/* Disparity map of one rectified pair (left view), device pointers, asynchronous.
 * Requirements: width, height >= N; 1 <= D <= min(width, 1024); the top pyramid level
 * at least N x N; pitch >= width; disp_pitch >= width; and the bound on summed
 * energies num_paths * (255 + min(T, p1 * (D - 1))) < 65535.
 * The launches of a pair are captured once per signature (sizes, buffers, parameters,
 * tables) into a CUDA graph that later calls replay; with MPV_NO_GRAPHS set in the
 * environment, or while profiling or dumping stages, they are launched directly.      */
mpv_status mpv_match(mpv_ctx *ctx, const uint8_t *left, const uint8_t *right,
                     int32_t width, int32_t height, int32_t pitch, uint16_t *disp,
                     int32_t disp_pitch, void *cuda_stream);

/* Same as mpv_match on HOST buffers: the call copies the pair to the device, matches,
 * copies the map back and synchronizes `cuda_stream` before returning.  Host buffers
 * may be pageable or pinned (pinned overlaps better).                                 */
mpv_status mpv_match_host(mpv_ctx *ctx, const uint8_t *left, const uint8_t *right,
                          int32_t width, int32_t height, int32_t pitch, uint16_t *disp,
                          int32_t disp_pitch, void *cuda_stream);

/* Matches n pairs of possibly different sizes and ranges in one submission.  Each pair
 * is validated first; if any is invalid nothing is launched.  For n > 1 the whole batch
 * is captured once as a CUDA graph in which the pairs run concurrently on the context's
 * worker streams (largest first), each with the launch shapes the autotuner chose for
 * its image shape (tuning an unseen shape runs its pair a few extra times first); the
 * graph is cached by the batch signature (sizes, ranges, pointers, parameters) and a
 * repeated batch costs one graph launch on `cuda_stream`.  Outputs are identical to
 * matching each pair alone.  Do not call it while `cuda_stream` is being captured.    */
mpv_status mpv_match_batch(mpv_ctx *ctx, const mpv_pair *pairs, int32_t n, void *cuda_stream);

/* Autotuner: times the candidate launch shapes of the matcher on `pair` (its buffers are
 * used and overwritten) and keeps the fastest for pairs of the same width, height and
 * range; *lanes (may be NULL) receives the chosen lanes per scan path of the
 * aggregation (4 or 8).  Synchronous.  Results do not depend on the choice.          */
mpv_status mpv_autotune(mpv_ctx *ctx, const mpv_pair *pair, int32_t *lanes);

/* Gradient-weighted TV penalty (Eq. EU: the TV term of a step scaled by e^{-|G|}).
 * slopes: host array of 256 integer jump slopes; the step from pixel p - r to p along a
 * scan direction then costs min(slopes[|I0(p) - I0(p - r)|] * |du|, T) instead of
 * min(p1 * |du|, T), I0 being the reference image of the view at the pyramid level.
 * Each slope must lie in [0, p1] of the parameters in force when matching (checked at
 * each match: MPV_ERR_INVALID_ARG otherwise).  The table is copied (to the device as
 * well); NULL switches the weighting off.  Applies to both merge modes.               */
mpv_status mpv_set_gradient_penalty(mpv_ctx *ctx, const int32_t *slopes);

/* Road detection on a disparity map (Section 3.5), asynchronous on cuda_stream; all
 * pointers are device pointers.
 *   disp: width x height uint16 disparities, rows disp_pitch elements apart; values not
 *         below max_disparity (MPV_INVALID) are not counted.
 *   vdisp (required, out): [height][max_disparity] uint32, the v-disparity (Eq. disp_map):
 *         vdisp[j][i] = number of pixels of row j with disparity i.
 *   udisp (optional, out): [width][max_disparity] uint32, the u-disparity (Eq. hy, read
 *         with the disparity index): udisp[j][i] = pixels of column j with disparity i.
 *   profile (out): [max_disparity] int32, the road's row P(i) for every disparity i: the
 *         path maximising sum_i vdisp[P(i)][i] under 0 < P(i) - P(i-1) < eta (Eqs. e and
 *         P_hat), ties to the smaller row; all -1 when no such path fits in the image.
 *   energy (out): one int64, the maximum (-1 when no path fits).
 * Limits: height <= 4096, max_disparity <= 1024, 2 <= eta <= 256; MPV_ERR_INVALID_ARG
 * otherwise.  The context keeps a scratch buffer for tall inputs.                      */
mpv_status mpv_road_detect(mpv_ctx *ctx, const uint16_t *disp, int32_t width, int32_t height,
                           int32_t disp_pitch, int32_t max_disparity, int32_t eta,
                           uint32_t *vdisp, uint32_t *udisp, int32_t *profile, int64_t *energy,
                           void *cuda_stream);

/* Loads the learned-proposal network (file written by paper_2001_09678_gb300/learn.py:
 * "MPVP", version 1, six layers of 3x3 convolutions, FP32 weights stored, converted to
 * BF16 on load).  With proposal = LEARNED (num_scales >= 2), a match computes the top
 * pyramid level's full-range cost, runs the network on it, and searches at the finest
 * level the window of `window` labels (default 17, i.e. centre +- 8) around the
 * prediction instead of seeding the intermediate levels.  The network's input channel
 * count must equal 2 + ceil(D / 2^(S-1)) (MPV_ERR_INVALID_ARG at match time
 * otherwise).  Invalid files return MPV_ERR_INVALID_ARG and keep the loaded network.  */
mpv_status mpv_load_proposal_weights(mpv_ctx *ctx, const char *path);

/* Network input of one pair, for training: the top pyramid level of `view` (0 = left
 * view, 1 = the mirrored, swapped pair) as 2 + D_top BF16 planes of W_top x H_top:
 * left/255 - 1/2, right/255 - 1/2, then the cost slice C(k)/255 for every label k.
 * Uses the context's pyramid parameters.  Asynchronous.                              */
mpv_status mpv_proposal_features(mpv_ctx *ctx, const uint8_t *left, const uint8_t *right,
                                 int32_t width, int32_t height, int32_t pitch, int32_t view,
                                 void *out, void *cuda_stream);

/* The learned proposal's raw prediction for one view (proposal = LEARNED, weights
 * loaded): disparity / D per pixel of the top pyramid level, FP32 [H_top][W_top] into
 * the device buffer out (sizes from mpv_level_info at level 0).  Asynchronous.         */
mpv_status mpv_proposal_predict(mpv_ctx *ctx, const uint8_t *left, const uint8_t *right,
                                int32_t width, int32_t height, int32_t pitch, int32_t view,
                                float *out, void *cuda_stream);

/* Of the last mpv_match with the learned proposal (read after mpv_sync): the pixels
 * whose winning label sits on their window's edge while the range continues past it,
 * and the pixels matched (both views), both counted on the network's windows.  A high
 * ratio means the windows missed; with fallback != MPV_FALLBACK_NONE the match itself
 * then re-matched the frame on the device (see fallback_edge_bp), and the output is
 * that of the fallback method.                                                        */
mpv_status mpv_proposal_stats(const mpv_ctx *ctx, uint64_t *edge_hits, uint64_t *pixels);

/* Learned-proposal frames matched by this context with a fallback configured (each
 * takes the decision) and how many of them fell back (read after mpv_sync; cumulative
 * since the context's creation).  The decision is taken on the device after the learned
 * frame's winner-take-all, so the call stays asynchronous: in the frame's cached CUDA
 * graph the fallback is the body of a conditional node that the decision sets (nothing
 * runs when it is not needed); launched directly (profiling, MPV_NO_GRAPHS, batches)
 * the fallback's launches are enqueued behind the decision and return at once unless
 * it opened them.                                                                     */
mpv_status mpv_proposal_fallbacks(const mpv_ctx *ctx, uint64_t *frames, uint64_t *fallbacks);

/* Waits for the context's last submitted work and returns any latched device error,
 * MPV_ERR_TIMEOUT among them: the last persistent batch ended by its bounded wait, or
 * the learned proposal network's wait for its tensor-core products ran out.            */
mpv_status mpv_sync(mpv_ctx *ctx);

/* Batches (mpv_match_batch with n > 1) run either through one persistent kernel over a
 * device work list or as a CUDA graph of per-pair launch sequences over worker streams.
 * The persistent kernel applies when every pair uses the summed merge with pyramid
 * windows, no gradient table, no top-level tiles, a jump radius ceil(T/p1) - 1 <= 2 and
 * label strides of 16, 32, 48 or 64 (and MPV_BATCH_STREAMS is not set in the
 * environment).  Each pair's stages become work items in per-group queues; a kernel CTA
 * claims an item only once the stage it depends on has completed, and the search for a
 * claimable item is the one device-side wait, bounded in clock cycles (about 2 s): when
 * it runs out the batch stops and mpv_sync returns MPV_ERR_TIMEOUT.  Once per set of
 * pair shapes the autotuner times the persistent kernel with each candidate shape
 * (lanes per scan path, work queues, cost blocks per item), then with 3 and 4 resident
 * blocks per SM (its register budget) for the best shape, and the stream graph, on the
 * batch itself, and keeps the fastest; all give the same bit-exact maps.
 * mpv_batch_info reports the path of the context's last batch (persistent 1 or 0), the
 * persistent shapes, the tuner's times in milliseconds per batch (0 when not tuned) and
 * the persistent kernel's resident blocks per SM.  Any output pointer may be NULL.     */
mpv_status mpv_batch_info(const mpv_ctx *ctx, int32_t *persistent, int32_t *lanes,
                          int32_t *queues, int32_t *cost_blocks, float *persistent_ms,
                          float *streams_ms, int32_t *occupancy);

/* Which batch path mpv_match_batch takes: MPV_BATCH_AUTO (default: the autotuner's
 * choice), MPV_BATCH_PERSISTENT (the persistent kernel wherever it applies) or
 * MPV_BATCH_STREAMS (always the stream graph).                                          */
#define MPV_BATCH_AUTO 0
#define MPV_BATCH_PERSISTENT 1
#define MPV_BATCH_STREAMS 2
mpv_status mpv_set_batch_mode(mpv_ctx *ctx, int32_t mode);

/* Test hook of the bounded wait: the next persistent batch makes one stage of its largest
 * pair wait for an item that never exists and gives its wait wait_cycles clock cycles;
 * that launch is not cached, and mpv_sync afterwards returns MPV_ERR_TIMEOUT.           */
mpv_status mpv_debug_batch_stall(mpv_ctx *ctx, int64_t wait_cycles);

/* Device bytes the context needs for a width x height pair at its parameters. */
mpv_status mpv_workspace_bytes(const mpv_ctx *ctx, int32_t width, int32_t height,
                               size_t *bytes);

/* Caps the workspace (bytes; 0 = no cap).  A match that needs more returns MPV_ERR_OOM. */
mpv_status mpv_set_workspace_limit(mpv_ctx *ctx, size_t bytes);

/* Stage outputs of one pyramid level of one view, for verification.  view 0 is the
 * left view, view 1 the right view (the matcher run on the mirrored, swapped pair).
 * Device outputs, each may be NULL: lo (uint16 W_l x H_l, window starts), cost
 * (uint16 W_l x H_l x Dw_l, u fastest), sum (uint32, same shape), disp (uint16 W_l x
 * H_l pre-check WTA map).  Synchronous.                                                */
mpv_status mpv_debug_stage(mpv_ctx *ctx, const uint8_t *left, const uint8_t *right,
                           int32_t width, int32_t height, int32_t pitch, int32_t view,
                           int32_t level, uint16_t *lo, uint16_t *cost, uint32_t *sum,
                           uint16_t *disp, void *cuda_stream);

/* Level geometry used by the matcher: width, height, full range D_l and window Dw_l of
 * level `level` (0 = coarsest) for a width x height pair.                            */
mpv_status mpv_level_info(const mpv_ctx *ctx, int32_t width, int32_t height, int32_t level,
                          int32_t *w, int32_t *h, int32_t *range, int32_t *window);

/* ---- Serving: continuous batching over camera streams (the serving loop) ------
 *
 * A server owns, per registered camera, resident device state (a matcher context whose
 * workspace keeps that frame size's pyramid levels and volumes allocated between frames,
 * device copies of the pair and map, pinned staging, a stream).  Frames are submitted
 * from HOST buffers and wait in a per-camera FIFO.  mpv_server_poll retires finished
 * frames (copying their maps to the caller's buffers) and admits waiting frames, oldest
 * first, while fewer than max_inflight frames run and the resident memory of the
 * admitted cameras fits hbm_budget (0 = no limit); idle cameras are evicted least
 * recently used first to make room.  Admitted frames of different cameras run
 * concurrently on the GPU.  The server is used from one host thread; nothing blocks on
 * the GPU.  Results equal mpv_match of the same pair alone.  A serving process should
 * load its kernels at start-up (CUDA_MODULE_LOADING=EAGER in its environment before CUDA
 * initialises): with lazy loading, a kernel's first launch while other frames are in
 * flight (a proposal's first fallback, say) held the host for tens of milliseconds.      */
typedef struct mpv_server mpv_server;

typedef struct {
    uint64_t request_id;
    int32_t camera;
    mpv_status status;      /* MPV_ERR_OOM: the camera cannot fit the budget at all    */
    double t_submit_ms;     /* host steady clock at submit                              */
    double t_start_ms;      /* admitted: copies and kernels enqueued                     */
    double t_done_ms;       /* the map reached pinned host memory (stream callback)      */
} mpv_completion;

mpv_status mpv_server_create(int device, const mpv_params *params, size_t hbm_budget,
                             int32_t max_inflight, mpv_server **out);
/* Learned window proposal for the cameras of a server: weights file as for
 * mpv_load_proposal_weights.  A camera whose range fits the network (2 + top-level range
 * input channels) matches with the learned proposal, the others with the pyramid; NULL
 * returns every camera to the pyramid.  Applies to cameras made resident afterwards
 * (call before the first submit).                                                    */
mpv_status mpv_server_set_proposal(mpv_server *server, const char *weights_path);

/* Registers a camera's frame geometry and range (validated as for mpv_match). */
mpv_status mpv_server_add_camera(mpv_server *srv, int32_t camera, int32_t width,
                                 int32_t height, int32_t max_disparity);
/* Queues a frame.  left/right (rows `pitch` bytes apart) and disp (rows disp_pitch
 * elements apart) are host buffers that must stay valid until the frame completes.   */
mpv_status mpv_server_submit(mpv_server *srv, int32_t camera, const uint8_t *left,
                             const uint8_t *right, int32_t pitch, uint16_t *disp,
                             int32_t disp_pitch, uint64_t request_id);
/* Retires and admits (see above); writes up to max completions to out, *n = count. */
mpv_status mpv_server_poll(mpv_server *srv, mpv_completion *out, int32_t max, int32_t *n);
/* Current in-flight and waiting frames, resident bytes, evictions so far and the largest
 * number of frames that were in flight at once.  Any output may be NULL.              */
mpv_status mpv_server_stats(const mpv_server *srv, int32_t *inflight, int32_t *waiting,
                            size_t *resident_bytes, uint64_t *evictions,
                            int32_t *peak_inflight);
/* Waits for in-flight frames, then releases everything; NULL is accepted. */
void mpv_server_destroy(mpv_server *srv);

/* ---- Learned window proposal: network kernels (training and inference) -------------
 *
 * The learned proposal (an extension; the paper has none) replaces the pyramid's
 * window seeding at the finest level by a small CNN evaluated at the top level: six
 * 3x3 convolutions, zero padding, 2 + D_top input channels (the top level's left and
 * right images and its full-range cost slice), 32 hidden channels with ReLU, one output
 * channel (disparity / D).  Activations and weights are BF16 (__nv_bfloat16 in device
 * memory, passed as void *), accumulation and gradients FP32.  Tensors are NCHW, device
 * pointers, asynchronous on cuda_stream.  Invalid sizes return MPV_ERR_INVALID_ARG.   */

/* out = conv3x3(in, weight[cout][cin][3][3]) + bias, optional ReLU; in is BF16, or FP32
 * when in_f32 = 1; cout is 32 or 1; out_bf16 and/or out_f32 receive the result.
 * BF16 input runs on the tensor cores (tcgen05, FP32 accumulation) while the operands
 * fit in shared memory (cin up to 208); its one device wait is bounded, and outputs of
 * tiles whose wait ran out are NaN.  Larger cin and FP32 input run on the CUDA cores.  */
mpv_status mpv_cnn_conv3x3(const void *in, int32_t in_f32, int32_t n, int32_t cin, int32_t h,
                           int32_t w, const void *weight, const float *bias, int32_t cout,
                           int32_t relu, void *out_bf16, float *out_f32, void *cuda_stream);
/* dweight[cout][cin][3][3] += sum over n,y,x of grad[n][co][y][x] in[n][ci][y+ky-1][x+kx-1];
 * dbias[cout] += sum of grad (dbias may be NULL).  Accumulates: zero them first.      */
mpv_status mpv_cnn_conv3x3_wgrad(const void *in, int32_t n, int32_t cin, const float *grad,
                                 int32_t cout, int32_t h, int32_t w, float *dweight,
                                 float *dbias, void *cuda_stream);
/* out[ci][co][2-ky][2-kx] = weight[co][ci][ky][kx] (BF16): the backward-data weights. */
mpv_status mpv_cnn_flip_transpose(const void *weight, int32_t cout, int32_t cin, void *out,
                                  void *cuda_stream);
/* out = grad where act > 0 else 0 (ReLU backward; act BF16). */
mpv_status mpv_cnn_relu_backward(const float *grad, const void *act, float *out, int64_t count,
                                 void *cuda_stream);
/* Huber loss with threshold delta, mean over count: grad = dloss/dpred; *loss (may be
 * NULL) is incremented by the mean loss.                                              */
mpv_status mpv_cnn_huber(const float *pred, const float *target, float delta, int64_t count,
                         float *grad, float *loss, void *cuda_stream);
/* One Adam step (bias-corrected, step >= 1) on FP32 weights; refreshes weight_bf16 when
 * not NULL.                                                                           */
mpv_status mpv_cnn_adam(float *weight, const float *grad, float *m, float *v, int64_t count,
                        float lr, float beta1, float beta2, float eps, int32_t step,
                        void *weight_bf16, void *cuda_stream);
mpv_status mpv_cnn_to_bf16(const float *in, void *out, int64_t count, void *cuda_stream);
/* Training target: mean of each factor x factor block of a full-resolution disparity
 * map, divided by max_disparity, at ceil(width/factor) x ceil(height/factor).        */
mpv_status mpv_cnn_target(const uint16_t *disp, int32_t disp_pitch, int32_t width,
                          int32_t height, int32_t factor, int32_t max_disparity, float *target,
                          void *cuda_stream);

/* Stages reported by the profiler. */
#define MPV_STAGE_PYRAMID 0     /* mirroring and 2x2 down-sampling                      */
#define MPV_STAGE_SEED 1        /* per-pixel windows of the finer levels                 */
#define MPV_STAGE_COST 2        /* SSIM cost volume                                      */
#define MPV_STAGE_AGGREGATE 3   /* directional Viterbi passes and their sum              */
#define MPV_STAGE_WTA 4         /* winner-take-all                                       */
#define MPV_STAGE_LR 5          /* left-right check                                      */
#define MPV_NUM_STAGES 6

/* on = 1: record a CUDA event pair around every kernel launch of later calls on the
 * launch's own stream; on = 0: stop recording and drop what was recorded.          */
mpv_status mpv_profile_enable(mpv_ctx *ctx, int32_t on);

/* Synchronizes the recorded work, then writes for each stage k < n the summed device
 * time ms[k] of its recorded launches and launches[k], the number of kernels the
 * library launched for it since the previous read (counted with profiling on or off),
 * and resets both.  Either array may be NULL.                                        */
mpv_status mpv_profile_read(mpv_ctx *ctx, double *ms, int64_t *launches, int32_t n);

/* ---- Matching without device allocation (the paper has no counterpart) -----------
 *
 * Some callers cannot call cudaMalloc: a host framework that owns a fixed device pool,
 * a real-time loop that must not allocate once running, a plug-in inside a process
 * whose device memory is budgeted by someone else.  mpv_match_noalloc runs the same
 * matcher as mpv_match with every scratch buffer taken from one fixed array of
 * MPV_NOALLOC_SCRATCH_BYTES in device global memory, declared in the library itself:
 * every GPU that loads the library holds that array until the process exits.  The call
 * allocates nothing (no cudaMalloc, no cudaFree, no allocating library routine) and
 * needs no context; the caller still owns the images and the output.
 *   - Uses the device that is current on the calling thread.  The first call on a
 *     device looks up the array's device address (cudaGetSymbolAddress); make that
 *     first call before any stream capture.
 *   - A pair whose scratch need exceeds MPV_NOALLOC_SCRATCH_BYTES is rejected with
 *     MPV_ERR_INVALID_ARG before anything is launched.  The need is the one
 *     mpv_workspace_bytes reports for the same parameters: per view (two with the
 *     left-right check) and level, two images (width rounded up to 16 bytes) and two
 *     uint16 maps, plus one cost volume of 1 byte and one summed volume of 2 bytes per
 *     pixel and label stride (the window rounded up to 16) at the largest level, each
 *     piece rounded up to 256 bytes; the layered merge (MPV_MERGE_PAPER) adds three more
 *     2-byte volumes per view.  So 640 x 480 at D = 64 with three scales and the
 *     left-right check fits with the summed merge (about 34 MB) but not with the layered
 *     merge (about 93 MB); 1280 x 720 at D = 128 (about 190 MB) does not fit.  The
 *     learned proposal and the right-view output are not available here.
 *   - Every call shares the one array, which keeps the previous call's contents (the
 *     call clears what must start at zero).  Calls that overlap on the GPU (other
 *     streams, other threads) race on it: serialize them on one stream.
 * Arguments as for mpv_match, plus the parameters to use (validated as by
 * mpv_set_params).                                                                     */
#define MPV_NOALLOC_SCRATCH_BYTES (64u << 20)
mpv_status mpv_match_noalloc(const mpv_params *params, const uint8_t *left,
                             const uint8_t *right, int32_t width, int32_t height,
                             int32_t pitch, uint16_t *disp, int32_t disp_pitch,
                             void *cuda_stream);

const char *mpv_status_string(mpv_status s);

/* Releases the context and its workspace; NULL is accepted. */
void mpv_destroy(mpv_ctx *ctx);

#ifdef __cplusplus
}
#endif
#endif
