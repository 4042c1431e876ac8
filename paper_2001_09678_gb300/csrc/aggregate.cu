// aggregate.cu -- directional Viterbi passes summed over 4 or 8 scan directions.
//
// Section 3.2 / Eq. e(p,u): along each scan direction r the energy of node (p,u) is its
// cost plus the cheapest predecessor node (p-r, v) plus the jump penalty
// eps(u,v) = min(p1 |u-v|, T), every node of the predecessor connected (full
// connectivity).  Section 3.3 evaluates that minimum in O(2m) by one upward and one
// downward sweep over the labels.  Labels are absolute disparities: a predecessor with a
// different window start connects through the penalty, and labels outside its window
// are virtual nodes (absent).  Energies are kept in the bounded form
//     L(p,u) = C(p,u) + M'(u) - min_v L(p-r,v),   M'(u) = min_v L(p-r,v) + eps(u,v),
// a per-pixel constant shift of the literal recursion that leaves every argmin unchanged
// and keeps every value small (at most 255 + T per pass); each pass adds L into the summed
// volume S, or, in the paper's layered merge, stores it min-normalised for the next layer.
//
// Three kernels:
//  * agg_stencil: 4 or 8 lanes own one scan path, each lane 2*KW consecutive labels packed
//    two per 32-bit register (16-bit energies, absent labels = the sentinel 16384).  When
//    the truncation makes every jump of more than R labels cost T (R = ceil(T/p1) - 1 <= 4;
//    the default p1 = 10, T = 30 gives R = 2), the two sweeps reduce to
//        M'(u) = min(min_{|d|<=R} L(p-r,u+d) + min(p1|d|, T), min_v L(p-r,v) + T),
//    packed add-min arithmetic over halo words from the neighbouring lanes.  The path's
//    minimum is exchanged through shared memory or by shuffles, a window shift between
//    consecutive pixels (pyramid levels) re-indexes the predecessor through shared memory,
//    and S is accumulated with 64-bit reductions of four packed labels.  While every path
//    of a warp is active its steps run without per-lane checks.  On levels small enough
//    to be resident at once, agg_rows_first starts the row paths (the W-step chains that
//    bound such levels) ahead of the other directions in one grid.  Its layer mode
//    runs one layer of the layered merge (Section 3.2), the left-to-right pass with doubled
//    upward jumps included; its sweep mode runs gradient-weighted slopes (Eq. EU) as
//    untruncated packed sweeps.
//  * agg_scan8: 8 lanes per path, int32 labels, the two sweeps as segmented prefix and
//    suffix minima across the lanes: the gradient and layered variants outside the packed
//    kernel's bounds or widths.
//  * agg_general: any window width: one warp per scan path, the sweeps written as prefix
//    minima  min_{v<=u} A(v) + p1 (u-v) = p1 u + min_{v<=u} (A(v) - p1 v)  (and the mirror
//    image), evaluated by shuffle scans over the lanes.
#include "agg_stencil.cuh"

namespace mpv {

namespace {

template <int G, int KW, int RM, bool WIN, bool BLK, bool LAYER, bool SWP, bool XM>
__global__ void __launch_bounds__(kStencilWarps * 32) agg_stencil(LevelArgs a, MergeArgs mg)
{
    if (a.gate && *a.gate == 0) return;
    using SM = StencilSmem<G, KW, RM, WIN, LAYER, SWP, kStencilWarps>;
    __shared__ __align__(16) unsigned char smem[SM::bytes];
    agg_stencil_body<G, KW, RM, WIN, BLK, LAYER, SWP, XM, kStencilWarps>(a, mg, blockIdx.x, blockIdx.y,
                                                                       blockIdx.z, threadIdx.x, smem);
}

template <int G, int KW, int RM, bool WIN, bool BLK, bool LAYER = false, bool SWP = false,
          bool XM = false>
void launch_stencil(const LevelArgs &a, cudaStream_t s, const MergeArgs &mg = MergeArgs{},
                    int ndirs = 0)
{
    const int maxp = a.W + a.H - 1;
    const int per_block = kStencilWarps * (32 / G);
    dim3 grid((maxp + per_block - 1) / per_block, ndirs ? ndirs : a.npaths, a.nviews);
    agg_stencil<G, KW, RM, WIN, BLK, LAYER, SWP, XM><<<grid, kStencilWarps * 32, 0, s>>>(a, mg);
}

// The summed pass of the 8-lane shape with the row (horizontal) paths first: one 1-D grid
// whose first nviews x 2 x nhb blocks run the two row directions of both views, the rest
// the other directions (2 .. npaths - 1, nbx blocks each).  Blocks start in index order, so
// the longest chains (W steps) start first.  The rows run agg_row_body on levels without
// windows and agg_stencil_body with them (measured at 1280x720, D = 128: 320x180 without
// windows 36.9 -> 34.8 us with the row body; 640x360 with windows 102.4 us with the
// stencil body, 112.7 us with the row body, whose separate code also has to be fetched).
template <bool WIN>
__global__ void __launch_bounds__(kStencilWarps * 32) agg_rows_first(LevelArgs a, MergeArgs mg,
                                                                   int nhb, int nbx)
{
    if (a.gate && *a.gate == 0) return;
    using SM = StencilSmem<8, 2, 2, WIN, false, false, kStencilWarps>;
    __shared__ __align__(16) unsigned char smem[SM::bytes];
    int b = blockIdx.x;
    const int nrow = a.nviews * 2 * nhb;
    int bx, by, view;
    if (b < nrow) {
        view = b / (2 * nhb);
        const int r = b - view * 2 * nhb;
        by = r / nhb;
        bx = r - by * nhb;
        if constexpr (!WIN) {
            if (by == 0) agg_row_body<1, WIN, kStencilWarps>(a, bx, view, threadIdx.x, smem);
            else agg_row_body<-1, WIN, kStencilWarps>(a, bx, view, threadIdx.x, smem);
            return;
        }
    } else {
        b -= nrow;
        const int per_view = (a.npaths - 2) * nbx;
        view = b / per_view;
        const int r = b - view * per_view;
        by = 2 + r / nbx;
        bx = r - (by - 2) * nbx;
    }
    agg_stencil_body<8, 2, 2, WIN, false, false, false, true, kStencilWarps>(
        a, mg, bx, by, view, threadIdx.x, smem);
}

// Whether the rows-first launch applies and pays: the level's blocks fit in about one and
// a half waves of the GPU, so the W-step row chains, not the throughput of the other
// directions, set the launch's time (measured at 1280x720, D = 128: 320x180 36.9 -> 34.8
// us, 640x360 108.5 -> 102.4 us; at 1280x720 itself, 2.2 waves, the library order is as
// fast or faster, 336 against 336-340 us).
template <bool WIN>
bool rows_first(const LevelArgs &a, int &nhb, int &nbx)
{
    if (a.npaths != 4 && a.npaths != 8) return false;
    constexpr int per_block = kStencilWarps * 4;   // 4 paths of 8 lanes per warp
    nhb = (a.H + per_block - 1) / per_block;
    nbx = (a.W + a.H - 1 + per_block - 1) / per_block;
    const int64_t blocks = (int64_t)a.nviews * (2 * nhb + (int64_t)(a.npaths - 2) * nbx);
    int dev = 0, nsm = 0, per_sm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, agg_rows_first<WIN>,
                                                      kStencilWarps * 32, 0) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return blocks * 2 <= (int64_t)3 * nsm * per_sm && blocks < 0x7FFFFFFF;
}

template <bool WIN>
bool launch_rows_first(const LevelArgs &a, cudaStream_t s)
{
    int nhb = 0, nbx = 0;
    if (!rows_first<WIN>(a, nhb, nbx)) return false;
    MergeArgs m{};
    m.dir0 = 0;
    m.ndirs = a.npaths;
    m.double_up_dir = -1;
    const int blocks = a.nviews * (2 * nhb + (a.npaths - 2) * nbx);
    agg_rows_first<WIN><<<blocks, kStencilWarps * 32, 0, s>>>(a, m, nhb, nbx);
    return true;
}

// Packed labels mark absent ones with the sentinel kInf16, which must exceed every cap
// min_v A(v) + Tu that a step forms.  Without windows the predecessor's best label carries
// over, so its minimum is at most a cost byte and the cap at most 255 + T.  With windows
// that label can lie outside the current window: the minimum then reaches 255 + Tu and the
// cap 255 + 2 Tu (Tu = T, or 2T for the doubled pass).  Beyond that the int32 kernels run.
bool packed_caps_ok(const LevelArgs &a, int up)
{
    return !a.v[0].lo || 255 + 2 * up * (int64_t)a.trunc < (int64_t)kInf16;
}

// windows (pyramid levels below the top) and tiles (the top level only) never meet
template <int G, int KW>
void launch_stencil_kw(const LevelArgs &a, cudaStream_t s)
{
    const bool win = a.v[0].lo != nullptr;
    const bool blk = a.block_cut > 0;
    // the shared-memory path minimum: measured faster on 8 lanes of two words without
    // padding labels, slower with one word per lane or with padding
    if constexpr (G == 8 && KW == 2) {
        if (a.Dw == a.Dws && a.radius <= 2) {
            if (!blk && (win ? launch_rows_first<true>(a, s) : launch_rows_first<false>(a, s)))
                return;
            if (win) launch_stencil<G, KW, 2, true, false, false, false, true>(a, s);
            else if (blk) launch_stencil<G, KW, 2, false, true, false, false, true>(a, s);
            else launch_stencil<G, KW, 2, false, false, false, false, true>(a, s);
            return;
        }
    }
    if (a.radius <= 2) {
        if (win) launch_stencil<G, KW, 2, true, false>(a, s);
        else if (blk) launch_stencil<G, KW, 2, false, true>(a, s);
        else launch_stencil<G, KW, 2, false, false>(a, s);
    } else if constexpr (KW >= 2) {    // halos of two words need two words per lane
        if (win) launch_stencil<G, KW, 4, true, false>(a, s);
        else if (blk) launch_stencil<G, KW, 4, false, true>(a, s);
        else launch_stencil<G, KW, 4, false, false>(a, s);
    }
}

// The gradient-weighted passes (a slope per step) as packed sweeps: 8 lanes per path for
// strides of 16 and 32 labels, while the sweeps' largest value, the sentinel plus the
// doubled slope (at most 2T) times the labels of a lane, stays below 2^16; a layer of the
// layered merge also needs its energies far below the sentinel.
bool sweep_ok(const LevelArgs &a, const MergeArgs &m)
{
    if (!m.lut || (a.Dws != 16 && a.Dws != 32)) return false;
    const int64_t K = a.Dws / 8, up = m.double_up_dir >= 0 ? 2 : 1;
    if ((int64_t)kInf16 + up * a.trunc * K >= 65536 || !packed_caps_ok(a, (int)up)) return false;
    return m.out_mode == 0 || 255 + 10 * (int64_t)a.trunc < (int64_t)kInf16;
}

template <int KW, bool LAYER>
void launch_sweep_kw(const LevelArgs &a, const MergeArgs &m, cudaStream_t s)
{
    // (the shared-memory path minimum measured faster in the layer mode only)
    if (a.v[0].lo)
        launch_stencil<kLanesWide, KW, 2, true, false, LAYER, true, LAYER>(a, s, m, m.ndirs);
    else if (a.block_cut > 0)
        launch_stencil<kLanesWide, KW, 2, false, true, LAYER, true, LAYER>(a, s, m, m.ndirs);
    else launch_stencil<kLanesWide, KW, 2, false, false, LAYER, true, LAYER>(a, s, m, m.ndirs);
}

void launch_sweep(const LevelArgs &a, const MergeArgs &m, cudaStream_t s)
{
    if (m.out_mode == 1) {
        if (a.Dws == 16) launch_sweep_kw<1, true>(a, m, s);
        else launch_sweep_kw<2, true>(a, m, s);
    } else {
        if (a.Dws == 16) launch_sweep_kw<1, false>(a, m, s);
        else launch_sweep_kw<2, false>(a, m, s);
    }
}

// ---------------------------------------------------------------------------------
// agg_general (general radius and width, per-step penalties, layered merge)
// ---------------------------------------------------------------------------------

constexpr int kScanWarps = 8;

// One warp per scan path, K labels per lane.  The envelope of the predecessor A with
// upward slope pu (u > v) and downward slope pd (u < v) is
//     M'(u) = min( pu u + min_{v<=u} (A(v) - pu v),   -pd u + min_{v>=u} (A(v) + pd v),
//                  min_{v<=u} A(v) + Tu,              min_{v>=u} A(v) + T )
// (Section 3.3's two sweeps as prefix/suffix minima over the lanes); with equal caps the
// last two terms are min_v A(v) + T.  The slope of a step is p1, or with a gradient
// table lut[|I0(p) - I0(p-r)|] (Eq. EU's weighting); the direction m.double_up_dir
// charges upward jumps twice (pu = 2P, Tu = 2T: the paper's left-to-right pass).
// Data term: the cost bytes, or the merge of the previous layer's two passes.  Output:
// the bounded energies added into S, or the per-pixel min-normalised energies stored
// into the direction's own volume (one layer of the paper's merge, Section 3.2).
template <int K>
__global__ void __launch_bounds__(kScanWarps * 32) agg_general(LevelArgs a, MergeArgs m)
{
    if (a.gate && *a.gate == 0) return;
    constexpr int NJ = 32 * K;                // labels covered by the warp
    const int view = blockIdx.z;
    const int dir = m.dir0 + blockIdx.y;
    const int dx = c_dirs[dir][0], dy = c_dirs[dir][1];
    const int W = a.W, H = a.H, Dw = a.Dw, Dws = a.Dws;
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int path = blockIdx.x * kScanWarps + warp;
    if (path >= num_paths_dir(dx, dy, W, H)) return;
    const ViewLevel &V = a.v[view];
    const int T = a.trunc;                    // finite: min(T, p1 (D_l - 1))
    const bool dbl = dir == m.double_up_dir;
    const int Tu = dbl ? 2 * T : T;
    // selected without dynamic indexing, which would copy the parameter arrays to the stack
    const uint16_t *qa = view ? m.qa[1] : m.qa[0];
    const uint16_t *qb = view ? m.qb[1] : m.qb[0];
    uint16_t *const *outs = view ? m.out[1] : m.out[0];
    uint16_t *out = (dir & 1) ? outs[1] : outs[0];

    extern __shared__ int sh[];
    int *pB = sh + warp * 4 * (NJ + 2);       // [NJ+1]: index j+1 holds the prefix minimum to j
    int *sC = pB + (NJ + 1);                  // [NJ+1]: index j holds the suffix minimum from j
    int *pA = sC + (NJ + 1);                  // the same two for A itself (asymmetric caps)
    int *sA = pA + (NJ + 1);

    int x, y;
    path_start(dx, dy, W, H, path, x, y);
    int A[K];
#pragma unroll
    for (int t = 0; t < K; ++t) A[t] = kInf;
    int prev_lo = 0, prev_i = 0;
    bool first = true;
    while (x >= 0 && x < W && y >= 0 && y < H) {
        const int64_t pix = (int64_t)y * W + x;
        const int cur_lo = V.lo ? (int)V.lo[pix] : 0;
        int c[K];
#pragma unroll
        for (int t = 0; t < K; ++t) {
            const int k = lane * K + t;
            int v = 0;
            if (k < Dw) {
                if (m.in_mode == 0) {
                    v = V.C[pix * Dws + k];
                } else {
                    const int ea = qa[pix * Dws + k], eb = qb[pix * Dws + k];
                    v = m.in_mode == 1 ? min(ea, eb) : (ea + eb) >> 1;
                }
            }
            c[t] = v;
        }
        const int cur_i = m.lut ? (int)V.I0[(int64_t)y * V.pitch0 + x] : 0;
        // entering a new tile of a split level: the path starts again here
        if (a.block_cut > 0 && !first &&
            (x / a.block_cut != (x - dx) / a.block_cut || y / a.block_cut != (y - dy) / a.block_cut))
            first = true;
        int L[K];
        if (first) {
#pragma unroll
            for (int t = 0; t < K; ++t) L[t] = c[t];
            first = false;
        } else {
            const int P = m.lut ? min(m.lut[abs(cur_i - prev_i) & 0xFF], T) : a.p1;
            const int pu = dbl ? 2 * P : P, pd = P;
            int mn = A[0];
#pragma unroll
            for (int t = 1; t < K; ++t) mn = min(mn, A[t]);
            const int amin = __reduce_min_sync(kFull, mn);
            // prefix minima of A(j) - pu j (and of A), suffix minima of A(j) + pd j (and of A)
            int pb[K], sc[K], pa[K], sa[K];
            int run = kInf, runa = kInf;
#pragma unroll
            for (int t = 0; t < K; ++t) {
                run = min(run, A[t] - pu * (lane * K + t));
                runa = min(runa, A[t]);
                pb[t] = run;
                pa[t] = runa;
            }
            int incl = run, incla = runa;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int v = __shfl_up_sync(kFull, incl, o);
                const int va = __shfl_up_sync(kFull, incla, o);
                if (lane >= o) {
                    incl = min(incl, v);
                    incla = min(incla, va);
                }
            }
            int excl = __shfl_up_sync(kFull, incl, 1);
            int excla = __shfl_up_sync(kFull, incla, 1);
            if (lane == 0) excl = excla = kInf;
#pragma unroll
            for (int t = 0; t < K; ++t) {
                pb[t] = min(pb[t], excl);
                pa[t] = min(pa[t], excla);
            }
            run = runa = kInf;
#pragma unroll
            for (int t = K - 1; t >= 0; --t) {
                run = min(run, A[t] + pd * (lane * K + t));
                runa = min(runa, A[t]);
                sc[t] = run;
                sa[t] = runa;
            }
            incl = run;
            incla = runa;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int v = __shfl_down_sync(kFull, incl, o);
                const int va = __shfl_down_sync(kFull, incla, o);
                if (lane + o < 32) {
                    incl = min(incl, v);
                    incla = min(incla, va);
                }
            }
            excl = __shfl_down_sync(kFull, incl, 1);
            excla = __shfl_down_sync(kFull, incla, 1);
            if (lane == 31) excl = excla = kInf;
#pragma unroll
            for (int t = 0; t < K; ++t) {
                sc[t] = min(sc[t], excl);
                sa[t] = min(sa[t], excla);
            }

            const int s = cur_lo - prev_lo;      // uniform across the warp
            if (s == 0) {
#pragma unroll
                for (int t = 0; t < K; ++t) {
                    const int j = lane * K + t;
                    int M = min(pu * j + pb[t], sc[t] - pd * j);
                    M = dbl ? min(M, min(pa[t] + Tu, sa[t] + T)) : min(M, amin + T);
                    L[t] = c[t] + M - amin;
                }
            } else {
#pragma unroll
                for (int t = 0; t < K; ++t) {
                    pB[lane * K + t + 1] = pb[t];
                    sC[lane * K + t] = sc[t];
                    pA[lane * K + t + 1] = pa[t];
                    sA[lane * K + t] = sa[t];
                }
                if (lane == 0) {
                    pB[0] = pA[0] = kInf;
                    sC[NJ] = sA[NJ] = kInf;
                }
                __syncwarp();
#pragma unroll
                for (int t = 0; t < K; ++t) {
                    const int jj = s + lane * K + t;  // label index in the predecessor window
                    const int pi = min(max(jj, -1), NJ - 1) + 1;
                    const int si = min(max(jj, 0), NJ);
                    int M = min(pu * jj + pB[pi], sC[si] - pd * jj);
                    M = dbl ? min(M, min(pA[pi] + Tu, sA[si] + T)) : min(M, amin + T);
                    L[t] = c[t] + M - amin;
                }
                __syncwarp();
            }
        }
        // padding labels: never a predecessor, add nothing, stored as 0
#pragma unroll
        for (int t = 0; t < K; ++t) {
            const int k = lane * K + t;
            if (k >= Dw) L[t] = 0;
        }
        if (m.out_mode == 0) {
            // S: packed 16-bit pairs
            uint16_t *sp = V.S + pix * Dws;
            if (K == 1) {
                const int up = __shfl_down_sync(kFull, L[0], 1);
                if ((lane & 1) == 0 && lane < Dws)
                    atomicAdd((unsigned int *)(sp + lane), (unsigned)L[0] | ((unsigned)up << 16));
            } else {
#pragma unroll
                for (int t = 0; t < K; t += 2) {
                    const int k = lane * K + t;
                    if (k < Dws)
                        atomicAdd((unsigned int *)(sp + k),
                                  (unsigned)L[t] | ((unsigned)L[t + 1] << 16));
                }
            }
        } else {
            int lm = kInf;
#pragma unroll
            for (int t = 0; t < K; ++t)
                if (lane * K + t < Dw) lm = min(lm, L[t]);
            const int lmin = __reduce_min_sync(kFull, lm);
            uint16_t *op = out + pix * Dws;
#pragma unroll
            for (int t = 0; t < K; ++t) {
                const int k = lane * K + t;
                if (k < Dws) op[k] = (uint16_t)(k < Dw ? L[t] - lmin : 0);
            }
        }
#pragma unroll
        for (int t = 0; t < K; ++t) {
            const int k = lane * K + t;
            A[t] = k < Dw ? L[t] : kInf;
        }
        prev_lo = cur_lo;
        prev_i = cur_i;
        x += dx;
        y += dy;
    }
}

template <int K>
void launch_general_k(const LevelArgs &a, const MergeArgs &m, cudaStream_t s)
{
    const int maxp = a.W + a.H - 1;
    dim3 grid((maxp + kScanWarps - 1) / kScanWarps, m.ndirs, a.nviews);
    const size_t smem = sizeof(int) * kScanWarps * 4 * (32 * K + 2);
    cudaFuncSetAttribute(agg_general<K>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    agg_general<K><<<grid, kScanWarps * 32, smem, s>>>(a, m);
}

}  // namespace

// ---------------------------------------------------------------------------------
// agg_scan8: the general passes with 8 lanes per scan path (4 paths per warp), K labels
// per lane as 32-bit integers, for strides of 8K labels.  Same arithmetic as agg_general
// (prefix minima of A(j) - pu j and suffix minima of A(j) + pd j, and of A itself for the
// asymmetric caps), with the scans over the path's 8 lanes (3 shuffle rounds) instead of
// a whole warp (5 rounds); re-indexing through shared memory when a window moved.
// ---------------------------------------------------------------------------------
constexpr int kScan8Warps = 4;

// Prefix minima over the path's G lanes of B(j) = A(j) - slope j (j = gl K + t): out[t] =
// min over labels up to this one; suffix minima of A(j) + slope j likewise from the end.
template <int K, int G>
__device__ __forceinline__ void scan8_prefix(const int (&A)[K], int slope, int gl, int (&out)[K])
{
    int run = kInf;
#pragma unroll
    for (int t = 0; t < K; ++t) {
        run = min(run, A[t] - slope * (gl * K + t));
        out[t] = run;
    }
    int incl = run;
#pragma unroll
    for (int o = 1; o < G; o <<= 1) {
        const int v = __shfl_up_sync(kFull, incl, o, G);
        if (gl >= o) incl = min(incl, v);
    }
    int excl = __shfl_up_sync(kFull, incl, 1, G);
    if (gl == 0) excl = kInf;
#pragma unroll
    for (int t = 0; t < K; ++t) out[t] = min(out[t], excl);
}

template <int K, int G>
__device__ __forceinline__ void scan8_suffix(const int (&A)[K], int slope, int gl, int (&out)[K])
{
    int run = kInf;
#pragma unroll
    for (int t = K - 1; t >= 0; --t) {
        run = min(run, A[t] + slope * (gl * K + t));
        out[t] = run;
    }
    int incl = run;
#pragma unroll
    for (int o = 1; o < G; o <<= 1) {
        const int v = __shfl_down_sync(kFull, incl, o, G);
        if (gl + o < G) incl = min(incl, v);
    }
    int excl = __shfl_down_sync(kFull, incl, 1, G);
    if (gl == G - 1) excl = kInf;
#pragma unroll
    for (int t = 0; t < K; ++t) out[t] = min(out[t], excl);
}

template <int K, bool WIN>
__global__ void __launch_bounds__(kScan8Warps * 32) agg_scan8(LevelArgs a, MergeArgs m)
{
    if (a.gate && *a.gate == 0) return;
    constexpr int G = 8, PPW = 32 / G, DWP = G * K, NJ = DWP;
    constexpr int PF = 4;                    // prefetch distance (steps)
    constexpr int QW = K / 2;                // 32-bit words of one u16 volume per lane
    const int view = blockIdx.z;
    const int dir = m.dir0 + blockIdx.y;
    const int dx = c_dirs[dir][0], dy = c_dirs[dir][1];
    const int W = a.W, H = a.H, Dw = a.Dw;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int gl = lane & (G - 1), grp = lane / G;
    const int path = (blockIdx.x * kScan8Warps + warp) * PPW + grp;
    const ViewLevel &V = a.v[view];
    const int T = a.trunc;
    const bool dbl = dir == m.double_up_dir;
    const int Tu = dbl ? 2 * T : T;
    const uint16_t *qa = view ? m.qa[1] : m.qa[0];
    const uint16_t *qb = view ? m.qb[1] : m.qb[0];
    uint16_t *const *outs = view ? m.out[1] : m.out[0];
    uint16_t *out = (dir & 1) ? outs[1] : outs[0];

    // per path: prefix/suffix minima for re-indexing, [4][NJ + 1]
    __shared__ int rbuf[WIN ? kScan8Warps * PPW * 4 * (NJ + 1) : 4];
    int *pB = rbuf + (WIN ? (warp * PPW + grp) * 4 * (NJ + 1) : 0);
    int *sC = pB + (NJ + 1), *pA = sC + (NJ + 1), *sA = pA + (NJ + 1);

    int x0 = 0, y0 = 0, n = 0;
    if (path < num_paths_dir(dx, dy, W, H)) {
        path_start(dx, dy, W, H, path, x0, y0);
        n = path_length(dx, dy, W, H, x0, y0);
    }
    const int nmax = __reduce_max_sync(kFull, n);
    const int64_t pix0 = (int64_t)y0 * W + x0, dpix = (int64_t)dy * W + dx;
    const int64_t ipix0 = (int64_t)y0 * V.pitch0 + x0, dipix = (int64_t)dy * V.pitch0 + dx;

    // prefetch ring: the data term words, the window start and the intensity of the next
    // PF pixels, loaded PF steps ahead with pinned loads
    // (zero until loaded: a slot past the end of a short path is never loaded, and its
    // intensity still indexes the slope table)
    uint32_t qr[PF][2 * QW > 1 ? 2 * QW : 1];
    uint32_t lr[PF], ir[PF];
#pragma unroll
    for (int u = 0; u < PF; ++u) {
        lr[u] = ir[u] = 0u;
#pragma unroll
        for (int j = 0; j < (2 * QW > 1 ? 2 * QW : 1); ++j) qr[u][j] = 0u;
    }
    auto issue = [&](int t, int slot) {
        const int64_t pix = pix0 + t * dpix;
        if (t < n && MPV_IN(a.err, pix >= 0 && pix < (int64_t)W * H, 8) &&
            MPV_IN(a.err, !m.lut || (ipix0 + t * dipix >= 0 &&
                                     ipix0 + t * dipix < (int64_t)V.pitch0 * H), 9)) {
            if (m.in_mode == 0) {
                const uint8_t *cp = V.C + pix * DWP + gl * K;
                if (K % 4 == 0) {
#pragma unroll
                    for (int j = 0; j < K / 4; ++j) qr[slot][j] = ld_pin_u32(cp + 4 * j);
                } else {
                    qr[slot][0] = ld_pin_u16(cp);
                }
            } else {
#pragma unroll
                for (int j = 0; j < QW; ++j) {
                    qr[slot][j] = ld_pin_u32(qa + pix * DWP + gl * K + 2 * j);
                    qr[slot][QW + j] = ld_pin_u32(qb + pix * DWP + gl * K + 2 * j);
                }
            }
            lr[slot] = V.lo ? ld_pin_u16(V.lo + pix) : 0u;
            ir[slot] = m.lut ? ld_pin_u8(V.I0 + ipix0 + t * dipix) : 0u;
        }
    };
#pragma unroll
    for (int u = 0; u < PF; ++u) issue(u, u);

    int A[K];
#pragma unroll
    for (int t = 0; t < K; ++t) A[t] = kInf;
    int prev_lo = 0, prev_i = 0;
    for (int t0 = 0; t0 < nmax; t0 += PF) {
#pragma unroll
        for (int u = 0; u < PF; ++u) {
            const int step = t0 + u;
            if (step >= nmax) break;
            const bool act = step < n;
            const int x = x0 + step * dx, y = y0 + step * dy;
            const int64_t pix = act ? pix0 + step * dpix : 0;
            const int cur_lo = (int)lr[u];
            const int cur_i = (int)ir[u];
            // data term of this lane's K labels
            int c[K];
            if (m.in_mode == 0) {
                if (K % 4 == 0) {
#pragma unroll
                    for (int t = 0; t < K; ++t) c[t] = (qr[u][t / 4] >> (8 * (t % 4))) & 0xFF;
                } else {
                    c[0] = qr[u][0] & 0xFF;
                    c[1 % K] = (qr[u][0] >> 8) & 0xFF;
                }
            } else {
#pragma unroll
                for (int t = 0; t < K; ++t) {
                    const int ea = (qr[u][t / 2] >> (16 * (t % 2))) & 0xFFFF;
                    const int eb = (qr[u][QW + t / 2] >> (16 * (t % 2))) & 0xFFFF;
                    c[t] = m.in_mode == 1 ? min(ea, eb) : (ea + eb) >> 1;
                }
            }
#pragma unroll
            for (int t = 0; t < K; ++t)
                if (gl * K + t >= Dw) c[t] = 0;
            issue(step + PF, u);
            bool first = step == 0;
            if (a.block_cut > 0 && !first &&
                (x / a.block_cut != (x - dx) / a.block_cut ||
                 y / a.block_cut != (y - dy) / a.block_cut))
                first = true;
            int L[K];
            if (__all_sync(kFull, first || !act)) {   // every path of the warp starts here
#pragma unroll
                for (int t = 0; t < K; ++t) L[t] = c[t];
            } else {
                // a path starting here (first pixel or tile edge): L = c below
                const int P = (m.lut && act &&
                               MPV_IN(a.err, cur_i >= 0 && cur_i < 256 && prev_i >= 0 &&
                                                 prev_i < 256, 12))
                                  ? min(m.lut[abs(cur_i - prev_i) & 0xFF], T)
                                  : a.p1;
                const int pu = dbl ? 2 * P : P, pd = P;
                int mn = A[0];
#pragma unroll
                for (int t = 1; t < K; ++t) mn = min(mn, A[t]);
#pragma unroll
                for (int o = 1; o < G; o <<= 1) mn = min(mn, __shfl_xor_sync(kFull, mn, o));
                const int amin = mn;
                int pb[K], sc[K], pa[K], sa[K];
                scan8_prefix<K, G>(A, pu, gl, pb);
                scan8_suffix<K, G>(A, pd, gl, sc);
                if (dbl) {   // the doubled pass's caps need the running minima of A itself
                    scan8_prefix<K, G>(A, 0, gl, pa);
                    scan8_suffix<K, G>(A, 0, gl, sa);
                } else {
#pragma unroll
                    for (int t = 0; t < K; ++t) pa[t] = sa[t] = kInf;
                }
                const int s = (WIN && act && !first) ? cur_lo - prev_lo : 0;
                if (WIN && __any_sync(kFull, s != 0)) {
#pragma unroll
                    for (int t = 0; t < K; ++t) {
                        pB[gl * K + t + 1] = pb[t];
                        sC[gl * K + t] = sc[t];
                        pA[gl * K + t + 1] = pa[t];
                        sA[gl * K + t] = sa[t];
                    }
                    if (gl == 0) {
                        pB[0] = pA[0] = kInf;
                        sC[NJ] = sA[NJ] = kInf;
                    }
                    __syncwarp();
#pragma unroll
                    for (int t = 0; t < K; ++t) {
                        const int jj = s + gl * K + t;   // label index in the predecessor window
                        const int pi = min(max(jj, -1), NJ - 1) + 1;
                        const int si = min(max(jj, 0), NJ);
                        int M = min(pu * jj + pB[pi], sC[si] - pd * jj);
                        M = dbl ? min(M, min(pA[pi] + Tu, sA[si] + T)) : min(M, amin + T);
                        L[t] = c[t] + M - amin;
                    }
                    __syncwarp();
                } else {
#pragma unroll
                    for (int t = 0; t < K; ++t) {
                        const int j = gl * K + t;
                        int M = min(pu * j + pb[t], sc[t] - pd * j);
                        M = dbl ? min(M, min(pa[t] + Tu, sa[t] + T)) : min(M, amin + T);
                        L[t] = c[t] + M - amin;
                    }
                }
                if (first) {
#pragma unroll
                    for (int t = 0; t < K; ++t) L[t] = c[t];
                }
            }
#pragma unroll
            for (int t = 0; t < K; ++t)
                if (gl * K + t >= Dw) L[t] = 0;
            if (m.out_mode == 0) {
                uint16_t *sp = V.S + pix * DWP + gl * K;
#pragma unroll
                for (int t = 0; t < K; t += 2)
                    if (act)
                        atomicAdd((unsigned int *)(sp + t),
                                  (unsigned)L[t] | ((unsigned)L[t + 1] << 16));
            } else {
                int lm = kInf;
#pragma unroll
                for (int t = 0; t < K; ++t)
                    if (gl * K + t < Dw) lm = min(lm, L[t]);
#pragma unroll
                for (int o = 1; o < G; o <<= 1) lm = min(lm, __shfl_xor_sync(kFull, lm, o));
                uint16_t *op = out + pix * DWP + gl * K;
#pragma unroll
                for (int t = 0; t < K; t += 2) {
                    const unsigned lo16 = gl * K + t < Dw ? (unsigned)(L[t] - lm) : 0u;
                    const unsigned hi16 = gl * K + t + 1 < Dw ? (unsigned)(L[t + 1] - lm) : 0u;
                    if (act) *(unsigned int *)(op + t) = lo16 | (hi16 << 16);
                }
            }
#pragma unroll
            for (int t = 0; t < K; ++t) A[t] = gl * K + t < Dw ? L[t] : kInf;
            prev_lo = cur_lo;
            prev_i = cur_i;
        }
    }
}

template <int K>
void launch_scan8_k(const LevelArgs &a, const MergeArgs &m, cudaStream_t s)
{
    const int maxp = a.W + a.H - 1;
    const int per_block = kScan8Warps * (32 / 8);
    dim3 grid((maxp + per_block - 1) / per_block, m.ndirs, a.nviews);
    if (a.v[0].lo)
        agg_scan8<K, true><<<grid, kScan8Warps * 32, 0, s>>>(a, m);
    else
        agg_scan8<K, false><<<grid, kScan8Warps * 32, 0, s>>>(a, m);
}

void launch_aggregate_general(const LevelArgs &a, const MergeArgs &m, cudaStream_t s)
{
    if (sweep_ok(a, m)) {
        launch_sweep(a, m, s);
        return;
    }
    // 8 lanes per path for the strides of 16, 32 and 64 labels
    switch (a.Dws) {
    case 16: launch_scan8_k<2>(a, m, s); return;
    case 32: launch_scan8_k<4>(a, m, s); return;
    case 64: launch_scan8_k<8>(a, m, s); return;
    default: break;
    }
    const int K = (a.Dw + 31) / 32;
    if (K <= 1) launch_general_k<1>(a, m, s);
    else if (K <= 2) launch_general_k<2>(a, m, s);
    else if (K <= 4) launch_general_k<4>(a, m, s);
    else if (K <= 8) launch_general_k<8>(a, m, s);
    else if (K <= 16) launch_general_k<16>(a, m, s);
    else launch_general_k<32>(a, m, s);
}

// ---------------------------------------------------------------------------------
// One layer of the layered merge: the packed stencil where its arithmetic holds (jumps
// beyond 4 labels truncated, no gradient table, strides of 16 or 32 labels, energies far
// below the packed sentinel), the doubled left-to-right pass and everything else through
// the general kernels.
// ---------------------------------------------------------------------------------
namespace {

bool layer_stencil_ok(const LevelArgs &a, const MergeArgs &m)
{
    return m.out_mode == 1 && !m.lut && a.radius <= 4 && (a.Dws == 16 || a.Dws == 32) &&
           255 + 10 * a.trunc < (int)kInf16;
}

template <int G, int KW>
void launch_layer_kw(const LevelArgs &a, const MergeArgs &m, cudaStream_t s)
{
    const bool win = a.v[0].lo != nullptr;
    const bool blk = a.block_cut > 0;
    if (a.radius <= 2) {
        if (win) launch_stencil<G, KW, 2, true, false, true, false, G == 8>(a, s, m, m.ndirs);
        else if (blk) launch_stencil<G, KW, 2, false, true, true, false, G == 8>(a, s, m, m.ndirs);
        else launch_stencil<G, KW, 2, false, false, true, false, G == 8>(a, s, m, m.ndirs);
    } else if constexpr (KW >= 2) {
        if (win) launch_stencil<G, KW, 4, true, false, true, false, G == 8>(a, s, m, m.ndirs);
        else if (blk) launch_stencil<G, KW, 4, false, true, true, false, G == 8>(a, s, m, m.ndirs);
        else launch_stencil<G, KW, 4, false, false, true, false, G == 8>(a, s, m, m.ndirs);
    }
}

void launch_layer_stencil(const LevelArgs &a, const MergeArgs &m, cudaStream_t s)
{
    if (a.Dws == 32) launch_layer_kw<kLanesWide, 2>(a, m, s);
    else if (a.radius <= 2) launch_layer_kw<kLanesWide, 1>(a, m, s);
    else launch_layer_kw<4, 2>(a, m, s);
}

}  // namespace

int launch_layer(const LevelArgs &a, const MergeArgs &m, cudaStream_t s)
{
    if (!layer_stencil_ok(a, m)) {
        launch_aggregate_general(a, m, s);
        return 1;
    }
    launch_layer_stencil(a, m, s);   // the doubled pass included (asymmetric stencil)
    return 1;
}

void launch_aggregate(const LevelArgs &a, cudaStream_t s)
{
    if (a.radius <= 4 && a.Dws <= 64 && packed_caps_ok(a, 1)) {
        const bool wide = a.lanes == kLanesWide;
        switch (a.Dws) {
        case 16:
            // 8 lanes of one word each for the radius-2 stencil, else 4 lanes of two words
            if (wide && a.radius <= 2) launch_stencil_kw<kLanesWide, 1>(a, s);
            else launch_stencil_kw<4, 2>(a, s);
            return;
        case 32:
            if (wide) launch_stencil_kw<kLanesWide, 32 / (2 * kLanesWide)>(a, s);
            else launch_stencil_kw<4, 4>(a, s);
            return;
        case 48: launch_stencil_kw<4, 6>(a, s); return;
        default:
            if (wide) launch_stencil_kw<kLanesWide, 64 / (2 * kLanesWide)>(a, s);
            else launch_stencil_kw<4, 8>(a, s);
            return;
        }
    }
    MergeArgs m{};
    m.in_mode = 0;
    m.out_mode = 0;
    m.dir0 = 0;
    m.ndirs = a.npaths;
    m.double_up_dir = -1;
    m.lut = nullptr;
    launch_aggregate_general(a, m, s);
}

}  // namespace mpv
