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
//    and S is accumulated with 64-bit reductions of four packed labels.  Its layer mode
//    runs one layer of the layered merge (Section 3.2), the left-to-right pass with doubled
//    upward jumps included; its sweep mode runs gradient-weighted slopes (Eq. EU) as
//    untruncated packed sweeps.
//  * agg_scan8: 8 lanes per path, int32 labels, the two sweeps as segmented prefix and
//    suffix minima across the lanes: the gradient and layered variants outside the packed
//    kernel's bounds or widths.
//  * agg_general: any window width: one warp per scan path, the sweeps written as prefix
//    minima  min_{v<=u} A(v) + p1 (u-v) = p1 u + min_{v<=u} (A(v) - p1 v)  (and the mirror
//    image), evaluated by shuffle scans over the lanes.
#include "mpv_internal.cuh"

namespace mpv {

namespace {

__constant__ int c_dirs[8][2] = {{1, 0}, {-1, 0}, {0, 1}, {0, -1},
                                 {1, 1}, {-1, -1}, {-1, 1}, {1, -1}};

constexpr unsigned kFull = 0xFFFFFFFFu;

__device__ __forceinline__ int num_paths_dir(int dx, int dy, int W, int H)
{
    if (dy == 0) return H;
    if (dx == 0) return W;
    return W + H - 1;
}

// First pixel of path i of direction (dx,dy): the pixels whose predecessor p - r lies
// outside the image.
__device__ __forceinline__ void path_start(int dx, int dy, int W, int H, int i, int &x, int &y)
{
    if (dy == 0) {
        x = dx > 0 ? 0 : W - 1;
        y = i;
    } else if (dx == 0) {
        x = i;
        y = dy > 0 ? 0 : H - 1;
    } else if (i < W) {
        x = i;
        y = dy > 0 ? 0 : H - 1;
    } else {
        x = dx > 0 ? 0 : W - 1;
        y = dy > 0 ? (i - W + 1) : (H - 2 - (i - W));
    }
}

// ---------------------------------------------------------------------------------
// agg_stencil
// ---------------------------------------------------------------------------------

constexpr int kStencilWarps = 4;            // warps per block
// lanes per scan path for 32- and 64-label strides when the tuning asks for the wide
// form (4 labels, resp. 8, per lane): more independent warps per SM hide the per-step
// dependency latency better than 4 lanes on large levels
constexpr int kLanesWide = 8;

// Prefetch loads of the scan paths.  Written as volatile asm so that the compiler keeps
// them where they are issued (PF steps ahead of their use) instead of re-issuing a
// read-only load next to its use.
__device__ __forceinline__ uint32_t ld_pin_u32(const void *p)
{
    uint32_t v;
    asm volatile("ld.global.nc.u32 %0, [%1];" : "=r"(v) : "l"(p));
    return v;
}
__device__ __forceinline__ uint2 ld_pin_u64(const void *p)
{
    uint2 v;
    asm volatile("ld.global.nc.v2.u32 {%0, %1}, [%2];" : "=r"(v.x), "=r"(v.y) : "l"(p));
    return v;
}
__device__ __forceinline__ uint32_t ld_pin_u8(const void *p)
{
    uint32_t v;
    asm volatile("ld.global.nc.u8 %0, [%1];" : "=r"(v) : "l"(p));
    return v;
}
__device__ __forceinline__ uint32_t ld_pin_u16(const void *p)
{
    unsigned short v;
    asm volatile("ld.global.nc.u16 %0, [%1];" : "=h"(v) : "l"(p));
    return v;
}

// (high half of a, low half of b): the word of labels shifted by one
__device__ __forceinline__ uint32_t shift1(uint32_t a, uint32_t b)
{
    return __byte_perm(a, b, 0x5432);
}

// Number of pixels of the path that starts at (x0,y0) in direction (dx,dy).
__device__ __forceinline__ int path_length(int dx, int dy, int W, int H, int x0, int y0)
{
    const int nx = dx > 0 ? W - x0 : (dx < 0 ? x0 + 1 : 0x7FFFFFFF);
    const int ny = dy > 0 ? H - y0 : (dy < 0 ? y0 + 1 : 0x7FFFFFFF);
    return min(nx, ny);
}

// floor((a + b) / 2) of each 16-bit half (the shift masked so that no bit crosses
// from the high half into the low half)
__device__ __forceinline__ uint32_t avg_u16x2(uint32_t a, uint32_t b)
{
    return (a & b) + (((a ^ b) >> 1) & 0x7FFF7FFFu);
}

// Packed energies of one lane minus the path's minimum m2 (both halves), padding labels
// as 0, stored as KW 32-bit words.
template <int KW>
__device__ __forceinline__ void store_normalised(uint16_t *dst, const uint32_t (&A)[KW], uint32_t m2,
                                                 const uint32_t (&keep)[KW], bool padded)
{
#pragma unroll
    for (int i = 0; i < KW; ++i) {
        uint32_t v = A[i] - m2;           // per half: A >= m2 on every kept label
        if (padded) v &= keep[i];
        ((uint32_t *)dst)[i] = v;
    }
}

// agg_stencil template parameters.
// G: lanes per scan path (4 or 8); KW: packed 32-bit words (2 labels each) per lane.
// RM: largest jump |d| handled explicitly.  The penalty of a jump of d labels is
// eps(d) = min(p1 d, T) for every d <= RM, so whenever the truncation dominates beyond
// RM (ceil(T/p1) - 1 <= RM) the stencil min over |d| <= RM plus the cap min_v A(v) + T
// is the full-connectivity minimum.  WIN: the level has per-pixel windows; a step whose
// window moved re-indexes the predecessor into the current window through shared memory.
// BLK: the level is split into independent block_cut x block_cut tiles (a scan path
// restarts where it enters a new tile); counters track the steps to the next tile edge.
// LAYER: one layer of the paper's layered merge - the data term is the cost bytes
// (mg.in_mode 0) or the previous layer's two passes merged by min (1) or floor mean (2),
// and the pass stores its per-pixel min-normalised energies into its own volume instead
// of adding into S (one step late, when the next step's minimum over the path's labels
// is known).  The pass mg.double_up_dir charges upward jumps twice (u > v: 2 min(p1 d, T));
// its envelope is
//     M'(u) = min( A(u), min_{1<=d<=RM} A(u-d) + 2 min(p1 d, T), A(u+d) + min(p1 d, T),
//                  min_v A(v) + 2T,  min_{v>=u} A(v) + T ),
// exact because every added term is at least one true term and every jump beyond RM is
// covered (upward ones by min_v A(v) + 2T, downward ones by the suffix minimum + T).  The
// suffix minimum is a packed scan over the lane's words and the path's lanes.
// SWP: the slope of each step comes from the gradient table (Eq. EU's weighting,
// lut[|I0(p) - I0(p-r)|]), so no fixed radius holds; the two sweeps of Section 3.3 are then
// evaluated untruncated in packed form,
//     F(u) = min_{v<=u} A(v) + pu (u-v),   G(u) = min_{v>=u} A(v) + pd (v-u),
// inside the lane by doubling (one label, then whole words) and across the path's lanes by
// a scan of the lanes' end values, and M'(u) = min(F(u), G(u), min_v A(v) + T) (plus the
// doubled pass's suffix term).  Sweep values never exceed the sentinel plus pu times the
// labels of a lane, which the dispatch keeps below 2^16.  With windows, the envelope is
// formed in the predecessor's frame and re-indexed; labels beyond the predecessor's window
// continue the sweeps linearly from its edge, capped.
// XM: the path minimum through shared memory instead of shuffles (8-lane paths; chosen at
// dispatch where measured faster).
template <int G, int KW, int RM, bool WIN, bool BLK, bool LAYER, bool SWP, bool XM>
__global__ void __launch_bounds__(kStencilWarps * 32) agg_stencil(LevelArgs a, MergeArgs mg)
{
    if (a.gate && *a.gate == 0) return;
    constexpr int kG = G;                    // lanes per scan path
    constexpr int kPathsPerWarp = 32 / kG;
    constexpr int HW = RM / 2;               // halo words per side
    constexpr int NE = KW + 2 * HW;          // words with halos
    constexpr int K = 2 * KW;                // labels per lane
    constexpr int DWP = kG * K;              // labels per path (= the volume stride)
    constexpr int PAD = (DWP + 4 * HW + 2 + 7) / 8 * 8;  // absent labels around a path
    constexpr int BUF = 2 * PAD + DWP;
    // prefetch distance (steps), measured: 12 for the summed pass with two words per lane
    // (8 lanes on 32 labels), 8 for the other shapes and for the layer and sweep modes
    // (each slower at 12), 4 for the widest lanes
    constexpr int PF = KW > 4 ? 4 : (KW == 2 && !LAYER && !SWP ? 12 : 8);
    constexpr int CW = KW >= 2 ? KW / 2 : 1; // 32-bit words of cost bytes per lane
    static_assert(kG == 4 || kG == 8, "paths of 4 or 8 lanes");

    __shared__ __align__(16) uint16_t rbuf[WIN ? kStencilWarps * kPathsPerWarp * BUF : 8];
    // suffix minima of the predecessor for the doubled pass: lower pad = the path's
    // minimum (every predecessor label lies above), upper pad absent
    __shared__ __align__(16) uint16_t sbuf[WIN && LAYER && !SWP ? kStencilWarps * kPathsPerWarp * BUF : 8];
    __shared__ int slut[SWP ? 256 : 1];      // the gradient table's slopes
    __shared__ __align__(16) uint32_t redbuf[2 * kStencilWarps * 32];   // path minima
    if (SWP) {
        for (int i = threadIdx.x; i < 256; i += blockDim.x) slut[i] = mg.lut[i];
        __syncthreads();
    }

    const int view = blockIdx.z, dir = mg.dir0 + blockIdx.y;
    // layered merge: the previous layer's pair (IN) and this pass's own volume (OUTN)
    const uint16_t *qa = view ? mg.qa[1] : mg.qa[0];
    const uint16_t *qb = view ? mg.qb[1] : mg.qb[0];
    uint16_t *const *outs = view ? mg.out[1] : mg.out[0];
    uint16_t *const outv = (dir & 1) ? outs[1] : outs[0];
    const int dx = c_dirs[dir][0], dy = c_dirs[dir][1];
    const int W = a.W, H = a.H, Dw = a.Dw;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int gl = lane & (kG - 1), grp = lane / kG;
    const int path = (blockIdx.x * kStencilWarps + warp) * kPathsPerWarp + grp;
    const ViewLevel &V = a.v[view];

    uint16_t *gb = rbuf + (WIN ? (warp * kPathsPerWarp + grp) * BUF : 0);
    uint16_t *sb = sbuf + (WIN && LAYER && !SWP ? (warp * kPathsPerWarp + grp) * BUF : 0);
    if (WIN) {
        for (int i = gl; i < BUF; i += kG) gb[i] = (uint16_t)kInf16;
        if (LAYER && !SWP)
            for (int i = gl; i < BUF; i += kG) sb[i] = (uint16_t)kInf16;
        __syncwarp();
    }

    const uint32_t INF2 = kInf16 * 0x10001u;
    const uint32_t T = (uint32_t)a.trunc, P1 = (uint32_t)a.p1;
    const uint32_t Tx2 = T * 0x10001u;
    const uint32_t E1 = min(P1, T) * 0x10001u, E2 = min(2 * P1, T) * 0x10001u;
    const uint32_t E3 = min(3 * P1, T) * 0x10001u, E4 = min(4 * P1, T) * 0x10001u;
    // the doubled pass (block-uniform): upward jumps and their cap cost twice
    const bool asym = LAYER && dir == mg.double_up_dir;
    const uint32_t up = asym ? 2u : 1u;
    const uint32_t U1 = E1 * up, U2 = E2 * up, U3 = E3 * up, U4 = E4 * up;
    const uint32_t Tcap = Tx2 * up;

    // labels at or beyond Dw are padding: never a predecessor, never summed
    const bool padded = Dw < DWP;
    uint32_t keep[KW];
#pragma unroll
    for (int i = 0; i < KW; ++i) {
        const int k0 = gl * K + 2 * i;
        keep[i] = (k0 < Dw ? 0x0000FFFFu : 0u) | (k0 + 1 < Dw ? 0xFFFF0000u : 0u);
    }

    int x0 = 0, y0 = 0, n = 0;
    if (path < num_paths_dir(dx, dy, W, H)) {
        path_start(dx, dy, W, H, path, x0, y0);
        n = path_length(dx, dy, W, H, x0, y0);
    }
    const int nmax = __reduce_max_sync(kFull, n);
    const int pix0 = y0 * W + x0;
    const int dpix = dy * W + dx;
    const uint8_t *cbase = V.C + gl * K;
    uint16_t *sbase = V.S + gl * K;
    const uint16_t *lob = V.lo;

    // prefetch ring (registers): cost bytes (or the previous layer's two words per
    // packed pair) and window start of the next PF steps
    constexpr int QW = LAYER ? KW : 1;
    const int IN = LAYER ? mg.in_mode : 0;
    constexpr bool OUTN = LAYER;
    uint32_t cq[PF][CW];
    uint32_t qaq[PF][QW], qbq[PF][QW];
    uint32_t lq[PF];
    // SWP: the reference intensity of the next PF pixels (zero until loaded: a slot past
    // the end of a short path is never loaded)
    uint32_t iq[PF];
#pragma unroll
    for (int u = 0; u < PF; ++u) iq[u] = 0u;
    const int64_t ipix0 = (int64_t)y0 * V.pitch0 + x0, dipix = (int64_t)dy * V.pitch0 + dx;
    auto issue = [&](int t, int slot) {
        if (t < n) {
            const int pix = pix0 + t * dpix;
            const uint8_t *src = cbase + (int64_t)pix * DWP;
            if (LAYER && IN) {
                const uint16_t *sa = qa + (int64_t)pix * DWP + gl * K;
                const uint16_t *sb = qb + (int64_t)pix * DWP + gl * K;
                if (KW % 2 == 0) {
#pragma unroll
                    for (int j = 0; j < KW; j += 2) {
                        const uint2 va = ld_pin_u64(sa + 2 * j), vb = ld_pin_u64(sb + 2 * j);
                        qaq[slot][j % QW] = va.x;
                        qaq[slot][(j + 1) % QW] = va.y;
                        qbq[slot][j % QW] = vb.x;
                        qbq[slot][(j + 1) % QW] = vb.y;
                    }
                } else {
#pragma unroll
                    for (int j = 0; j < KW; ++j) {
                        qaq[slot][j % QW] = ld_pin_u32(sa + 2 * j);
                        qbq[slot][j % QW] = ld_pin_u32(sb + 2 * j);
                    }
                }
            } else if (KW == 1) {
                cq[slot][0] = ld_pin_u16(src);
            } else if (CW % 2 == 0) {
#pragma unroll
                for (int j = 0; j < CW; j += 2) {
                    const uint2 v = ld_pin_u64(src + 4 * j);
                    cq[slot][j] = v.x;
                    cq[slot][j + 1] = v.y;
                }
            } else {
#pragma unroll
                for (int j = 0; j < CW; ++j) cq[slot][j] = ld_pin_u32(src + 4 * j);
            }
            lq[slot] = WIN ? ld_pin_u16(lob + pix) : 0u;
            if (SWP) iq[slot] = ld_pin_u8(V.I0 + ipix0 + t * dipix);
        }
    };
#pragma unroll
    for (int u = 0; u < PF; ++u) issue(u, u);

    uint32_t A[KW];
#pragma unroll
    for (int i = 0; i < KW; ++i) A[i] = INF2;   // no predecessor: L = C at the first pixel
    int prev_lo = -1;
    int prev_i = 0;
    // steps to the next tile edge in x and in y (BLK)
    const int B = a.block_cut;
    int cx = 0x7FFFFFFF, cy = 0x7FFFFFFF;
    if (BLK) {
        if (dx > 0) cx = B - x0 % B;
        if (dx < 0) cx = x0 % B + 1;
        if (dy > 0) cy = B - y0 % B;
        if (dy < 0) cy = y0 % B + 1;
    }

    for (int t0 = 0; t0 < nmax; t0 += PF) {
#pragma unroll
        for (int u = 0; u < PF; ++u) {
            const int t = t0 + u;
            if (t >= nmax) break;
            const bool act = t < n;
            const int pix = pix0 + t * dpix;
            uint32_t c[KW];
            if (LAYER && IN) {
#pragma unroll
                for (int i = 0; i < KW; ++i)
                    c[i] = IN == 1 ? __vminu2(qaq[u][i % QW], qbq[u][i % QW])
                                   : avg_u16x2(qaq[u][i % QW], qbq[u][i % QW]);
            } else if (KW == 1) {
                c[0] = __byte_perm(cq[u][0], 0u, 0x4140);
            } else {
#pragma unroll
                for (int j = 0; j < CW; ++j) {
                    c[2 * j] = __byte_perm(cq[u][j], 0u, 0x4140);
                    c[(2 * j + 1) % KW] = __byte_perm(cq[u][j], 0u, 0x4342);
                }
            }
            const int cur_lo = (int)lq[u];
            const int cur_i = (int)iq[u];
            issue(t + PF, u);

            // this step's window shift, known from the prefetched window starts: a path whose
            // window moved re-indexes through shared memory (the whole warp does, when any of
            // its paths moved); voted here, ahead of the shuffles that depend on A
            const int s = (WIN && act && prev_lo >= 0) ? cur_lo - prev_lo : 0;
            const bool moved = WIN && __any_sync(kFull, s != 0);

            // minimum of the predecessor over the path's lanes, in both halves
            uint32_t m2 = A[0];
#pragma unroll
            for (int i = 1; i < KW; ++i) m2 = __vminu2(m2, A[i]);
            m2 = __vminu2(m2, __byte_perm(m2, m2, 0x1032));
            uint32_t lm = m2;                 // this lane's minimum
            if constexpr (!XM || kG != 8) {
#pragma unroll
                for (int o = 1; o < kG; o <<= 1) m2 = __vminu2(m2, __shfl_xor_sync(kFull, m2, o));
            } else {
                // the 8 lane minima of the path through shared memory (one store, one warp
                // barrier, two 16-byte loads) instead of three dependent shuffles: the
                // exchange is on every step's dependent chain.  Double-buffered by step
                // parity, so a lane's next store never meets a read of this step.
                uint32_t *rw = redbuf + ((t & 1) * kStencilWarps + warp) * 32;
                rw[lane] = lm;
                __syncwarp();
                const uint4 *g4 = (const uint4 *)(rw + grp * kG);
                const uint4 q0 = g4[0];
                const uint32_t r = __vminu2(__vminu2(q0.x, q0.y), __vminu2(q0.z, q0.w));
                const uint4 q1 = g4[1];
                m2 = __vminu2(r, __vminu2(__vminu2(q1.x, q1.y), __vminu2(q1.z, q1.w)));
            }
            if (OUTN && t > 0 && t - 1 < n)   // the previous pixel, normalised by its minimum
                store_normalised<KW>(outv + (int64_t)(pix - dpix) * DWP + gl * K, A, m2, keep,
                                     padded);
            if (BLK && t > 0) {   // entering a new tile: the path starts again here
                --cx;
                --cy;
                const bool cut = cx == 0 || cy == 0;
                if (cx == 0) cx = B;
                if (cy == 0) cy = B;
                if (cut) {
#pragma unroll
                    for (int i = 0; i < KW; ++i) A[i] = INF2;
                    m2 = INF2;
                    lm = INF2;
                }
            }
            const uint32_t cap = m2 + Tcap;

            // doubled pass: suffix minima SA(u) = min_{v>=u} A(v), first over the lanes
            // above (exclusive scan of the lane minima), then down the lane's own words
            uint32_t SA[KW];
            if (asym) {
                uint32_t ex = __shfl_down_sync(kFull, lm, 1, kG);
                if (gl == kG - 1) ex = INF2;
#pragma unroll
                for (int o = 1; o < kG; o <<= 1) {
                    const uint32_t v = __shfl_down_sync(kFull, ex, o, kG);
                    if (gl + o < kG) ex = __vminu2(ex, v);
                }
#pragma unroll
                for (int i = KW - 1; i >= 0; --i) {
                    const uint32_t v = __vminu2(A[i], ex);               // (min(lo,r), min(hi,r))
                    SA[i] = __vminu2(v, __byte_perm(v, v, 0x3232));     // low half also <= high
                    ex = __byte_perm(SA[i], SA[i], 0x1010);
                }
            }

            if constexpr (!SWP) {
                // predecessor words around this lane's labels, HW halo words per side
                uint32_t E[NE];
#pragma unroll
                for (int i = 0; i < KW; ++i) E[HW + i] = A[i];
#pragma unroll
                for (int h = 0; h < HW; ++h) {
                    const uint32_t l = __shfl_up_sync(kFull, A[KW - HW + h], 1, kG);
                    const uint32_t r = __shfl_down_sync(kFull, A[h], 1, kG);
                    E[h] = gl == 0 ? INF2 : l;
                    E[HW + KW + h] = gl == kG - 1 ? INF2 : r;
                }
                if (moved) {   // re-index the predecessor
                    uint32_t *gw = (uint32_t *)(gb + PAD + gl * K);
#pragma unroll
                    for (int i = 0; i < KW; ++i) gw[i] = A[i];
                    if (LAYER && asym) {
                        uint32_t *sw = (uint32_t *)(sb + PAD + gl * K);
#pragma unroll
                        for (int i = 0; i < KW; ++i) sw[i] = SA[i];
                        uint32_t *sl = (uint32_t *)(sb + PAD - DWP);
                        for (int w = gl; w < DWP / 2; w += kG) sl[w] = m2;
                    }
                    __syncwarp();
                    const int sc = min(max(s, -(DWP + 2 * HW)), DWP + 2 * HW);
                    const int j0 = PAD + gl * K - 2 * HW + sc;
                    const uint32_t *gwords = (const uint32_t *)gb + (j0 >> 1);
                    const uint32_t sel = (j0 & 1) ? 0x5432u : 0x3210u;
                    uint32_t Wd[NE + 1];
#pragma unroll
                    for (int i = 0; i <= NE; ++i) Wd[i] = gwords[i];
#pragma unroll
                    for (int w = 0; w < NE; ++w) E[w] = __byte_perm(Wd[w], Wd[w + 1], sel);
                    if (LAYER && asym) {
                        // current label j reads the predecessor's suffix minimum at j + s:
                        // below its window every label is above (the minimum), beyond it none
                        const int s2 = min(max(s, -DWP), DWP);
                        const int j1 = PAD + gl * K + s2;
                        const uint32_t *swords = (const uint32_t *)sb + (j1 >> 1);
                        const uint32_t sel2 = (j1 & 1) ? 0x5432u : 0x3210u;
                        uint32_t Sd[KW + 1];
#pragma unroll
                        for (int i = 0; i <= KW; ++i) Sd[i] = swords[i];
#pragma unroll
                        for (int i = 0; i < KW; ++i) SA[i] = __byte_perm(Sd[i], Sd[i + 1], sel2);
                    }
                    __syncwarp();
                }

                uint32_t SH[NE - 1];
#pragma unroll
                for (int j = 0; j < NE - 1; ++j) SH[j] = shift1(E[j], E[j + 1]);

#pragma unroll
                for (int i = 0; i < KW; ++i) {
                    const int e = HW + i;
                    // words below e hold smaller labels: jumps up into (u, u+1)
                    uint32_t m = __vminu2(E[e], cap);
                    m = __viaddmin_u16x2(SH[e - 1], U1, m);
                    m = __viaddmin_u16x2(SH[e], E1, m);
                    m = __viaddmin_u16x2(E[e - 1], U2, m);
                    m = __viaddmin_u16x2(E[e + 1], E2, m);
                    if (RM >= 4) {
                        m = __viaddmin_u16x2(SH[e - 2], U3, m);
                        m = __viaddmin_u16x2(SH[e + 1], E3, m);
                        m = __viaddmin_u16x2(E[e - 2], U4, m);
                        m = __viaddmin_u16x2(E[e + 2], E4, m);
                    }
                    if (asym) m = __viaddmin_u16x2(SA[i], Tx2, m);
                    uint32_t L = c[i] + m - m2;      // per half: no carry, no borrow
                    if (padded) {
                        L &= keep[i];
                        A[i] = L | (INF2 & ~keep[i]);
                    } else {
                        A[i] = L;
                    }
                    c[i] = L;
                }
            } else {
                uint32_t Mv[KW];   // the envelope M'(u) of this lane's labels
                // this step's slopes: the table at the intensity step, at most T
                const uint32_t P =
                    (act && t > 0) ? min((uint32_t)slut[abs(cur_i - prev_i) & 0xFF], T) : P1;
                const uint32_t Pu = P * up, Pd = P;
                const uint32_t Cu1 = Pu * 0x10001u, Cd1 = Pd * 0x10001u;
                uint32_t F[KW], Gd[KW];
                // inside the lane: neighbours one label away, then whole words
#pragma unroll
                for (int w = 0; w < KW; ++w) {
                    // (absent, first label) and (last label, absent) at the lane's ends
                    const uint32_t xl =
                        w == 0 ? __byte_perm(A[0], INF2, 0x1054) : shift1(A[w - 1], A[w]);
                    const uint32_t xr =
                        w == KW - 1 ? __byte_perm(A[KW - 1], INF2, 0x7632) : shift1(A[w], A[w + 1]);
                    F[w] = __viaddmin_u16x2(xl, Cu1, A[w]);
                    Gd[w] = __viaddmin_u16x2(xr, Cd1, A[w]);
                }
#pragma unroll
                for (int mw = 1; mw < KW; mw <<= 1) {
#pragma unroll
                    for (int w = KW - 1; w >= mw; --w)
                        F[w] = __viaddmin_u16x2(F[w - mw], Cu1 * (2 * mw), F[w]);
#pragma unroll
                    for (int w = 0; w + mw < KW; ++w)
                        Gd[w] = __viaddmin_u16x2(Gd[w + mw], Cd1 * (2 * mw), Gd[w]);
                }
                // across the lanes: F at the last label below this lane, G at the first label
                // above it (scans of the lanes' end values, K labels per lane step)
                int xf = __shfl_up_sync(kFull, (int)(F[KW - 1] >> 16), 1, kG);
                int xg = __shfl_down_sync(kFull, (int)(Gd[0] & 0xFFFFu), 1, kG);
                if (gl == 0) xf = (int)kInf16;
                if (gl == kG - 1) xg = (int)kInf16;
                const int su = (int)Pu * K, sd = (int)Pd * K;
#pragma unroll
                for (int o = 1; o < kG; o <<= 1) {
                    const int vf = __shfl_up_sync(kFull, xf, o, kG);
                    const int vg = __shfl_down_sync(kFull, xg, o, kG);
                    if (gl >= o) xf = min(xf, vf + su * o);
                    if (gl + o < kG) xg = min(xg, vg + sd * o);
                }
                const uint32_t xfp = (uint32_t)xf * 0x10001u, xgp = (uint32_t)xg * 0x10001u;
#pragma unroll
                for (int w = 0; w < KW; ++w) {
                    // distances from the label below the lane (2w+1, 2w+2) and to the label
                    // above it (K-2w, K-2w-1)
                    const uint32_t du = (2u * w + 1) | ((2u * w + 2) << 16);
                    const uint32_t dd = (uint32_t)(K - 2 * w) | ((uint32_t)(K - 2 * w - 1) << 16);
                    F[w] = __viaddmin_u16x2(xfp, Pu * du, F[w]);
                    Gd[w] = __viaddmin_u16x2(xgp, Pd * dd, Gd[w]);
                    Mv[w] = __vminu2(__vminu2(F[w], Gd[w]), cap);
                    if (asym) Mv[w] = __viaddmin_u16x2(SA[w], Tx2, Mv[w]);
                }
                if (moved) {   // re-index the envelope
                    const int base = lane & ~(kG - 1);
                    const int ftop = __shfl_sync(kFull, (int)(F[KW - 1] >> 16), base + kG - 1);
                    const int gbot = __shfl_sync(kFull, (int)(Gd[0] & 0xFFFFu), base);
                    uint32_t *gw = (uint32_t *)(gb + PAD + gl * K);
#pragma unroll
                    for (int i = 0; i < KW; ++i) gw[i] = Mv[i];
                    __syncwarp();
                    const int s2 = min(max(s, -DWP), DWP);
                    const int j1 = PAD + gl * K + s2;
                    const uint32_t *mwords = (const uint32_t *)gb + (j1 >> 1);
                    const uint32_t sel = (j1 & 1) ? 0x5432u : 0x3210u;
                    uint32_t Wd[KW + 1];
#pragma unroll
                    for (int i = 0; i <= KW; ++i) Wd[i] = mwords[i];
#pragma unroll
                    for (int i = 0; i < KW; ++i) Mv[i] = __byte_perm(Wd[i], Wd[i + 1], sel);
                    __syncwarp();
                    // labels outside the predecessor's window: F continued above its top
                    // label, G below its first, each capped
                    const int q0 = gl * K + s;
                    if (q0 < 0 || q0 + K > DWP) {
                        const int m2s = (int)(m2 & 0xFFFFu);
                        const int capu = m2s + (int)(T * up), capd = m2s + (int)T;
#pragma unroll
                        for (int i = 0; i < KW; ++i) {
                            uint32_t h2[2] = {Mv[i] & 0xFFFFu, Mv[i] >> 16};
#pragma unroll
                            for (int h = 0; h < 2; ++h) {
                                const int q = q0 + 2 * i + h;
                                if (q >= DWP)
                                    h2[h] = (uint32_t)min(ftop + (int)Pu * (q - DWP + 1), capu);
                                else if (q < 0)
                                    h2[h] = (uint32_t)min(gbot + (int)Pd * (-q), capd);
                            }
                            Mv[i] = h2[0] | (h2[1] << 16);
                        }
                    }
                }
#pragma unroll
                for (int i = 0; i < KW; ++i) {
                    uint32_t L = c[i] + Mv[i] - m2;      // per half: no carry, no borrow
                    if (padded) {
                        L &= keep[i];
                        A[i] = L | (INF2 & ~keep[i]);
                    } else {
                        A[i] = L;
                    }
                    c[i] = L;
                }
            }
            if (act && !OUTN) {
                if (KW % 2 == 0) {
                    unsigned long long *sp = (unsigned long long *)(sbase + (int64_t)pix * DWP);
#pragma unroll
                    for (int j = 0; j < KW / 2; ++j)
                        atomicAdd(sp + j, ((unsigned long long)c[2 * j + 1] << 32) | c[2 * j]);
                } else {
                    unsigned int *sp = (unsigned int *)(sbase + (int64_t)pix * DWP);
#pragma unroll
                    for (int j = 0; j < KW; ++j) atomicAdd(sp + j, c[j]);
                }
            }
            prev_lo = cur_lo;
            prev_i = cur_i;
        }
    }
    if (OUTN) {   // the last pixel of the longest paths: nothing follows to store it
        uint32_t m2 = A[0];
#pragma unroll
        for (int i = 1; i < KW; ++i) m2 = __vminu2(m2, A[i]);
        m2 = __vminu2(m2, __byte_perm(m2, m2, 0x1032));
#pragma unroll
        for (int o = 1; o < kG; o <<= 1) m2 = __vminu2(m2, __shfl_xor_sync(kFull, m2, o));
        if (n > 0 && n == nmax)
            store_normalised<KW>(outv + (int64_t)(pix0 + (n - 1) * dpix) * DWP + gl * K, A, m2,
                                 keep, padded);
    }
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
        if (t < n) {
            const int64_t pix = pix0 + t * dpix;
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
                const int P = (m.lut && act) ? min(m.lut[abs(cur_i - prev_i) & 0xFF], T) : a.p1;
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
