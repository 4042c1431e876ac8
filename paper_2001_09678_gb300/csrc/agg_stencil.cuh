// agg_stencil.cuh -- the packed-stencil directional passes (see aggregate.cu), as a device
// function of (block index, thread index) shared by the stand-alone kernel and the batch
// scheduler's persistent kernel.  NW: warps of the block that runs it.
#pragma once
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

constexpr int kStencilWarps = 4;            // warps per block of the stand-alone kernel
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
// Shared memory of one block of agg_stencil_body: the re-indexing buffers (rbuf; sbuf for
// the doubled pass of a layer), the gradient table (slut) and the path minima (redbuf).
template <int G, int KW, int RM, bool WIN, bool LAYER, bool SWP, int NW>
struct StencilSmem {
    static constexpr int kPathsPerWarp = 32 / G;
    static constexpr int HW = RM / 2;
    static constexpr int DWP = G * 2 * KW;
    static constexpr int PAD = (DWP + 4 * HW + 2 + 7) / 8 * 8;
    static constexpr int BUF = 2 * PAD + DWP;
    static constexpr int nr = WIN ? NW * kPathsPerWarp * BUF : 8;              // uint16
    static constexpr int ns = WIN && LAYER && !SWP ? NW * kPathsPerWarp * BUF : 8;
    static constexpr int nl = SWP ? 256 : 1;                                   // int
    static constexpr int nm = 2 * NW * 32;                                     // uint32
    // byte offsets in one 16-byte aligned block
    static constexpr size_t off_s = (2 * (size_t)nr + 15) / 16 * 16;
    static constexpr size_t off_l = off_s + (2 * (size_t)ns + 15) / 16 * 16;
    static constexpr size_t off_m = off_l + (4 * (size_t)nl + 15) / 16 * 16;
    static constexpr size_t bytes = off_m + 4 * (size_t)nm;
};

template <int G, int KW, int RM, bool WIN, bool BLK, bool LAYER, bool SWP, bool XM, int NW>
__device__ __forceinline__ void agg_stencil_body(const LevelArgs &a, const MergeArgs &mg, int bx,
                                                 int by, int bz, int tid, unsigned char *smem)
{
    using SM = StencilSmem<G, KW, RM, WIN, LAYER, SWP, NW>;
    constexpr int kG = G;                    // lanes per scan path
    constexpr int kPathsPerWarp = 32 / kG;
    constexpr int HW = RM / 2;               // halo words per side
    constexpr int NE = KW + 2 * HW;          // words with halos
    constexpr int K = 2 * KW;                // labels per lane
    constexpr int DWP = kG * K;              // labels per path (= the volume stride)
    constexpr int PAD = SM::PAD;             // absent labels around a path
    constexpr int BUF = SM::BUF;
    // prefetch distance (steps), measured: 10 for the summed pass with two words per lane
    // (8 lanes on 32 labels; 8, 12 and 16 slower), 8 for the other shapes and for the layer
    // and sweep modes (each slower at 12), 4 for the widest lanes
    constexpr int PF = KW > 4 ? 4 : (KW == 2 && !LAYER && !SWP ? 10 : 8);
    constexpr int CW = KW >= 2 ? KW / 2 : 1; // 32-bit words of cost bytes per lane
    static_assert(kG == 4 || kG == 8, "paths of 4 or 8 lanes");

    uint16_t *rbuf = (uint16_t *)smem;
    // suffix minima of the predecessor for the doubled pass: lower pad = the path's
    // minimum (every predecessor label lies above), upper pad absent
    uint16_t *sbuf = (uint16_t *)(smem + SM::off_s);
    int *slut = (int *)(smem + SM::off_l);   // the gradient table's slopes
    uint32_t *redbuf = (uint32_t *)(smem + SM::off_m);   // path minima
    if (SWP) {
        for (int i = tid; i < 256; i += (NW * 32)) slut[i] = mg.lut[i];
        __syncthreads();
    }

    const int view = bz, dir = mg.dir0 + by;
    // layered merge: the previous layer's pair (IN) and this pass's own volume (OUTN)
    const uint16_t *qa = view ? mg.qa[1] : mg.qa[0];
    const uint16_t *qb = view ? mg.qb[1] : mg.qb[0];
    uint16_t *const *outs = view ? mg.out[1] : mg.out[0];
    uint16_t *const outv = (dir & 1) ? outs[1] : outs[0];
    const int dx = c_dirs[dir][0], dy = c_dirs[dir][1];
    const int W = a.W, H = a.H, Dw = a.Dw;
    const int lane = tid & 31, warp = tid >> 5;
    const int gl = lane & (kG - 1), grp = lane / kG;
    const int path = (bx * NW + warp) * kPathsPerWarp + grp;
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
    auto issue = [&](int t, int slot, bool guard) {
        const int pix = pix0 + t * dpix;
        if ((!guard || t < n) && MPV_IN(a.err, pix >= 0 && pix < W * H, 1) &&
            MPV_IN(a.err, !SWP || (ipix0 + t * dipix >= 0 &&
                                   ipix0 + t * dipix < (int64_t)V.pitch0 * H), 2)) {
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
    for (int u = 0; u < PF; ++u) issue(u, u, true);

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

    // One step of the scan (step t, ring slot u = t mod PF).  GUARD: a path of the warp may
    // end within the next PF steps, so the step and its load are checked per lane; before
    // that (t + PF below the warp's shortest path) every lane is active and every next load
    // lies on its path, and the chunks run as straight-line code without the checks.
    auto step = [&](const int u, const int t, const bool GUARD) {
        const bool act = !GUARD || t < n;
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
        issue(t + PF, u, GUARD);

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
            uint32_t *rw = redbuf + ((t & 1) * NW + warp) * 32;
            rw[lane] = lm;
            __syncwarp();
            const uint4 *g4 = (const uint4 *)(rw + grp * kG);
            const uint4 q0 = g4[0];
            const uint4 q1 = g4[1];
            // 3-input packed minima: two dependent levels instead of three
            const uint32_t r0 = __vimin3_u16x2(q0.x, q0.y, q0.z);
            const uint32_t r1 = __vimin3_u16x2(q0.w, q1.x, q1.y);
            m2 = __vimin3_u16x2(r0, r1, __vminu2(q1.z, q1.w));
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
                const bool wok = MPV_IN(a.err, j0 >= 0 && (j0 >> 1) + NE < BUF / 2, 3);
#pragma unroll
                for (int i = 0; i <= NE; ++i) Wd[i] = wok ? gwords[i] : INF2;
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
                    const bool sok = MPV_IN(a.err, j1 >= 0 && (j1 >> 1) + KW < BUF / 2, 4);
#pragma unroll
                    for (int i = 0; i <= KW; ++i) Sd[i] = sok ? swords[i] : INF2;
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
                // words below e hold smaller labels: jumps up into (u, u+1); the cap
                // (which waits for the path minimum) enters last
                uint32_t m;
                if constexpr (!LAYER) {
                    // equal slopes both ways: the two neighbours d labels away share
                    // their penalty, min(A(u-d), A(u+d)) + eps(d) (no half reaches 2^16)
                    m = __viaddmin_u16x2(__vminu2(SH[e - 1], SH[e]), E1, E[e]);
                    m = __viaddmin_u16x2(__vminu2(E[e - 1], E[e + 1]), E2, m);
                    if (RM >= 4) {
                        m = __viaddmin_u16x2(__vminu2(SH[e - 2], SH[e + 1]), E3, m);
                        m = __viaddmin_u16x2(__vminu2(E[e - 2], E[e + 2]), E4, m);
                    }
                } else {
                    m = __viaddmin_u16x2(SH[e - 1], U1, E[e]);
                    m = __viaddmin_u16x2(SH[e], E1, m);
                    m = __viaddmin_u16x2(E[e - 1], U2, m);
                    m = __viaddmin_u16x2(E[e + 1], E2, m);
                    if (RM >= 4) {
                        m = __viaddmin_u16x2(SH[e - 2], U3, m);
                        m = __viaddmin_u16x2(SH[e + 1], E3, m);
                        m = __viaddmin_u16x2(E[e - 2], U4, m);
                        m = __viaddmin_u16x2(E[e + 2], E4, m);
                    }
                }
                if (asym) m = __viaddmin_u16x2(SA[i], Tx2, m);
                m = __vminu2(m, cap);
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
                (act && t > 0 && MPV_IN(a.err, cur_i >= 0 && cur_i < 256 && prev_i >= 0 &&
                                                    prev_i < 256, 6))
                    ? min((uint32_t)slut[abs(cur_i - prev_i) & 0xFF], T)
                    : P1;
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
                const bool mok = MPV_IN(a.err, j1 >= 0 && (j1 >> 1) + KW < BUF / 2, 5);
#pragma unroll
                for (int i = 0; i <= KW; ++i) Wd[i] = mok ? mwords[i] : INF2;
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
        if (act && !OUTN && MPV_IN(a.err, pix >= 0 && pix < W * H, 7)) {
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
    };
    const int nmin = __reduce_min_sync(kFull, n);
    const int T1 = nmin >= 2 * PF ? (nmin - PF) / PF * PF : 0;
    for (int t0 = 0; t0 < T1; t0 += PF) {
#pragma unroll
        for (int u = 0; u < PF; ++u) step(u, t0 + u, false);
    }
    for (int t0 = T1; t0 < nmax; t0 += PF) {
#pragma unroll
        for (int u = 0; u < PF; ++u) {
            if (t0 + u >= nmax) break;
            step(u, t0 + u, true);
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

// ---------------------------------------------------------------------------------
// agg_row_body: the summed pass along image rows (directions (1,0) and (-1,0)), 8 lanes of
// two packed words per path, radius 2, no padding labels.  Every path of these directions
// has exactly W steps, and the cost, window-start and reduction addresses of a prefetch
// chunk's steps are one chunk pointer plus constant offsets (fewer instructions per step
// than agg_stencil_body's computed addresses).  The arithmetic is agg_stencil_body's
// (summed pass, path minimum through shared memory, neighbour terms paired), so the
// results are the same bit for bit.  The rows are the longest scan chains of a level (W
// steps); on small levels, where the whole launch is resident at once, their per-step
// latency sets the launch's time.  Lanes of rows past the image read the last row and add
// nothing.
// ---------------------------------------------------------------------------------
template <int DX, bool WIN, int NW>
__device__ __forceinline__ void agg_row_body(const LevelArgs &a, int bx, int view, int tid,
                                             unsigned char *smem)
{
    using SM = StencilSmem<8, 2, 2, WIN, false, false, NW>;
    constexpr int kG = 8, KW = 2, K = 4, DWP = 32, PPW = 4, NE = KW + 2, PF = 12;
    constexpr int PAD = SM::PAD, BUF = SM::BUF;
    const int lane = tid & 31, warp = tid >> 5;
    const int gl = lane & (kG - 1), grp = lane / kG;
    const int W = a.W, H = a.H;
    const int path0 = (bx * NW + warp) * PPW;
    if (path0 >= H) return;   // (warp-uniform)
    const bool valid = path0 + grp < H;
    const int y = valid ? path0 + grp : H - 1;
    const ViewLevel &V = a.v[view];
    const int64_t pix0 = (int64_t)y * W + (DX > 0 ? 0 : W - 1);
    const uint8_t *cp = V.C + pix0 * DWP + gl * K;
    uint16_t *sp = V.S + pix0 * DWP + gl * K;
    const uint16_t *lp = WIN ? V.lo + pix0 : nullptr;
    uint16_t *gb = (uint16_t *)smem + (WIN ? (warp * PPW + grp) * BUF : 0);
    uint32_t *redbuf = (uint32_t *)(smem + SM::off_m);
    if (WIN) {
        for (int i = gl; i < BUF; i += kG) gb[i] = (uint16_t)kInf16;
        __syncwarp();
    }
    const uint32_t INF2 = kInf16 * 0x10001u;
    const uint32_t T = (uint32_t)a.trunc, P1 = (uint32_t)a.p1;
    const uint32_t Tx2 = T * 0x10001u;
    const uint32_t E1 = min(P1, T) * 0x10001u, E2 = min(2 * P1, T) * 0x10001u;

    // prefetch ring: cost bytes and window start of the next PF steps
    uint32_t cq[PF], lq[PF];
#pragma unroll
    for (int u = 0; u < PF; ++u) {
        lq[u] = 0u;
        if (u < W) {
            cq[u] = ld_pin_u32(cp + u * DX * DWP);
            if (WIN) lq[u] = ld_pin_u16(lp + u * DX);
        }
    }
    uint32_t A[KW];
#pragma unroll
    for (int i = 0; i < KW; ++i) A[i] = INF2;   // no predecessor: L = C at the first pixel
    int prev_lo = WIN ? (int)lq[0] : 0;         // (no shift at the first pixel)

    // step t = t0 + u of the chunk at cpt/spt/lpt (the pixel of step t0); pre: the slot's
    // next load (step t + PF) lies inside the row
    auto step = [&](const int u, const bool pre, const uint8_t *cpt, uint16_t *spt,
                    const uint16_t *lpt) {
        uint32_t c[KW];
        c[0] = __byte_perm(cq[u], 0u, 0x4140);
        c[1] = __byte_perm(cq[u], 0u, 0x4342);
        const int cur_lo = WIN ? (int)lq[u] : 0;
        if (pre) {
            cq[u] = ld_pin_u32(cpt + (u + PF) * DX * DWP);
            if (WIN) lq[u] = ld_pin_u16(lpt + (u + PF) * DX);
        }
        const int s = WIN ? cur_lo - prev_lo : 0;
        const bool moved = WIN && __any_sync(kFull, s != 0);

        // the path's minimum: the lanes' minima through shared memory (double-buffered by
        // step parity; PF is even, so the parity of t is that of u)
        uint32_t m2 = __vminu2(A[0], A[1]);
        m2 = __vminu2(m2, __byte_perm(m2, m2, 0x1032));
        {
            uint32_t *rw = redbuf + ((u & 1) * NW + warp) * 32;
            rw[lane] = m2;
            __syncwarp();
            const uint4 *g4 = (const uint4 *)(rw + grp * kG);
            const uint4 q0 = g4[0];
            const uint4 q1 = g4[1];
            const uint32_t r0 = __vimin3_u16x2(q0.x, q0.y, q0.z);
            const uint32_t r1 = __vimin3_u16x2(q0.w, q1.x, q1.y);
            m2 = __vimin3_u16x2(r0, r1, __vminu2(q1.z, q1.w));
        }
        const uint32_t cap = m2 + Tx2;

        uint32_t E[NE];
        E[1] = A[0];
        E[2] = A[1];
        {
            const uint32_t l = __shfl_up_sync(kFull, A[KW - 1], 1, kG);
            const uint32_t r = __shfl_down_sync(kFull, A[0], 1, kG);
            E[0] = gl == 0 ? INF2 : l;
            E[NE - 1] = gl == kG - 1 ? INF2 : r;
        }
        if (WIN && moved) {   // re-index the predecessor into this pixel's window
            uint32_t *gw = (uint32_t *)(gb + PAD + gl * K);
            gw[0] = A[0];
            gw[1] = A[1];
            __syncwarp();
            const int sc = min(max(s, -(DWP + 2)), DWP + 2);
            const int j0 = PAD + gl * K - 2 + sc;
            const uint32_t *gwords = (const uint32_t *)gb + (j0 >> 1);
            const uint32_t sel = (j0 & 1) ? 0x5432u : 0x3210u;
            const bool wok = MPV_IN(a.err, j0 >= 0 && (j0 >> 1) + NE < BUF / 2, 3);
            uint32_t Wd[NE + 1];
#pragma unroll
            for (int i = 0; i <= NE; ++i) Wd[i] = wok ? gwords[i] : INF2;
#pragma unroll
            for (int w = 0; w < NE; ++w) E[w] = __byte_perm(Wd[w], Wd[w + 1], sel);
            __syncwarp();
        }
        uint32_t SH[NE - 1];
#pragma unroll
        for (int j = 0; j < NE - 1; ++j) SH[j] = shift1(E[j], E[j + 1]);
#pragma unroll
        for (int i = 0; i < KW; ++i) {
            const int e = 1 + i;
            uint32_t m = __viaddmin_u16x2(__vminu2(SH[e - 1], SH[e]), E1, E[e]);
            m = __viaddmin_u16x2(__vminu2(E[e - 1], E[e + 1]), E2, m);
            m = __vminu2(m, cap);
            const uint32_t L = c[i] + m - m2;   // per half: no carry, no borrow
            A[i] = L;
            c[i] = L;
        }
        if (valid) {
            unsigned long long *d = (unsigned long long *)(spt + u * DX * DWP);
            atomicAdd(d, ((unsigned long long)c[1] << 32) | c[0]);
        }
        prev_lo = cur_lo;
    };

    // whole chunks whose next loads stay inside the row, then the last one or two chunks
    const int T1 = W >= 2 * PF ? (W - PF) / PF * PF : 0;
    for (int t0 = 0; t0 < T1; t0 += PF) {
        const uint8_t *cpt = cp + (int64_t)t0 * DX * DWP;
        uint16_t *spt = sp + (int64_t)t0 * DX * DWP;
        const uint16_t *lpt = WIN ? lp + (int64_t)t0 * DX : nullptr;
#pragma unroll
        for (int u = 0; u < PF; ++u) step(u, true, cpt, spt, lpt);
    }
    for (int t0 = T1; t0 < W; t0 += PF) {
        const uint8_t *cpt = cp + (int64_t)t0 * DX * DWP;
        uint16_t *spt = sp + (int64_t)t0 * DX * DWP;
        const uint16_t *lpt = WIN ? lp + (int64_t)t0 * DX : nullptr;
#pragma unroll
        for (int u = 0; u < PF; ++u) {
            if (t0 + u >= W) break;
            step(u, t0 + u + PF < W, cpt, spt, lpt);
        }
    }
}

}  // namespace

}  // namespace mpv
