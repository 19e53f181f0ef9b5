// molt_strided_nb.cuh -- strided-axis powers D^p u (float32 sweeps) with one
// exchange per sweep between neighbouring segments (sm_103a).
//
// Layout as k_strided: lane = one of 32 neighbouring lines (every global
// access coalesced), warp = a segment of RPT consecutive points of those
// lines, the segments of a line over the warps of a CTA and the CTAs of a
// thread-block cluster.
//
// The operator (Sec. 2, the two recurrences of L^{-1} in the difference form
// of D): e = anti-causal(causal(q)) plus the boundary terms A d^j + B d^{n-1-j}.
// The causal and anti-causal recurrences decay by d = e^{-nu} per point, so a
// value RPT points away enters a segment's results multiplied by d^RPT.  When
// d^{RPT-1} <= 2^-30 (far below float32 rounding) every inflow a segment needs
// comes from its two neighbours alone:
//   * each segment runs both halves of its causal recurrence with zero inflow
//     and publishes four numbers: E = y0 at its last point, y0 at the one
//     before, and the zero-inflow anti-causal sums ER0 = sum_k d^k y0_k,
//     ER1 = sum_{k>=1} d^(k-1) y0_k;
//   * after ONE barrier it reads E, y0 of its left neighbour (its causal
//     inflow) and ER0, ER1 of its right neighbour, which with its own E give
//     the right neighbour's first two values e_{a+RPT}, e_{a+RPT+1} exactly to
//     the truncation (the right inflow is linear in E: ER = ER0 + G E);
//   * it corrects its causal values for the inflow (y_k += yin d^(k+1)), runs
//     the anti-causal recurrence from e_{a+RPT}, and forms the halos of the
//     next sweep (its left neighbour's last two e values follow from E, y0 and
//     its own first e value) without a second exchange.
// The Dirichlet coefficients reduce to A = -e_0 / (1 - mu^2) and
// B = -y_{n-1} / (1 - mu^2) (mu = d^{n-1} <= d^{2 RPT - 1} is negligible), so
// only the two end segments apply them; periodic images reduce to the wrapped
// neighbour.  The full-carry kernel (k_strided, three exchanges per sweep)
// serves every other decay.
#pragma once
#include "molt_regs.cuh"
#include "molt_tma.cuh"

namespace molt {

// Shared memory of one CTA: the exchange slots [2][S][4][32], then (STAGE
// != 0) the tile barrier and the tile: the pair level's rows a0-2 .. a0+S RPT+1
// of the CTA's 32 lines (STAGE & 1; nbox boxes of box_rows rows for hi and for
// lo), or only the output rows a0 .. a0+S RPT-1 (STAGE == 2).  STAGE & 2
// stages each output power in the tile and writes it with one tensor store.
__host__ __device__ inline size_t strided_nb_slot_bytes(int S) { return (size_t)2 * S * 4 * 32 * sizeof(float); }
__host__ __device__ inline size_t strided_nb_tile_off(int S) { return (strided_nb_slot_bytes(S) + 8 + 127) & ~(size_t)127; }
__host__ __device__ inline size_t strided_nb_smem(int S, int rpt = 0, int stage = 0, int nbox = 0, int box_rows = 0)
{
    if (stage == 0) return strided_nb_slot_bytes(S);
    const size_t out_rows = (size_t)S * rpt, in_rows = (stage & 1) ? (size_t)2 * nbox * box_rows : 0;
    return strided_nb_tile_off(S) + (in_rows > out_rows ? in_rows : out_rows) * 32 * sizeof(float);
}

// The exchange of one sweep between neighbouring segments of a line: each
// warp publishes its four numbers in slot buffer `buf` ([2][S][4][32] floats
// per CTA, a peer CTA's through distributed shared memory), one CTA or
// cluster barrier, then it reads its left neighbour's E, y0 and its right
// neighbour's ER0, ER1.  Sweeps alternate the buffer: a segment reads the
// numbers of sweep p before it reaches the barrier of sweep p + 1, so two
// buffers suffice.  Periodic lines wrap; Dirichlet ends have no neighbour.
template <int BC>
struct NbXch {
    float *slots;
    cg::cluster_group &cl;
    int S, K, w, lane, sl, sr, buf = 0;
    bool hasL, hasR;
    __device__ __forceinline__ NbXch(float *slots_, cg::cluster_group &cl_, int S_, int K_, int w_, int lane_, int seg, int Gd)
        : slots(slots_), cl(cl_), S(S_), K(K_), w(w_), lane(lane_), sl(seg - 1), sr(seg + 1)
    {
        if (BC == BC_PERIODIC) {
            if (sl < 0) sl = Gd - 1;
            if (sr >= Gd) sr = 0;
        }
        const bool full = seg < Gd;
        hasL = full && sl >= 0;
        hasR = full && sr < Gd;
    }
    __device__ __forceinline__ const float *slot(int sg) const
    {
        const float *p = slots + ((size_t)buf * S + sg % S) * 128;
        return K > 1 ? cl.map_shared_rank(p, sg / S) : p;
    }
    __device__ __forceinline__ void operator()(float E, float Y2, float ER0, float ER1, float &EL, float &Y2L, float &ER0R,
                               float &ER1R)
    {
        float *mine = slots + ((size_t)buf * S + w) * 128;
        mine[lane] = E;
        mine[32 + lane] = Y2;
        mine[64 + lane] = ER0;
        mine[96 + lane] = ER1;
        if (K > 1) cl.sync();
        else __syncthreads();
        if (hasL) {
            const float *q = slot(sl);
            EL = q[lane];
            Y2L = q[32 + lane];
        }
        if (hasR) {
            const float *q = slot(sr);
            ER0R = q[64 + lane];
            ER1R = q[96 + lane];
        }
    }
};

// One application of D on a segment with one neighbour exchange (the algebra
// above; the powers kernel below carries the same steps inline, where they
// compile to fewer registers).  MODE as seg_make_q: 0 z holds s (the first
// power: hl1 = s at a-1, hr0 = s at a+RPT), 1 s = second difference of z, 2
// the same plus cu r; 3 z holds q itself (the solve alone: the transposed
// operator).
// hl2, hl1, hr0, hr1: z at a-2, a-1, a+RPT, a+RPT+1 on entry, e there on exit.
// xch(E, Y2, ER0, ER1, EL, Y2L, ER0R, ER1R) publishes this segment's four
// numbers, waits for the neighbours' and returns theirs (zeros where there is
// no neighbour).
template <int BC, int RPT, int MODE, class RF, class XCH>
__device__ __forceinline__ void strided_sweep_nb(float (&z)[RPT], RF r, float cu, const AxisDev &A, const NbConsts &nc,
                                                 bool full, bool left_end, bool right_end, bool hasL, bool hasR,
                                                 XCH &&xch, float &hl2, float &hl1, float &hr0, float &hr1)
{
    constexpr int H = RPT / 2;
    const float d = A.fd, c1 = A.fc1, c2 = A.fc2, inv = A.finv;
    if constexpr (MODE != 3) {
        float zl2 = hl2, zl1 = hl1, zr0 = hr0, zr1 = hr1;
        if (BC == BC_DIRICHLET) end_ghosts<float, RPT, MODE>(z, left_end, right_end, zl2, zl1, zr0, zr1);
        seg_make_q<float, RPT, MODE>(z, zl2, zl1, zr0, zr1, r, cu, c1, c2);
        if (BC == BC_DIRICHLET) end_zero<float, RPT>(z, left_end, right_end);
    }
    if (!full) {
#pragma unroll
        for (int k = 0; k < RPT; ++k) z[k] = 0.f;
    }

    // both halves of the causal recurrence with zero inflow; ERb and the
    // chain-A part of ER1 on the way
    float ya = z[0], yb = z[H], ra1 = 0.f, rb = yb, pw = 1.f;
#pragma unroll
    for (int k = 1; k < H; ++k) {
        ya = d * ya + z[k];
        yb = d * yb + z[H + k];
        z[k] = ya;
        z[H + k] = yb;
        const float pbk = pw * d;     // chain A weighs y_k by d^(k-1), chain B by d^k
        ra1 += pw * ya;
        rb += pbk * yb;
        pw = pbk;
    }
    const float E1 = ya;                                // zero-inflow y at H-1
    const float E = yb + E1 * nc.dH;                    // ... at RPT-1
    const float Y2 = z[RPT - 2] + E1 * nc.dH1;          // ... at RPT-2
    const float ER1 = ra1 + nc.dH1 * (rb + E1 * nc.GH);
    const float ER0 = z[0] + d * ER1;
    float EL = 0.f, Y2L = 0.f, ER0R = 0.f, ER1R = 0.f;
    xch(E, Y2, ER0, ER1, EL, Y2L, ER0R, ER1R);

    // true causal values: chain A from the left neighbour's y at a-1,
    // chain B from the corrected y at H-1
    const float cB = E1 + EL * nc.dH;
    float pk = d;
#pragma unroll
    for (int k = 0; k < H; ++k) {
        z[k] += EL * pk;
        z[H + k] += cB * pk;
        pk *= d;
    }
    const float ER2 = rb + cB * nc.GH;                  // sum_j d^j y_{H+j}
    const float eout = hasR ? ER0R + nc.G * E : 0.f;    // e at a+RPT
    const float er1 = hasR ? ER1R + nc.G1 * E : 0.f;    // e at a+RPT+1
    float acc = d * eout;
    if (right_end) acc -= z[RPT - 1] * inv;             // B' d^{n-1-j} through the inflow
    seg_bwd_scan2<float, RPT>(z, d, nc.dH, acc, ER2);
    if (left_end) seg_add_left2<float, RPT>(z, d, nc.dH, -z[0] * inv);

    // halos of the next sweep: e at a-1, a-2 from the left neighbour's
    // last causal values and this segment's first e; e at a+RPT, a+RPT+1
    hl1 = hasL ? EL + d * z[0] : 0.f;
    hl2 = hasL ? Y2L + d * hl1 : 0.f;
    hr0 = eout;
    hr1 = er1;
}

// KM: 0 = powers D^p u, p = 1..P, into pr.out[p-1] (r = second difference of
// the pair level u formed here).  Launch: grid (column groups, K), clusters
// of K CTAs along y, S warps per CTA, strided_nb_smem(S) bytes.
template <int BC, int RPT, int STAGE>
__global__ void __launch_bounds__(256, 2) k_strided_nb(AxisDev A, LineSet LS, ProgParams pr, NbConsts nc,
                                                      const __grid_constant__ TmaMaps tm)
{
    pdl_enter();
    static_assert(RPT % 2 == 0 && RPT >= 8, "segment length");
    constexpr int H = RPT / 2;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float *slots = reinterpret_cast<float *>(smem_raw);          // [2][S][4][32]
    cg::cluster_group cl = cg::this_cluster();
    const int S = LS.S, K = LS.K;
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int krank = K > 1 ? (int)cl.block_rank() : 0;
    const int n = A.n, Gd = n / RPT;
    const int seg = krank * S + w, a = seg * RPT;
    const bool full = seg < Gd;
    const float d = A.fd, c1 = A.fc1, c2 = A.fc2, inv = A.finv;

    const int64_t line = (int64_t)blockIdx.x * 32 + lane;
    const bool valid = line < LS.nlines;
    const bool io = valid && full;
    const int64_t lbase = valid ? (line % LS.inner) + (line / LS.inner) * LS.inner * (int64_t)n : 0;
    const int64_t st = LS.stride;

    // neighbouring segments: periodic lines wrap, Dirichlet ends have none
    int sl = seg - 1, sr = seg + 1;
    if (BC == BC_PERIODIC) {
        if (sl < 0) sl = Gd - 1;
        if (sr >= Gd) sr = 0;
    }
    const bool hasL = full && sl >= 0, hasR = full && sr < Gd;
    const bool left_end = BC == BC_DIRICHLET && seg == 0, right_end = BC == BC_DIRICHLET && seg == Gd - 1;
    auto slot = [&](int buf, int sg) -> const float * {
        const float *p = slots + ((size_t)buf * S + sg % S) * 128;
        return K > 1 ? cl.map_shared_rank(p, sg / S) : p;
    };

    // tile of the CTA's lines: 32 lines from column x0 of outer slice z0
    const int64_t line0 = (int64_t)blockIdx.x * 32;
    const int x0 = (int)(line0 % LS.inner), z0 = (int)(line0 / LS.inner);
    const int a0 = krank * S * RPT;
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem_raw + strided_nb_slot_bytes(S));
    float *tile = reinterpret_cast<float *>(smem_raw + strided_nb_tile_off(S));
    if constexpr (STAGE & 1) {
        if (threadIdx.x == 0) {
            mbar_init(bar, 1);
            mbar_expect_tx(bar, (uint32_t)(2 * tm.nbox * tm.box_rows * 32 * sizeof(float)));
            for (int b = 0; b < tm.nbox; ++b) {
                tma_load_3d(tile + (size_t)b * tm.box_rows * 32, &tm.in_hi, x0, a0 - 2 + b * tm.box_rows, z0, bar);
                tma_load_3d(tile + (size_t)(tm.nbox + b) * tm.box_rows * 32, &tm.in_lo, x0, a0 - 2 + b * tm.box_rows,
                            z0, bar);
            }
        }
        __syncthreads();                                   // the barrier is initialised before anyone waits on it
    }

    // r = accurate second difference of u along the line (Dirichlet end
    // nodes take the neighbouring interior centre)
    float z[RPT];
    float rl = 0.f, rr = 0.f;
    if constexpr (STAGE & 1) {
        mbar_wait_or_flag(bar, 0);
        // tile row of line point j: j - (a0 - 2); rows outside the line came
        // in as zeros: periodic lines take their wrapped rows from global
        // memory, Dirichlet ends replace the values that used them
        const float *Th = tile + (size_t)(w * RPT) * 32 + lane;
        const float *Tl = tile + (size_t)(tm.nbox * tm.box_rows + w * RPT) * 32 + lane;
        float hm = Th[0], lm = Tl[0], h0 = Th[32], l0 = Tl[32];
        if (BC == BC_PERIODIC && io && seg == 0) {
            const float *Hp = (const float *)pr.u_hi + lbase, *Lp = (const float *)pr.u_lo + lbase;
            hm = Hp[(int64_t)(n - 2) * st];
            lm = Lp[(int64_t)(n - 2) * st];
            h0 = Hp[(int64_t)(n - 1) * st];
            l0 = Lp[(int64_t)(n - 1) * st];
        }
#pragma unroll
        for (int k = 0; k <= RPT + 1; ++k) {
            float hp = Th[(k + 2) * 32], lp = Tl[(k + 2) * 32];
            if (BC == BC_PERIODIC && k >= RPT && io && seg == Gd - 1) {
                const float *Hp = (const float *)pr.u_hi + lbase, *Lp = (const float *)pr.u_lo + lbase;
                hp = Hp[(int64_t)(k - RPT) * st];
                lp = Lp[(int64_t)(k - RPT) * st];
            }
            const float v = sdiff_pair(hm, h0, hp, lm, l0, lp);   // centre a + k - 1
            if (k == 0) rl = v;
            else if (k == RPT + 1) rr = v;
            else z[k - 1] = v;
            hm = h0;
            h0 = hp;
            lm = l0;
            l0 = lp;
        }
        if (!io) {
#pragma unroll
            for (int k = 0; k < RPT; ++k) z[k] = 0.f;
        }
    } else {
        if (io) strided_r_pair<BC, RPT>(pr, lbase, st, a, n, z, rl, rr);
        else {
#pragma unroll
            for (int k = 0; k < RPT; ++k) z[k] = 0.f;
        }
    }
    if (BC == BC_DIRICHLET) {
        if (left_end) z[0] = z[1];
        if (right_end) z[RPT - 1] = z[RPT - 2];
    }
    float hl2 = 0.f, hl1 = rl, hr0 = rr, hr1 = 0.f;   // sweep 1 (z = s): s at a-1 and a+RPT

    for (int p = 1; p <= pr.P; ++p) {
        float zl2 = hl2, zl1 = hl1, zr0 = hr0, zr1 = hr1;
        if (p == 1) {
            if (BC == BC_DIRICHLET) end_ghosts<float, RPT, 0>(z, left_end, right_end, zl2, zl1, zr0, zr1);
            seg_make_q<float, RPT, 0>(z, zl2, zl1, zr0, zr1, [](int) { return 0.f; }, 0.f, c1, c2);
        } else {
            if (BC == BC_DIRICHLET) end_ghosts<float, RPT, 1>(z, left_end, right_end, zl2, zl1, zr0, zr1);
            seg_make_q<float, RPT, 1>(z, zl2, zl1, zr0, zr1, [](int) { return 0.f; }, 0.f, c1, c2);
        }
        if (BC == BC_DIRICHLET) end_zero<float, RPT>(z, left_end, right_end);
        if (!full) {
#pragma unroll
            for (int k = 0; k < RPT; ++k) z[k] = 0.f;
        }

        // both halves of the causal recurrence with zero inflow; ERb and the
        // chain-A part of ER1 on the way
        float ya = z[0], yb = z[H], ra1 = 0.f, rb = yb, pw = 1.f;
#pragma unroll
        for (int k = 1; k < H; ++k) {
            ya = d * ya + z[k];
            yb = d * yb + z[H + k];
            z[k] = ya;
            z[H + k] = yb;
            const float pbk = pw * d;     // chain A weighs y_k by d^(k-1), chain B by d^k
            ra1 += pw * ya;
            rb += pbk * yb;
            pw = pbk;
        }
        const float E1 = ya;                                // zero-inflow y at H-1
        const float E = yb + E1 * nc.dH;                    // ... at RPT-1
        const float Y2 = z[RPT - 2] + E1 * nc.dH1;          // ... at RPT-2
        const float ER1 = ra1 + nc.dH1 * (rb + E1 * nc.GH);
        const float ER0 = z[0] + d * ER1;

        float *mine = slots + ((size_t)(p & 1) * S + w) * 128;
        mine[lane] = E;
        mine[32 + lane] = Y2;
        mine[64 + lane] = ER0;
        mine[96 + lane] = ER1;
        if (K > 1) cl.sync();
        else __syncthreads();
        float EL = 0.f, Y2L = 0.f, ER0R = 0.f, ER1R = 0.f;
        if (hasL) {
            const float *q = slot(p & 1, sl);
            EL = q[lane];
            Y2L = q[32 + lane];
        }
        if (hasR) {
            const float *q = slot(p & 1, sr);
            ER0R = q[64 + lane];
            ER1R = q[96 + lane];
        }

        // true causal values: chain A from the left neighbour's y at a-1,
        // chain B from the corrected y at H-1
        const float cB = E1 + EL * nc.dH;
        float pk = d;
#pragma unroll
        for (int k = 0; k < H; ++k) {
            z[k] += EL * pk;
            z[H + k] += cB * pk;
            pk *= d;
        }
        const float ER2 = rb + cB * nc.GH;                  // sum_j d^j y_{H+j}
        const float eout = hasR ? ER0R + nc.G * E : 0.f;    // e at a+RPT
        const float er1 = hasR ? ER1R + nc.G1 * E : 0.f;    // e at a+RPT+1
        float acc = d * eout;
        if (right_end) acc -= z[RPT - 1] * inv;             // B' d^{n-1-j} through the inflow
        seg_bwd_scan2<float, RPT>(z, d, nc.dH, acc, ER2);
        if (left_end) seg_add_left2<float, RPT>(z, d, nc.dH, -z[0] * inv);

        // halos of the next sweep: e at a-1, a-2 from the left neighbour's
        // last causal values and this segment's first e; e at a+RPT, a+RPT+1
        hl1 = hasL ? EL + d * z[0] : 0.f;
        hl2 = hasL ? Y2L + d * hl1 : 0.f;
        hr0 = eout;
        hr1 = er1;

        float *o = reinterpret_cast<float *>(pr.out[p - 1]);
        if constexpr (STAGE & 2) {
            if (o != nullptr) {
                // the previous power's store has read the tile before it is
                // written again; then one tensor store per box
                if (threadIdx.x == 0) tma_store_wait_read();
                __syncthreads();
                float *T = tile + (size_t)(w * RPT) * 32 + lane;
#pragma unroll
                for (int k = 0; k < RPT; ++k) T[k * 32] = z[k];
                fence_proxy_async();
                __syncthreads();
                if (threadIdx.x == 0) {
                    const int orows = S * RPT, ob = orows > 256 ? 256 : orows;
                    for (int y = 0; y < orows; y += ob) tma_store_3d(&tm.out[p - 1], x0, a0 + y, z0, tile + (size_t)y * 32);
                    tma_store_commit();
                }
            }
        } else if (o != nullptr && io) {
            float *po = o + lbase + (int64_t)a * st;
#pragma unroll
            for (int k = 0; k < RPT; ++k) { *po = z[k]; po += st; }
        }
    }
    if constexpr (STAGE & 2) {
        if (threadIdx.x == 0) tma_store_wait_all();    // the tile outlives the stores that read it
    }
    // peers read this CTA's slots after the last exchange: no CTA of the
    // cluster exits before every one of them is past those reads
    if (K > 1) cl.sync();
}

// Shared memory of the Horner kernel: the exchange slots, r ([S][RPT][32]),
// then (GT) the tile barrier and the g tiles ([ng][tile_rows][32], rows
// a0-2 .. of the CTA's 32 lines, 128-byte aligned).
__host__ __device__ inline size_t strided_nb_h_bar_off(int S, int rpt)
{
    return strided_nb_slot_bytes(S) + (size_t)S * rpt * 32 * sizeof(float);
}
__host__ __device__ inline size_t strided_nb_h_smem(int S, int rpt, int ng, bool gt, int tile_rows = 0)
{
    return strided_nb_h_bar_off(S, rpt) + (gt ? 128 + (size_t)ng * tile_rows * 32 * sizeof(float) : 0);
}

// The Horner pass with several outputs (the 3D y pass, Sec. 4: the ADI
// factors of F grouped by the power of D_y):
//   out_o = sum_{t=0..P} D^t (sum_q coef[o][t][q] g_q + cu[o][t] u)
// evaluated as Horner in t, each application of D with one neighbour
// exchange; the u terms enter through r, the accurate second difference of
// the pair level u, formed once and kept in shared memory (the t = 0 term of
// u is left to the x pass).  GT: the CTA's rows of the g fields (two halo
// rows on each side) are copied into shared memory once by TMA tensor loads
// on an mbarrier, while r is formed, instead of read from global memory for
// every output and every power.  Launch as k_strided_nb, strided_nb_h_smem
// bytes.
template <int BC, int RPT, bool GT>
__global__ void __launch_bounds__(256, 2) k_strided_nb_h(AxisDev A, LineSet LS, ProgParams pr, NbConsts nc,
                                                        const __grid_constant__ TmaGMaps tg)
{
    pdl_enter();
    static_assert(RPT % 2 == 0 && RPT >= 8, "segment length");
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float *slots = reinterpret_cast<float *>(smem_raw);          // [2][S][4][32]
    cg::cluster_group cl = cg::this_cluster();
    const int S = LS.S, K = LS.K;
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int krank = K > 1 ? (int)cl.block_rank() : 0;
    const int n = A.n, Gd = n / RPT;
    const int seg = krank * S + w, a = seg * RPT;
    const bool full = seg < Gd;
    const int64_t line = (int64_t)blockIdx.x * 32 + lane;
    const bool valid = line < LS.nlines;
    const bool io = valid && full;
    const int64_t lbase = valid ? (line % LS.inner) + (line / LS.inner) * LS.inner * (int64_t)n : 0;
    const int64_t st = LS.stride;
    NbXch<BC> xch(slots, cl, S, K, w, lane, seg, Gd);
    const bool left_end = BC == BC_DIRICHLET && seg == 0, right_end = BC == BC_DIRICHLET && seg == Gd - 1;
    const int P = pr.P, ng = pr.ng;
    float *rs = reinterpret_cast<float *>(smem_raw + strided_nb_slot_bytes(S)) + (size_t)w * RPT * 32 + lane;
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem_raw + strided_nb_h_bar_off(S, RPT));
    float *gtile = reinterpret_cast<float *>(smem_raw + strided_nb_h_bar_off(S, RPT) + 128);
    const int trows = tg.nbox * tg.box_rows;

    if constexpr (GT) {
        // tile row j of field q is line point a0 - 2 + j of the CTA's 32
        // lines (column x0 of outer slice z0); rows outside the line come in
        // as zeros (periodic halos are read from global memory below,
        // Dirichlet end halos are replaced by the end ghosts)
        if (threadIdx.x == 0) {
            const int64_t line0 = (int64_t)blockIdx.x * 32;
            const int x0 = (int)(line0 % LS.inner), z0 = (int)(line0 / LS.inner);
            const int a0 = krank * S * RPT;
            mbar_init(bar, 1);
            mbar_expect_tx(bar, (uint32_t)(ng * trows * 32 * sizeof(float)));
            for (int q = 0; q < ng; ++q)
                for (int b = 0; b < tg.nbox; ++b)
                    tma_load_3d(gtile + ((size_t)q * trows + (size_t)b * tg.box_rows) * 32, &tg.g[q], x0,
                                a0 - 2 + b * tg.box_rows, z0, bar);
        }
        __syncthreads();                                   // the barrier is initialised before anyone waits on it
    }
    // r = accurate second difference of u along the line (Dirichlet end
    // nodes take the neighbouring interior centre)
    float z[RPT];
    float rl = 0.f, rr = 0.f;
    if (io) strided_r_pair<BC, RPT>(pr, lbase, st, a, n, z, rl, rr);
    else {
#pragma unroll
        for (int k = 0; k < RPT; ++k) z[k] = 0.f;
    }
    if (BC == BC_DIRICHLET) {
        if (left_end) z[0] = z[1];
        if (right_end) z[RPT - 1] = z[RPT - 2];
    }
#pragma unroll
    for (int k = 0; k < RPT; ++k) rs[k * 32] = z[k];
    if constexpr (GT) mbar_wait_or_flag(bar, 0);       // the g tiles have landed
    const auto rfun = [&](int k) { return k < 0 ? rl : (k >= RPT ? rr : rs[k * 32]); };

    for (int o = 0; o < pr.nout; ++o) {
#pragma unroll
        for (int k = 0; k < RPT; ++k) z[k] = 0.f;
        float hl2 = 0.f, hl1 = 0.f, hr0 = 0.f, hr1 = 0.f;   // z at a-2, a-1, a+RPT, a+RPT+1
        for (int t = P; t >= 0; --t) {
            const int cf = (o * (P + 1) + t) * ng;
            if (io) {
                for (int q = 0; q < ng; ++q) {
                    const float cq = pr.coef32[cf + q];
                    if (cq == 0.f) continue;
                    if constexpr (GT) {
                        const float *T = gtile + ((size_t)q * trows + w * RPT) * 32 + lane;   // row of a-2
                        float gl2 = T[0], gl1 = T[32], gr0 = T[(RPT + 2) * 32], gr1 = T[(RPT + 3) * 32];
                        if (BC == BC_PERIODIC && (seg == 0 || seg == Gd - 1)) {
                            const float *G = reinterpret_cast<const float *>(pr.g[q]) + lbase;
                            if (seg == 0) {
                                gl2 = G[(int64_t)(n - 2) * st];
                                gl1 = G[(int64_t)(n - 1) * st];
                            }
                            if (seg == Gd - 1) {
                                gr0 = G[0];
                                gr1 = G[st];
                            }
                        }
                        hl2 += cq * gl2;
                        hl1 += cq * gl1;
#pragma unroll
                        for (int k = 0; k < RPT; ++k) z[k] += cq * T[(k + 2) * 32];
                        hr0 += cq * gr0;
                        hr1 += cq * gr1;
                    } else {
                        const float *G = reinterpret_cast<const float *>(pr.g[q]) + lbase;
                        hl2 += cq * G[wrap_or_clamp<BC>(a - 2, n) * st];
                        hl1 += cq * G[wrap_or_clamp<BC>(a - 1, n) * st];
                        const float *pg = G + (int64_t)a * st;
#pragma unroll
                        for (int k = 0; k < RPT; ++k) { z[k] += cq * *pg; pg += st; }
                        hr0 += cq * G[wrap_or_clamp<BC>(a + RPT, n) * st];
                        hr1 += cq * G[wrap_or_clamp<BC>(a + RPT + 1, n) * st];
                    }
                }
            }
            if (t == 0) break;
            xch.buf ^= 1;
            strided_sweep_nb<BC, RPT, 2>(z, rfun, pr.cu32[o * (P + 1) + t], A, nc, full, left_end, right_end, xch.hasL,
                                         xch.hasR, xch, hl2, hl1, hr0, hr1);
        }
        float *ob = reinterpret_cast<float *>(pr.out[o]);
        if (io) {
            float *po = ob + lbase + (int64_t)a * st;
#pragma unroll
            for (int k = 0; k < RPT; ++k) { *po = z[k]; po += st; }
        }
    }
    if (K > 1) cl.sync();       // peers may still read this CTA's slots
}

// Powers of the transposed operator, (D^T)^p u for p = 1..P (Dirichlet lines,
// the adjoint step's y pass), with one neighbour exchange per sweep: D^T w =
// Delta^T C^T S w (post_T), where S, the solve of the difference form, is
// the same recurrence pair with its Dirichlet terms (strided_sweep_nb, MODE 3,
// on w with its end values dropped) and the halos of e that post_T needs are
// the exchange's.  u = the level's pair summed.  Launch as k_strided_nb.
template <int RPT>
__global__ void __launch_bounds__(256, 2) k_strided_nb_T(AxisDev A, LineSet LS, ProgParams pr, NbConsts nc)
{
    static_assert(RPT % 2 == 0 && RPT >= 8, "segment length");
    pdl_enter();
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float *slots = reinterpret_cast<float *>(smem_raw);          // [2][S][4][32]
    cg::cluster_group cl = cg::this_cluster();
    const int S = LS.S, K = LS.K;
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int krank = K > 1 ? (int)cl.block_rank() : 0;
    const int n = A.n, Gd = n / RPT;
    const int seg = krank * S + w, a = seg * RPT;
    const bool full = seg < Gd;
    const int64_t line = (int64_t)blockIdx.x * 32 + lane;
    const bool valid = line < LS.nlines;
    const bool io = valid && full;
    const int64_t lbase = valid ? (line % LS.inner) + (line / LS.inner) * LS.inner * (int64_t)n : 0;
    const int64_t st = LS.stride;
    NbXch<BC_DIRICHLET> xch(slots, cl, S, K, w, lane, seg, Gd);
    const bool left_end = seg == 0, right_end = seg == Gd - 1;
    const float c1 = A.fc1, c2 = A.fc2;

    float z[RPT];
    {
        const float *H = reinterpret_cast<const float *>(pr.u_hi) + lbase;
        const float *L = reinterpret_cast<const float *>(pr.u_lo) + lbase;
#pragma unroll
        for (int k = 0; k < RPT; ++k) z[k] = io ? H[(int64_t)(a + k) * st] + L[(int64_t)(a + k) * st] : 0.f;
    }
    const auto no_r = [](int) { return 0.f; };
    const int kl = n - 1 - a;
    for (int p = 1; p <= pr.P; ++p) {
        // interior rows only, the solve with one exchange, interior rows only
#pragma unroll
        for (int k = 0; k < RPT; ++k) z[k] = (k < kl && (seg > 0 || k > 0)) ? z[k] : 0.f;
        float hl2 = 0.f, hl1 = 0.f, hr0 = 0.f, hr1 = 0.f;
        xch.buf = p & 1;
        strided_sweep_nb<BC_DIRICHLET, RPT, 3>(z, no_r, 0.f, A, nc, full, left_end, right_end, xch.hasL, xch.hasR,
                                               xch, hl2, hl1, hr0, hr1);
#pragma unroll
        for (int k = 0; k < RPT; ++k) z[k] = (k < kl && (seg > 0 || k > 0)) ? z[k] : 0.f;
        if (left_end || right_end) post_T<float, RPT, true>(z, hl2, hl1, hr0, hr1, c1, c2, a, n);
        else post_T<float, RPT, false>(z, hl2, hl1, hr0, hr1, c1, c2, a, n);
        float *o = reinterpret_cast<float *>(pr.out[p - 1]);
        if (o != nullptr && io) {
            float *po = o + lbase + (int64_t)a * st;
#pragma unroll
            for (int k = 0; k < RPT; ++k) { *po = z[k]; po += st; }
        }
    }
    if (K > 1) cl.sync();       // peers may still read this CTA's slots
}

}  // namespace molt
