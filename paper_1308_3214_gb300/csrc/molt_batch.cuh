// molt_batch.cuh -- many independent 2D Dirichlet problems of uneven size in
// one launch per pass.
//
// A step of problem i is the 2D pass plan of Sec. 4 (eq. Full_2D expanded in
// the per-axis D_gamma): a y pass forming g_k = D_y^{k+1} u (k < P_i), then an
// x pass evaluating F = sum_t D_x^t (f_t0 u + sum_k f_t,k+1 g_k) by Horner's
// rule with the level combination u^{n+1} = ea u^n + eb u^{n-1} + ec F fused
// in (eq. update_P).  Each pass runs every problem in a few launches over
// flat work lists:
//
//  * x pass: one warp per row; the rows of all problems form the list (the
//    problem of a row is looked up, its constants copied to shared memory).
//    A lane owns a segment of RPT_i points, RPT_i the smallest of 4..32 with
//    32 RPT_i >= nx_i, so short rows keep most lanes busy; the row's input
//    fields are copied once into shared memory with cp.async.
//  * y pass: a cluster of K_i CTAs of kBatchYSeg warps per group of 32
//    neighbouring columns (lane = column, warp = segment of RPT_i rows,
//    kBatchYSeg K_i RPT_i >= ny_i), one launch per cluster size; carries cross
//    the segments through shared and distributed shared memory, or one
//    neighbour exchange per sweep where that is exact (batch_cols_nb).
//
// Line lengths are arbitrary: the segment routines' RAG variants handle the
// last point anywhere in a segment.  Fields live in an internal layout whose
// rows are padded to a multiple of 4 points (16-byte aligned vectors); the
// padding carries zeros and is never read as data.
#pragma once
#include "molt_regs.cuh"
#include "molt_recv.cuh"

namespace molt {

constexpr int BMAXP = 5;            // highest P of a batched problem
constexpr int kBatchYSeg = 4;       // y pass: warps (segments) per CTA; a column group takes a
                                    // cluster of ky such CTAs
constexpr int kBatchDpowPad = 64;   // table entries past d^n (read, multiplied by zero, by the exchange)
constexpr int kBatchMaxN = 1024;    // longest line of a batched problem

struct BatchProb {
    AxisDev ax, ay;                  // per-axis constants (dm[] for rpt_x / rpt_y)
    long long off;                   // first element in the internal layout (multiple of 64)
    int pitch;                       // row pitch of the internal layout (multiple of 4, >= nx)
    int P;
    int rpt_x, rpt_y;                // segment lengths of the x and y passes
    int row0;                        // first global row of the problem in the x-pass list
    int pad_;
    double cu[BMAXP + 1];            // x Horner weights of u, t = 0..P
    double coef[BMAXP + 1][BMAXP];   // x Horner weights of g_k, t = 0..P, k < P
    float cu32[BMAXP + 1];           // float32 copies (batch_mirror)
    float coef32[BMAXP + 1][BMAXP];
    // y pass with one neighbour exchange per sweep (float32; batch_cols_nb):
    // ynb = 1 where exact to rounding; the constants of rpt_y and of the
    // ragged last segment (its last point at kl = (ny - 1) mod rpt_y)
    NbConsts nby;
    float nbGL, nbG1L;               // sum_{k<=kl} d^(2k+1), sum_{1<=k<=kl} d^(2k)
    float nbdk, nbdk1, nbdkp;        // d^kl, d^(kl-1) (0 when kl = 0), d^(kl+1)
    int ynb;
    int ky;                          // y pass: CTAs (of kBatchYSeg warps) per column group

    template <class T> __device__ T ccu(int t) const
    {
        if constexpr (sizeof(T) == 4) return cu32[t];
        else return cu[t];
    }
    template <class T> __device__ T ccoef(int t, int k) const
    {
        if constexpr (sizeof(T) == 4) return coef32[t][k];
        else return coef[t][k];
    }
};

// fills a problem's float32 copies (after any change to its constants)
inline void batch_mirror(BatchProb &pb)
{
    axis_mirror(pb.ax);
    axis_mirror(pb.ay);
    for (int t = 0; t <= BMAXP; ++t) {
        pb.cu32[t] = (float)pb.cu[t];
        for (int k = 0; k < BMAXP; ++k) pb.coef32[t][k] = (float)pb.coef[t][k];
    }
}
static_assert(sizeof(BatchProb) % 16 == 0, "BatchProb is copied in 8-byte words into 16-byte aligned slots");

struct BatchPass {
    const BatchProb *probs;
    const int *row_prob;     // x pass: problem of every global row
    const int2 *items;       // y pass: (problem, first column)
    int row_begin;           // x pass: first row of the list
    int nitems;              // x pass: end of the rows; y pass: column groups
    ProgParams pr;           // levels, ea / eb / ec, g[k] planes (internal layout)
};

// field buffers of the one-warp x kernel: LARGE rows take 32-point segments,
// the others at most 16 (a buffer holds a row in the padded segment layout)
template <class T, bool LARGE>
struct BatchX {
    static constexpr int VN = VecOf<T>::n;
    static constexpr int RMAX = LARGE ? 32 : 16;     // largest x segment
    static constexpr int LINE = 32 * (RMAX + VN);    // elements of one field buffer
};

// copy a struct of 8-byte words with the lanes of one warp
template <class S>
__device__ __forceinline__ void warp_copy(S *dst, const S *src, int lane)
{
    static_assert(sizeof(S) % 8 == 0, "word copy");
    const unsigned long long *s = reinterpret_cast<const unsigned long long *>(src);
    unsigned long long *d = reinterpret_cast<unsigned long long *>(dst);
    for (int i = lane; i < (int)(sizeof(S) / 8); i += 32) d[i] = __ldg(s + i);
}

__device__ __forceinline__ float vfirst(const float4 &v) { return v.x; }
__device__ __forceinline__ float vlast(const float4 &v) { return v.w; }
__device__ __forceinline__ double vfirst(const double2 &v) { return v.x; }
__device__ __forceinline__ double vlast(const double2 &v) { return v.y; }

// second difference of 2 consecutive points given their outer neighbours
__device__ __forceinline__ double2 sdiff2(const double2 &h, double hl, double hr)
{
    return make_double2((h.y - h.x) - (h.x - hl), (hr - h.y) - (h.y - h.x));
}

// ---------------------------------------------------------------------------
// x pass: one row
// ---------------------------------------------------------------------------
// ADJ: the transposed Horner pass, F^T = sum_t (D_x^T)^t (f_t0 u + sum_k f_tk g_k)
// with g_k = (D_y^T)^{k+1} u; u itself (not its second difference) is kept
// in registers.
template <class T, int RPT, bool ADJ>
__device__ __forceinline__ void batch_row(const BatchProb &pb, const ProgParams &pr, int row, int lane, T *B)
{
    using St = ContigStage<T, RPT>;
    using V = typename VecOf<T>::type;
    constexpr int VN = VecOf<T>::n;
    constexpr int NVL = RPT / VN;                    // vectors per lane of a full segment row
    constexpr bool pair = sizeof(T) == 4;
    constexpr int LB = BatchX<T, (RPT > 16)>::LINE;
    static_assert(RPT % VN == 0 && RPT >= 4 && RPT <= BatchX<T, true>::RMAX, "segment length");
    const AxisDev &A = pb.ax;
    const int n = A.n;
    const int64_t base = pb.off + (int64_t)row * pb.pitch;
    const int nvec = (n + VN - 1) / VN;              // within the padded pitch
    const int ng = pb.P;
    if (lane == 0) {
        const unsigned bytes = (unsigned)(nvec * 16);    // whole 16-byte vectors inside the pitch
        prefetch_l2(reinterpret_cast<const T *>(pr.u_hi) + base, bytes);
        if (pair) prefetch_l2(reinterpret_cast<const T *>(pr.u_lo) + base, bytes);
        // field 0 is copied only once r has left its buffer: into L2 now
        if (ng > 0) prefetch_l2(reinterpret_cast<const T *>(pr.g[0]) + base, bytes);
        if (pr.feb != 0.f) {
            prefetch_l2(reinterpret_cast<const T *>(pr.up_hi) + base, bytes);
            if (pair) prefetch_l2(reinterpret_cast<const T *>(pr.up_lo) + base, bytes);
        }
    }

    // 1. fields 1..ng-1 -> shared memory (asynchronous); field 0 after r
    auto copy_field = [&](int k) {
        const V *src = reinterpret_cast<const V *>(reinterpret_cast<const T *>(pr.g[k]) + base);
        T *dst = B + k * LB;
#pragma unroll
        for (int i = 0; i < NVL; ++i) {
            const int v = lane + 32 * i;
            if (v < nvec) cp_async16(dst + St::pos(VN * v), src + v);
        }
    };
    for (int k = 1; k < ng; ++k) copy_field(k);
    cp_async_commit();

    // 2. r = accurate second difference of u, coalesced, in chunks of up to
    //    4 vectors per lane (all loads of a chunk in flight together);
    //    buffer 0 stages it
    T *R = B;
    {
        const T *H = reinterpret_cast<const T *>(pr.u_hi) + base;
        const T *Lo = pair ? reinterpret_cast<const T *>(pr.u_lo) + base : H;
        const V *H4 = reinterpret_cast<const V *>(H), *L4 = reinterpret_cast<const V *>(Lo);
        constexpr int CR = NVL < 4 ? NVL : 4;
#pragma unroll
        for (int i0 = 0; i0 < NVL; i0 += CR) {
            V h[CR], l[CR];
            T hx[CR], lx[CR];        // lane 0: the point before the chunk; lane 31: the point after it
#pragma unroll
            for (int i = 0; i < CR; ++i) {
                const int v = lane + 32 * (i0 + i);
                if (v < nvec) {
                    h[i] = __ldg(H4 + v);
                    if (pair) l[i] = __ldg(L4 + v);
                } else {
                    h[i] = V{};
                    l[i] = V{};
                }
                int j = (lane == 0) ? VN * v - 1 : VN * v + VN;
                j = j < 0 ? 0 : (j > n - 1 ? n - 1 : j);
                hx[i] = 0;
                lx[i] = 0;
                if ((lane == 0 || lane == 31) && v < nvec) {
                    hx[i] = __ldg(H + j);
                    if (pair) lx[i] = __ldg(Lo + j);
                }
            }
            __syncwarp();
#pragma unroll
            for (int i = 0; i < CR; ++i) {
                const int v = lane + 32 * (i0 + i);
                T hl = __shfl_up_sync(0xffffffffu, vlast(h[i]), 1), hr = __shfl_down_sync(0xffffffffu, vfirst(h[i]), 1);
                T ll = 0, lr = 0;
                if (pair) {
                    ll = __shfl_up_sync(0xffffffffu, vlast(l[i]), 1);
                    lr = __shfl_down_sync(0xffffffffu, vfirst(l[i]), 1);
                }
                hl = (lane == 0) ? hx[i] : hl;
                ll = (lane == 0) ? lx[i] : ll;
                hr = (lane == 31) ? hx[i] : hr;
                lr = (lane == 31) ? lx[i] : lr;
                if (v < nvec) {
                    V r;
                    if constexpr (ADJ) {
                        r = h[i];
                        if constexpr (pair) {
                            T *e = reinterpret_cast<T *>(&r);
                            const T *lo4 = reinterpret_cast<const T *>(&l[i]);
#pragma unroll
                            for (int cc = 0; cc < VN; ++cc) e[cc] += lo4[cc];
                        }
                    } else {
                        if constexpr (pair) r = sdiff4(h[i], l[i], hl, ll, hr, lr);
                        else r = sdiff2(h[i], hl, hr);
                        if (v == 0) r.x = r.y;         // Dirichlet: the end node takes the interior centre
                    }
                    *reinterpret_cast<V *>(R + St::pos(VN * v)) = r;
                }
            }
        }
        __syncwarp();
    }
    T r[RPT];
    stage_to_regs<T, RPT>(R, r, lane, false);
    __syncwarp();
    copy_field(0);
    cp_async_commit();
    cp_async_wait_all();
    __syncwarp();

    // 3. Horner in D_x with the fields from shared memory
    T z[RPT];
#pragma unroll
    for (int k = 0; k < RPT; ++k) z[k] = 0;
    for (int t = pb.P; t >= 0; --t) {
        for (int k = 0; k < ng; ++k) {
            const T c = pb.ccoef<T>(t, k);
            if (c == (T)0) continue;
            const V *seg = reinterpret_cast<const V *>(B + k * LB + lane * St::SST);
#pragma unroll
            for (int q = 0; q < RPT / VN; ++q) {
                const V y = seg[q];
                const T *e = reinterpret_cast<const T *>(&y);
#pragma unroll
                for (int cc = 0; cc < VN; ++cc) z[VN * q + cc] += c * e[cc];
            }
        }
        if (t == 0) break;
        if (ADJ) warp_sweep_T<T, RPT>(z, r, pb.ccu<T>(t), A, lane);
        else warp_sweep_rreg<T, BC_DIRICHLET, RPT, true>(z, r, pb.ccu<T>(t), A, lane);
    }

    // 4. F -> coalesced side -> next level; padding points get F = 0
    __syncwarp();
    regs_to_stage<T, RPT>(B, z, lane);
    __syncwarp();
    constexpr int CH = NVL > 4 ? 4 : NVL;
#pragma unroll
    for (int i0 = 0; i0 < NVL; i0 += CH) {
        V F[CH];
#pragma unroll
        for (int i = 0; i < CH; ++i) {
            const int v = lane + 32 * (i0 + i);
            F[i] = V{};
            if (v < nvec) {
                F[i] = *CoalescedSide<T, RPT>::at(B, v * VN);
                T *e = reinterpret_cast<T *>(&F[i]);
#pragma unroll
                for (int cc = 0; cc < VN; ++cc) e[cc] = (VN * v + cc < n) ? e[cc] : (T)0;
            }
        }
        level_batch<T, CH>(pr, base, lane, i0, nvec, F);
    }
}

// LARGE: rows of 513..1024 points (32-point segments; the segment, its r and
// the sweep temporaries need more than 128 registers); else rows of up to
// 512 points at two CTAs per SM.  Rows [row_begin, nitems) of the list.
template <class T, bool LARGE, bool ADJ>
__global__ void __launch_bounds__(256, LARGE ? 1 : 2) k_batch_x(BatchPass bp, int nbuf)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, W = blockDim.x >> 5;
    BatchProb *pbs = reinterpret_cast<BatchProb *>(smem_raw) + warp;
    T *B = reinterpret_cast<T *>(smem_raw + (size_t)W * sizeof(BatchProb)) + (size_t)warp * nbuf * BatchX<T, LARGE>::LINE;
    int cur = -1;
    for (int r = bp.row_begin + blockIdx.x * W + warp; r < bp.nitems; r += gridDim.x * W) {
        const int p = __ldg(bp.row_prob + r);
        if (p != cur) {
            __syncwarp();
            warp_copy(pbs, bp.probs + p, lane);
            __syncwarp();
            cur = p;
        }
        const BatchProb &pb = *pbs;
        const int row = r - pb.row0;
        if (LARGE) {
            batch_row<T, 32, ADJ>(pb, bp.pr, row, lane, B);
        } else {
            switch (pb.rpt_x) {
            case 4: batch_row<T, 4, ADJ>(pb, bp.pr, row, lane, B); break;
            case 8: batch_row<T, 8, ADJ>(pb, bp.pr, row, lane, B); break;
            default: batch_row<T, 16, ADJ>(pb, bp.pr, row, lane, B); break;
            }
        }
        __syncwarp();
    }
}

// ---------------------------------------------------------------------------
// x pass: long rows split over the W warps of one CTA
// ---------------------------------------------------------------------------
// A row of 32 (W-1) RPT < n <= 32 W RPT points: thread t = 32 warp + lane
// owns segment t (points t RPT .. t RPT + RPT - 1); the last point falls in
// the last warp.  The steps are those of batch_row with the thread index in
// place of the lane and the halos and carries between the warps through
// shared memory (row_sweep / row_sweep_T).
template <class T, int RPT, int W, bool ADJ>
__device__ __forceinline__ void batch_row_split(const BatchProb &pb, const ProgParams &pr, int row, int t, T *B,
                                                RowSlots<T, W> &sl)
{
    using St = ContigStage<T, RPT>;
    using V = typename VecOf<T>::type;
    constexpr int VN = VecOf<T>::n;
    constexpr int NT = 32 * W;
    constexpr int NVL = RPT / VN;                    // vectors per thread of a full row
    constexpr bool pair = sizeof(T) == 4;
    constexpr int LB = NT * St::SST;                 // one field buffer
    static_assert(RPT % VN == 0 && RPT >= 4, "segment length");
    const int warp = t >> 5, lane = t & 31;
    const AxisDev &A = pb.ax;
    const int n = A.n;
    const int64_t base = pb.off + (int64_t)row * pb.pitch;
    const int nvec = (n + VN - 1) / VN;              // within the padded pitch
    const int ng = pb.P;
    if (t == 0) {
        const unsigned bytes = (unsigned)(nvec * 16);
        prefetch_l2(reinterpret_cast<const T *>(pr.u_hi) + base, bytes);
        if (pair) prefetch_l2(reinterpret_cast<const T *>(pr.u_lo) + base, bytes);
        if (ng > 0) prefetch_l2(reinterpret_cast<const T *>(pr.g[0]) + base, bytes);   // copied after r
        if (pr.feb != 0.f) {
            prefetch_l2(reinterpret_cast<const T *>(pr.up_hi) + base, bytes);
            if (pair) prefetch_l2(reinterpret_cast<const T *>(pr.up_lo) + base, bytes);
        }
    }

    // 1. fields 1..ng-1 -> shared memory (asynchronous); field 0 after r
    auto copy_field = [&](int k) {
        const V *src = reinterpret_cast<const V *>(reinterpret_cast<const T *>(pr.g[k]) + base);
        T *dst = B + k * LB;
#pragma unroll
        for (int i = 0; i < NVL; ++i) {
            const int v = t + NT * i;
            if (v < nvec) cp_async16(dst + St::pos(VN * v), src + v);
        }
    };
    for (int k = 1; k < ng; ++k) copy_field(k);
    cp_async_commit();

    // 2. r (ADJ: u) coalesced over the CTA, staged in buffer 0
    T *R = B;
    {
        const T *H = reinterpret_cast<const T *>(pr.u_hi) + base;
        const T *Lo = pair ? reinterpret_cast<const T *>(pr.u_lo) + base : H;
        const V *H4 = reinterpret_cast<const V *>(H), *L4 = reinterpret_cast<const V *>(Lo);
        constexpr int CR = NVL < 4 ? NVL : 4;
#pragma unroll
        for (int i0 = 0; i0 < NVL; i0 += CR) {
            V h[CR], l[CR];
            T hx[CR], lx[CR];        // lane 0: the point before its vector; lane 31: the point after it
#pragma unroll
            for (int i = 0; i < CR; ++i) {
                const int v = t + NT * (i0 + i);
                if (v < nvec) {
                    h[i] = __ldg(H4 + v);
                    if (pair) l[i] = __ldg(L4 + v);
                } else {
                    h[i] = V{};
                    l[i] = V{};
                }
                int j = (lane == 0) ? VN * v - 1 : VN * v + VN;
                j = j < 0 ? 0 : (j > n - 1 ? n - 1 : j);
                hx[i] = 0;
                lx[i] = 0;
                if (!ADJ && (lane == 0 || lane == 31) && v < nvec) {
                    hx[i] = __ldg(H + j);
                    if (pair) lx[i] = __ldg(Lo + j);
                }
            }
            __syncwarp();
#pragma unroll
            for (int i = 0; i < CR; ++i) {
                const int v = t + NT * (i0 + i);
                T hl = __shfl_up_sync(0xffffffffu, vlast(h[i]), 1), hr = __shfl_down_sync(0xffffffffu, vfirst(h[i]), 1);
                T ll = 0, lr = 0;
                if (pair) {
                    ll = __shfl_up_sync(0xffffffffu, vlast(l[i]), 1);
                    lr = __shfl_down_sync(0xffffffffu, vfirst(l[i]), 1);
                }
                hl = (lane == 0) ? hx[i] : hl;
                ll = (lane == 0) ? lx[i] : ll;
                hr = (lane == 31) ? hx[i] : hr;
                lr = (lane == 31) ? lx[i] : lr;
                if (v < nvec) {
                    V r;
                    if constexpr (ADJ) {
                        r = h[i];
                        if constexpr (pair) {
                            T *e = reinterpret_cast<T *>(&r);
                            const T *lo4 = reinterpret_cast<const T *>(&l[i]);
#pragma unroll
                            for (int cc = 0; cc < VN; ++cc) e[cc] += lo4[cc];
                        }
                    } else {
                        if constexpr (pair) r = sdiff4(h[i], l[i], hl, ll, hr, lr);
                        else r = sdiff2(h[i], hl, hr);
                        if (v == 0) r.x = r.y;         // Dirichlet: the end node takes the interior centre
                    }
                    *reinterpret_cast<V *>(R + St::pos(VN * v)) = r;
                } else {
                    *reinterpret_cast<V *>(R + St::pos(VN * v)) = V{};
                }
            }
        }
    }
    __syncthreads();
    T r[RPT];
    stage_to_regs<T, RPT>(R, r, t, false);
    if (!ADJ) {
        if (lane == 0) sl.rhalo[warp][0] = r[0];
        if (lane == 31) sl.rhalo[warp][1] = r[RPT - 1];
    }
    __syncthreads();                                 // every thread is done with R
    copy_field(0);
    cp_async_commit();
    T rl = 0, rr = 0;
    if (!ADJ) {
        rl = __shfl_up_sync(0xffffffffu, r[RPT - 1], 1);
        rr = __shfl_down_sync(0xffffffffu, r[0], 1);
        if (lane == 0) rl = (warp > 0) ? sl.rhalo[warp - 1][1] : r[0];
        if (lane == 31) rr = (warp < W - 1) ? sl.rhalo[warp + 1][0] : r[RPT - 1];
    }
    cp_async_wait_all();
    __syncthreads();

    // 3. Horner in D_x with the fields from shared memory
    T z[RPT];
#pragma unroll
    for (int k = 0; k < RPT; ++k) z[k] = 0;
    for (int tt = pb.P; tt >= 0; --tt) {
        for (int k = 0; k < ng; ++k) {
            const T c = pb.ccoef<T>(tt, k);
            if (c == (T)0) continue;
            const V *seg = reinterpret_cast<const V *>(B + k * LB + t * St::SST);
#pragma unroll
            for (int q = 0; q < NVL; ++q) {
                const V y = seg[q];
                const T *e = reinterpret_cast<const T *>(&y);
#pragma unroll
                for (int cc = 0; cc < VN; ++cc) z[VN * q + cc] += c * e[cc];
            }
        }
        if (tt == 0) break;
        if (ADJ) row_sweep_T<T, RPT, W>(z, r, pb.ccu<T>(tt), A, lane, warp, sl);
        else row_sweep<T, BC_DIRICHLET, RPT, W, true>(z, r, rl, rr, pb.ccu<T>(tt), A, lane, warp, sl);
    }

    // 4. F -> coalesced side -> next level; padding points get F = 0
    __syncthreads();                                 // every thread is done reading the fields
    regs_to_stage<T, RPT>(B, z, t);
    __syncthreads();
    constexpr int CH = NVL > 4 ? 4 : NVL;
#pragma unroll
    for (int i0 = 0; i0 < NVL; i0 += CH) {
        V F[CH];
#pragma unroll
        for (int i = 0; i < CH; ++i) {
            const int v = t + NT * (i0 + i);
            F[i] = V{};
            if (v < nvec) {
                F[i] = *CoalescedSide<T, RPT>::at(B, v * VN);
                T *e = reinterpret_cast<T *>(&F[i]);
#pragma unroll
                for (int cc = 0; cc < VN; ++cc) e[cc] = (VN * v + cc < n) ? e[cc] : (T)0;
            }
        }
        level_batch<T, CH, NT>(pr, base, t, i0, nvec, F);
    }
}

// Rows [row_begin, nitems) of the list, one CTA of W warps per row (rows of
// 32 (W-1) RPT < n <= 32 W RPT points).  Float: ten CTAs per SM at RPT = 16
// (96 registers, no spills; 20 warps in flight against 16 at eight CTAs),
// sixteen at RPT = 8 (64 registers).
template <class T, int RPT, int W, bool ADJ>
__global__ void __launch_bounds__(32 * W, sizeof(T) == 4 ? (RPT <= 8 ? 16 : 10) : 4) k_batch_xs(BatchPass bp)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    BatchProb &pb = *reinterpret_cast<BatchProb *>(smem_raw);
    RowSlots<T, W> &sl = *reinterpret_cast<RowSlots<T, W> *>(smem_raw + sizeof(BatchProb));
    T *B = reinterpret_cast<T *>(smem_raw + sizeof(BatchProb) + row_slots_bytes<T, W>());
    const int r = bp.row_begin + (int)blockIdx.x;
    if (r >= bp.nitems) return;
    const int p = __ldg(bp.row_prob + r);
    {
        const unsigned long long *src = reinterpret_cast<const unsigned long long *>(bp.probs + p);
        unsigned long long *dst = reinterpret_cast<unsigned long long *>(&pb);
        for (int i = threadIdx.x; i < (int)(sizeof(BatchProb) / 8); i += 32 * W) dst[i] = __ldg(src + i);
    }
    __syncthreads();
    batch_row_split<T, RPT, W, ADJ>(pb, bp.pr, r - pb.row0, threadIdx.x, B, sl);
}

// ---------------------------------------------------------------------------
// y pass: one group of 32 columns
// ---------------------------------------------------------------------------
// r = accurate second difference of u at rows a-1 .. a+RPT of one column,
// every row index clamped into the problem (the last segment may be partial)
template <int RPT>
__device__ __forceinline__ void bcol_r_rag(const ProgParams &pr, int64_t lbase, int64_t st, int a, int n,
                                           float (&r)[RPT], float &rl, float &rr)
{
    const float *H = (const float *)pr.u_hi + lbase, *L = (const float *)pr.u_lo + lbase;
    auto row = [&](int j) { return (int64_t)(j < 0 ? 0 : (j > n - 1 ? n - 1 : j)) * st; };
    float hm = H[row(a - 2)], lm = L[row(a - 2)], h0 = H[row(a - 1)], l0 = L[row(a - 1)];
#pragma unroll
    for (int k = 0; k <= RPT + 1; ++k) {
        const int64_t j = row(a + k);
        const float hp = H[j], lp = L[j];
        const float v = sdiff_pair(hm, h0, hp, lm, l0, lp);
        if (k == 0) rl = v; else if (k == RPT + 1) rr = v; else r[k - 1] = v;
        hm = h0; h0 = hp; lm = l0; l0 = lp;
    }
}

template <int RPT>
__device__ __forceinline__ void bcol_r_rag(const ProgParams &pr, int64_t lbase, int64_t st, int a, int n,
                                           double (&r)[RPT], double &rl, double &rr)
{
    const double *U = (const double *)pr.u_hi + lbase;
    auto row = [&](int j) { return (int64_t)(j < 0 ? 0 : (j > n - 1 ? n - 1 : j)) * st; };
    double um = U[row(a - 2)], u0 = U[row(a - 1)];
#pragma unroll
    for (int k = 0; k <= RPT + 1; ++k) {
        const double up = U[row(a + k)];
        const double v = (up - u0) - (u0 - um);
        if (k == 0) rl = v; else if (k == RPT + 1) rr = v; else r[k - 1] = v;
        um = u0; u0 = up;
    }
}

// The solve of the difference form on this thread's segment of a Dirichlet
// column of any length: z holds q on entry (zero past the line and at the
// end nodes), e on exit.  rag: the segment holds the last point (0 <= kl <
// RPT) or the one before it (kl == RPT); YL carries y_{n-1} of every lane
// from the segment that holds the last point to all segments.
template <class T, int RPT>
__device__ __forceinline__ void bsolve(const StridedCtx<T> &c, const AxisDev &A, T (&z)[RPT], int kl, bool rag, T *YL)
{
    const T d = c.d;
    constexpr bool TWO = RPT >= 16;              // two-chain recurrences on the segments without the line's end
    const T dH = TWO ? c.dpg[RPT / 2] : (T)0;
    T E1 = 0, ER2 = 0;
    const T E = (TWO && !rag) ? seg_fwd_reduce2<T, RPT>(z, d, dH, E1) : seg_fwd_reduce<T, RPT>(z, d);
    T yin, ytot;
    strided_causal<T, RPT>(c, E, yin, ytot);
    if (!c.full) yin = 0;
    T ylast = 0;
    T ER;
    if (rag) ER = seg_fwd_scan<T, RPT, true>(z, d, yin, kl, &ylast);
    else if (TWO) ER = seg_fwd_scan2<T, RPT>(z, d, dH, yin, E1, ER2);
    else ER = seg_fwd_scan<T, RPT>(z, d, yin);
    if (rag && kl < RPT) YL[c.lane] = ylast;
    T eout, e00;
    strided_anticausal<T, RPT>(c, ER, eout, e00);      // its barrier publishes YL
    const T yl = peer_of(c, YL, (c.Gd - 1) / c.S)[c.lane];   // written by the CTA holding the last point
    const T mu = A.cmu<T>(), inv = A.cinv<T>();
    const T Acoef = (mu * yl - e00) * inv;
    const T Z = (mu * e00 - yl) * inv;
    const T acc = d * eout + ((c.full && kl >= RPT) ? c.dpg[kl + 1 - RPT] * Z : (T)0);
    if (rag) seg_bwd_scan<T, RPT, true>(z, d, acc, kl, Z);
    else if (TWO) seg_bwd_scan2<T, RPT>(z, d, dH, acc, ER2);
    else seg_bwd_scan<T, RPT>(z, d, acc);
    if (c.full) {
        if (TWO && !rag) seg_add_left2<T, RPT>(z, d, dH, Acoef * c.dpg[c.a]);
        else seg_add_left<T, RPT>(z, d, Acoef * c.dpg[c.a]);
    }
}

// One application of D on this thread's segment (MODE as in seg_make_q)
template <class T, int RPT, int MODE>
__device__ __forceinline__ void bsweep(const StridedCtx<T> &c, const AxisDev &A, T (&z)[RPT], T l2, T l1, T r0,
                                       T r1, int kl, bool rag, T *YL)
{
    const bool left = c.seg == 0;
    end_ghosts<T, RPT, MODE>(z, left, false, l2, l1, r0, r1);
    const T c1 = A.cc1<T>(), c2 = A.cc2<T>();
    auto rz = [&](int) { return (T)0; };
    if (rag) seg_make_q<T, RPT, MODE, true>(z, l2, l1, r0, r1, rz, (T)0, c1, c2, kl);
    else seg_make_q<T, RPT, MODE, false>(z, l2, l1, r0, r1, rz, (T)0, c1, c2);
    end_zero<T, RPT>(z, left, false);
    if (!c.full) {
#pragma unroll
        for (int k = 0; k < RPT; ++k) z[k] = 0;
    }
    bsolve<T, RPT>(c, A, z, kl, rag, YL);
}

// zero at the end nodes and past the line (interior rows only)
template <class T, int RPT>
__device__ __forceinline__ void interior_only(const StridedCtx<T> &c, T (&z)[RPT], int kl, bool rag)
{
    if (c.seg == 0) z[0] = 0;
    if (rag) {
#pragma unroll
        for (int k = 0; k < RPT; ++k) z[k] = (k < kl) ? z[k] : (T)0;
    }
    if (!c.full) {
#pragma unroll
        for (int k = 0; k < RPT; ++k) z[k] = 0;
    }
}

// One application of D^T on this thread's segment (see post_T)
template <class T, int RPT>
__device__ __forceinline__ void bsweep_T(const StridedCtx<T> &c, const AxisDev &A, T (&z)[RPT], int kl, bool rag,
                                         T *YL, int hbuf)
{
    interior_only<T, RPT>(c, z, kl, rag);
    bsolve<T, RPT>(c, A, z, kl, rag, YL);
    interior_only<T, RPT>(c, z, kl, rag);
    T l2, l1, r0, r1;
    strided_halos<T, BC_DIRICHLET, RPT>(c, z, l2, l1, r0, r1, hbuf);
    const T c1 = A.cc1<T>(), c2 = A.cc2<T>();
    if (c.seg == 0 || rag) post_T<T, RPT, true>(z, l2, l1, r0, r1, c1, c2, c.a, c.n);
    else post_T<T, RPT, false>(z, l2, l1, r0, r1, c1, c2, c.a, c.n);
}

// level value at rows a .. a+RPT-1 of one column (pairs summed in T), rows
// past the line read as zero
template <class T, int RPT>
__device__ __forceinline__ void bcol_level(const ProgParams &pr, int64_t lbase, int64_t st, int a, int n, T (&z)[RPT])
{
    const T *H = (const T *)pr.u_hi + lbase;
    const T *L = (const T *)pr.u_lo + lbase;
#pragma unroll
    for (int k = 0; k < RPT; ++k) {
        const int j = a + k;
        const int64_t o = (int64_t)(j < n ? j : n - 1) * st;
        T v = H[o];
        if constexpr (sizeof(T) == 4) v += L[o];
        z[k] = (j < n) ? v : (T)0;
    }
}

template <class T, int RPT, bool ADJ>
__device__ __forceinline__ void batch_cols(const BatchProb &pb, const ProgParams &pr, int col0, StridedCtx<T> &c, T *YL)
{
    const AxisDev &A = pb.ay;
    const int n = A.n;
    c.n = n;
    c.d = A.cd<T>();
    c.dR = A.cdm<T>(0);
    c.dpg = dpow_of<T>(A);
    c.Gd = (n + RPT - 1) / RPT;
    strided_cta_consts<T, RPT>(c);
    c.a = c.seg * RPT;
    c.full = c.seg < c.Gd;
    const int kl = n - 1 - c.a;
    const bool rag = c.full && kl <= RPT;
    const int col = col0 + c.lane;
    const bool io = c.full && col < pb.ax.n;
    const int64_t lbase = pb.off + (io ? col : 0);
    const int64_t st = pb.pitch;

    T z[RPT];
    if (ADJ) {
        // powers of D_y^T applied to the level
        if (io) bcol_level<T, RPT>(pr, lbase, st, c.a, n, z);
        else {
#pragma unroll
            for (int k = 0; k < RPT; ++k) z[k] = 0;
        }
        for (int p = 1; p <= pb.P; ++p) {
            bsweep_T<T, RPT>(c, A, z, kl, rag, YL, p & 1);
            if (io) {
                T *po = reinterpret_cast<T *>(pr.out[p - 1]) + lbase + (int64_t)c.a * st;
#pragma unroll
                for (int k = 0; k < RPT; ++k) {
                    if (k <= kl) *po = z[k];
                    po += st;
                }
            }
        }
        return;
    }
    T rl = 0, rr = 0;
    if (io) {
        if (rag) bcol_r_rag<RPT>(pr, lbase, st, c.a, n, z, rl, rr);
        else strided_r_pair<BC_DIRICHLET, RPT>(pr, lbase, st, c.a, n, z, rl, rr);
    } else {
#pragma unroll
        for (int k = 0; k < RPT; ++k) z[k] = 0;
    }
    if (c.seg == 0) z[0] = z[1];                   // Dirichlet: the end node takes the interior centre

    for (int p = 1; p <= pb.P; ++p) {
        if (p == 1) {
            bsweep<T, RPT, 0>(c, A, z, (T)0, rl, rr, (T)0, kl, rag, YL);
        } else {
            T l2, l1, r0, r1;
            strided_halos<T, BC_DIRICHLET, RPT>(c, z, l2, l1, r0, r1, p & 1);
            bsweep<T, RPT, 1>(c, A, z, l2, l1, r0, r1, kl, rag, YL);
        }
        if (io) {
            T *po = reinterpret_cast<T *>(pr.out[p - 1]) + lbase + (int64_t)c.a * st;
#pragma unroll
            for (int k = 0; k < RPT; ++k) {
                if (k <= kl) *po = z[k];
                po += st;
            }
        }
    }
}

// The powers D_y^p u of one group of 32 columns with ONE exchange per sweep
// between neighbouring segments (the algebra of k_strided_nb: each segment
// runs its causal recurrence with zero inflow, publishes E, y0(RPT-2), ER0,
// ER1, and after one barrier corrects itself from its neighbours' numbers),
// for columns of any length: the last segment holds the line's last point
// at kl and is ragged (zeros past it; with kl = 0 the segment before it is
// ragged too, so that it never reads past the line).  The right boundary
// term B' = -y_{n-1} / (1 - mu^2) of the Dirichlet line enters at the last
// point; the last segment also publishes its zero-inflow y at kl, so that its
// left neighbour forms B' (linear in its own E) and takes the term into its
// inflow.  Valid when d^(RPT-1) <= 2^-30 and the line has more than two
// segments (ynb, set on the host).  Float32 only.
template <int RPT>
__device__ __forceinline__ void batch_cols_nb(const BatchProb &pb, const ProgParams &pr, int col0, int w, int lane,
                                              float *slots, int S, int K, int krank, cg::cluster_group &cl)
{
    constexpr int H = RPT / 2;
    constexpr bool TWO = RPT >= 8;                  // two-chain recurrences on the full segments
    const AxisDev &A = pb.ay;
    const NbConsts &nc = pb.nby;
    const int n = A.n, Gd = (n + RPT - 1) / RPT, Ld = Gd - 1;
    const int seg = krank * S + w, a = seg * RPT;
    const bool full = seg < Gd;
    const int kl = n - 1 - a;
    const bool rag = full && kl <= RPT;
    const bool left_end = seg == 0, last = seg == Ld;
    // a segment's slots ([2][S][5][32] per CTA), in its CTA of the cluster
    auto slot = [&](int buf, int sg) -> float * {
        float *q = slots + ((size_t)buf * S + sg % S) * 160;
        return K > 1 ? cl.map_shared_rank(q, sg / S) : q;
    };
    const bool hasL = full && seg > 0, hasR = full && seg < Ld, rlast = seg == Ld - 1;
    const int col = col0 + lane;
    const bool io = full && col < pb.ax.n;
    const int64_t lbase = pb.off + (io ? col : 0);
    const int64_t st = pb.pitch;
    const float d = A.fd, c1 = A.fc1, c2 = A.fc2, inv = A.finv;

    float z[RPT];
    float rl = 0.f, rr = 0.f;
    if (io) {
        if (rag) bcol_r_rag<RPT>(pr, lbase, st, a, n, z, rl, rr);
        else strided_r_pair<BC_DIRICHLET, RPT>(pr, lbase, st, a, n, z, rl, rr);
    } else {
#pragma unroll
        for (int k = 0; k < RPT; ++k) z[k] = 0.f;
    }
    if (seg == 0) z[0] = z[1];                      // Dirichlet: the end node takes the interior centre
    float hl2 = 0.f, hl1 = rl, hr0 = rr, hr1 = 0.f;  // sweep 1 (z = s): s at a-1 and a+RPT
    auto noR = [](int) { return 0.f; };

    for (int p = 1; p <= pb.P; ++p) {
        float zl2 = hl2, zl1 = hl1, zr0 = hr0, zr1 = hr1;
        if (p == 1) {
            end_ghosts<float, RPT, 0>(z, left_end, false, zl2, zl1, zr0, zr1);
            if (rag) seg_make_q<float, RPT, 0, true>(z, zl2, zl1, zr0, zr1, noR, 0.f, c1, c2, kl);
            else seg_make_q<float, RPT, 0, false>(z, zl2, zl1, zr0, zr1, noR, 0.f, c1, c2);
        } else {
            end_ghosts<float, RPT, 1>(z, left_end, false, zl2, zl1, zr0, zr1);
            if (rag) seg_make_q<float, RPT, 1, true>(z, zl2, zl1, zr0, zr1, noR, 0.f, c1, c2, kl);
            else seg_make_q<float, RPT, 1, false>(z, zl2, zl1, zr0, zr1, noR, 0.f, c1, c2);
        }
        end_zero<float, RPT>(z, left_end, false);
        if (!full) {
#pragma unroll
            for (int k = 0; k < RPT; ++k) z[k] = 0.f;
        }

        // the causal recurrence with zero inflow (ragged segments: one chain,
        // zero past the last point); E, Y2 = zero-inflow y at RPT-1, RPT-2
        float E1 = 0.f, rb = 0.f, ER1 = 0.f, YL0 = 0.f, E, Y2;
        if (TWO && !rag) {
            float ya = z[0], yb = z[H], ra1 = 0.f, pw = 1.f;
            rb = yb;
#pragma unroll
            for (int k = 1; k < H; ++k) {
                ya = d * ya + z[k];
                yb = d * yb + z[H + k];
                z[k] = ya;
                z[H + k] = yb;
                const float pbk = pw * d;            // chain A weighs y_k by d^(k-1), chain B by d^k
                ra1 += pw * ya;
                rb += pbk * yb;
                pw = pbk;
            }
            E1 = ya;
            E = yb + E1 * nc.dH;
            Y2 = z[RPT - 2] + E1 * nc.dH1;
            ER1 = ra1 + nc.dH1 * (rb + E1 * nc.GH);
        } else {
            float y = 0.f, pw = 1.f;
#pragma unroll
            for (int k = 0; k < RPT; ++k) {
                y = d * y + z[k];
                const float yo = (!rag || k <= kl) ? y : 0.f;
                YL0 = (k == kl) ? y : YL0;
                z[k] = yo;
                if (k > 0) {
                    ER1 += pw * yo;
                    pw *= d;
                }
            }
            E = z[RPT - 1];
            Y2 = z[RPT - 2];
        }
        const float ER0 = z[0] + d * ER1;

        float *mine = slots + ((size_t)(p & 1) * S + w) * 160;
        mine[lane] = E;
        mine[32 + lane] = Y2;
        mine[64 + lane] = ER0;
        mine[96 + lane] = ER1;
        mine[128 + lane] = YL0;
        if (K > 1) cl.sync();
        else __syncthreads();
        float EL = 0.f, Y2L = 0.f, ER0R = 0.f, ER1R = 0.f, YLR = 0.f;
        if (hasL) {
            const float *q = slot(p & 1, seg - 1);
            EL = q[lane];
            Y2L = q[32 + lane];
        }
        if (hasR) {
            const float *q = slot(p & 1, seg + 1);
            ER0R = q[64 + lane];
            ER1R = q[96 + lane];
            YLR = q[128 + lane];
        }

        // true causal values: chain A from the left neighbour's y at a-1,
        // chain B from the corrected y at H-1
        float ER2 = 0.f;
        if (TWO && !rag) {
            const float cB = E1 + EL * nc.dH;
            float pk = d;
#pragma unroll
            for (int k = 0; k < H; ++k) {
                z[k] += EL * pk;
                z[H + k] += cB * pk;
                pk *= d;
            }
            ER2 = rb + cB * nc.GH;                   // sum_j d^j y_{H+j}
        } else {
            float pk = d;
#pragma unroll
            for (int k = 0; k < RPT; ++k) {
                if (!rag || k <= kl) z[k] += EL * pk;
                pk *= d;
            }
        }

        // the right inflow: e at a+RPT and a+RPT+1, with the line's B' term
        // when the right neighbour holds the last point
        float eout = 0.f, er1 = 0.f;
        if (hasR) {
            if (rlast) {
                const float Bp = -(YLR + E * pb.nbdkp) * inv;
                eout = ER0R + pb.nbGL * E + Bp * pb.nbdk;
                er1 = ER1R + pb.nbG1L * E + Bp * pb.nbdk1;
            } else {
                eout = ER0R + nc.G * E;
                er1 = ER1R + nc.G1 * E;
            }
        }
        const float acc = d * eout;
        if (TWO && !rag) {
            seg_bwd_scan2<float, RPT>(z, d, nc.dH, acc, ER2);
        } else {
            const float Zr = last ? -(YL0 + EL * pb.nbdkp) * inv : 0.f;   // B' at the last point
            seg_bwd_scan<float, RPT, true>(z, d, acc, rag ? kl : RPT, Zr);
        }
        if (left_end) {
            if (TWO && !rag) seg_add_left2<float, RPT>(z, d, nc.dH, -z[0] * inv);
            else seg_add_left<float, RPT>(z, d, -z[0] * inv);
        }

        // halos of the next sweep
        hl1 = hasL ? EL + d * z[0] : 0.f;
        hl2 = hasL ? Y2L + d * hl1 : 0.f;
        hr0 = eout;
        hr1 = er1;

        if (io) {
            float *po = reinterpret_cast<float *>(pr.out[p - 1]) + lbase + (int64_t)a * st;
#pragma unroll
            for (int k = 0; k < RPT; ++k) {
                if (k <= kl) *po = z[k];
                po += st;
            }
        }
    }
}

// One column group (32 neighbouring columns of one problem, the work-list
// item of blockIdx.x) per cluster of ky = gridDim.y CTAs of kBatchYSeg warps;
// warp w of cluster rank k owns segment k kBatchYSeg + w of rpt_y rows.  The
// launch takes the items of one cluster size; small CTAs (four per SM at 128
// registers) let the loads of some column groups overlap the sweeps of
// others.  Float32 forward passes exchange once per sweep between
// neighbouring segments where that is exact (batch_cols_nb), the others
// carry through every segment (batch_cols).
// ADJ: powers of D_y^T (the adjoint step) instead of D_y.
template <class T, bool ADJ>
__global__ void __launch_bounds__(32 * kBatchYSeg, sizeof(T) == 4 ? 4 : 2) k_batch_y(BatchPass bp)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    cg::cluster_group cl = cg::this_cluster();
    const int2 item = bp.items[blockIdx.x];
    // the problem's constants are read where they are used (through L1): a
    // copy of the whole table entry would cost each short-lived CTA a round trip
    const BatchProb &pbs = bp.probs[item.x];
    const int K = (int)gridDim.y;
    StridedCtx<T> c{cl};
    c.S = kBatchYSeg;
    c.K = K;
    c.krank = K > 1 ? (int)cl.block_rank() : 0;
    c.w = threadIdx.x >> 5;
    c.lane = threadIdx.x & 31;
    c.seg = c.krank * c.S + c.w;
    bool done = false;
    if constexpr (sizeof(T) == 4 && !ADJ) {
        if (pbs.ynb) {
            float *slots = reinterpret_cast<float *>(smem_raw);
            switch (pbs.rpt_y) {
            case 4: batch_cols_nb<4>(pbs, bp.pr, item.y, c.w, c.lane, slots, c.S, K, c.krank, cl); break;
            case 8: batch_cols_nb<8>(pbs, bp.pr, item.y, c.w, c.lane, slots, c.S, K, c.krank, cl); break;
            case 16: batch_cols_nb<16>(pbs, bp.pr, item.y, c.w, c.lane, slots, c.S, K, c.krank, cl); break;
            case 32: batch_cols_nb<32>(pbs, bp.pr, item.y, c.w, c.lane, slots, c.S, K, c.krank, cl); break;
            default: batch_cols_nb<64>(pbs, bp.pr, item.y, c.w, c.lane, slots, c.S, K, c.krank, cl); break;
            }
            done = true;
        }
    }
    if (!done) {
        T *p = reinterpret_cast<T *>(smem_raw);
        c.sl.E = p;
        c.sl.ER = p + c.S * 32;
        c.sl.H = p + 2 * c.S * 32;
        c.sl.Tot = p + 10 * c.S * 32;
        T *YL = reinterpret_cast<T *>(smem_raw + strided_slot_bytes(c.S, sizeof(T)));
        switch (pbs.rpt_y) {
        case 4: batch_cols<T, 4, ADJ>(pbs, bp.pr, item.y, c, YL); break;
        case 8: batch_cols<T, 8, ADJ>(pbs, bp.pr, item.y, c, YL); break;
        case 16: batch_cols<T, 16, ADJ>(pbs, bp.pr, item.y, c, YL); break;
        case 32: batch_cols<T, 32, ADJ>(pbs, bp.pr, item.y, c, YL); break;
        default:
            if constexpr (sizeof(T) == 4) batch_cols<T, 64, ADJ>(pbs, bp.pr, item.y, c, YL);
            break;
        }
    }
    // peers read this CTA's shared memory after the last exchange: no CTA
    // of the cluster exits before all of them are past those reads
    if (K > 1) cl.sync();
}

inline size_t batch_y_smem(size_t tsize)
{
    const size_t full = strided_slot_bytes(kBatchYSeg, tsize) + 32 * tsize;
    const size_t nb = (size_t)2 * kBatchYSeg * 5 * 32 * sizeof(float);   // batch_cols_nb's slots
    return full > nb ? full : nb;
}
inline size_t batch_x_smem(size_t tsize, int W, int nbuf, bool large)
{
    const size_t rmax = large ? BatchX<float, true>::RMAX : BatchX<float, false>::RMAX;
    return (size_t)W * (sizeof(BatchProb) + (size_t)nbuf * 32 * (rmax + 16 / tsize) * tsize);
}
// k_batch_xs: the problem, the exchange slots and nbuf fields of one row
// (32 W segments of RPT + 16 / tsize elements)
inline size_t batch_xs_smem(size_t tsize, int RPT, int W, int nbuf)
{
    const size_t slots = tsize == 4 ? row_slots_bytes<float, 8>() : row_slots_bytes<double, 8>();
    return sizeof(BatchProb) + slots + (size_t)nbuf * 32 * W * (RPT + 16 / tsize) * tsize;
}

// ---------------------------------------------------------------------------
// packed float64 fields (problem after problem, rows of nx points) <->
// internal layout (padded rows; float32 pairs or float64)
// ---------------------------------------------------------------------------
template <class T>
__global__ void __launch_bounds__(256, 8) k_batch_pack(const BatchProb *probs, const int *row_prob, const long long *uoff, int nrows,
                             const double *__restrict__ x, T *__restrict__ hi, T *__restrict__ lo)
{
    // a warp converts a row 128 points at a time, lane + 32 c for c = 0..3:
    // every load and store instruction of the warp covers one contiguous
    // span (256 bytes of float64, 128 of float32), whatever the alignment of
    // the packed row; the padding of the internal row is written as zeros
    const int lane = threadIdx.x & 31;
    const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, nw = (gridDim.x * blockDim.x) >> 5;
    for (int r = gw; r < nrows; r += nw) {
        const int p = __ldg(row_prob + r);
        const BatchProb *pb = probs + p;
        const int nx = __ldg(&pb->ax.n), pitch = __ldg(&pb->pitch);
        const int row = r - __ldg(&pb->row0);
        const double *src = x + __ldg(uoff + p) + (int64_t)row * nx;
        const int64_t dst = __ldg(&pb->off) + (int64_t)row * pitch;
#pragma unroll 2
        for (int j0 = lane; j0 < pitch; j0 += 128) {
            double v[4];
#pragma unroll
            for (int c = 0; c < 4; ++c) v[c] = (j0 + 32 * c < nx) ? __ldg(src + j0 + 32 * c) : 0.0;
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                const int j = j0 + 32 * c;
                if (j < pitch) {
                    if constexpr (sizeof(T) == 4) {
                        float h, l;                  // the pair split of the single-problem levels
                        split_pair(v[c], h, l);
                        hi[dst + j] = h;
                        lo[dst + j] = l;
                    } else {
                        hi[dst + j] = v[c];
                    }
                }
            }
        }
    }
}

// x = level (+ add, a packed field, when given); the same warp-per-row
// traversal as k_batch_pack
template <class T>
__global__ void __launch_bounds__(256, 8) k_batch_unpack(const BatchProb *probs, const int *row_prob, const long long *uoff, int nrows,
                               const T *__restrict__ hi, const T *__restrict__ lo, double *__restrict__ x,
                               const double *__restrict__ add)
{
    const int lane = threadIdx.x & 31;
    const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, nw = (gridDim.x * blockDim.x) >> 5;
    for (int r = gw; r < nrows; r += nw) {
        const int p = __ldg(row_prob + r);
        const BatchProb *pb = probs + p;
        const int nx = __ldg(&pb->ax.n), pitch = __ldg(&pb->pitch);
        const int row = r - __ldg(&pb->row0);
        const int64_t u0 = __ldg(uoff + p) + (int64_t)row * nx;
        double *dstp = x + u0;
        const int64_t src = __ldg(&pb->off) + (int64_t)row * pitch;
        for (int j0 = lane; j0 < nx; j0 += 128) {
            double v[4];
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                const int j = j0 + 32 * c;
                v[c] = 0.0;
                if (j < nx) {
                    if constexpr (sizeof(T) == 4) v[c] = join_pair(__ldg(hi + src + j), __ldg(lo + src + j));
                    else v[c] = __ldg(hi + src + j);
                    if (add) v[c] += __ldg(add + u0 + j);
                }
            }
#pragma unroll
            for (int c = 0; c < 4; ++c)
                if (j0 + 32 * c < nx) dstp[j0 + 32 * c] = v[c];
        }
    }
}

}  // namespace molt
