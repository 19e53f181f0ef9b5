// molt_regs.cuh -- register-resident line sweeps (sm_103a).
//
// Every thread owns one segment of RPT consecutive points of one line in
// registers.  The operator D (see molt_kernels.cuh for the difference form)
// runs on the segment with a sliding 5-point window, a causal reduction, a
// carry exchange, a causal scan fused with the anti-causal reduction, a
// second exchange and the anti-causal scan; the Dirichlet term A' d^j is
// added last.  Two layouts share these segment routines:
//
//  * k_contig  (contiguous axis x): one warp per line, lane s owns points
//    [s*RPT, (s+1)*RPT).  Carries and halos travel by warp shuffles.  Global
//    memory is read and written coalesced (lane = consecutive points) and
//    turned into the segment layout through a per-warp shared staging buffer
//    whose segment stride RPT + 16 B keeps both the coalesced side and the
//    per-lane 16-byte side free of bank conflicts.
//  * k_strided (axes y, z): lane = one of 32 neighbouring lines, so every
//    global access is coalesced as it is; the segments of a line are spread
//    over the warps of a CTA and, for long lines, over the CTAs of a thread
//    block cluster.  Carries and halos travel through shared memory and, across
//    the cluster, through distributed shared memory.
#pragma once
#include <cooperative_groups.h>
#include <type_traits>
#include "molt_kernels.cuh"

namespace molt {

namespace cg = cooperative_groups;

// ---------------------------------------------------------------------------
// per-segment arithmetic
// ---------------------------------------------------------------------------
template <class T> struct VecOf;
template <> struct VecOf<float> { using type = float4; static constexpr int n = 4; };
template <> struct VecOf<double> { using type = double2; static constexpr int n = 2; };

// q_k = c1 s_k + c2 (s_{k-1} + s_{k+1}) from a sliding window.  MODE 0: z
// already holds s; MODE 1: s = second difference of z; MODE 2: s = second
// difference of z + cu r.  zl2, zl1 = z at a-2, a-1; zr0, zr1 = z at a+RPT,
// a+RPT+1 (MODE 0: zl1 = s_{a-1}, zr0 = s_{a+RPT}).  r(k) supplies r at a+k
// for k in [-1, RPT].  Dirichlet ends are handled by the caller: ghost values
// in the halos (end_ghosts) and q = 0 at the end nodes (end_zero).
// RAG (Dirichlet lines whose last point n-1 may sit anywhere): kl = n-1-a is
// the local index of the last point; s_{n-1} is replaced by s_{n-2} in
// q_{n-2} (the one-sided end interpolant) and q = 0 from the last point on.
template <class T, int RPT, int MODE, bool RAG = false, class RF>
__device__ __forceinline__ void seg_make_q(T (&z)[RPT], T zl2, T zl1, T zr0, T zr1, RF r, T cu, T c1, T c2,
                                           int kl = 0)
{
    T sm1, s0, zk, zp1;
    if (MODE == 0) {
        sm1 = zl1;
        s0 = z[0];
    } else {
        zk = z[0];
        zp1 = z[1];
        sm1 = (zk - zl1) - (zl1 - zl2);
        s0 = (zp1 - zk) - (zk - zl1);
        if (MODE == 2) { sm1 += cu * r(-1); s0 += cu * r(0); }
    }
#pragma unroll
    for (int k = 0; k < RPT; ++k) {
        T sp1;
        if (MODE == 0) {
            sp1 = (k + 1 < RPT) ? z[k + 1] : zr0;
        } else {
            const T zp2 = (k + 2 < RPT) ? z[k + 2] : (k + 2 == RPT ? zr0 : zr1);
            sp1 = (zp2 - zp1) - (zp1 - zk);
            if (MODE == 2) sp1 += cu * r(k + 1);
            zk = zp1;
            zp1 = zp2;
        }
        if (RAG) sp1 = (k == kl - 1) ? s0 : sp1;
        z[k] = c1 * s0 + c2 * (sm1 + sp1);
        if (RAG) z[k] = (k < kl) ? z[k] : (T)0;
        sm1 = s0;
        s0 = sp1;
    }
}

// Dirichlet: the one-sided interpolants of the end cells make s_0 = s_1 and
// s_{n-1} = s_{n-2}; with the quadratic-extrapolation ghosts
// z_{-1} = 3 z_0 - 3 z_1 + z_2 and z_n = 3 z_{n-1} - 3 z_{n-2} + z_{n-3}
// the plain second difference gives exactly that.  MODE 0 (z = s, whose ends
// were duplicated when formed) takes the ghost s_{-1} = s_0, s_n = s_{n-1}.
template <class T, int RPT, int MODE>
__device__ __forceinline__ void end_ghosts(const T (&z)[RPT], bool left, bool right, T &zl2, T &zl1, T &zr0, T &zr1)
{
    if (left) {
        zl1 = (MODE == 0) ? z[0] : (T)3 * (z[0] - z[1]) + z[2];
        zl2 = zl1;
    }
    if (right) {
        zr0 = (MODE == 0) ? z[RPT - 1] : (T)3 * (z[RPT - 1] - z[RPT - 2]) + z[RPT - 3];
        zr1 = zr0;
    }
}

// Dirichlet: no interior equation at the end nodes (e = 0 there)
template <class T, int RPT>
__device__ __forceinline__ void end_zero(T (&z)[RPT], bool left, bool right)
{
    if (left) z[0] = 0;
    if (right) z[RPT - 1] = 0;
}

template <class T, int RPT>
__device__ __forceinline__ T seg_fwd_reduce(const T (&q)[RPT], T d)
{
    T E = 0;
#pragma unroll
    for (int k = 0; k < RPT; ++k) E = d * E + q[k];
    return E;
}

// y_k = d y_{k-1} + q_k from y = y_{a-1}; returns ER = sum_k d^k y_k.
// RAG: y = 0 past the last point kl (so that the zero-inflow anti-causal
// value at n-1 is y_{n-1} itself), and ylast = y_{n-1} when kl is local.
template <class T, int RPT, bool RAG = false>
__device__ __forceinline__ T seg_fwd_scan(T (&z)[RPT], T d, T y, int kl = 0, T *ylast = nullptr)
{
    T ER = 0, pw = 1, yl = 0;
#pragma unroll
    for (int k = 0; k < RPT; ++k) {
        y = d * y + z[k];
        const T yo = (!RAG || k <= kl) ? y : (T)0;
        if (RAG) yl = (k == kl) ? y : yl;
        z[k] = yo;
        ER += pw * yo;
        pw *= d;
    }
    if (RAG) *ylast = yl;
    return ER;
}

// e_k = d e_{k+1} + y_k with acc = d e_{a+RPT} on entry.  RAG: the right
// boundary term B' d^{n-1-j} enters at the last point kl as Zr.
template <class T, int RPT, bool RAG = false>
__device__ __forceinline__ void seg_bwd_scan(T (&z)[RPT], T d, T acc, int kl = 0, T Zr = 0)
{
#pragma unroll
    for (int k = RPT - 1; k >= 0; --k) {
        T e = acc + z[k];
        if (RAG) e += (k == kl) ? Zr : (T)0;
        acc = d * e;
        z[k] = e;
    }
}

// Two-chain forms of the three recurrences (segments of RPT >= 16, no
// ragged end): the halves [0, H) and [H, RPT) advance together, which halves
// the length of the dependent chains.  The second half of the causal scan
// starts from y_{H-1} = d^H yin + E1 (E1 = the first half's zero-inflow total
// from the reduction); the first half of the anti-causal scan starts from
// d e_H = d ER2 + d^{RPT-H} acc (ER2 = sum_j d^j y_{H+j} from the causal scan).
template <class T, int RPT>
__device__ __forceinline__ T seg_fwd_reduce2(const T (&q)[RPT], T d, T dH, T &E1)
{
    constexpr int H = RPT / 2;
    T a = 0, b = 0;
#pragma unroll
    for (int k = 0; k < H; ++k) {
        a = d * a + q[k];
        b = d * b + q[H + k];
    }
    E1 = a;
    return dH * a + b;
}

template <class T, int RPT>
__device__ __forceinline__ T seg_fwd_scan2(T (&z)[RPT], T d, T dH, T y, T E1, T &ER2)
{
    constexpr int H = RPT / 2;
    T ya = y, yb = dH * y + E1, ra = 0, rb = 0, pw = 1;
#pragma unroll
    for (int k = 0; k < H; ++k) {
        ya = d * ya + z[k];
        yb = d * yb + z[H + k];
        z[k] = ya;
        z[H + k] = yb;
        ra += pw * ya;
        rb += pw * yb;
        pw *= d;
    }
    ER2 = rb;
    return ra + dH * rb;
}

// dHc = d^{RPT-H}
template <class T, int RPT>
__device__ __forceinline__ void seg_bwd_scan2(T (&z)[RPT], T d, T dHc, T acc, T ER2)
{
    constexpr int H = RPT / 2;
    T accb = acc, acca = d * ER2 + dHc * acc;
#pragma unroll
    for (int k = H - 1; k >= 0; --k) {
        const T eb = accb + z[H + k];
        const T ea = acca + z[k];
        accb = d * eb;
        acca = d * ea;
        z[H + k] = eb;
        z[k] = ea;
    }
}

template <class T, int RPT>
__device__ __forceinline__ void seg_add_left2(T (&z)[RPT], T d, T dH, T w0)
{
    constexpr int H = RPT / 2;
    T wa = w0, wb = w0 * dH;
#pragma unroll
    for (int k = 0; k < H; ++k) {
        z[k] += wa;
        z[H + k] += wb;
        wa *= d;
        wb *= d;
    }
}

// z_k += A' d^{a+k}, given w0 = A' d^a
template <class T, int RPT>
__device__ __forceinline__ void seg_add_left(T (&z)[RPT], T d, T w0)
{
#pragma unroll
    for (int k = 0; k < RPT; ++k) {
        z[k] += w0;
        w0 *= d;
    }
}

// ---------------------------------------------------------------------------
// contiguous axis: one warp per line
// ---------------------------------------------------------------------------
template <class T, int RPT>
struct ContigStage {
    static constexpr int VN = VecOf<T>::n;
    static constexpr int SST = RPT + VN;       // segment stride (elements)
    static constexpr int LINE = 32 * SST;      // one line in the staging layout
    __device__ static int pos(int g) { return (g / RPT) * SST + (g % RPT); }
};

template <class T, int BC, int RPT, bool RAG>
__device__ __forceinline__ void warp_solve(T (&z)[RPT], const AxisDev &A, int lane);

// One application of D on a line held by a warp (lane = segment).  The line
// has n = RPT * (Ld + 1) points; lanes past Ld hold zeros.  RAG (Dirichlet
// only): any n <= 32 RPT; lane Ld = (n-1)/RPT holds the last point.
template <class T, int BC, int RPT, int MODE, bool RAG = false, class RF>
__device__ __forceinline__ void warp_sweep_core(T (&z)[RPT], RF rfun, T cu, const AxisDev &A, int lane)
{
    static_assert(!RAG || BC == BC_DIRICHLET, "ragged lines are Dirichlet lines");
    const int n = A.n;
    const T d = A.cd<T>();
    const int Ld = RAG ? (n - 1) / RPT : n / RPT - 1;
    const bool full = lane <= Ld;
    const int a = lane * RPT;
    const int kl = n - 1 - a;

    // Lanes diverge in the predicated per-lane code; __shfl_sync pairs lanes by
    // mask, not by call site, so the warp is reconverged before every group of
    // shuffles (consecutive sweeps otherwise exchanged values across sweeps).
    __syncwarp();
    T zl1 = __shfl_up_sync(0xffffffffu, z[RPT - 1], 1);
    T zl2 = __shfl_up_sync(0xffffffffu, z[RPT - 2], 1);
    T zr0 = __shfl_down_sync(0xffffffffu, z[0], 1);
    T zr1 = __shfl_down_sync(0xffffffffu, z[1], 1);
    if (BC == BC_PERIODIC) {
        const T w1 = __shfl_sync(0xffffffffu, z[RPT - 1], Ld), w2 = __shfl_sync(0xffffffffu, z[RPT - 2], Ld);
        const T v0 = __shfl_sync(0xffffffffu, z[0], 0), v1 = __shfl_sync(0xffffffffu, z[1], 0);
        zl1 = (lane == 0) ? w1 : zl1;
        zl2 = (lane == 0) ? w2 : zl2;
        zr0 = (lane == Ld) ? v0 : zr0;
        zr1 = (lane == Ld) ? v1 : zr1;
    } else {
        end_ghosts<T, RPT, MODE>(z, lane == 0, !RAG && lane == Ld, zl2, zl1, zr0, zr1);
    }
    const T c1 = A.cc1<T>(), c2 = A.cc2<T>();
    seg_make_q<T, RPT, MODE, RAG>(z, zl2, zl1, zr0, zr1, rfun, cu, c1, c2, kl);
    if (BC == BC_DIRICHLET) end_zero<T, RPT>(z, lane == 0, !RAG && lane == Ld);
#pragma unroll
    for (int k = 0; k < RPT; ++k) z[k] = full ? z[k] : (T)0;
    warp_solve<T, BC, RPT, RAG>(z, A, lane);
}

// The solve of the difference form on a warp's line: z holds q on entry
// (zero past the line) and e on exit, (1 + d^2) e_j - d (e_{j-1} + e_{j+1})
// = q_j with the homogeneous boundary terms (Dirichlet: e = 0 at both end
// nodes; periodic: all images).
template <class T, int BC, int RPT, bool RAG>
__device__ __forceinline__ void warp_solve(T (&z)[RPT], const AxisDev &A, int lane)
{
    const int n = A.n;
    const T d = A.cd<T>();
    const int Ld = RAG ? (n - 1) / RPT : n / RPT - 1;
    const bool full = lane <= Ld;
    const int a = lane * RPT;
    const int kl = n - 1 - a;

    // causal carries: Kogge-Stone over lanes with multipliers d^{RPT 2^k};
    // all shuffles of a group run before any lane-dependent branch
    constexpr bool TWO = !RAG && RPT >= 16;
    const T *dpg = dpow_of<T>(A);
    const T dH = TWO ? dpg[RPT / 2] : (T)0;
    T E1 = 0, ER2 = 0;
    const T E = TWO ? seg_fwd_reduce2<T, RPT>(z, d, dH, E1) : seg_fwd_reduce<T, RPT>(z, d);
    __syncwarp();
    T x = E;
#pragma unroll
    for (int k = 0; k < 5; ++k) {
        const T y = __shfl_up_sync(0xffffffffu, x, 1 << k);
        x = (lane >= (1 << k)) ? x + A.cdm<T>(k) * y : x;
    }
    T yin = __shfl_up_sync(0xffffffffu, x, 1);
    const T tot = __shfl_sync(0xffffffffu, x, Ld);              // zero-inflow y_{n-1}
    yin = (lane == 0) ? (T)0 : yin;
    if (BC == BC_PERIODIC)
        yin += full ? dpg[a] * (tot * A.cinv<T>()) : (T)0;          // images to the left
    yin = full ? yin : (T)0;                                     // lanes past the line stay zero
    T ylast = 0;
    const T ER = TWO ? seg_fwd_scan2<T, RPT>(z, d, dH, yin, E1, ER2) : seg_fwd_scan<T, RPT, RAG>(z, d, yin, kl, &ylast);

    // anti-causal carries
    __syncwarp();
    T xb = ER;
#pragma unroll
    for (int k = 0; k < 5; ++k) {
        const T t = __shfl_down_sync(0xffffffffu, xb, 1 << k);
        xb = (lane + (1 << k) < 32) ? xb + A.cdm<T>(k) * t : xb;
    }
    T exclb = __shfl_down_sync(0xffffffffu, xb, 1);
    const T e00 = __shfl_sync(0xffffffffu, xb, 0);              // zero-inflow e_0
    const T yl = __shfl_sync(0xffffffffu, RAG ? ylast : z[RPT - 1], Ld);   // y_{n-1}
    exclb = (lane == 31) ? (T)0 : exclb;
    T Z, Acoef = 0;
    if (BC == BC_DIRICHLET) {
        const T mu = A.cmu<T>(), inv = A.cinv<T>();
        Acoef = (mu * yl - e00) * inv;
        Z = (mu * e00 - yl) * inv;
    } else {
        Z = d * e00 * A.cinv<T>();
    }
    // B' d^{n-1-j}: through the inflow of every segment that ends before the
    // last point; RAG injects it at the last point itself
    const bool before = RAG ? lane < Ld : full;
    const int ia = full ? a : 0, ib = before ? n - a - RPT : 0;   // table indices in [0, n]
    const T acc = d * exclb + (before ? dpg[ib] * Z : (T)0);
    if constexpr (TWO) seg_bwd_scan2<T, RPT>(z, d, dH, acc, ER2);
    else seg_bwd_scan<T, RPT, RAG>(z, d, acc, kl, Z);
    if (BC == BC_DIRICHLET && full) {
        if constexpr (TWO) seg_add_left2<T, RPT>(z, d, dH, Acoef * dpg[ia]);
        else seg_add_left<T, RPT>(z, d, Acoef * dpg[ia]);
    }
    __syncwarp();
}

// D on the warp's line; MODE 2 takes r from the staging layout in shared memory
template <class T, int BC, int RPT, int MODE>
__device__ __forceinline__ void warp_sweep(T (&z)[RPT], const T *rline, T cu, const AxisDev &A, int lane)
{
    using St = ContigStage<T, RPT>;
    if (MODE == 2) {
        const int n = A.n, a = lane * RPT;
        const T *rs = rline + lane * St::SST;
        const int jl = a == 0 ? (BC == BC_PERIODIC ? n - 1 : 0) : a - 1;
        const int jr = a + RPT >= n ? (BC == BC_PERIODIC ? 0 : n - 1) : a + RPT;
        const T rl = rline[St::pos(min(jl, n - 1))], rr = rline[St::pos(min(jr, n - 1))];
        warp_sweep_core<T, BC, RPT, 2>(z, [&](int k) { return k < 0 ? rl : (k >= RPT ? rr : rs[k]); }, cu, A, lane);
    } else {
        warp_sweep_core<T, BC, RPT, MODE>(z, [&](int) { return (T)0; }, (T)0, A, lane);
    }
}

// D on the warp's line, MODE 2 with r held in registers (segment layout)
template <class T, int BC, int RPT, bool RAG = false>
__device__ __forceinline__ void warp_sweep_rreg(T (&z)[RPT], const T (&r)[RPT], T cu, const AxisDev &A, int lane)
{
    const int n = A.n;
    const int Ld = RAG ? (n - 1) / RPT : n / RPT - 1;
    __syncwarp();
    T rl = __shfl_up_sync(0xffffffffu, r[RPT - 1], 1);
    T rr = __shfl_down_sync(0xffffffffu, r[0], 1);
    const T wl = __shfl_sync(0xffffffffu, r[RPT - 1], Ld), wr = __shfl_sync(0xffffffffu, r[0], 0);
    if (BC == BC_PERIODIC) {
        rl = (lane == 0) ? wl : rl;
        rr = (lane == Ld) ? wr : rr;
    }
    warp_sweep_core<T, BC, RPT, 2, RAG>(z, [&](int k) { return k < 0 ? rl : (k >= RPT ? rr : r[k]); }, cu, A, lane);
}

// ---------------------------------------------------------------------------
// Transpose of D (Dirichlet).  In the difference form D = S C Delta: Delta the
// second difference with the end rows duplicated (s_0 = s_1, s_{n-1} =
// s_{n-2}), C the stencil q_j = c1 s_j + c2 (s_{j-1} + s_{j+1}) on the interior
// rows, S the solve with e = 0 at both end nodes.  S is symmetric (the
// interior system is symmetric Toeplitz and the end rows and columns are
// dropped), so D^T w = Delta^T C^T S w: the same solve on w with its end values
// dropped, then t = c1 e + c2 (e_{j-1} + e_{j+1}) (e zero outside the interior),
// the end rows folded in (t'_1 = t_1 + t_0, t'_{n-2} = t_{n-2} + t_{n-1} with
// t_0 = c2 e_1, t_{n-1} = c2 e_{n-2}; t' = 0 at and past the ends), and the
// second difference of t'.
// ---------------------------------------------------------------------------
// z <- second difference of t' on a segment [a, a + RPT), given e there and
// its halos e_{a-2}, e_{a-1}, e_{a+RPT}, e_{a+RPT+1}.  EDGE: the segment may
// touch an end of the line (else t' = t throughout).
template <class T, int RPT, bool EDGE>
__device__ __forceinline__ void post_T(T (&z)[RPT], T el2, T el1, T er0, T er1, T c1, T c2, int a, int n)
{
    auto E = [&](int k) -> T {
        return k < 0 ? (k == -1 ? el1 : el2) : (k >= RPT ? (k == RPT ? er0 : er1) : z[(k >= 0 && k < RPT) ? k : 0]);
    };
    auto tp = [&](int k) -> T {
        const T ek = E(k);
        T t = c1 * ek + c2 * (E(k - 1) + E(k + 1));
        if (EDGE) {
            const int j = a + k;
            t += ((j == 1) ? c2 * ek : (T)0) + ((j == n - 2) ? c2 * ek : (T)0);
            t = (j >= 1 && j <= n - 2) ? t : (T)0;
        }
        return t;
    };
    T tm = tp(-1), t0 = tp(0);
#pragma unroll
    for (int k = 0; k < RPT; ++k) {
        const T tn = tp(k + 1);          // reads e at k .. k+2: z[k] is still e here
        z[k] = (tn - t0) - (t0 - tm);
        tm = t0;
        t0 = tn;
    }
}

// D^T (z + cu u) on the warp's line (any n <= 32 RPT; lane = segment)
template <class T, int RPT>
__device__ __forceinline__ void warp_sweep_T(T (&z)[RPT], const T (&u)[RPT], T cu, const AxisDev &A, int lane)
{
    const int n = A.n, a = lane * RPT, kl = n - 1 - a;
#pragma unroll
    for (int k = 0; k < RPT; ++k) {
        const T q = z[k] + cu * u[k];
        z[k] = (k < kl && (lane > 0 || k > 0)) ? q : (T)0;     // interior rows only
    }
    warp_solve<T, BC_DIRICHLET, RPT, true>(z, A, lane);
#pragma unroll
    for (int k = 0; k < RPT; ++k) z[k] = (k < kl && (lane > 0 || k > 0)) ? z[k] : (T)0;
    __syncwarp();
    T el2 = __shfl_up_sync(0xffffffffu, z[RPT - 2], 1), el1 = __shfl_up_sync(0xffffffffu, z[RPT - 1], 1);
    T er0 = __shfl_down_sync(0xffffffffu, z[0], 1), er1 = __shfl_down_sync(0xffffffffu, z[1], 1);
    el2 = (lane == 0) ? (T)0 : el2;
    el1 = (lane == 0) ? (T)0 : el1;
    er0 = (lane == 31) ? (T)0 : er0;
    er1 = (lane == 31) ? (T)0 : er1;
    post_T<T, RPT, true>(z, el2, el1, er0, er1, A.cc1<T>(), A.cc2<T>(), a, n);
    __syncwarp();
}

// stage (coalesced side) -> registers (segment side)
template <class T, int RPT>
__device__ __forceinline__ void stage_to_regs(const T *st, T (&z)[RPT], int lane, bool add)
{
    using V = typename VecOf<T>::type;
    constexpr int VN = VecOf<T>::n;
    const V *p = reinterpret_cast<const V *>(st + lane * ContigStage<T, RPT>::SST);
#pragma unroll
    for (int q = 0; q < RPT / VN; ++q) {
        V v = p[q];
        const T *e = reinterpret_cast<const T *>(&v);
#pragma unroll
        for (int c = 0; c < VN; ++c) z[q * VN + c] = add ? z[q * VN + c] + e[c] : e[c];
    }
}

template <class T, int RPT>
__device__ __forceinline__ void regs_to_stage(T *st, const T (&z)[RPT], int lane)
{
    using V = typename VecOf<T>::type;
    constexpr int VN = VecOf<T>::n;
    V *p = reinterpret_cast<V *>(st + lane * ContigStage<T, RPT>::SST);
#pragma unroll
    for (int q = 0; q < RPT / VN; ++q) {
        V v;
        T *e = reinterpret_cast<T *>(&v);
#pragma unroll
        for (int c = 0; c < VN; ++c) e[c] = z[q * VN + c];
        p[q] = v;
    }
}

// next time level of a vector of VN consecutive elements starting at i:
// u_next = ea u + eb u_prev + ec F
__device__ __forceinline__ void level_vec(const ProgParams &p, int64_t i, const float4 &F)
{
    const float4 uh = *reinterpret_cast<const float4 *>((const float *)p.u_hi + i);
    const float4 ul = *reinterpret_cast<const float4 *>((const float *)p.u_lo + i);
    float4 ph = make_float4(0.f, 0.f, 0.f, 0.f), pl = ph;
    if (p.feb != 0.f) {
        ph = *reinterpret_cast<const float4 *>((const float *)p.up_hi + i);
        pl = *reinterpret_cast<const float4 *>((const float *)p.up_lo + i);
    }
    const float ea = p.fea, eb = p.feb, ec = p.fec;
    float4 nh, nl;
    level_pair(uh.x, ul.x, ph.x, pl.x, F.x, ea, eb, ec, nh.x, nl.x);
    level_pair(uh.y, ul.y, ph.y, pl.y, F.y, ea, eb, ec, nh.y, nl.y);
    level_pair(uh.z, ul.z, ph.z, pl.z, F.z, ea, eb, ec, nh.z, nl.z);
    level_pair(uh.w, ul.w, ph.w, pl.w, F.w, ea, eb, ec, nh.w, nl.w);
    *reinterpret_cast<float4 *>((float *)p.un_hi + i) = nh;
    *reinterpret_cast<float4 *>((float *)p.un_lo + i) = nl;
}
__device__ __forceinline__ void level_vec(const ProgParams &p, int64_t i, const double2 &F)
{
    const double2 u = *reinterpret_cast<const double2 *>((const double *)p.u_hi + i);
    double2 v;
    v.x = p.ea * u.x + p.ec * F.x;
    v.y = p.ea * u.y + p.ec * F.y;
    if (p.feb != 0.f) {
        const double2 q = *reinterpret_cast<const double2 *>((const double *)p.up_hi + i);
        v.x += p.eb * q.x;
        v.y += p.eb * q.y;
    }
    *reinterpret_cast<double2 *>((double *)p.un_hi + i) = v;
}

// level combination of CH vectors per thread (v = lane + NT (i0 + i) with NT
// threads over the row), all loads issued before any store
template <class T, int CH, int NT = 32> struct LevelBatch;
template <int CH, int NT> struct LevelBatch<float, CH, NT> {
    __device__ static void run(const ProgParams &p, int64_t base, int lane, int i0, int nvec, const float4 (&F)[CH])
    {
        const float4 *__restrict__ UH = reinterpret_cast<const float4 *>((const float *)p.u_hi + base);
        const float4 *__restrict__ UL = reinterpret_cast<const float4 *>((const float *)p.u_lo + base);
        const float4 *__restrict__ PH = reinterpret_cast<const float4 *>((const float *)p.up_hi + base);
        const float4 *__restrict__ PL = reinterpret_cast<const float4 *>((const float *)p.up_lo + base);
        float4 uh[CH], ul[CH], ph[CH], pl[CH];
        const bool prev = p.feb != 0.f;
#pragma unroll
        for (int i = 0; i < CH; ++i) {
            const int v = lane + NT * (i0 + i);
            if (v < nvec) {
                uh[i] = __ldg(UH + v);
                ul[i] = __ldg(UL + v);
                ph[i] = prev ? __ldg(PH + v) : make_float4(0.f, 0.f, 0.f, 0.f);
                pl[i] = prev ? __ldg(PL + v) : make_float4(0.f, 0.f, 0.f, 0.f);
            }
        }
        const float ea = p.fea, eb = p.feb, ec = p.fec;
        float4 *NH = reinterpret_cast<float4 *>((float *)p.un_hi + base);
        float4 *NL = reinterpret_cast<float4 *>((float *)p.un_lo + base);
#pragma unroll
        for (int i = 0; i < CH; ++i) {
            const int v = lane + NT * (i0 + i);
            if (v < nvec) {
                float4 nh, nl;
                level_pair(uh[i].x, ul[i].x, ph[i].x, pl[i].x, F[i].x, ea, eb, ec, nh.x, nl.x);
                level_pair(uh[i].y, ul[i].y, ph[i].y, pl[i].y, F[i].y, ea, eb, ec, nh.y, nl.y);
                level_pair(uh[i].z, ul[i].z, ph[i].z, pl[i].z, F[i].z, ea, eb, ec, nh.z, nl.z);
                level_pair(uh[i].w, ul[i].w, ph[i].w, pl[i].w, F[i].w, ea, eb, ec, nh.w, nl.w);
                NH[v] = nh;
                NL[v] = nl;
            }
        }
    }
};
template <int CH, int NT> struct LevelBatch<double, CH, NT> {
    __device__ static void run(const ProgParams &p, int64_t base, int lane, int i0, int nvec, const double2 (&F)[CH])
    {
        const double2 *__restrict__ U = reinterpret_cast<const double2 *>((const double *)p.u_hi + base);
        const double2 *__restrict__ Q = reinterpret_cast<const double2 *>((const double *)p.up_hi + base);
        double2 u[CH], q[CH];
        const bool prev = p.eb != 0.0;
#pragma unroll
        for (int i = 0; i < CH; ++i) {
            const int v = lane + NT * (i0 + i);
            if (v < nvec) {
                u[i] = __ldg(U + v);
                q[i] = prev ? __ldg(Q + v) : make_double2(0.0, 0.0);
            }
        }
        double2 *N = reinterpret_cast<double2 *>((double *)p.un_hi + base);
#pragma unroll
        for (int i = 0; i < CH; ++i) {
            const int v = lane + NT * (i0 + i);
            if (v < nvec) {
                double2 r;
                r.x = p.ea * u[i].x + p.ec * F[i].x + p.eb * q[i].x;
                r.y = p.ea * u[i].y + p.ec * F[i].y + p.eb * q[i].y;
                N[v] = r;
            }
        }
    }
};
template <class T, int CH, int NT = 32, class V>
__device__ __forceinline__ void level_batch(const ProgParams &p, int64_t base, int lane, int i0, int nvec, const V (&F)[CH])
{
    LevelBatch<T, CH, NT>::run(p, base, lane, i0, nvec, F);
}

template <class V> __device__ __forceinline__ V vfma(typename std::remove_reference<decltype(V().x)>::type c, const V &a, const V &b);
template <> __device__ __forceinline__ float4 vfma<float4>(float c, const float4 &a, const float4 &b)
{
    return make_float4(b.x + c * a.x, b.y + c * a.y, b.z + c * a.z, b.w + c * a.w);
}
template <> __device__ __forceinline__ double2 vfma<double2>(double c, const double2 &a, const double2 &b)
{
    return make_double2(b.x + c * a.x, b.y + c * a.y);
}

// Coalesced side of the staging buffer: a lane covers vectors of VN
// consecutive elements g = VN*(lane + 32 i).  Segment boundaries are
// multiples of RPT (a multiple of VN), so a vector never straddles two
// segments and sits 16-byte aligned at pos(g).
template <class T, int RPT>
struct CoalescedSide {
    using V = typename VecOf<T>::type;
    static constexpr int VN = VecOf<T>::n;
    static constexpr int NV = RPT;                 // vectors per lane in a full line (32*RPT/(32*VN)*VN)
    __device__ static V *at(T *st, int g) { return reinterpret_cast<V *>(st + ContigStage<T, RPT>::pos(g)); }
};

// stage <- stage + sum_k coef[k] g_k[base + .] over the line (coalesced),
// one pass per field with a non-zero weight; every lane first issues all the
// loads of its share of the row (up to RPT/VN vectors) so that they are in
// flight together, then accumulates.
template <class T, int RPT>
__device__ __forceinline__ void stage_accumulate(T *stage, const ProgParams &pr, size_t cf, int64_t base, int n,
                                                 int lane)
{
    using V = typename VecOf<T>::type;
    constexpr int VN = VecOf<T>::n;
    constexpr int NV = RPT / VN;                    // vectors per lane (n <= 32*RPT)
    const int nvec = n / VN;                        // n is a multiple of RPT, hence of VN
    for (int k = 0; k < pr.ng; ++k) {
        const T ck = prog_coef<T>(pr, cf + k);
        if (ck == (T)0) continue;
        const V *__restrict__ src = reinterpret_cast<const V *>(reinterpret_cast<const T *>(pr.g[k]) + base);
        V buf[NV];
#pragma unroll
        for (int i = 0; i < NV; ++i) {
            const int v = lane + 32 * i;
            if (v < nvec) buf[i] = __ldg(src + v);
        }
#pragma unroll
        for (int i = 0; i < NV; ++i) {
            const int v = lane + 32 * i;
            if (v < nvec) {
                V *d = CoalescedSide<T, RPT>::at(stage, v * VN);
                *d = vfma<V>(ck, buf[i], *d);
            }
        }
    }
}

// r = accurate second difference of u along the line, formed in the segment
// layout from u staged in shared memory (hi plane in `stage`, lo in `rline`
// for float32 pairs); result left in z and written to rline.
template <class T, int BC, int RPT>
__device__ __forceinline__ void contig_r(T (&z)[RPT], T *stage, T *rline, const ProgParams &pr, int64_t base, int n,
                                         int lane)
{
    using St = ContigStage<T, RPT>;
    using V = typename VecOf<T>::type;
    constexpr int VN = VecOf<T>::n;
    const int nvec = n / VN;
    const bool pair = sizeof(T) == 4;
    constexpr int NV = RPT / VN;
    {
        const V *__restrict__ H = reinterpret_cast<const V *>(reinterpret_cast<const T *>(pr.u_hi) + base);
        V buf[NV];
#pragma unroll
        for (int i = 0; i < NV; ++i) if (lane + 32 * i < nvec) buf[i] = __ldg(H + lane + 32 * i);
#pragma unroll
        for (int i = 0; i < NV; ++i) if (lane + 32 * i < nvec) *CoalescedSide<T, RPT>::at(stage, (lane + 32 * i) * VN) = buf[i];
    }
    if (pair) {
        const V *__restrict__ Lo = reinterpret_cast<const V *>(reinterpret_cast<const T *>(pr.u_lo) + base);
        V buf[NV];
#pragma unroll
        for (int i = 0; i < NV; ++i) if (lane + 32 * i < nvec) buf[i] = __ldg(Lo + lane + 32 * i);
#pragma unroll
        for (int i = 0; i < NV; ++i) if (lane + 32 * i < nvec) *CoalescedSide<T, RPT>::at(rline, (lane + 32 * i) * VN) = buf[i];
    }
    __syncwarp();
    const int a = lane * RPT;
    const int Ld = n / RPT - 1;
    const bool full = lane <= Ld;
    auto wrapc = [&](int j) { return BC == BC_PERIODIC ? (j < 0 ? j + n : (j >= n ? j - n : j)) : min(max(j, 0), n - 1); };
    const int jl = wrapc(a - 1), jr = wrapc(a + RPT);
    // hi part
    stage_to_regs<T, RPT>(stage, z, lane, false);
    {
        T hm = stage[St::pos(jl)], hp = stage[St::pos(jr)];
        T prev = hm, cur = z[0];
#pragma unroll
        for (int k = 0; k < RPT; ++k) {
            const T next = (k + 1 < RPT) ? z[k + 1] : hp;
            const T sd = (next - cur) - (cur - prev);
            prev = cur;
            cur = next;
            z[k] = sd;
        }
    }
    if (pair) {
        // lo part straight from shared memory (keeps register use at one line)
        const T *ls = rline + lane * St::SST;
        T prev = rline[St::pos(jl)], cur = ls[0];
        const T lp = rline[St::pos(jr)];
#pragma unroll
        for (int k = 0; k < RPT; ++k) {
            const T next = (k + 1 < RPT) ? ls[k + 1] : lp;
            const T sd = (next - cur) - (cur - prev);
            prev = cur;
            cur = next;
            z[k] = z[k] + sd;
        }
    }
    if (BC == BC_DIRICHLET) {          // end nodes take the neighbouring interior centre
        if (lane == 0) z[0] = z[1];
        if (lane == Ld) z[RPT - 1] = z[RPT - 2];
    }
    if (!full) {
#pragma unroll
        for (int k = 0; k < RPT; ++k) z[k] = 0;
    }
    __syncwarp();
    regs_to_stage<T, RPT>(rline, z, lane);
    __syncwarp();
}

template <class T, int BC, int RPT, int WARPS>
__global__ void __launch_bounds__(32 * WARPS, 3) k_contig(AxisDev A, LineSet LS, ProgParams pr)
{
    pdl_enter();
    static_assert(RPT >= 4 && RPT % VecOf<T>::n == 0, "segment length");
    using St = ContigStage<T, RPT>;
    using V = typename VecOf<T>::type;
    constexpr int VN = VecOf<T>::n;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    T *stage = reinterpret_cast<T *>(smem_raw) + (size_t)warp * 2 * St::LINE;
    T *rline = stage + St::LINE;
    const int n = A.n;
    const int64_t L = (int64_t)blockIdx.x * WARPS + warp;
    if (L >= LS.nlines) return;
    const int64_t base = L * (int64_t)n;   // contiguous axis
    const int nvec = n / VN;

    T z[RPT];
    contig_r<T, BC, RPT>(z, stage, rline, pr, base, n, lane);

    if (pr.mode == 0) {
        // powers: the first sweep starts from s = r
        for (int p = 1; p <= pr.P; ++p) {
            if (p == 1) warp_sweep<T, BC, RPT, 0>(z, rline, (T)0, A, lane);
            else warp_sweep<T, BC, RPT, 1>(z, rline, (T)0, A, lane);
            if (pr.out[p - 1] != nullptr) {
                regs_to_stage<T, RPT>(stage, z, lane);
                __syncwarp();
                V *o = reinterpret_cast<V *>(reinterpret_cast<T *>(pr.out[p - 1]) + base);
#pragma unroll 4
                for (int v = lane; v < nvec; v += 32) o[v] = *CoalescedSide<T, RPT>::at(stage, v * VN);
                __syncwarp();
            }
        }
        return;
    }
    const int P = pr.P, ng = pr.ng;
#pragma unroll
    for (int k = 0; k < RPT; ++k) z[k] = 0;
    for (int t = P; t >= 0; --t) {
        if (ng > 0 || t == 0) {
            regs_to_stage<T, RPT>(stage, z, lane);
            __syncwarp();
            if (ng > 0) stage_accumulate<T, RPT>(stage, pr, (size_t)t * ng, base, n, lane);
            __syncwarp();
            if (t == 0) break;
            stage_to_regs<T, RPT>(stage, z, lane, false);
            __syncwarp();
        }
        warp_sweep<T, BC, RPT, 2>(z, rline, prog_cu<T>(pr, t), A, lane);
    }
    // out = stage (coalesced side): level combination or plain store
    if (pr.epi) {
        constexpr int NV = RPT / VN;
        constexpr int CH = NV > 4 ? 4 : NV;          // vectors per lane per batch
#pragma unroll
        for (int i0 = 0; i0 < NV; i0 += CH) {
            V F[CH];
#pragma unroll
            for (int i = 0; i < CH; ++i) {
                const int v = lane + 32 * (i0 + i);
                if (v < nvec) F[i] = *CoalescedSide<T, RPT>::at(stage, v * VN);
            }
            level_batch<T, CH>(pr, base, lane, i0, nvec, F);
        }
    } else {
        V *o = reinterpret_cast<V *>(reinterpret_cast<T *>(pr.out[0]) + base);
#pragma unroll 4
        for (int v = lane; v < nvec; v += 32) o[v] = *CoalescedSide<T, RPT>::at(stage, v * VN);
    }
}

// ---------------------------------------------------------------------------
// contiguous axis, float32 Horner pass with the input fields resident
// ---------------------------------------------------------------------------
// Each warp copies the NG input rows of its line into shared memory once,
// with cp.async (16-byte pieces, coalesced global side, padded segment
// layout in shared memory), while it forms r = second difference of u in
// registers from coalesced 16-byte loads.  All Horner steps then read the
// fields from shared memory: a row costs a handful of memory round trips
// instead of one per field and step.
__device__ __forceinline__ void cp_async16(void *smem_dst, const void *gsrc)
{
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem_dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }

// Bulk prefetch of [p, p + bytes) into L2 (16-byte aligned, bytes a multiple
// of 16): the level rows the epilogue reads long after the row starts are
// fetched while the row is being swept, at no register or shared-memory cost.
__device__ __forceinline__ void prefetch_l2(const void *p, unsigned bytes)
{
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;\n" ::"l"(p), "r"(bytes) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// second difference of a pair field at 4 consecutive points, given the
// points left (before .x) and right (after .w)
__device__ __forceinline__ float4 sdiff4(const float4 &h, const float4 &l, float hl, float ll, float hr, float lr)
{
    float4 r;
    r.x = sdiff_pair(hl, h.x, h.y, ll, l.x, l.y);
    r.y = sdiff_pair(h.x, h.y, h.z, l.x, l.y, l.z);
    r.z = sdiff_pair(h.y, h.z, h.w, l.y, l.z, l.w);
    r.w = sdiff_pair(h.z, h.w, hr, l.z, l.w, lr);
    return r;
}

// Up to 4 warps per CTA (the warps per CTA are a launch choice: blockDim.x / 32)
template <int BC, int RPT, int NB>
__global__ void __launch_bounds__(128) k_contig_res(AxisDev A, LineSet LS, ProgParams pr)
{
    pdl_enter();
    static_assert(RPT % 4 == 0 && RPT >= 8, "segment length");
    using T = float;
    using St = ContigStage<T, RPT>;
    constexpr int NVL = RPT / 4;                 // vectors per lane when n = 32*RPT
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    T *B = reinterpret_cast<T *>(smem_raw) + (size_t)warp * NB * St::LINE;   // NB field buffers
    T *R = B;                                    // staging for r before field 0 lands there
    const int n = A.n;
    const int64_t L = (int64_t)blockIdx.x * (blockDim.x >> 5) + warp;
    if (L >= LS.nlines) return;
    const int64_t base = L * (int64_t)n;
    const int nvec = n / 4;
    const int ng = pr.ng;
    if (lane == 0) {
        const unsigned bytes = (unsigned)n * 4u;          // n is a multiple of RPT >= 8
        prefetch_l2((const float *)pr.u_hi + base, bytes);
        prefetch_l2((const float *)pr.u_lo + base, bytes);
        if (pr.feb != 0.f) {
            prefetch_l2((const float *)pr.up_hi + base, bytes);
            prefetch_l2((const float *)pr.up_lo + base, bytes);
        }
    }

    // 1. fields 1..ng-1 -> shared memory (asynchronous); field 0 after r
    auto copy_field = [&](int k) {
        const float4 *src = reinterpret_cast<const float4 *>(reinterpret_cast<const T *>(pr.g[k]) + base);
        T *dst = B + k * St::LINE;
#pragma unroll
        for (int i = 0; i < NVL; ++i) {
            const int v = lane + 32 * i;
            if (v < nvec) cp_async16(dst + St::pos(4 * v), src + v);
        }
    };
    for (int k = 1; k < ng; ++k) copy_field(k);
    cp_async_commit();

    // 2. r = second difference of u (pair levels), coalesced, into R; every
    //    load of the row (and of the points just past each 128-point chunk)
    //    is issued before any is used
    {
        const T *H = reinterpret_cast<const T *>(pr.u_hi) + base, *Lo = reinterpret_cast<const T *>(pr.u_lo) + base;
        const float4 *H4 = reinterpret_cast<const float4 *>(H), *L4 = reinterpret_cast<const float4 *>(Lo);
        float4 h[NVL], l[NVL];
        float hx[NVL], lx[NVL];        // lane 0: point before the chunk; lane 31: point after it
#pragma unroll
        for (int i = 0; i < NVL; ++i) {
            const int v = lane + 32 * i;
            if (v < nvec) { h[i] = __ldg(H4 + v); l[i] = __ldg(L4 + v); }
            else { h[i] = make_float4(0.f, 0.f, 0.f, 0.f); l[i] = h[i]; }
            int j = (lane == 0) ? 4 * v - 1 : 4 * v + 4;
            if (BC == BC_PERIODIC) j = j < 0 ? j + n : (j >= n ? j - n : j);
            else j = j < 0 ? 0 : (j > n - 1 ? n - 1 : j);
            hx[i] = 0.f; lx[i] = 0.f;
            if ((lane == 0 || lane == 31) && v < nvec) { hx[i] = __ldg(H + j); lx[i] = __ldg(Lo + j); }
        }
#pragma unroll
        for (int i = 0; i < NVL; ++i) {
            const int v = lane + 32 * i;
            float hl = __shfl_up_sync(0xffffffffu, h[i].w, 1), ll = __shfl_up_sync(0xffffffffu, l[i].w, 1);
            float hr = __shfl_down_sync(0xffffffffu, h[i].x, 1), lr = __shfl_down_sync(0xffffffffu, l[i].x, 1);
            const int g0 = 4 * v;
            // the last vector of the line may sit in any lane: its right neighbour is past the line
            const bool last = (g0 + 4 == n);
            if (lane == 0) { hl = hx[i]; ll = lx[i]; }
            if (lane == 31) { hr = hx[i]; lr = lx[i]; }
            if (last && lane != 31) {
                const int j = (BC == BC_PERIODIC) ? 0 : n - 1;
                hr = H[j]; lr = Lo[j];
            }
            if (v < nvec) {
                float4 r = sdiff4(h[i], l[i], hl, ll, hr, lr);
                if (BC == BC_DIRICHLET) {            // end nodes take the neighbouring interior centre
                    if (g0 == 0) r.x = r.y;
                    if (last) r.w = r.z;
                }
                *reinterpret_cast<float4 *>(R + St::pos(g0)) = r;
            }
        }
        __syncwarp();
    }
    // r to registers (segment layout); then field 0 may overwrite the staging
    T r[RPT];
    stage_to_regs<T, RPT>(R, r, lane, false);
    __syncwarp();
    if (ng > 0) copy_field(0);
    cp_async_commit();
    cp_async_wait_all();
    __syncwarp();

    // 3. Horner in D_x with the fields from shared memory
    const int P = pr.P;
    T z[RPT];
#pragma unroll
    for (int k = 0; k < RPT; ++k) z[k] = 0;
    for (int t = P; t >= 0; --t) {
        for (int k = 0; k < ng; ++k) {
            const T c = prog_coef<T>(pr, (size_t)t * ng + k);
            if (c == (T)0) continue;
            const float4 *seg = reinterpret_cast<const float4 *>(B + k * St::LINE + lane * St::SST);
#pragma unroll
            for (int q = 0; q < RPT / 4; ++q) {
                const float4 y = seg[q];
                z[4 * q] += c * y.x;
                z[4 * q + 1] += c * y.y;
                z[4 * q + 2] += c * y.z;
                z[4 * q + 3] += c * y.w;
            }
        }
        if (t == 0) break;
        warp_sweep_rreg<T, BC, RPT>(z, r, prog_cu<T>(pr, t), A, lane);
    }

    // 4. F (segment layout) -> coalesced side -> next level
    T *S0 = B;                                   // the first buffer is free now
    __syncwarp();
    regs_to_stage<T, RPT>(S0, z, lane);
    __syncwarp();
    if (pr.epi) {
        constexpr int CH = NVL > 8 ? 8 : NVL;
#pragma unroll
        for (int i0 = 0; i0 < NVL; i0 += CH) {
            float4 F[CH];
#pragma unroll
            for (int i = 0; i < CH; ++i) {
                const int v = lane + 32 * (i0 + i);
                if (v < nvec) F[i] = *CoalescedSide<T, RPT>::at(S0, v * 4);
            }
            level_batch<T, CH>(pr, base, lane, i0, nvec, F);
        }
    } else {
        float4 *o = reinterpret_cast<float4 *>(reinterpret_cast<T *>(pr.out[0]) + base);
#pragma unroll 4
        for (int v = lane; v < nvec; v += 32) o[v] = *CoalescedSide<T, RPT>::at(S0, v * 4);
    }
}

// ---------------------------------------------------------------------------
// contiguous axis, float32 Horner pass, one row per CTA of W warps
// ---------------------------------------------------------------------------
// one neighbour exchange per sweep (molt_strided_nb.cuh explains the algebra)
// ---------------------------------------------------------------------------
// Constants of the neighbour exchange, float32 copies of float64 values:
// G = d sum_{j<RPT} d^2j, G1 = d^2 sum_{j<RPT-1} d^2j, GH = d sum_{j<H} d^2j,
// dH = d^H, dH1 = d^(H-1) with H = RPT/2.
struct NbConsts {
    float G, G1, GH, dH, dH1;
    float dR, dR1, dR2, dRp1;   // d^RPT, d^(RPT-1), d^(RPT-2), d^(RPT+1) (two-hop exchange)
};

// True when the neighbour exchange is exact to well below float32 rounding
// for a line of n points with segments of rpt points and decay d.
inline bool strided_nb_exact(double d, int n, int rpt, int log2_limit = 30)
{
    if (rpt < 4 || n % rpt != 0 || n / rpt < 2) return false;
    return std::pow(d, (double)(rpt - 1)) <= std::ldexp(1.0, -log2_limit);
}

inline NbConsts strided_nb_consts(double d, int rpt)
{
    const int H = rpt / 2;
    double g = 0.0, g1 = 0.0, gh = 0.0, p = 1.0;
    for (int j = 0; j < rpt; ++j) {
        if (j < rpt - 1) g1 += p;
        if (j < H) gh += p;
        g += p;
        p *= d * d;
    }
    NbConsts c;
    c.G = (float)(d * g);
    c.G1 = (float)(d * d * g1);
    c.GH = (float)(d * gh);
    c.dH = (float)std::pow(d, (double)H);
    c.dH1 = (float)std::pow(d, (double)(H - 1));
    c.dR = (float)std::pow(d, (double)rpt);
    c.dR1 = (float)std::pow(d, (double)(rpt - 1));
    c.dR2 = (float)std::pow(d, (double)(rpt - 2));
    c.dRp1 = (float)std::pow(d, (double)(rpt + 1));
    return c;
}

// ---------------------------------------------------------------------------
// A row of n = 32 W RPT points is split over the W warps of a CTA: warp w holds
// points [32 w RPT, 32 (w+1) RPT), lane = segment of RPT points.  Each warp
// runs the single-warp sweep on its part; halos and the causal and anti-causal
// carries between the warps of the row pass through a few shared-memory slots
// (three CTA barriers per sweep).  A row then costs about 1/W of the
// single-warp latency, and the shorter segments need fewer registers, so more
// rows are in flight per SM.
template <class T, int W>
struct RowSlots {
    T halo[W][4];    // per warp: z at its first two and last two points
    T rhalo[W][2];   // per warp: r at its first and last point
    T tc[W];         // per warp: zero-inflow causal total (y at its last point)
    T ta[W];         // per warp: zero-inflow anti-causal total (e at its first point)
    T yl;            // y_{n-1} of the row with zero inflow
    T nb[2][W][8];   // neighbour exchange, per warp (two sets, alternating by sweep): lane 31's
                     // E, y0(RPT-2); lane 0's ER0, ER1; two hops also lane 30's E, lane 0's E,
                     // lane 1's ER0
};

// Neighbours of the thread's segment: z at a-2, a-1 (left) and a+RPT,
// a+RPT+1 (right), by shuffles inside the warp and through shared memory
// across warps.  WRAP: the row's ends see each other (periodic); else the
// outer halos of the row are left as the shuffles give them (the caller
// replaces them).
template <class T, int RPT, int W, bool WRAP>
__device__ __forceinline__ void row_halos(const T (&z)[RPT], int lane, int warp, RowSlots<T, W> &sl, T &zl2, T &zl1,
                                          T &zr0, T &zr1)
{
    __syncwarp();
    zl1 = __shfl_up_sync(0xffffffffu, z[RPT - 1], 1);
    zl2 = __shfl_up_sync(0xffffffffu, z[RPT - 2], 1);
    zr0 = __shfl_down_sync(0xffffffffu, z[0], 1);
    zr1 = __shfl_down_sync(0xffffffffu, z[1], 1);
    if (lane == 0) { sl.halo[warp][0] = z[0]; sl.halo[warp][1] = z[1]; }
    if (lane == 31) { sl.halo[warp][2] = z[RPT - 2]; sl.halo[warp][3] = z[RPT - 1]; }
    __syncthreads();
    if (lane == 0 && (warp > 0 || WRAP)) {
        const int wl = warp > 0 ? warp - 1 : W - 1;
        zl2 = sl.halo[wl][2];
        zl1 = sl.halo[wl][3];
    }
    if (lane == 31 && (warp < W - 1 || WRAP)) {
        const int wr = warp < W - 1 ? warp + 1 : 0;
        zr0 = sl.halo[wr][0];
        zr1 = sl.halo[wr][1];
    }
}

// The solve of the difference form on a row held by the W warps of a CTA
// (thread 32 warp + lane owns segment a = (32 warp + lane) RPT): z holds q on
// entry (zero past the row) and e on exit.  Carries: Kogge-Stone inside each
// warp, then a short serial pass over the W warp totals in shared memory.
// RAG (Dirichlet): the row's last point n-1 may sit anywhere in the last warp
// (n > 32 (W-1) RPT); the segment routines' ragged variants handle it.
template <class T, int BC, int RPT, int W, bool RAG>
__device__ __forceinline__ void row_solve(T (&z)[RPT], const AxisDev &A, int lane, int warp, RowSlots<T, W> &sl)
{
    static_assert(!RAG || BC == BC_DIRICHLET, "ragged rows are Dirichlet rows");
    const int n = A.n;
    const T d = A.cd<T>();
    const int seg = warp * 32 + lane, a = seg * RPT;
    const int Ld = RAG ? (n - 1) / RPT : 32 * W - 1;  // segment holding the last point
    const int kl = n - 1 - a;
    const bool full = seg <= Ld;
    const T *dpg = dpow_of<T>(A);

    constexpr bool TWO = !RAG && RPT >= 16;
    const T dH = TWO ? dpg[RPT / 2] : (T)0;
    T E1 = 0, ER2 = 0;
    const T E = TWO ? seg_fwd_reduce2<T, RPT>(z, d, dH, E1) : seg_fwd_reduce<T, RPT>(z, d);
    __syncwarp();
    T x = E;
#pragma unroll
    for (int k = 0; k < 5; ++k) {
        const T y = __shfl_up_sync(0xffffffffu, x, 1 << k);
        x = (lane >= (1 << k)) ? x + A.cdm<T>(k) * y : x;
    }
    T yin = __shfl_up_sync(0xffffffffu, x, 1);
    yin = (lane == 0) ? (T)0 : yin;
    if (lane == 31) sl.tc[warp] = x;
    __syncthreads();
    const T DW = dpg[32 * RPT];                      // decay over one warp's points
    T cin = 0, tot = 0;
#pragma unroll
    for (int w2 = 0; w2 < W; ++w2) {
        cin = (w2 == warp) ? tot : cin;
        tot = DW * tot + sl.tc[w2];
    }
    yin += dpg[lane * RPT] * cin;
    if (BC == BC_PERIODIC) yin += dpg[a] * (tot * A.cinv<T>());       // images to the left
    if (RAG) yin = full ? yin : (T)0;
    T ylast = 0;
    const T ER = TWO ? seg_fwd_scan2<T, RPT>(z, d, dH, yin, E1, ER2) : seg_fwd_scan<T, RPT, RAG>(z, d, yin, kl, &ylast);

    // anti-causal carries
    __syncwarp();
    T xb = ER;
#pragma unroll
    for (int k = 0; k < 5; ++k) {
        const T t = __shfl_down_sync(0xffffffffu, xb, 1 << k);
        xb = (lane + (1 << k) < 32) ? xb + A.cdm<T>(k) * t : xb;
    }
    T exclb = __shfl_down_sync(0xffffffffu, xb, 1);
    exclb = (lane == 31) ? (T)0 : exclb;
    if (lane == 0) sl.ta[warp] = xb;
    if (RAG) {
        if (kl >= 0 && kl < RPT) sl.yl = ylast;
    } else if (warp == W - 1 && lane == 31) {
        sl.yl = z[RPT - 1];
    }
    __syncthreads();
    T cinb = 0, e00 = 0;
#pragma unroll
    for (int w2 = W - 1; w2 >= 0; --w2) {
        cinb = (w2 == warp) ? e00 : cinb;
        e00 = DW * e00 + sl.ta[w2];
    }
    exclb += dpg[(31 - lane) * RPT] * cinb;
    T Z, Acoef = 0;
    if (BC == BC_DIRICHLET) {
        const T mu = A.cmu<T>(), inv = A.cinv<T>(), yl = sl.yl;
        Acoef = (mu * yl - e00) * inv;
        Z = (mu * e00 - yl) * inv;
    } else {
        Z = d * e00 * A.cinv<T>();
    }
    // B' d^{n-1-j}: through the inflow of every segment that ends before the
    // last point; RAG injects it at the last point itself
    const bool before = RAG ? seg < Ld : true;
    const T acc = d * exclb + (before ? dpg[before ? n - a - RPT : 0] * Z : (T)0);
    if constexpr (TWO) seg_bwd_scan2<T, RPT>(z, d, dH, acc, ER2);
    else seg_bwd_scan<T, RPT, RAG>(z, d, acc, kl, Z);
    if (BC == BC_DIRICHLET && full) {
        if constexpr (TWO) seg_add_left2<T, RPT>(z, d, dH, Acoef * dpg[a]);
        else seg_add_left<T, RPT>(z, d, Acoef * dpg[a]);
    }
    __syncwarp();
}

// One application of D (MODE 2: z + cu r, r the second difference of u in
// registers with its row neighbours rl, rr) on a row split over W warps
template <class T, int BC, int RPT, int W, bool RAG = false>
__device__ __forceinline__ void row_sweep(T (&z)[RPT], const T (&r)[RPT], T rl, T rr, T cu, const AxisDev &A, int lane,
                                          int warp, RowSlots<T, W> &sl)
{
    const int n = A.n;
    const int seg = warp * 32 + lane, a = seg * RPT;
    const int Ld = RAG ? (n - 1) / RPT : 32 * W - 1;
    const int kl = n - 1 - a;
    const T c1 = A.cc1<T>(), c2 = A.cc2<T>();
    T zl2, zl1, zr0, zr1;
    row_halos<T, RPT, W, BC == BC_PERIODIC>(z, lane, warp, sl, zl2, zl1, zr0, zr1);
    if (BC == BC_DIRICHLET) end_ghosts<T, RPT, 2>(z, seg == 0, !RAG && seg == Ld, zl2, zl1, zr0, zr1);
    seg_make_q<T, RPT, 2, RAG>(z, zl2, zl1, zr0, zr1, [&](int k) { return k < 0 ? rl : (k >= RPT ? rr : r[k]); }, cu,
                               c1, c2, kl);
    if (BC == BC_DIRICHLET) end_zero<T, RPT>(z, seg == 0, !RAG && seg == Ld);
    if (RAG && seg > Ld) {
#pragma unroll
        for (int k = 0; k < RPT; ++k) z[k] = 0;
    }
    row_solve<T, BC, RPT, W, RAG>(z, A, lane, warp, sl);
}

// One application of D (MODE 2: s = the second difference of z plus cu r) on
// a row split over W warps with ONE neighbour exchange: the algebra of
// k_strided_nb (molt_strided_nb.cuh) with the neighbours at lane -+ 1 by
// shuffles and across warps through the slots, one CTA barrier.  For rows
// with d^(RPT-1) <= 2^-27 (the dropped inflows below 1/8 of a float32 unit in
// the last place).  hl2, hl1, hr0, hr1: z at a-2, a-1, a+RPT, a+RPT+1 on
// entry; e there on exit (the caller adds the next Horner term to both).
template <int BC, int RPT, int W>
__device__ __forceinline__ void row_sweep_nb(float (&z)[RPT], const float (&r)[RPT], float rl, float rr, float cu,
                                             const AxisDev &A, const NbConsts &nc, int lane, int warp,
                                             RowSlots<float, W> &sl, int buf, float &hl2, float &hl1, float &hr0,
                                             float &hr1)
{
    constexpr int H = RPT / 2;
    constexpr int NSEG = 32 * W;
    const int seg = warp * 32 + lane;
    const bool left_end = BC == BC_DIRICHLET && seg == 0, right_end = BC == BC_DIRICHLET && seg == NSEG - 1;
    const float d = A.fd, c1 = A.fc1, c2 = A.fc2, inv = A.finv;
    float zl2 = hl2, zl1 = hl1, zr0 = hr0, zr1 = hr1;
    if (BC == BC_DIRICHLET) end_ghosts<float, RPT, 2>(z, left_end, right_end, zl2, zl1, zr0, zr1);
    seg_make_q<float, RPT, 2>(z, zl2, zl1, zr0, zr1, [&](int k) { return k < 0 ? rl : (k >= RPT ? rr : r[k]); }, cu,
                              c1, c2);
    if (BC == BC_DIRICHLET) end_zero<float, RPT>(z, left_end, right_end);

    // both halves of the causal recurrence with zero inflow
    float ya = z[0], yb = z[H], ra1 = 0.f, rb = yb, pw = 1.f;
#pragma unroll
    for (int k = 1; k < H; ++k) {
        ya = d * ya + z[k];
        yb = d * yb + z[H + k];
        z[k] = ya;
        z[H + k] = yb;
        const float pbk = pw * d;
        ra1 += pw * ya;
        rb += pbk * yb;
        pw = pbk;
    }
    const float E1 = ya;
    const float E = yb + E1 * nc.dH;
    const float Y2 = z[RPT - 2] + E1 * nc.dH1;
    const float ER1 = ra1 + nc.dH1 * (rb + E1 * nc.GH);
    const float ER0 = z[0] + d * ER1;

    // the exchange: lane -+ 1 by shuffles, the neighbouring warps' end lanes
    // through the slots
    __syncwarp();
    float EL = __shfl_up_sync(0xffffffffu, E, 1), Y2L = __shfl_up_sync(0xffffffffu, Y2, 1);
    float ER0R = __shfl_down_sync(0xffffffffu, ER0, 1), ER1R = __shfl_down_sync(0xffffffffu, ER1, 1);
    if (lane == 31) { sl.nb[buf][warp][0] = E; sl.nb[buf][warp][1] = Y2; }
    if (lane == 0) { sl.nb[buf][warp][2] = ER0; sl.nb[buf][warp][3] = ER1; }
    __syncthreads();
    if (lane == 0) {
        const int wl = warp > 0 ? warp - 1 : W - 1;
        EL = sl.nb[buf][wl][0];
        Y2L = sl.nb[buf][wl][1];
    }
    if (lane == 31) {
        const int wr = warp < W - 1 ? warp + 1 : 0;
        ER0R = sl.nb[buf][wr][2];
        ER1R = sl.nb[buf][wr][3];
    }
    const bool hasL = !left_end, hasR = !right_end;
    if (!hasL) { EL = 0.f; Y2L = 0.f; }
    if (!hasR) { ER0R = 0.f; ER1R = 0.f; }

    const float cB = E1 + EL * nc.dH;
    float pk = d;
#pragma unroll
    for (int k = 0; k < H; ++k) {
        z[k] += EL * pk;
        z[H + k] += cB * pk;
        pk *= d;
    }
    const float ER2 = rb + cB * nc.GH;
    const float eout = hasR ? ER0R + nc.G * E : 0.f;
    const float er1 = hasR ? ER1R + nc.G1 * E : 0.f;
    float acc = d * eout;
    if (right_end) acc -= z[RPT - 1] * inv;
    seg_bwd_scan2<float, RPT>(z, d, nc.dH, acc, ER2);
    if (left_end) seg_add_left2<float, RPT>(z, d, nc.dH, -z[0] * inv);
    hl1 = hasL ? EL + d * z[0] : 0.f;
    hl2 = hasL ? Y2L + d * hl1 : 0.f;
    hr0 = eout;
    hr1 = er1;
}

// Two hops (segments of 16 points, where d^RPT is not yet negligible but
// d^(2 RPT - 1) <= 2^-27): the inflows from l-1, l-2 and l+1, l+2, the
// Dirichlet corrections reaching into the second segment from each end.
// Same interface as row_sweep_nb.
template <int BC, int RPT, int W>
__device__ __forceinline__ void row_sweep_nb2(float (&z)[RPT], const float (&r)[RPT], float rl, float rr, float cu,
                                              const AxisDev &A, const NbConsts &nc, int lane, int warp,
                                              RowSlots<float, W> &sl, int buf, float &hl2, float &hl1, float &hr0,
                                              float &hr1)
{
    constexpr int H = RPT / 2;
    constexpr int NSEG = 32 * W;
    constexpr bool DIR = BC == BC_DIRICHLET;
    const int seg = warp * 32 + lane;
    const bool left_end = DIR && seg == 0, right_end = DIR && seg == NSEG - 1;
    const float d = A.fd, c1 = A.fc1, c2 = A.fc2, inv = A.finv;
    float zl2 = hl2, zl1 = hl1, zr0 = hr0, zr1 = hr1;
    if (DIR) end_ghosts<float, RPT, 2>(z, left_end, right_end, zl2, zl1, zr0, zr1);
    seg_make_q<float, RPT, 2>(z, zl2, zl1, zr0, zr1, [&](int k) { return k < 0 ? rl : (k >= RPT ? rr : r[k]); }, cu,
                              c1, c2);
    if (DIR) end_zero<float, RPT>(z, left_end, right_end);

    float ya = z[0], yb = z[H], ra1 = 0.f, rb = yb, pw = 1.f;
#pragma unroll
    for (int k = 1; k < H; ++k) {
        ya = d * ya + z[k];
        yb = d * yb + z[H + k];
        z[k] = ya;
        z[H + k] = yb;
        const float pbk = pw * d;
        ra1 += pw * ya;
        rb += pbk * yb;
        pw = pbk;
    }
    const float E1 = ya;
    const float E = yb + E1 * nc.dH;
    const float Y2 = z[RPT - 2] + E1 * nc.dH1;
    const float ER1 = ra1 + nc.dH1 * (rb + E1 * nc.GH);
    const float ER0 = z[0] + d * ER1;

    __syncwarp();
    constexpr unsigned F = 0xffffffffu;
    float EL = __shfl_up_sync(F, E, 1), EL2 = __shfl_up_sync(F, E, 2), Y2L = __shfl_up_sync(F, Y2, 1);
    const float ER0L = __shfl_up_sync(F, ER0, 1);
    float ER = __shfl_down_sync(F, E, 1), ER0R = __shfl_down_sync(F, ER0, 1), ER1R = __shfl_down_sync(F, ER1, 1);
    float ER0R2 = __shfl_down_sync(F, ER0, 2);
    float *mine = sl.nb[buf][warp];
    if (lane == 31) { mine[0] = E; mine[1] = Y2; }
    if (lane == 30) mine[4] = E;
    if (lane == 0) { mine[2] = ER0; mine[3] = ER1; mine[5] = E; }
    if (lane == 1) mine[6] = ER0;
    __syncthreads();
    const float *prev = sl.nb[buf][warp > 0 ? warp - 1 : W - 1], *next = sl.nb[buf][warp < W - 1 ? warp + 1 : 0];
    if (lane == 0) { EL = prev[0]; Y2L = prev[1]; EL2 = prev[4]; }
    if (lane == 1) EL2 = prev[0];
    if (lane == 31) { ER = next[5]; ER0R = next[2]; ER1R = next[3]; ER0R2 = next[6]; }
    if (lane == 30) ER0R2 = next[2];
    const bool hasL = !(DIR && seg < 1), hasL2 = !(DIR && seg < 2);
    const bool hasR = !(DIR && seg > NSEG - 2), hasR2 = !(DIR && seg > NSEG - 3);
    EL = hasL ? EL : 0.f;
    Y2L = hasL ? Y2L : 0.f;
    EL2 = hasL2 ? EL2 : 0.f;

    const float yin = EL + nc.dR * EL2;                     // causal value at a-1
    const float cB = E1 + yin * nc.dH;
    float pk = d;
#pragma unroll
    for (int k = 0; k < H; ++k) {
        z[k] += yin * pk;
        z[H + k] += cB * pk;
        pk *= d;
    }
    const float Cl = E + nc.dR * EL;                        // causal value at a+RPT-1
    const float ER2n = hasR2 ? ER0R2 + nc.G * ER : 0.f;      // anti-causal sum of segment l+2
    float eout = hasR ? ER0R + nc.G * Cl + nc.dR * ER2n : 0.f;
    float er1 = hasR ? ER1R + nc.G1 * Cl + nc.dR1 * ER2n : 0.f;
    float acc = d * eout;
    if (DIR && seg == NSEG - 1) {
        acc -= z[RPT - 1] * inv;                               // B' = -y_{n-1} / (1 - mu^2)
    } else if (DIR && seg == NSEG - 2) {
        const float Bc = -(ER + nc.dR * E) * inv;             // y_{n-1} from the last segment's E
        acc += Bc * nc.dR;
        eout += Bc * nc.dR1;
        er1 += Bc * nc.dR2;
    }
    const float ER2 = rb + cB * nc.GH;
    seg_bwd_scan2<float, RPT>(z, d, nc.dH, acc, ER2);
    float Ac = 0.f;
    if (DIR && seg == 0) {
        Ac = -z[0] * inv;                                       // A' = -e_0 / (1 - mu^2)
        seg_add_left2<float, RPT>(z, d, nc.dH, Ac);
    } else if (DIR && seg == 1) {
        Ac = -(ER0L + nc.dR * (ER0 + nc.G * EL)) * inv;        // e_0 from the first segment's sums
        seg_add_left2<float, RPT>(z, d, nc.dH, Ac * nc.dR);
    }
    if (DIR && seg == 1) {
        hl1 = yin + d * (z[0] - Ac * nc.dR) + Ac * nc.dR1;
        hl2 = Y2L + d * (hl1 - Ac * nc.dR1) + Ac * nc.dR2;
    } else {
        hl1 = hasL ? yin + d * z[0] : 0.f;
        hl2 = hasL ? Y2L + EL2 * nc.dR1 + d * hl1 : 0.f;
    }
    hr0 = eout;
    hr1 = er1;
    if (DIR && seg == 0) {
        hr0 += Ac * nc.dR;
        hr1 += Ac * nc.dRp1;
    }
}

// D^T (z + cu u) on a Dirichlet row split over W warps (the transposed
// difference form of post_T; any n with 32 (W-1) RPT < n <= 32 W RPT)
template <class T, int RPT, int W>
__device__ __forceinline__ void row_sweep_T(T (&z)[RPT], const T (&u)[RPT], T cu, const AxisDev &A, int lane, int warp,
                                            RowSlots<T, W> &sl)
{
    const int n = A.n, seg = warp * 32 + lane, a = seg * RPT, kl = n - 1 - a;
#pragma unroll
    for (int k = 0; k < RPT; ++k) {
        const T q = z[k] + cu * u[k];
        z[k] = (k < kl && (seg > 0 || k > 0)) ? q : (T)0;      // interior rows only
    }
    row_solve<T, BC_DIRICHLET, RPT, W, true>(z, A, lane, warp, sl);
#pragma unroll
    for (int k = 0; k < RPT; ++k) z[k] = (k < kl && (seg > 0 || k > 0)) ? z[k] : (T)0;
    T el2, el1, er0, er1;
    row_halos<T, RPT, W, false>(z, lane, warp, sl, el2, el1, er0, er1);
    const bool first = seg == 0, last = seg == 32 * W - 1;
    el2 = first ? (T)0 : el2;
    el1 = first ? (T)0 : el1;
    er0 = last ? (T)0 : er0;
    er1 = last ? (T)0 : er1;
    post_T<T, RPT, true>(z, el2, el1, er0, er1, A.cc1<T>(), A.cc2<T>(), a, n);
    __syncwarp();
}

template <class T, int W>
__host__ __device__ constexpr size_t row_slots_bytes() { return (sizeof(RowSlots<T, W>) + 15) & ~(size_t)15; }

// ADJ (Dirichlet): the transposed Horner pass of the adjoint step,
// F^T = sum_t (D_x^T)^t (f_t0 u + sum_k f_tk g_k) with g_k = (D_y^T)^{k+1} u;
// u itself (pairs summed) takes the place of its second difference.
// Four warps per row: seven CTAs per SM (72 registers, 31 KB of shared
// memory each at RPT = 16 and three fields), so that the 2048 rows of a
// 2048^2 grid run in two waves over the 152 SMs instead of two and a quarter.
template <int BC, int RPT, int NB, int W, bool ADJ = false, bool NBX = false>
__global__ void __launch_bounds__(32 * W, W == 2 ? 8 : (W == 4 ? 7 : 4)) k_contig_rows(AxisDev A, LineSet LS, ProgParams pr,
                                                                                       NbConsts nc)
{
    pdl_enter();
    static_assert(RPT % 4 == 0 && RPT >= 8, "segment length");
    static_assert(!ADJ || BC == BC_DIRICHLET, "the transposed pass is for Dirichlet rows");
    using T = float;
    using St = ContigStage<T, RPT>;
    constexpr int NT = 32 * W;                        // threads (segments) of one row
    constexpr int LINE = NT * St::SST;                // one field of the row in the segment layout
    constexpr int NVL = RPT / 4;                      // 16-byte vectors per thread
    extern __shared__ __align__(16) unsigned char smem_raw[];
    RowSlots<T, W> &sl = *reinterpret_cast<RowSlots<T, W> *>(smem_raw);
    T *B = reinterpret_cast<T *>(smem_raw + row_slots_bytes<T, W>());
    const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
    const int n = A.n;                                // == NT * RPT
    const int ng = pr.ng;
    // one row per CTA, or (gridDim.x < rows) persistent CTAs that walk the
    // rows with a stride of the grid and stream the next row into L2 while
    // they work on this one, so that DRAM stays busy through the sweeps
    for (int64_t row = blockIdx.x; row < LS.nlines; row += gridDim.x) {
    if (row != (int64_t)blockIdx.x) __syncthreads();  // the previous row is done with the buffers and slots
    const int64_t base = row * (int64_t)n;
    if (t == 0) {
        const unsigned bytes = (unsigned)n * 4u;
        prefetch_l2((const float *)pr.u_hi + base, bytes);
        prefetch_l2((const float *)pr.u_lo + base, bytes);
        // field 0 is copied only once r has left its buffer: into L2 now
        if (ng > 0) prefetch_l2(reinterpret_cast<const float *>(pr.g[0]) + base, bytes);
        if (pr.feb != 0.f) {
            prefetch_l2((const float *)pr.up_hi + base, bytes);
            prefetch_l2((const float *)pr.up_lo + base, bytes);
        }
        const int64_t nx = row + gridDim.x;
        if (nx < LS.nlines) {
            const int64_t nb = nx * (int64_t)n;
            prefetch_l2((const float *)pr.u_hi + nb, bytes);
            prefetch_l2((const float *)pr.u_lo + nb, bytes);
            for (int k = 0; k < ng; ++k) prefetch_l2(reinterpret_cast<const float *>(pr.g[k]) + nb, bytes);
            if (pr.feb != 0.f) {
                prefetch_l2((const float *)pr.up_hi + nb, bytes);
                prefetch_l2((const float *)pr.up_lo + nb, bytes);
            }
        }
    }
    auto copy_field = [&](int k) {
        const float4 *src = reinterpret_cast<const float4 *>(reinterpret_cast<const T *>(pr.g[k]) + base);
        T *dst = B + k * LINE;
#pragma unroll
        for (int i = 0; i < NVL; ++i) {
            const int v = t + NT * i;
            cp_async16(dst + St::pos(4 * v), src + v);
        }
    };
    for (int k = 1; k < ng; ++k) copy_field(k);
    cp_async_commit();

    // r = accurate second difference of u (pairs), coalesced over the CTA;
    // buffer 0 stages it in the segment layout
    T *R = B;
    {
        const T *H = reinterpret_cast<const T *>(pr.u_hi) + base, *Lo = reinterpret_cast<const T *>(pr.u_lo) + base;
        const float4 *H4 = reinterpret_cast<const float4 *>(H), *L4 = reinterpret_cast<const float4 *>(Lo);
        float4 h[NVL], l[NVL];
        float hx[NVL], lx[NVL];      // lane 0: the point before its vector; lane 31: the point after it
#pragma unroll
        for (int i = 0; i < NVL; ++i) {
            const int v = t + NT * i;
            h[i] = __ldg(H4 + v);
            l[i] = __ldg(L4 + v);
            int j = (lane == 0) ? 4 * v - 1 : 4 * v + 4;
            if (BC == BC_PERIODIC) j = j < 0 ? j + n : (j >= n ? j - n : j);
            else j = j < 0 ? 0 : (j > n - 1 ? n - 1 : j);
            hx[i] = 0.f;
            lx[i] = 0.f;
            if (lane == 0 || lane == 31) { hx[i] = __ldg(H + j); lx[i] = __ldg(Lo + j); }
        }
        __syncwarp();
#pragma unroll
        for (int i = 0; i < NVL; ++i) {
            const int v = t + NT * i;
            float hl = __shfl_up_sync(0xffffffffu, h[i].w, 1), ll = __shfl_up_sync(0xffffffffu, l[i].w, 1);
            float hr = __shfl_down_sync(0xffffffffu, h[i].x, 1), lr = __shfl_down_sync(0xffffffffu, l[i].x, 1);
            hl = (lane == 0) ? hx[i] : hl;
            ll = (lane == 0) ? lx[i] : ll;
            hr = (lane == 31) ? hx[i] : hr;
            lr = (lane == 31) ? lx[i] : lr;
            float4 rv;
            if constexpr (ADJ) {
                rv = make_float4(h[i].x + l[i].x, h[i].y + l[i].y, h[i].z + l[i].z, h[i].w + l[i].w);
            } else {
                rv = sdiff4(h[i], l[i], hl, ll, hr, lr);
                if (BC == BC_DIRICHLET) {            // end nodes take the neighbouring interior centre
                    if (v == 0) rv.x = rv.y;
                    if (4 * v + 4 == n) rv.w = rv.z;
                }
            }
            *reinterpret_cast<float4 *>(R + St::pos(4 * v)) = rv;
        }
    }
    __syncthreads();
    T r[RPT];
    stage_to_regs<T, RPT>(R, r, t, false);
    if (lane == 0) sl.rhalo[warp][0] = r[0];
    if (lane == 31) sl.rhalo[warp][1] = r[RPT - 1];
    __syncthreads();                                  // every thread is done with R
    if (ng > 0) copy_field(0);
    cp_async_commit();
    float rl = __shfl_up_sync(0xffffffffu, r[RPT - 1], 1), rr = __shfl_down_sync(0xffffffffu, r[0], 1);
    if (lane == 0) rl = (warp > 0) ? sl.rhalo[warp - 1][1] : (BC == BC_PERIODIC ? sl.rhalo[W - 1][1] : r[0]);
    if (lane == 31) rr = (warp < W - 1) ? sl.rhalo[warp + 1][0] : (BC == BC_PERIODIC ? sl.rhalo[0][0] : r[RPT - 1]);
    cp_async_wait_all();
    __syncthreads();

    // Horner in D_x with the fields from shared memory
    T z[RPT];
#pragma unroll
    for (int k = 0; k < RPT; ++k) z[k] = 0;
    // NBX: z's halos ride along (the sweeps form e's, each Horner term adds
    // the fields' values there); positions a-2, a-1, a+RPT, a+RPT+1
    float hz[4] = {0.f, 0.f, 0.f, 0.f};
    int hpos[4] = {0, 0, 0, 0};
    bool hin[4] = {false, false, false, false};
    if constexpr (NBX) {
        const int a = t * RPT;
        const int g[4] = {a - 2, a - 1, a + RPT, a + RPT + 1};
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            int gi = g[i];
            if (BC == BC_PERIODIC) gi = gi < 0 ? gi + n : (gi >= n ? gi - n : gi);
            hin[i] = gi >= 0 && gi < n;
            hpos[i] = hin[i] ? St::pos(gi) : 0;
        }
    }
    for (int tt = pr.P; tt >= 0; --tt) {
        for (int k = 0; k < ng; ++k) {
            const T c = prog_coef<T>(pr, (size_t)tt * ng + k);
            if (c == (T)0) continue;
            const float4 *sg = reinterpret_cast<const float4 *>(B + k * LINE + t * St::SST);
#pragma unroll
            for (int q = 0; q < RPT / 4; ++q) {
                const float4 y = sg[q];
                z[4 * q] += c * y.x;
                z[4 * q + 1] += c * y.y;
                z[4 * q + 2] += c * y.z;
                z[4 * q + 3] += c * y.w;
            }
            if constexpr (NBX) {
#pragma unroll
                for (int i = 0; i < 4; ++i) hz[i] += hin[i] ? c * B[k * LINE + hpos[i]] : 0.f;
            }
        }
        if (tt == 0) break;
        if constexpr (ADJ) row_sweep_T<T, RPT, W>(z, r, prog_cu<T>(pr, tt), A, lane, warp, sl);
        else if constexpr (NBX && W == 2)
            row_sweep_nb<BC, RPT, W>(z, r, rl, rr, prog_cu<T>(pr, tt), A, nc, lane, warp, sl, tt & 1, hz[0], hz[1],
                                     hz[2], hz[3]);
        else if constexpr (NBX)
            row_sweep_nb2<BC, RPT, W>(z, r, rl, rr, prog_cu<T>(pr, tt), A, nc, lane, warp, sl, tt & 1, hz[0], hz[1],
                                      hz[2], hz[3]);
        else row_sweep<T, BC, RPT, W>(z, r, rl, rr, prog_cu<T>(pr, tt), A, lane, warp, sl);
    }

    // F -> coalesced side -> next level
    __syncthreads();                                  // every thread is done reading the fields
    regs_to_stage<T, RPT>(B, z, t);
    __syncthreads();
    const float4 *UH = reinterpret_cast<const float4 *>((const float *)pr.u_hi + base);
    const float4 *UL = reinterpret_cast<const float4 *>((const float *)pr.u_lo + base);
    const float4 *PH = reinterpret_cast<const float4 *>((const float *)pr.up_hi + base);
    const float4 *PL = reinterpret_cast<const float4 *>((const float *)pr.up_lo + base);
    float4 *NH = reinterpret_cast<float4 *>((float *)pr.un_hi + base);
    float4 *NL = reinterpret_cast<float4 *>((float *)pr.un_lo + base);
    const bool prev = pr.feb != 0.f;
    const float ea = pr.fea, eb = pr.feb, ec = pr.fec;
    constexpr int CH = NVL > 4 ? 4 : NVL;
#pragma unroll
    for (int i0 = 0; i0 < NVL; i0 += CH) {
        float4 uh[CH], ul[CH], ph[CH], pl[CH];
#pragma unroll
        for (int i = 0; i < CH; ++i) {
            const int v = t + NT * (i0 + i);
            uh[i] = __ldg(UH + v);
            ul[i] = __ldg(UL + v);
            ph[i] = prev ? __ldg(PH + v) : make_float4(0.f, 0.f, 0.f, 0.f);
            pl[i] = prev ? __ldg(PL + v) : make_float4(0.f, 0.f, 0.f, 0.f);
        }
#pragma unroll
        for (int i = 0; i < CH; ++i) {
            const int v = t + NT * (i0 + i);
            const float4 F = *CoalescedSide<T, RPT>::at(B, 4 * v);
            float4 nh, nl;
            level_pair(uh[i].x, ul[i].x, ph[i].x, pl[i].x, F.x, ea, eb, ec, nh.x, nl.x);
            level_pair(uh[i].y, ul[i].y, ph[i].y, pl[i].y, F.y, ea, eb, ec, nh.y, nl.y);
            level_pair(uh[i].z, ul[i].z, ph[i].z, pl[i].z, F.z, ea, eb, ec, nh.z, nl.z);
            level_pair(uh[i].w, ul[i].w, ph[i].w, pl[i].w, F.w, ea, eb, ec, nh.w, nl.w);
            NH[v] = nh;
            NL[v] = nl;
        }
    }
    }   // rows
}

// ---------------------------------------------------------------------------
// strided axes: lanes = 32 neighbouring lines, segments over warps and CTAs
// ---------------------------------------------------------------------------
template <class T>
struct StridedSlots {
    T *E;      // [S][32] causal segment reductions
    T *ER;     // [S][32] anti-causal segment reductions
    T *H;      // [2][S][4][32] first two / last two values of each segment, two sets
    T *Tot;    // [2][32] CTA totals (causal, anti-causal)
};

__host__ __device__ inline size_t strided_slot_bytes(int S, size_t tsize) { return (10 * (size_t)S * 32 + 64) * tsize; }

template <class T>
struct StridedCtx {
    cg::cluster_group cl;
    StridedSlots<T> sl;
    const T *dpg;
    T d, dR;            // e^{-nu}, d^RPT
    T dS, dL;           // cta_mult: decay across a full CTA and across the last CTA with data
    int n, S, K, w, lane, krank, seg, a, Gd, kL;
    bool full;
};

template <class T>
__device__ __forceinline__ T *peer_of(const StridedCtx<T> &c, T *p, int r)
{
    return c.K > 1 ? c.cl.map_shared_rank(p, r) : p;
}

template <class T>
__device__ __forceinline__ void csync(const StridedCtx<T> &c)
{
    if (c.K > 1) c.cl.sync();
    else __syncthreads();
}

// decay across the data segments of CTA k of the line: d^{S RPT} for the
// CTAs before the last one holding data (kL), d^{len} for that one (dL),
// 1 past it
template <class T>
__device__ __forceinline__ T cta_mult(const StridedCtx<T> &c, int k)
{
    return k < c.kL ? c.dS : (k == c.kL ? c.dL : (T)1);
}

// per-kernel constants of cta_mult
template <class T, int RPT>
__device__ __forceinline__ void strided_cta_consts(StridedCtx<T> &c)
{
    c.kL = c.Gd > 0 ? (c.Gd - 1) / c.S : 0;
    c.dS = c.kL > 0 ? c.dpg[c.S * RPT] : (T)1;          // read only when a full CTA precedes the last
    c.dL = c.dpg[(c.Gd - c.kL * c.S) * RPT];           // <= n + RPT - 1 (tables padded past d^n)
}

// Exchanges across the segments of a line.  The totals of the warps of this
// CTA (shared memory) and of the cluster's CTAs (distributed shared memory)
// are combined by short recurrences; the loads of a group of them are issued
// together (KMAX = 8 CTAs, SMAX = 16 warps at most), so that their latencies
// overlap instead of adding up.
constexpr int kXchKMax = 8, kXchSMax = 16;

// causal exchange: y at a-1 (zero inflow) and the line's y_{n-1}.  A line
// inside one CTA (K = 1) needs one barrier: every warp combines the totals
// itself, in the order the cluster path's warp 0 uses (the same values).
template <class T, int RPT>
__device__ __forceinline__ void strided_causal(const StridedCtx<T> &c, T E, T &yin, T &ytot)
{
    c.sl.E[c.w * 32 + c.lane] = E;
    __syncthreads();
    if (c.K == 1) {
        T acc = 0, all = 0;
#pragma unroll
        for (int v0 = 0; v0 < kXchSMax; v0 += 4) {
            T ev[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) ev[i] = v0 + i < c.S ? c.sl.E[(v0 + i) * 32 + c.lane] : (T)0;
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                if (v0 + i < c.w) acc = c.dR * acc + ev[i];
                if (v0 + i < c.S) all = ((v0 + i) < c.Gd ? c.dR : (T)1) * all + ev[i];
            }
        }
        yin = acc;
        ytot = all;
        return;
    }
    if (c.w == 0) {
        T acc = 0;
#pragma unroll
        for (int v0 = 0; v0 < kXchSMax; v0 += 4) {
            T ev[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) ev[i] = v0 + i < c.S ? c.sl.E[(v0 + i) * 32 + c.lane] : (T)0;
#pragma unroll
            for (int i = 0; i < 4; ++i)
                if (v0 + i < c.S) acc = ((c.krank * c.S + v0 + i) < c.Gd ? c.dR : (T)1) * acc + ev[i];
        }
        c.sl.Tot[c.lane] = acc;
    }
    csync(c);
    T tv[kXchKMax];
#pragma unroll
    for (int k2 = 0; k2 < kXchKMax; ++k2) tv[k2] = k2 < c.K ? peer_of(c, c.sl.Tot, k2)[c.lane] : (T)0;
    T cin = 0, tot = 0;
#pragma unroll
    for (int k2 = 0; k2 < kXchKMax; ++k2)
        if (k2 < c.K) {
            cin = (k2 == c.krank) ? tot : cin;
            tot = cta_mult<T>(c, k2) * tot + tv[k2];
        }
    T acc = cin;
#pragma unroll
    for (int v0 = 0; v0 < kXchSMax; v0 += 4) {
        T ev[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) ev[i] = v0 + i < c.w ? c.sl.E[(v0 + i) * 32 + c.lane] : (T)0;
#pragma unroll
        for (int i = 0; i < 4; ++i)
            if (v0 + i < c.w) acc = c.dR * acc + ev[i];
    }
    yin = acc;
    ytot = tot;
}

// anti-causal exchange: zero-inflow e just past the segment, and e_0 (one
// barrier for a line inside one CTA, as above)
template <class T, int RPT>
__device__ __forceinline__ void strided_anticausal(const StridedCtx<T> &c, T ER, T &eout, T &e0)
{
    c.sl.ER[c.w * 32 + c.lane] = ER;
    __syncthreads();
    if (c.K == 1) {
        T acc = 0, all = 0;
#pragma unroll
        for (int v0 = kXchSMax - 1; v0 >= 0; v0 -= 4) {
            T ev[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) ev[i] = v0 - i < c.S ? c.sl.ER[(v0 - i) * 32 + c.lane] : (T)0;
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const T f = (v0 - i) < c.Gd ? c.dR : (T)1;
                if (v0 - i > c.w && v0 - i < c.S) acc = f * acc + ev[i];
                if (v0 - i < c.S) all = f * all + ev[i];
            }
        }
        eout = acc;
        e0 = all;
        return;
    }
    if (c.w == 0) {
        T acc = 0;
#pragma unroll
        for (int v0 = kXchSMax - 1; v0 >= 0; v0 -= 4) {
            T ev[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) ev[i] = v0 - i < c.S ? c.sl.ER[(v0 - i) * 32 + c.lane] : (T)0;
#pragma unroll
            for (int i = 0; i < 4; ++i)
                if (v0 - i < c.S) acc = ((c.krank * c.S + v0 - i) < c.Gd ? c.dR : (T)1) * acc + ev[i];
        }
        c.sl.Tot[32 + c.lane] = acc;
    }
    csync(c);
    T tv[kXchKMax];
#pragma unroll
    for (int k2 = 0; k2 < kXchKMax; ++k2) tv[k2] = k2 < c.K ? peer_of(c, c.sl.Tot, k2)[32 + c.lane] : (T)0;
    T cin = 0, tot = 0;
#pragma unroll
    for (int k2 = kXchKMax - 1; k2 >= 0; --k2)
        if (k2 < c.K) {
            cin = (k2 == c.krank) ? tot : cin;
            tot = cta_mult<T>(c, k2) * tot + tv[k2];
        }
    T acc = cin;
#pragma unroll
    for (int v0 = kXchSMax - 1; v0 >= 0; v0 -= 4) {
        T ev[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) ev[i] = (v0 - i > c.w && v0 - i < c.S) ? c.sl.ER[(v0 - i) * 32 + c.lane] : (T)0;
#pragma unroll
        for (int i = 0; i < 4; ++i)
            if (v0 - i > c.w && v0 - i < c.S)
                acc = ((c.krank * c.S + v0 - i) < c.Gd ? c.dR : (T)1) * acc + ev[i];
    }
    eout = acc;
    e0 = tot;
}

// halo exchange: z at a-2, a-1 and a+RPT, a+RPT+1
template <class T, int BC, int RPT>
__device__ __forceinline__ void strided_halos(const StridedCtx<T> &c, const T (&z)[RPT], T &l2, T &l1, T &r0, T &r1,
                                              int buf)
{
    T *Hb = c.sl.H + buf * c.S * 128;
    T *H = Hb + c.w * 128;
    H[c.lane] = z[0];
    H[32 + c.lane] = z[1];
    H[64 + c.lane] = z[RPT - 2];
    H[96 + c.lane] = z[RPT - 1];
    csync(c);
    int gl = c.seg - 1, gr = c.seg + 1;
    if (BC == BC_PERIODIC) {
        if (gl < 0) gl = c.Gd - 1;
        if (gr >= c.Gd) gr = 0;
    }
    l2 = l1 = r0 = r1 = 0;
    if (gl >= 0) {
        const T *Hl = peer_of(c, Hb, gl / c.S) + (gl % c.S) * 128;
        l2 = Hl[64 + c.lane];
        l1 = Hl[96 + c.lane];
    }
    if (gr < c.Gd) {
        const T *Hr = peer_of(c, Hb, gr / c.S) + (gr % c.S) * 128;
        r0 = Hr[c.lane];
        r1 = Hr[32 + c.lane];
    }
    // two alternating slot sets: a set is written again only after two more
    // cluster barriers (the causal and anti-causal exchanges of the sweep),
    // by which time every reader is done with it
}

template <class T, int BC, int RPT>
__device__ __forceinline__ void strided_solve(const StridedCtx<T> &c, const AxisDev &A, T (&z)[RPT]);

// One application of D on this thread's segment.  MODE as in seg_make_q;
// halos l2, l1, r0, r1 as exchanged (MODE 0: l1 = s_{a-1}, r0 = s_{a+RPT}).
template <class T, int BC, int RPT, int MODE>
__device__ __forceinline__ void strided_sweep(const StridedCtx<T> &c, const AxisDev &A, T (&z)[RPT], T cu,
                                              T l2, T l1, T r0, T r1, const T *rs, T rl, T rr)
{
    const bool left = c.seg == 0, right = c.seg == c.Gd - 1;
    if (BC == BC_DIRICHLET) end_ghosts<T, RPT, MODE>(z, left, right, l2, l1, r0, r1);
    const T c1 = A.cc1<T>(), c2 = A.cc2<T>();
    if (MODE == 2)
        seg_make_q<T, RPT, 2>(z, l2, l1, r0, r1, [&](int k) { return k < 0 ? rl : (k >= RPT ? rr : rs[k * 32]); },
                              cu, c1, c2);
    else
        seg_make_q<T, RPT, MODE>(z, l2, l1, r0, r1, [&](int) { return (T)0; }, (T)0, c1, c2);
    if (BC == BC_DIRICHLET) end_zero<T, RPT>(z, left, right);
    if (!c.full) {
#pragma unroll
        for (int k = 0; k < RPT; ++k) z[k] = 0;
    }
    strided_solve<T, BC, RPT>(c, A, z);
}

// The solve of the difference form on this thread's segment of a strided
// line of whole segments: z holds q on entry (zero in segments past the
// line), e on exit (Dirichlet: e = 0 at both end nodes; periodic: images)
template <class T, int BC, int RPT>
__device__ __forceinline__ void strided_solve(const StridedCtx<T> &c, const AxisDev &A, T (&z)[RPT])
{
    const T d = c.d;
    const T dH = c.dpg[RPT / 2];
    T E1, ER2;
    const T E = seg_fwd_reduce2<T, RPT>(z, d, dH, E1);
    T yin, ytot;
    strided_causal<T, RPT>(c, E, yin, ytot);
    if (BC == BC_PERIODIC && c.full) yin += c.dpg[c.a] * (ytot * A.cinv<T>());
    if (!c.full) yin = 0;                                          // segments past the line stay zero
    const T ER = seg_fwd_scan2<T, RPT>(z, d, dH, yin, E1, ER2);
    T eout, e00;
    strided_anticausal<T, RPT>(c, ER, eout, e00);
    T Z, Acoef = 0;
    if (BC == BC_DIRICHLET) {
        const T mu = A.cmu<T>(), inv = A.cinv<T>();
        Acoef = (mu * ytot - e00) * inv;     // ytot = zero-inflow y_{n-1}
        Z = (mu * e00 - ytot) * inv;
    } else {
        Z = d * e00 * A.cinv<T>();
    }
    const T acc = d * eout + (c.full ? c.dpg[c.n - c.a - RPT] * Z : (T)0);
    seg_bwd_scan2<T, RPT>(z, d, dH, acc, ER2);
    if (BC == BC_DIRICHLET && c.full) seg_add_left2<T, RPT>(z, d, dH, Acoef * c.dpg[c.a]);
}

// One application of D^T (Dirichlet) on this thread's segment of a strided
// line of whole segments (the transposed difference form of post_T): the
// solve on the interior values, then t' and its second difference with the
// neighbouring segments' e as halos.  hbuf: halo slot set (alternating).
template <class T, int RPT>
__device__ __forceinline__ void strided_sweep_T(const StridedCtx<T> &c, const AxisDev &A, T (&z)[RPT], int hbuf)
{
    const int kl = c.n - 1 - c.a;
#pragma unroll
    for (int k = 0; k < RPT; ++k) z[k] = (k < kl && (c.seg > 0 || k > 0)) ? z[k] : (T)0;   // interior rows only
    strided_solve<T, BC_DIRICHLET, RPT>(c, A, z);
#pragma unroll
    for (int k = 0; k < RPT; ++k) z[k] = (k < kl && (c.seg > 0 || k > 0)) ? z[k] : (T)0;
    T l2, l1, r0, r1;
    strided_halos<T, BC_DIRICHLET, RPT>(c, z, l2, l1, r0, r1, hbuf);
    const T c1 = A.cc1<T>(), c2 = A.cc2<T>();
    if (c.seg == 0 || c.seg == c.Gd - 1) post_T<T, RPT, true>(z, l2, l1, r0, r1, c1, c2, c.a, c.n);
    else post_T<T, RPT, false>(z, l2, l1, r0, r1, c1, c2, c.a, c.n);
}

// second differences r of u at points a-1 .. a+RPT of one strided line, from
// one pass over rows a-2 .. a+RPT+1 (rows wrapped or clamped into the line;
// the clamped Dirichlet end values are fixed by the caller)
template <int BC>
__device__ __forceinline__ int64_t wrap_or_clamp(int j, int n)
{
    if (BC == BC_PERIODIC) { if (j < 0) j += n; else if (j >= n) j -= n; }
    else j = j < 0 ? 0 : (j > n - 1 ? n - 1 : j);
    return (int64_t)j;
}

template <int BC, int RPT>
__device__ __forceinline__ void strided_r_pair(const ProgParams &pr, int64_t lbase, int64_t st, int a, int n,
                                               float (&r)[RPT], float &rl, float &rr)
{
    const float *H = (const float *)pr.u_hi + lbase, *L = (const float *)pr.u_lo + lbase;
    const int64_t jm2 = wrap_or_clamp<BC>(a - 2, n) * st, jm1 = wrap_or_clamp<BC>(a - 1, n) * st;
    float hm = H[jm2], lm = L[jm2], h0 = H[jm1], l0 = L[jm1];
    const float *ph = H + (int64_t)a * st, *pl = L + (int64_t)a * st;
#pragma unroll
    for (int k = 0; k <= RPT + 1; ++k) {
        float hp, lp;
        if (k < RPT) {
            hp = *ph; lp = *pl;
            ph += st; pl += st;
        } else {
            const int64_t j = wrap_or_clamp<BC>(a + k, n) * st;
            hp = H[j]; lp = L[j];
        }
        const float v = sdiff_pair(hm, h0, hp, lm, l0, lp);     // centre a + k - 1
        if (k == 0) rl = v; else if (k == RPT + 1) rr = v; else r[k - 1] = v;
        hm = h0; h0 = hp; lm = l0; l0 = lp;
    }
}

template <int BC, int RPT>
__device__ __forceinline__ void strided_r_pair(const ProgParams &pr, int64_t lbase, int64_t st, int a, int n,
                                               double (&r)[RPT], double &rl, double &rr)
{
    const double *U = (const double *)pr.u_hi + lbase;
    double um = U[wrap_or_clamp<BC>(a - 2, n) * st], u0 = U[wrap_or_clamp<BC>(a - 1, n) * st];
    const double *pu = U + (int64_t)a * st;
#pragma unroll
    for (int k = 0; k <= RPT + 1; ++k) {
        double up;
        if (k < RPT) { up = *pu; pu += st; }
        else up = U[wrap_or_clamp<BC>(a + k, n) * st];
        const double v = (up - u0) - (u0 - um);
        if (k == 0) rl = v; else if (k == RPT + 1) rr = v; else r[k - 1] = v;
        um = u0; u0 = up;
    }
}

// KM: 0 powers D^p u, 1 Horner with several outputs, 2 powers (D^T)^p u
// (Dirichlet; the adjoint step)
template <class T, int BC, int RPT, int KM>
__global__ void __launch_bounds__(256, 2) k_strided(AxisDev A, LineSet LS, ProgParams pr)
{
    pdl_enter();
    extern __shared__ __align__(16) unsigned char smem_raw[];
    StridedCtx<T> c{cg::this_cluster()};
    c.S = LS.S;
    c.K = LS.K;
    c.w = threadIdx.x >> 5;
    c.lane = threadIdx.x & 31;
    c.krank = LS.K > 1 ? (int)c.cl.block_rank() : 0;
    c.n = A.n;
    c.d = A.cd<T>();
    c.dR = A.cdm<T>(0);
    c.dpg = dpow_of<T>(A);
    c.Gd = A.n / RPT;
    strided_cta_consts<T, RPT>(c);
    c.seg = c.krank * c.S + c.w;
    c.a = c.seg * RPT;
    c.full = c.seg < c.Gd;
    {
        T *p = reinterpret_cast<T *>(smem_raw);
        c.sl.E = p;
        c.sl.ER = p + c.S * 32;
        c.sl.H = p + 2 * c.S * 32;
        c.sl.Tot = p + 10 * c.S * 32;
    }
    T *rbuf = reinterpret_cast<T *>(smem_raw + strided_slot_bytes(c.S, sizeof(T)));   // [S][RPT][32]
    const int n = c.n, a = c.a;

    const int64_t line = (int64_t)blockIdx.x * 32 + c.lane;
    const bool valid = line < LS.nlines;
    const bool io = valid && c.full;
    const int64_t lbase = valid ? (line % LS.inner) + (line / LS.inner) * LS.inner * (int64_t)n : 0;
    const int64_t st = LS.stride;

    T z[RPT];
    if constexpr (KM == 2) {
        static_assert(BC == BC_DIRICHLET, "the transposed powers are for Dirichlet lines");
        // the level value itself (pairs summed), then its powers of D^T
        const T *H = reinterpret_cast<const T *>(pr.u_hi) + lbase, *L = reinterpret_cast<const T *>(pr.u_lo) + lbase;
#pragma unroll
        for (int k = 0; k < RPT; ++k) {
            T v = 0;
            if (io) {
                v = H[(int64_t)(a + k) * st];
                if constexpr (sizeof(T) == 4) v += L[(int64_t)(a + k) * st];
            }
            z[k] = v;
        }
        for (int p = 1; p <= pr.P; ++p) {
            strided_sweep_T<T, RPT>(c, A, z, p & 1);
            T *o = reinterpret_cast<T *>(pr.out[p - 1]);
            if (o != nullptr && io) {
                T *po = o + lbase + (int64_t)a * st;
#pragma unroll
                for (int k = 0; k < RPT; ++k) { *po = z[k]; po += st; }
            }
        }
        if (c.K > 1) c.cl.sync();       // see the powers path below
        return;
    }

    // r = accurate second difference of u along the line (Dirichlet end
    // nodes use the neighbouring interior centre)
    T rl = 0, rr = 0;
    if (io) strided_r_pair<BC, RPT>(pr, lbase, st, a, n, z, rl, rr);
    else {
#pragma unroll
        for (int k = 0; k < RPT; ++k) z[k] = 0;
    }
    if (BC == BC_DIRICHLET) {
        if (c.seg == 0) z[0] = z[1];
        if (c.seg == c.Gd - 1) z[RPT - 1] = z[RPT - 2];
    }

    if (KM == 0) {
        // powers; the first sweep starts from s = r
        for (int p = 1; p <= pr.P; ++p) {
            if (p == 1) {
                strided_sweep<T, BC, RPT, 0>(c, A, z, (T)0, (T)0, rl, rr, (T)0, nullptr, (T)0, (T)0);
            } else {
                T l2, l1, r0, r1;
                strided_halos<T, BC, RPT>(c, z, l2, l1, r0, r1, p & 1);
                strided_sweep<T, BC, RPT, 1>(c, A, z, (T)0, l2, l1, r0, r1, nullptr, (T)0, (T)0);
            }
            T *o = reinterpret_cast<T *>(pr.out[p - 1]);
            if (o != nullptr && io) {
                T *po = o + lbase + (int64_t)a * st;
#pragma unroll
                for (int k = 0; k < RPT; ++k) { *po = z[k]; po += st; }
            }
        }
        // peers read this CTA's shared memory after the last exchange: no CTA
        // of the cluster exits before all of them are past those reads
        if (c.K > 1) c.cl.sync();
        return;
    }

    // Horner: r kept on chip, lane-interleaved
    T *rs = rbuf + (size_t)c.w * RPT * 32 + c.lane;
#pragma unroll
    for (int k = 0; k < RPT; ++k) rs[k * 32] = z[k];
    const int P = pr.P, ng = pr.ng;
    int hpar = 0;
    for (int o = 0; o < pr.nout; ++o) {
        const size_t cfo = (size_t)o * (P + 1) * ng;
#pragma unroll
        for (int k = 0; k < RPT; ++k) z[k] = 0;
        for (int t = P; t >= 0; --t) {
            const size_t cf = cfo + (size_t)t * ng;
            if (io) {
                for (int q = 0; q < ng; ++q) {
                    const T cq = prog_coef<T>(pr, cf + q);
                    if (cq == (T)0) continue;
                    const T *gq = reinterpret_cast<const T *>(pr.g[q]) + lbase + (int64_t)a * st;
#pragma unroll
                    for (int k = 0; k < RPT; ++k) { z[k] += cq * *gq; gq += st; }
                }
            }
            if (t == 0) break;
            T l2, l1, r0, r1;
            strided_halos<T, BC, RPT>(c, z, l2, l1, r0, r1, hpar);
            hpar ^= 1;
            strided_sweep<T, BC, RPT, 2>(c, A, z, prog_cu<T>(pr, (size_t)o * (P + 1) + t), l2, l1, r0, r1, rs, rl, rr);
        }
        T *ob = reinterpret_cast<T *>(pr.out[o]);
        if (io) {
            T *po = ob + lbase + (int64_t)a * st;
#pragma unroll
            for (int k = 0; k < RPT; ++k) { *po = z[k]; po += st; }
        }
    }
    if (c.K > 1) c.cl.sync();       // see the powers path: peers may still read this CTA's slots
}

}  // namespace molt
