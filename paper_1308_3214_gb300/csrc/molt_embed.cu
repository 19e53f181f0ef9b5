// molt_embed.cu -- embedded boundaries (Sec. 4.3): the 2D scheme on a domain
// cut out of a grid, its lines being "line objects" (the interior grid nodes
// of a grid line plus a boundary point at each end, off the grid).  Float64.
//
// L^{-1} on a line object of m interior nodes: nodes x_0 = a, x_1..x_m (spacing
// h, x_1 = a + ga), x_{m+1} = b = x_m + gb; the data at a and b are zero.
//   J^L_k = (alpha/2) int_{x_{k-1}}^{x_k} e^{-alpha (x_k - y)} p(y) dy,
//   J^R_k = (alpha/2) int_{x_k}^{x_{k+1}} e^{-alpha (y - x_k)} p(y) dy,
// p the quadratic through x_{k-1}, x_k, x_{k+1} (moved one node inward where
// that node does not exist), integrated exactly; I^L_k = e^{-alpha(x_k -
// x_{k-1})} I^L_{k-1} + J^L_k from I^L_0 = 0, I^R likewise from the right;
// w = I^L + I^R + A e^{-alpha (x - a)} + B e^{-alpha (b - x)} with w(a) = w(b)
// = 0.  Cells between grid nodes take the axis' uniform weights; the cells
// and stencils that touch a boundary point take per-line weights computed on
// the host in float64.
//
// The kernel: one warp per line object; the line's two partial sums sit in
// shared memory (the increments overwrite the line's values in place); each
// lane owns a chunk of consecutive nodes, and both recurrences run as
// chunked scans of affine maps (a lane's chunk maps the inflow y to P y + Q;
// a 5-step shuffle scan composes them).
// A line is read and written in place in the caller's layout: x lines with
// stride 1, y lines with stride nx (the 4 warps of a CTA take 4 neighbouring
// columns, which share the 32-byte sectors of each row).
#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

#include "molt.h"
#include "molt_internal.h"

namespace {

constexpr int kObjMaxM = 2046;             // interior nodes of a line object at most
constexpr int kObjWarps = 4;               // line objects (warps) per CTA
constexpr int kObjThreads32 = 128;         // threads per line object in the float32 sweep
constexpr int kObjCpb[2] = {1, 4};         // float32 sweep: line objects per CTA, contiguous / strided axis

struct ObjLine {
    long long base;     // element index of the first interior node
    int m;              // interior nodes
    int pad_;
    double dA, dB;      // e^{-alpha ga}, e^{-alpha gb}
    double rA, rB;      // dA / d, dB / d (d = e^{-alpha h})
    double mu, inv;     // e^{-alpha (b - a)}, 1 / (1 - mu^2)
    double wl[6];       // J^R_0, J^L_1, J^R_1 as weights on (u_1, u_2)
    double wr[6];       // J^L_{m+1}, J^L_m, J^R_m as weights on (u_m, u_{m-1})
};

struct ObjAxis {
    long long stride;   // element stride along the lines (1 for x, nx for y)
    double d;           // e^{-alpha h}
    double uL[3];       // uniform J^L_k weights on (u_{k-1}, u_k, u_{k+1})
    double uR[3];       // uniform J^R_k weights on (u_{k-1}, u_k, u_{k+1})
    const double *dpow; // d^k, k = 0..kObjMaxM
};

enum : int { OBJ_LINV = 0, OBJ_D = 1, OBJ_SUB = 2 };

// inclusive scan of affine maps y -> p y + q over the lanes (lane order =
// application order when FWD, reversed otherwise)
template <bool FWD>
__device__ __forceinline__ void affine_scan(double &p, double &q, int lane)
{
#pragma unroll
    for (int k = 1; k < 32; k <<= 1) {
        const double pp = FWD ? __shfl_up_sync(0xffffffffu, p, k) : __shfl_down_sync(0xffffffffu, p, k);
        const double qq = FWD ? __shfl_up_sync(0xffffffffu, q, k) : __shfl_down_sync(0xffffffffu, q, k);
        const bool take = FWD ? lane >= k : lane + k < 32;
        if (take) {                               // this lane's maps follow the other's
            q = qq * p + q;
            p = pp * p;
        }
    }
}

template <bool FWD>
__device__ __forceinline__ void affine_scan32(float &p, float &q, int lane)
{
#pragma unroll
    for (int k = 1; k < 32; k <<= 1) {
        const float pp = FWD ? __shfl_up_sync(0xffffffffu, p, k) : __shfl_down_sync(0xffffffffu, p, k);
        const float qq = FWD ? __shfl_up_sync(0xffffffffu, q, k) : __shfl_down_sync(0xffffffffu, q, k);
        const bool take = FWD ? lane >= k : lane + k < 32;
        if (take) {
            q = qq * p + q;
            p = pp * p;
        }
    }
}

// out[k] (interior node k of every line) = w = L^{-1} in (OBJ_LINV),
// in - w (OBJ_D) or sub - w (OBJ_SUB); accum adds it to out instead.  slot:
// shared-memory elements per line array (>= the longest line's m + 2; two
// arrays per warp).
__global__ void __launch_bounds__(32 * kObjWarps) k_obj_sweep(ObjAxis ax, const ObjLine *lines, int nlines,
                                                             const double *__restrict__ in, double *out,
                                                             const double *sub, int mode, int accum, int slot)
{
    extern __shared__ __align__(16) double sm[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    double *L = sm + (size_t)warp * 2 * slot;
    double *R = L + slot;
    const double d = ax.d;
    for (int li = blockIdx.x * kObjWarps + warp; li < nlines; li += gridDim.x * kObjWarps) {
        const ObjLine &ln = lines[li];
        const int m = ln.m, N = m + 1;
        const long long base = ln.base;
        const double dA = ln.dA, dB = ln.dB;
        __syncwarp();
        // the line's values into R (zero at the boundary points)
        const long long st = ax.stride;
        for (int k = lane; k <= N; k += 32) R[k] = (k >= 1 && k <= m) ? in[base + (k - 1) * st] : 0.0;
        __syncwarp();
        // chunk of nodes [k0, k1) of this lane
        const int s = (N + 1 + 31) / 32;
        const int k0 = min(lane * s, N + 1), k1 = min(k0 + s, N + 1);
        // values the increments need from outside the lane's chunk, read before
        // any lane overwrites R
        const double u1 = R[1], u2 = R[2], um = R[m], um1 = R[m - 1];
        double a = (k0 >= 1 && k0 <= N) ? R[k0 - 1] : 0.0;      // u_{k-1}
        double b = (k0 <= N) ? R[k0] : 0.0;                     // u_k
        const double after = (k1 <= N) ? R[k1] : 0.0;          // u_{k1}
        __syncwarp();
        // increments, in place: L[k] = J^L_k (L[0] = 0), R[k] = J^R_k (R[N] = 0)
        for (int k = k0; k < k1; ++k) {
            const double c = (k + 1 < k1) ? R[k + 1] : after;     // u_{k+1}, not yet overwritten
            double jl = 0.0, jr = 0.0;
            if (k == 1) jl = ln.wl[2] * u1 + ln.wl[3] * u2;
            else if (k == N) jl = ln.wr[0] * um + ln.wr[1] * um1;
            else if (k == m) jl = ln.wr[2] * um + ln.wr[3] * um1;
            else if (k > 1) jl = ax.uL[0] * a + ax.uL[1] * b + ax.uL[2] * c;
            if (k == 0) jr = ln.wl[0] * u1 + ln.wl[1] * u2;
            else if (k == 1) jr = ln.wl[4] * u1 + ln.wl[5] * u2;
            else if (k == m) jr = ln.wr[4] * um + ln.wr[5] * um1;
            else if (k < m) jr = ax.uR[0] * a + ax.uR[1] * b + ax.uR[2] * c;
            L[k] = jl;
            R[k] = jr;
            a = b;
            b = c;
        }
        __syncwarp();
        // causal: I^L_k = e_k I^L_{k-1} + J^L_k, e_1 = dA, e_N = dB, else d; the
        // chunk's decay is d^{k1-k0} with the end cells' factors swapped in
        {
            double q = 0.0;
            for (int k = k0; k < k1; ++k) {
                const double e = (k == 1) ? dA : (k == N ? dB : d);
                q = e * q + L[k];
            }
            double p = ax.dpow[k1 - k0];
            if (k0 <= 1 && 1 < k1) p *= ln.rA;
            if (k0 <= N && N < k1) p *= ln.rB;
            affine_scan<true>(p, q, lane);
            double y = __shfl_up_sync(0xffffffffu, q, 1);
            y = (lane == 0) ? 0.0 : y;
            for (int k = k0; k < k1; ++k) {
                const double e = (k == 1) ? dA : (k == N ? dB : d);
                y = e * y + L[k];
                L[k] = y;
            }
        }
        // anti-causal: I^R_k = f_k I^R_{k+1} + J^R_k, f_0 = dA, f_m = dB, else d
        // (the chunk holding N passes no inflow on: every later chunk is empty)
        {
            double q = 0.0;
            for (int k = k1 - 1; k >= k0; --k) {
                const double f = (k == 0) ? dA : (k == m ? dB : d);
                const double r = (k == N) ? 0.0 : R[k];
                q = f * q + r;
            }
            double p = ax.dpow[k1 - k0];
            if (k0 <= 0 && 0 < k1) p *= ln.rA;
            if (k0 <= m && m < k1) p *= ln.rB;
            affine_scan<false>(p, q, lane);
            double y = __shfl_down_sync(0xffffffffu, q, 1);
            y = (lane == 31) ? 0.0 : y;
            for (int k = k1 - 1; k >= k0; --k) {
                const double f = (k == 0) ? dA : (k == m ? dB : d);
                const double r = (k == N) ? 0.0 : R[k];
                y = (k == N) ? 0.0 : f * y + r;
                R[k] = y;
            }
        }
        __syncwarp();
        // homogeneous terms: w(a) = I^R_0 + A + mu B = 0, w(b) = I^L_N + mu A + B = 0
        const double r0 = -R[0], r1 = -L[N];
        const double Acoef = (r0 - ln.mu * r1) * ln.inv;
        const double Bcoef = (r1 - ln.mu * r0) * ln.inv;
        for (int k = 1 + lane; k <= m; k += 32) {
            const double w = L[k] + R[k] + Acoef * dA * ax.dpow[k - 1] + Bcoef * dB * ax.dpow[m - k];
            double res = w;
            const long long at = base + (k - 1) * st;
            if (mode == OBJ_D) res = in[at] - w;
            else if (mode == OBJ_SUB) res = sub[at] - w;
            double *o = out + at;
            *o = accum ? *o + res : res;
        }
    }
}

constexpr int kCombMax = 8;
struct CombTerms {
    int n;
    double c[kCombMax];
    const double *x[kCombMax];
};

// out = sum_t c_t x_t (out may be one of the x_t)
__global__ void __launch_bounds__(256) k_obj_combine(CombTerms t, double *out, int64_t N)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
        double v = 0.0;
        for (int k = 0; k < t.n; ++k) v += t.c[k] * t.x[k][i];
        out[i] = v;
    }
}

// ---------------------------------------------------------------------------
// float32 sweeps: the difference form of D on a line object
// ---------------------------------------------------------------------------
// With g_k the decay of cell k (between x_{k-1} and x_k) and e = D v, the two
// recurrences and the boundary terms give, at every interior node k = 1..N-1,
//   T_k - g_{k+1} T_{k+1} = q_k,   T_k = (e_k - g_k e_{k-1}) / (1 - g_k^2),
// with e = 0 at both boundary points; q_k is local in v and vanishes on
// linear data, so it is a combination of second divided differences:
//   q_k = ge s_{k-1} + gc s_k + ge s_{k+1} on the uniform interior
//   (s_t = v_{t-1} - 2 v_t + v_{t+1}, the divided difference times h^2), and
//   two per-line coefficients on rows 1 and N-1, whose end triples (a, x_1,
//   x_2) and (x_{m-1}, x_m, b) have their own spacings.
// The anti-causal recurrence gives T from T_N = 0, the causal one e from
// e_0 = 0, and the homogeneous solutions A' e^{-alpha (x - a)} + B'
// e^{-alpha (b - x)} restore e_N = 0.  D v then never subtracts two nearly
// equal numbers, so float32 sweeps keep their accuracy (D v << v for smooth
// fields); the input's second differences come from float32 pairs when the
// input is a time level.
struct ObjLineF {
    long long base;     // element index of the first interior node
    int m, pad_;
    float dA, dB;       // decays of the end cells
    float rA, rB;       // dA / d, dB / d
    float cA, cB;       // 1 - dA^2, 1 - dB^2
    float mu, inv;      // e^{-alpha (b - a)}, 1 / (1 - mu^2)
    float g11, g12;     // row 1: q_1 = g11 s_1 + g12 s_2
    float gNa, gNb;     // row N-1: q_m = gNa s_{m-1} + gNb s_m
    float p1, q1;       // s_1 = p1 (v_2 - v_1) - q1 v_1 (v_2 = 0 when m = 1)
    float pm, qm;       // s_m = pm (0 - v_m) - qm (v_m - v_{m-1})
};

struct ObjAxisF {
    long long stride;
    float d, c;         // e^{-alpha h}, 1 - d^2
    float gc, ge;       // uniform rows
    const float *dpow;  // d^k
};

enum : int { OBJF_D = 0, OBJF_LINV = 1, OBJF_BOTH = 2 };

// MODE OBJF_D: out = D v; OBJF_LINV: out = v - D v (= L^{-1} v); OBJF_BOTH:
// out = D v and out2 = v - D v (and out3 = D v when given).  accum adds to
// out.  PAIR: v is a float32 pair level (in = hi, lo = lo plane), else a
// float32 field.
// A CTA takes CPB consecutive line objects at a time, kObjThreads32 threads
// per line.  Loads and stores run over grid positions along the lines, the
// CPB lines interleaved, so that on the strided axis (consecutive lines =
// adjacent columns) a row's CPB values are read and written together.  In the
// recurrences each thread reduces a chunk of its group's line, the chunk maps
// are composed over the lanes of a warp (shuffles) and over the group's warps
// (their totals in shared memory), and each chunk is re-run from its carry.
// slot: elements per line array (>= m + 2), four arrays per line.
template <bool PAIR, int CPB>
__global__ void __launch_bounds__(kObjThreads32 * CPB) k_obj_sweep32(ObjAxisF ax, const ObjLineF *lines, int nlines,
                                                                    const float *__restrict__ in,
                                                                    const float *__restrict__ lo, float *out,
                                                                    float *out2, float *out3, int mode, int accum,
                                                                    int slot)
{
    constexpr int NW = kObjThreads32 / 32, NT = kObjThreads32 * CPB;
    extern __shared__ __align__(16) float smf[];
    __shared__ float2 totA[CPB][NW], totC[CPB][NW];   // warp totals of the two recurrences
    __shared__ long long l_base[CPB], l_pos[CPB];      // first interior node: element, position on the line's axis
    __shared__ int l_m[CPB];
    __shared__ float l_Ad[CPB], l_Bd[CPB];
    const int tid = threadIdx.x;
    const int grp = tid / kObjThreads32, gt = tid % kObjThreads32, warp = gt >> 5, lane = gt & 31;
    const int ij = tid % CPB, ii = tid / CPB;           // interleaved load/store mapping: line, position
    const long long st = ax.stride;
    const float d = ax.d, c = ax.c;
    for (int gb = blockIdx.x * CPB; gb < nlines; gb += gridDim.x * CPB) {
        __syncthreads();
        if (tid < CPB) {
            const int li = gb + tid;
            const bool ok = li < nlines;
            l_m[tid] = ok ? lines[li].m : 0;
            l_base[tid] = ok ? lines[li].base : 0;
            l_pos[tid] = (ok && CPB > 1) ? lines[li].base / st : 0;
        }
        __syncthreads();
        long long p_lo = l_pos[0], p_hi = l_pos[0] + l_m[0] - 1;
#pragma unroll
        for (int j = 1; j < CPB; ++j)
            if (l_m[j] > 0) {
                p_lo = min(p_lo, l_pos[j]);
                p_hi = max(p_hi, l_pos[j] + l_m[j] - 1);
            }
        {
            const int mj = l_m[ij];
            const long long bj = l_base[ij], pj = l_pos[ij];
            float *Hj = smf + (size_t)ij * 4 * slot, *Lj = Hj + slot;
            for (long long r = p_lo + ii; r <= p_hi; r += NT / CPB) {
                const long long k = r - pj + 1;
                if (k >= 1 && k <= mj) {
                    Hj[k] = in[bj + (k - 1) * st];
                    Lj[k] = PAIR ? lo[bj + (k - 1) * st] : 0.f;
                }
            }
            if (ii == 0) { Hj[0] = 0.f; Lj[0] = 0.f; Hj[mj + 1] = 0.f; Lj[mj + 1] = 0.f; }
        }
        __syncthreads();
        // the recurrences of line grp
        const int li = gb + grp;
        const int m = l_m[grp], N = m + 1;
        float *H = smf + (size_t)grp * 4 * slot;
        float *Lo = H + slot;        // lo plane (PAIR)
        float *S = Lo + slot;        // second differences s_t
        float *Q = S + slot;         // q_k, then T_k, then e_k
        const ObjLineF &ln = lines[li < nlines ? li : 0];
        // second differences s_t, t = 1..m (end triples with their spacings)
        for (int t = 1 + gt; t <= m; t += kObjThreads32) {
            float sv;
            if (t == 1 || t == m) {
                // differences of the pair values, then the end triple's weights
                const float v1h = H[t], v1l = Lo[t];
                const float dn = __fadd_rn(__fsub_rn(H[t + 1], v1h), __fsub_rn(Lo[t + 1], v1l));   // v_{t+1} - v_t
                const float dp = __fadd_rn(__fsub_rn(v1h, H[t - 1]), __fsub_rn(v1l, Lo[t - 1]));   // v_t - v_{t-1}
                if (t == 1) sv = ln.p1 * dn - ln.q1 * dp;
                else sv = ln.pm * dn - ln.qm * dp;
            } else {
                sv = PAIR ? molt::sdiff_pair(H[t - 1], H[t], H[t + 1], Lo[t - 1], Lo[t], Lo[t + 1])
                          : (H[t + 1] - H[t]) - (H[t] - H[t - 1]);
            }
            S[t] = sv;
        }
        __syncthreads();
        for (int k = 1 + gt; k <= m; k += kObjThreads32) {
            float q;
            if (k == 1) q = ln.g11 * S[1] + (m >= 2 ? ln.g12 * S[2] : 0.f);
            else if (k == m) q = ln.gNa * S[m - 1] + ln.gNb * S[m];
            else q = ax.ge * (S[k - 1] + S[k + 1]) + ax.gc * S[k];
            Q[k] = q;
        }
        if (gt == 0) { Q[0] = 0.f; Q[N] = 0.f; }
        __syncthreads();
        const int s = (N + kObjThreads32) / kObjThreads32;      // ceil((N + 1) / threads)
        const int k0 = m > 0 ? min(gt * s, N + 1) : 0, k1 = m > 0 ? min(k0 + s, N + 1) : 0;
        // anti-causal: T_k = q_k + g_{k+1} T_{k+1}, T_N = 0 (g_N = dB); a
        // thread's chunk reads and writes only its own entries of Q
        {
            float qq = 0.f;
            for (int k = k1 - 1; k >= k0; --k) {
                const float g = (k == N - 1) ? ln.dB : d;
                qq = (k == N) ? 0.f : g * qq + Q[k];
            }
            float p = ax.dpow[k1 - k0];
            if (k0 <= N - 1 && N - 1 < k1) p *= ln.rB;
            affine_scan32<false>(p, qq, lane);
            if (lane == 0) totA[grp][warp] = make_float2(p, qq);
            __syncthreads();
            float yin = 0.f;                                     // carry from the warps to the right
            for (int w = NW - 1; w > warp; --w) yin = totA[grp][w].x * yin + totA[grp][w].y;
            const float pn = __shfl_down_sync(0xffffffffu, p, 1), qn = __shfl_down_sync(0xffffffffu, qq, 1);
            float y = (lane == 31) ? yin : pn * yin + qn;
            for (int k = k1 - 1; k >= k0; --k) {
                const float g = (k == N - 1) ? ln.dB : d;
                y = (k == N) ? 0.f : g * y + Q[k];
                Q[k] = y;
            }
        }
        // causal: e_k = g_k e_{k-1} + (1 - g_k^2) T_k, e_0 = 0 (g_1 = dA, g_N = dB)
        {
            float qq = 0.f;
            for (int k = k0; k < k1; ++k) {
                const float g = (k == 1) ? ln.dA : (k == N ? ln.dB : d);
                const float cg = (k == 1) ? ln.cA : (k == N ? ln.cB : c);
                qq = (k == 0) ? 0.f : g * qq + cg * Q[k];
            }
            float p = ax.dpow[k1 - k0];
            if (k0 <= 1 && 1 < k1) p *= ln.rA;
            if (k0 <= N && N < k1) p *= ln.rB;
            affine_scan32<true>(p, qq, lane);
            if (lane == 31) totC[grp][warp] = make_float2(p, qq);
            __syncthreads();
            float yin = 0.f;                                     // carry from the warps to the left
            for (int w = 0; w < warp; ++w) yin = totC[grp][w].x * yin + totC[grp][w].y;
            const float pp = __shfl_up_sync(0xffffffffu, p, 1), qp = __shfl_up_sync(0xffffffffu, qq, 1);
            float y = (lane == 0) ? yin : pp * yin + qp;
            for (int k = k0; k < k1; ++k) {
                const float g = (k == 1) ? ln.dA : (k == N ? ln.dB : d);
                const float cg = (k == 1) ? ln.cA : (k == N ? ln.cB : c);
                y = (k == 0) ? 0.f : g * y + cg * Q[k];
                Q[k] = y;
            }
        }
        __syncthreads();
        // e += A' e^{-alpha (x - a)} + B' e^{-alpha (b - x)} with e_0 = e_N = 0
        if (gt == 0 && m > 0) {
            const float Bp = -Q[N] * ln.inv, Ap = -Bp * ln.mu;
            l_Ad[grp] = Ap * ln.dA;
            l_Bd[grp] = Bp * ln.dB;
        }
        __syncthreads();
        {
            const int mj = l_m[ij];
            const long long bj = l_base[ij], pj = l_pos[ij];
            const float *Hj = smf + (size_t)ij * 4 * slot, *Lj = Hj + slot, *Qj = Hj + 3 * slot;
            const float Ad = l_Ad[ij], Bd = l_Bd[ij];
            for (long long r = p_lo + ii; r <= p_hi; r += NT / CPB) {
                const long long kk = r - pj + 1;
                if (kk >= 1 && kk <= mj) {
                    const int k = (int)kk;
                    const float e = Qj[k] + Ad * ax.dpow[k - 1] + Bd * ax.dpow[mj - k];
                    const float v = Hj[k] + Lj[k];
                    const long long at = bj + (k - 1) * st;
                    const float rr = (mode == OBJF_LINV) ? v - e : e;
                    out[at] = accum ? out[at] + rr : rr;
                    if (mode == OBJF_BOTH) {
                        out2[at] = v - e;
                        if (out3) out3[at] = e;
                    }
                }
            }
        }
    }
}

// out = sum_t c_t x_t in float32 (the partial sums of F)
struct CombTermsF {
    int n;
    float c[kCombMax];
    const float *x[kCombMax];
};
// Both kernels below touch the interior nodes only, row by row (the line
// objects of the contiguous axis): outside the domain every field stays zero.
__global__ void __launch_bounds__(256) k_obj_combine32(CombTermsF t, const ObjLineF *rows, int nrows, float *out)
{
    for (int li = blockIdx.x; li < nrows; li += gridDim.x) {
        const long long base = rows[li].base;
        const int m = rows[li].m;
        for (int k = threadIdx.x; k < m; k += blockDim.x) {
            const long long i = base + k;
            float v = 0.f;
            for (int j = 0; j < t.n; ++j) v += t.c[j] * t.x[j][i];
            out[i] = v;
        }
    }
}

// next level in pair arithmetic: (nh, nl) = a u + b up + c (F + sum_t c_t x_t)
__global__ void __launch_bounds__(256) k_obj_level32(CombTermsF t, const ObjLineF *rows, int nrows, const float *uh,
                                                     const float *ul, const float *ph, const float *pl, float a,
                                                     float b, float cF, float *nh, float *nl)
{
    for (int li = blockIdx.x; li < nrows; li += gridDim.x) {
        const long long base = rows[li].base;
        const int m = rows[li].m;
        for (int k = threadIdx.x; k < m; k += blockDim.x) {
            const long long i = base + k;
            float F = 0.f;
            for (int j = 0; j < t.n; ++j) F += t.c[j] * t.x[j][i];
            float h, l;
            molt::level_pair(uh[i], ul[i], b != 0.f ? ph[i] : 0.f, b != 0.f ? pl[i] : 0.f, F, a, b, cF, h, l);
            nh[i] = h;
            nl[i] = l;
        }
    }
}

// ---------------------------------------------------------------------------
// host constants
// ---------------------------------------------------------------------------
// int_0^nu t^k e^{-t} dt, k = 0, 1, 2: the power series below 1 (the closed
// forms cancel for short cells), the closed forms above
double exp_moment(int k, double nu)
{
    if (nu < 1.0) {
        double term = std::pow(nu, k + 1), sum = 0.0;   // term = (-1)^i nu^{k+1+i} / i!
        for (int i = 0; i < 60; ++i) {
            const double t = term / (double)(k + 1 + i);
            sum += t;
            if (std::fabs(t) < 1e-18 * std::fabs(sum)) break;
            term *= -nu / (double)(i + 1);
        }
        return sum;
    }
    const double e = std::exp(-nu);
    if (k == 0) return -std::expm1(-nu);
    if (k == 1) return 1.0 - (1.0 + nu) * e;
    return 2.0 - (2.0 + nu * (2.0 + nu)) * e;
}

// w[i] = (alpha/2) int_0^len e^{-alpha s} l_i(s) ds, l_i the Lagrange basis of
// the nodes s_0, s_1, s_2 (s measured from the destination node into the cell).
// With t = alpha s: l_i = (t^2 - alpha (sa + sb) t + alpha^2 sa sb) / (alpha^2
// (s_i - sa)(s_i - sb)) and ds = dt / alpha.
void obj_cell_weights(const double s[3], double len, double alpha, double w[3])
{
    const double nu = alpha * len;
    const double M0 = exp_moment(0, nu), M1 = exp_moment(1, nu), M2 = exp_moment(2, nu);
    for (int i = 0; i < 3; ++i) {
        const double sa = s[(i + 1) % 3], sb = s[(i + 2) % 3];
        const double num = M2 - alpha * (sa + sb) * M1 + alpha * alpha * sa * sb * M0;
        w[i] = num / (2.0 * alpha * alpha * (s[i] - sa) * (s[i] - sb));
    }
}

// the per-line constants of a line object of m interior nodes
ObjLine make_line(long long base, int m, double h, double ga, double gb, double alpha)
{
    ObjLine L{};
    L.base = base;
    L.m = m;
    const double x1 = ga, xm = ga + (double)(m - 1) * h, b = xm + gb;
    const double x2 = (m >= 2) ? ga + h : b;              // node 2 (b itself when m = 1)
    const double xm1 = (m >= 2) ? xm - h : 0.0;           // node m - 1 (a itself when m = 1)
    L.dA = std::exp(-alpha * ga);
    L.dB = std::exp(-alpha * gb);
    L.rA = std::exp(-alpha * (ga - h));
    L.rB = std::exp(-alpha * (gb - h));
    L.mu = std::exp(-alpha * b);
    L.inv = 1.0 / (-std::expm1(-2.0 * alpha * b));
    double w[3];
    {   // J^R_0: destination a, cell [a, x_1], nodes a, x_1, x_2
        const double s[3] = {0.0, x1, x2};
        obj_cell_weights(s, x1, alpha, w);
        L.wl[0] = w[1]; L.wl[1] = w[2];
    }
    {   // J^L_1: destination x_1, cell [a, x_1], nodes a, x_1, x_2
        const double s[3] = {x1, 0.0, x1 - x2};
        obj_cell_weights(s, x1, alpha, w);
        L.wl[2] = w[1]; L.wl[3] = w[2];
    }
    {   // J^R_1: destination x_1, cell [x_1, x_2], nodes a, x_1, x_2
        const double s[3] = {-x1, 0.0, x2 - x1};
        obj_cell_weights(s, x2 - x1, alpha, w);
        L.wl[4] = w[1]; L.wl[5] = w[2];
    }
    {   // J^L_{m+1}: destination b, cell [x_m, b], nodes x_{m-1}, x_m, b
        const double s[3] = {b - xm1, b - xm, 0.0};
        obj_cell_weights(s, b - xm, alpha, w);
        L.wr[0] = w[1]; L.wr[1] = w[0];
    }
    {   // J^L_m: destination x_m, cell [x_{m-1}, x_m], nodes x_{m-1}, x_m, b
        const double s[3] = {xm - xm1, 0.0, xm - b};
        obj_cell_weights(s, xm - xm1, alpha, w);
        L.wr[2] = w[1]; L.wr[3] = w[0];
    }
    {   // J^R_m: destination x_m, cell [x_m, b], nodes x_{m-1}, x_m, b
        const double s[3] = {xm1 - xm, 0.0, b - xm};
        obj_cell_weights(s, b - xm, alpha, w);
        L.wr[4] = w[1]; L.wr[5] = w[0];
    }
    return L;
}


// Row k (1 <= k <= N-1) of the difference form as weights on the node
// values v_0..v_N (beta, a dense vector): (v_k - g_k v_{k-1})/(1 - g_k^2) -
// g_{k+1}(v_{k+1} - g_{k+1} v_k)/(1 - g_{k+1}^2) minus the same combination of
// the increments, J^L_k - g_k J^R_{k-1} over (1 - g_k^2), ..., + J^R_k.  x: node
// positions x_0..x_N; the increments use the quadrature rule of the line.
std::vector<double> diff_row(const std::vector<double> &x, int k, double alpha)
{
    const int N = (int)x.size() - 1;
    std::vector<double> b(N + 1, 0.0);
    auto g = [&](int j) { return std::exp(-alpha * (x[j] - x[j - 1])); };   // decay of cell j
    auto add_JL = [&](int j, double c) {   // c J^L_j: cell [x_{j-1}, x_j], destination x_j
        const int c0 = (j + 1 <= N) ? j - 1 : j - 2;
        double ts[3], w[3];
        for (int i = 0; i < 3; ++i) ts[i] = x[j] - x[c0 + i];
        obj_cell_weights(ts, x[j] - x[j - 1], alpha, w);
        for (int i = 0; i < 3; ++i) b[c0 + i] += c * w[i];
    };
    auto add_JR = [&](int j, double c) {   // c J^R_j: cell [x_j, x_{j+1}], destination x_j
        const int c0 = (j - 1 >= 0) ? j - 1 : j;
        double ts[3], w[3];
        for (int i = 0; i < 3; ++i) ts[i] = x[c0 + i] - x[j];
        obj_cell_weights(ts, x[j + 1] - x[j], alpha, w);
        for (int i = 0; i < 3; ++i) b[c0 + i] += c * w[i];
    };
    const double gk = g(k), gk1 = g(k + 1), ik = 1.0 / (1.0 - gk * gk), ik1 = 1.0 / (1.0 - gk1 * gk1);
    b[k] += ik + gk1 * gk1 * ik1;
    b[k - 1] -= gk * ik;
    b[k + 1] -= gk1 * ik1;
    add_JL(k, -ik);
    add_JR(k - 1, gk * ik);
    add_JL(k + 1, gk1 * ik1);
    add_JR(k, -gk1 * gk1 * ik1);
    add_JR(k, -1.0);
    return b;
}

// weight of v_j in the second divided difference over the nodes t-1, t, t+1
double ddiff_w(const std::vector<double> &x, int t, int j)
{
    const double a = x[t - 1], c = x[t], e = x[t + 1];
    if (j == t - 1) return 2.0 / ((a - c) * (a - e));
    if (j == t) return 2.0 / ((c - a) * (c - e));
    return 2.0 / ((e - a) * (e - c));
}

// node positions of a line object (x_0 = a = 0)
std::vector<double> obj_positions(int m, double h, double ga, double gb)
{
    std::vector<double> x(m + 2);
    x[0] = 0.0;
    for (int j = 1; j <= m; ++j) x[j] = ga + (double)(j - 1) * h;
    x[m + 1] = x[m] + gb;
    return x;
}

// the float32 constants of a line object.  The rows 1 and N-1 of the
// difference form are computed in float64 from the increments and written
// as weights on the second divided differences (scaled by h^2): a row
// vanishes on linear data, so node 0 (node N) carries only s_1 (s_m), node
// 3 (node N-3) only s_2 (s_{m-1}).
ObjLineF make_line32(long long base, int m, double h, double ga, double gb, double alpha)
{
    ObjLineF L{};
    L.base = base;
    L.m = m;
    const std::vector<double> x = obj_positions(m, h, ga, gb);
    const int N = m + 1;
    const double b = x[N];
    L.dA = (float)std::exp(-alpha * ga);
    L.dB = (float)std::exp(-alpha * gb);
    L.rA = (float)std::exp(-alpha * (ga - h));
    L.rB = (float)std::exp(-alpha * (gb - h));
    L.cA = (float)(-std::expm1(-2.0 * alpha * ga));
    L.cB = (float)(-std::expm1(-2.0 * alpha * gb));
    L.mu = (float)std::exp(-alpha * b);
    L.inv = (float)(1.0 / (-std::expm1(-2.0 * alpha * b)));
    const double h2 = h * h;
    // s_1 = h^2 divided difference over (x_0, x_1, x_2) = p1 (v_2 - v_1) - q1 (v_1 - v_0)
    L.p1 = (float)(2.0 * h2 / ((x[2] - x[0]) * (x[2] - x[1])));
    L.q1 = (float)(2.0 * h2 / ((x[2] - x[0]) * (x[1] - x[0])));
    L.pm = (float)(2.0 * h2 / ((x[N] - x[m - 1]) * (x[N] - x[m])));
    L.qm = (float)(2.0 * h2 / ((x[N] - x[m - 1]) * (x[m] - x[m - 1])));
    const std::vector<double> b1 = diff_row(x, 1, alpha);
    L.g11 = (float)(b1[0] / ddiff_w(x, 1, 0) / h2);
    L.g12 = m >= 2 ? (float)(b1[3] / ddiff_w(x, 2, 3) / h2) : 0.f;
    const std::vector<double> bm = diff_row(x, m, alpha);
    L.gNb = (float)(bm[N] / ddiff_w(x, m, N) / h2);
    L.gNa = m >= 2 ? (float)(bm[N - 3] / ddiff_w(x, m - 1, N - 3) / h2) : 0.f;
    return L;
}

// the uniform rows: ge s_{k-1} + gc s_k + ge s_{k+1}, from a uniform line
void uniform_rows32(double h, double alpha, float &gc, float &ge)
{
    const int m = 9, k = 5;
    const std::vector<double> x = obj_positions(m, h, h, h);
    const std::vector<double> bk = diff_row(x, k, alpha);
    const double e = bk[k - 2] / ddiff_w(x, k - 1, k - 2);
    const double c = (bk[k - 1] - e * ddiff_w(x, k - 1, k - 1)) / ddiff_w(x, k, k - 1);
    ge = (float)(e / (h * h));
    gc = (float)(c / (h * h));
}

}  // namespace

using namespace molt;

struct mol_embed_ctx {
    int64_t nx = 0, ny = 0, N = 0;
    double hx = 0, hy = 0, alpha = 0, beta = 0;
    int P = 1;
    std::vector<double> tw;             // weights of C^m D^{p-m}: tw[p * 8 + m]
    ObjAxis ax[2]{};                    // x lines (rows), y lines (columns)
    ObjLine *lines[2] = {nullptr, nullptr};
    int nlines[2] = {0, 0};
    double *dpow[2] = {nullptr, nullptr};
    double *V[kMaxP + 1] = {};          // V[1..P]: the Table 3 auxiliaries
    double *tmp = nullptr, *t1 = nullptr, *lev = nullptr, *Fb = nullptr;
    double *io[2] = {nullptr, nullptr}; // device copies of mol_embed_solve_host
    std::vector<void *> allocs;
    int smem = 0, grid = 1, slot = 2;     // sweep launch: shared memory, CTAs, elements per line array
    int smem32[2] = {0, 0}, grid32[2] = {1, 1};   // float32 sweep launch per axis
    int64_t launches = 0;
    std::string err;
    bool timing = false;                // per-kind CUDA events (0 x sweeps, 1 y sweeps, 2 combinations)
    int prec = 0;                       // MOL_FP64 or MOL_MIXED (float32 sweeps, float32-pair levels)
    ObjAxisF ax32[2]{};
    ObjLineF *lines32[2] = {nullptr, nullptr};
    float *dpow32[2] = {nullptr, nullptr};
    float *V32[kMaxP + 1] = {};
    float *tmp32 = nullptr, *t132 = nullptr, *t232 = nullptr, *t332 = nullptr, *Fb32 = nullptr;
    float *lh[3] = {nullptr, nullptr, nullptr}, *ll[3] = {nullptr, nullptr, nullptr};   // pair levels
    std::vector<cudaEvent_t> ev_pool;
    struct Rec { int kind; cudaEvent_t a, b; };
    std::vector<Rec> recs;
};

namespace {

mol_status efail(mol_embed_ctx *e, mol_status st, const std::string &msg)
{
    if (e) e->err = msg;
    else set_global_error(msg);
    return st;
}

#define ECK(expr, what)                                                                   \
    do {                                                                                  \
        cudaError_t e_ = (expr);                                                          \
        if (e_ != cudaSuccess) return efail(e, MOL_ECUDA, std::string(what) + ": " + cudaGetErrorString(e_)); \
    } while (0)

mol_status ealloc(mol_embed_ctx *e, void **p, size_t bytes)
{
    if (alloc_injected_failure())
        return efail(e, MOL_ENOMEM, "device allocation of " + std::to_string(bytes) + " bytes failed (injected)");
    cudaError_t r = cudaMalloc(p, bytes);
    if (r != cudaSuccess) {
        cudaGetLastError();
        return efail(e, MOL_ENOMEM, "device allocation of " + std::to_string(bytes) + " bytes failed");
    }
    e->allocs.push_back(*p);
    return MOL_OK;
}

void efree_all(mol_embed_ctx *e)
{
    for (auto &r : e->recs) { e->ev_pool.push_back(r.a); e->ev_pool.push_back(r.b); }
    e->recs.clear();
    for (cudaEvent_t v : e->ev_pool) cudaEventDestroy(v);
    e->ev_pool.clear();
    for (void *p : e->allocs) cudaFree(p);
    e->allocs.clear();
}

cudaEvent_t take_event(mol_embed_ctx *e)
{
    if (!e->ev_pool.empty()) {
        cudaEvent_t v = e->ev_pool.back();
        e->ev_pool.pop_back();
        return v;
    }
    cudaEvent_t v = nullptr;
    return cudaEventCreate(&v) == cudaSuccess ? v : nullptr;
}

// events around one launch of the given kind while pass timing is on
struct Timed {
    mol_embed_ctx *e;
    int kind;
    cudaStream_t s;
    cudaEvent_t a = nullptr, b = nullptr;
    Timed(mol_embed_ctx *e_, int k, cudaStream_t s_) : e(e_), kind(k), s(s_)
    {
        if (!e->timing) return;
        a = take_event(e);
        b = take_event(e);
        if (a) cudaEventRecord(a, s);
    }
    ~Timed()
    {
        if (!a || !b) return;
        cudaEventRecord(b, s);
        e->recs.push_back({kind, a, b});
    }
};

// one sweep along axis a (0: the rows, 1: the columns of the field)
mol_status sweep(mol_embed_ctx *e, int a, const double *in, double *out, int mode, int accum, const double *sub,
                 cudaStream_t s)
{
    if (e->nlines[a] == 0) return MOL_OK;
    const int grid = std::min(e->grid, (e->nlines[a] + kObjWarps - 1) / kObjWarps);
    Timed t(e, a, s);
    k_obj_sweep<<<grid, 32 * kObjWarps, e->smem, s>>>(e->ax[a], e->lines[a], e->nlines[a], in, out, sub, mode,
                                                        accum, e->slot);
    ++e->launches;
    ECK(cudaGetLastError(), "line-object sweep");
    return MOL_OK;
}

mol_status combine(mol_embed_ctx *e, const CombTerms &t, double *out, cudaStream_t s)
{
    const int64_t blocks = std::min<int64_t>((e->N + 255) / 256, 4096);
    Timed tm(e, 2, s);
    k_obj_combine<<<(unsigned)blocks, 256, 0, s>>>(t, out, e->N);
    ++e->launches;
    ECK(cudaGetLastError(), "combine");
    return MOL_OK;
}

#define EST(expr)                              \
    do {                                       \
        mol_status st_ = (expr);               \
        if (st_ != MOL_OK) return st_;         \
    } while (0)

// out = C v = L_y^{-1} D_x v + L_x^{-1} D_y v   (eq. C_def_ADI)
mol_status apply_C(mol_embed_ctx *e, const double *v, double *out, cudaStream_t s)
{
    EST(sweep(e, 0, v, e->t1, OBJ_D, 0, nullptr, s));          // t1 = D_x v
    EST(sweep(e, 1, e->t1, out, OBJ_LINV, 0, nullptr, s));     // out = L_y^{-1} t1
    EST(sweep(e, 1, v, e->t1, OBJ_D, 0, nullptr, s));          // t1 = D_y v
    return sweep(e, 0, e->t1, out, OBJ_LINV, 1, nullptr, s);   // out += L_x^{-1} t1
}

// out = D v = v - L_x^{-1} L_y^{-1} v   (eq. D_def_ADI)
mol_status apply_Dadi(mol_embed_ctx *e, const double *v, double *out, cudaStream_t s)
{
    EST(sweep(e, 1, v, e->t1, OBJ_LINV, 0, nullptr, s));       // t1 = L_y^{-1} v
    return sweep(e, 0, e->t1, out, OBJ_SUB, 0, v, s);          // out = v - L_x^{-1} t1
}

// lev = ea u + eb up + ec F[u]   (eq. Full_2D, terms in Table 3 order: after
// stage p, V[k] = C^{p-k+1} D^{k-1} u)
mol_status run_update(mol_embed_ctx *e, const double *u, const double *up, double *out, double ea, double eb,
                      double ec, cudaStream_t s)
{
    const int P = e->P;
    for (int p = 1; p <= P; ++p) {
        if (p == 1) {
            EST(apply_C(e, u, e->V[1], s));
        } else {
            EST(apply_Dadi(e, e->V[p - 1], e->V[p], s));
            for (int k = 1; k < p; ++k) {
                EST(apply_C(e, e->V[k], e->tmp, s));
                std::swap(e->V[k], e->tmp);
            }
        }
        // the stage-1 term tw_11 C u is still in tmp after stage 2 (whose only C
        // swaps V_1 out): with P > 1 it joins stage 2's sum, no pass of its own
        if (p == 1 && P > 1) continue;
        CombTerms t{};
        const bool last = p == P;
        if (p == 2) { t.c[t.n] = (last ? ec : 1.0) * e->tw[1 * 8 + 1]; t.x[t.n++] = e->tmp; }
        if (p > 2) { t.c[t.n] = last ? ec : 1.0; t.x[t.n++] = e->Fb; }
        for (int k = 1; k <= p; ++k) {
            t.c[t.n] = (last ? ec : 1.0) * e->tw[p * 8 + (p - k + 1)];
            t.x[t.n++] = e->V[k];
        }
        if (last) {
            if (ea != 0.0) { t.c[t.n] = ea; t.x[t.n++] = u; }
            if (eb != 0.0) { t.c[t.n] = eb; t.x[t.n++] = up; }
        }
        EST(combine(e, t, last ? out : e->Fb, s));
    }
    return MOL_OK;
}

// ---- float32 sweeps (MOL_MIXED) ----
// one difference-form sweep along axis a; lo: the lo plane when in is a pair level
mol_status sweep32(mol_embed_ctx *e, int a, const float *in, const float *lo, float *out, float *out2, int mode,
                   int accum, cudaStream_t s, float *out3 = nullptr)
{
    if (e->nlines[a] == 0) return MOL_OK;
    const int cpb = kObjCpb[a];
    const int grid = std::min(e->grid32[a], (e->nlines[a] + cpb - 1) / cpb);
    Timed t(e, a, s);
    auto launch = [&](auto kern) {
        kern<<<grid, kObjThreads32 * cpb, e->smem32[a], s>>>(e->ax32[a], e->lines32[a], e->nlines[a], in, lo, out,
                                                             out2, out3, mode, accum, e->slot);
    };
    if (cpb == 1) {
        if (lo) launch(k_obj_sweep32<true, 1>);
        else launch(k_obj_sweep32<false, 1>);
    } else {
        if (lo) launch(k_obj_sweep32<true, kObjCpb[1]>);
        else launch(k_obj_sweep32<false, kObjCpb[1]>);
    }
    ++e->launches;
    ECK(cudaGetLastError(), "line-object sweep (float32)");
    return MOL_OK;
}

// out = C v (eq. C_def_ADI) with L^{-1} = 1 - D: D_x v - D_y D_x v + D_y v - D_x D_y v.
// dyv: D_y v when an earlier sweep has formed it, else null.
mol_status apply_C32(mol_embed_ctx *e, const float *v, const float *vlo, float *out, cudaStream_t s,
                     const float *dyv = nullptr)
{
    EST(sweep32(e, 0, v, vlo, e->t132, nullptr, OBJF_D, 0, s));               // t1 = D_x v
    EST(sweep32(e, 1, e->t132, nullptr, out, nullptr, OBJF_LINV, 0, s));      // out = L_y^{-1} t1
    if (!dyv) {
        EST(sweep32(e, 1, v, vlo, e->t132, nullptr, OBJF_D, 0, s));           // t1 = D_y v
        dyv = e->t132;
    }
    return sweep32(e, 0, dyv, nullptr, out, nullptr, OBJF_LINV, 1, s);       // out += L_x^{-1} D_y v
}

// out = D v (eq. D_def_ADI) = v - L_x^{-1} L_y^{-1} v = D_y v + D_x (L_y^{-1} v); dyv, when
// given, receives D_y v as well
mol_status apply_D32(mol_embed_ctx *e, const float *v, float *out, cudaStream_t s, float *dyv = nullptr)
{
    EST(sweep32(e, 1, v, nullptr, out, e->t232, OBJF_BOTH, 0, s, dyv));       // out = D_y v, t2 = L_y^{-1} v
    return sweep32(e, 0, e->t232, nullptr, out, nullptr, OBJF_D, 1, s);       // out += D_x t2
}

mol_status combine32(mol_embed_ctx *e, const CombTermsF &t, float *out, cudaStream_t s)
{
    if (e->nlines[0] == 0) return MOL_OK;
    Timed tm(e, 2, s);
    k_obj_combine32<<<std::min(e->nlines[0], e->grid32[0]), 256, 0, s>>>(t, e->lines32[0], e->nlines[0], out);
    ++e->launches;
    ECK(cudaGetLastError(), "combine (float32)");
    return MOL_OK;
}

// F[u] of the pair level (uh, ul), Table 3 order as run_update.  With nh
// set: (nh, nl) = ea u + eb up + ec F in pair arithmetic; else F (float32)
// into F32.
mol_status run_update32(mol_embed_ctx *e, const float *uh, const float *ul, const float *ph, const float *pl,
                        float *nh, float *nl, float *F32, float ea, float eb, float ec, cudaStream_t s)
{
    const int P = e->P;
    for (int p = 1; p <= P; ++p) {
        if (p == 1) {
            EST(apply_C32(e, uh, ul, e->V32[1], s));
        } else {
            // D_y V_{p-1} serves both D V_{p-1} and C V_{p-1}: formed once
            EST(apply_D32(e, e->V32[p - 1], e->V32[p], s, e->t332));
            for (int k = 1; k < p; ++k) {
                EST(apply_C32(e, e->V32[k], nullptr, e->tmp32, s, k == p - 1 ? e->t332 : nullptr));
                std::swap(e->V32[k], e->tmp32);
            }
        }
        // F's partial sum.  The terms of stage 1 are tw_11 C u alone, and C u
        // is still in tmp32 after stage 2 (whose only C swaps V_1 out), so
        // with P > 1 they join the sum of stage 2 instead of a pass of their own
        if (p == 1 && P > 1) continue;
        CombTermsF t{};
        if (p == 2) { t.c[t.n] = (float)e->tw[1 * 8 + 1]; t.x[t.n++] = e->tmp32; }
        if (p > 2) { t.c[t.n] = 1.f; t.x[t.n++] = e->Fb32; }
        for (int k = 1; k <= p; ++k) {
            t.c[t.n] = (float)e->tw[p * 8 + (p - k + 1)];
            t.x[t.n++] = e->V32[k];
        }
        if (p < P || !nh) {
            EST(combine32(e, t, p < P ? e->Fb32 : F32, s));
        } else {
            if (e->nlines[0] == 0) continue;
            Timed tm(e, 2, s);
            k_obj_level32<<<std::min(e->nlines[0], e->grid32[0]), 256, 0, s>>>(t, e->lines32[0], e->nlines[0], uh, ul,
                                                                                ph, pl, ea, eb, ec, nh, nl);
            ++e->launches;
            ECK(cudaGetLastError(), "level update (float32 pairs)");
        }
    }
    return MOL_OK;
}

mol_status to_pair(mol_embed_ctx *e, const double *x, int k, cudaStream_t s)
{
    ECK(launch_to_pair(x, e->lh[k], e->ll[k], e->N, s), "level conversion");
    ++e->launches;
    return MOL_OK;
}

mol_status from_pair(mol_embed_ctx *e, int k, double *x, cudaStream_t s)
{
    ECK(launch_from_pair(e->lh[k], e->ll[k], x, e->N, s), "level conversion");
    ++e->launches;
    return MOL_OK;
}

mol_status check_dev(mol_embed_ctx *e, const void *p, const char *name)
{
    if (!p) return efail(e, MOL_EINVAL, std::string(name) + " is NULL");
    cudaPointerAttributes at{};
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return efail(e, MOL_EINVAL, std::string(name) + ": not a CUDA pointer");
    }
    if (at.type != cudaMemoryTypeDevice && at.type != cudaMemoryTypeManaged)
        return efail(e, MOL_EINVAL, std::string(name) + " must be device memory");
    return MOL_OK;
}

}  // namespace

extern "C" {

mol_status mol_embed_create(const mol_embed_geom *g, double c, double dt, double beta, int P, mol_prec prec,
                            mol_embed *out)
{
    if (!out) return efail(nullptr, MOL_EINVAL, "out is NULL");
    *out = nullptr;
    if (!g) return efail(nullptr, MOL_EINVAL, "geometry is NULL");
    if (g->nx < 3 || g->ny < 3 || g->nx > (1 << 15) || g->ny > (1 << 15))
        return efail(nullptr, MOL_EINVAL, "nx and ny must be in 3..32768");
    if (!(g->hx > 0) || !(g->hy > 0) || !std::isfinite(g->hx) || !std::isfinite(g->hy))
        return efail(nullptr, MOL_EINVAL, "hx and hy must be positive");
    if (!g->row_lo || !g->row_hi || !g->row_gap_lo || !g->row_gap_hi || !g->col_lo || !g->col_hi ||
        !g->col_gap_lo || !g->col_gap_hi)
        return efail(nullptr, MOL_EINVAL, "geometry arrays must not be NULL");
    if (P < 1 || P > kMaxP) return efail(nullptr, MOL_EINVAL, "P must be in 1..5");
    if (prec != MOL_FP64 && prec != MOL_MIXED) return efail(nullptr, MOL_EINVAL, "unknown precision");
    if (!(c > 0) || !(dt > 0) || !std::isfinite(c) || !std::isfinite(dt))
        return efail(nullptr, MOL_EINVAL, "c and dt must be positive");
    const double bmax = beta_max_of(P);
    if (beta <= 0) beta = bmax;
    if (beta > bmax * (1.0 + 1e-12))
        return efail(nullptr, MOL_EUNSTABLE, "beta above beta_max(P): the scheme is not A-stable");

    const int64_t nx = g->nx, ny = g->ny;
    // lines, and the agreement of rows and columns on the interior nodes
    std::vector<int> seen((size_t)(nx * ny), 0);
    int64_t maxm = 1;
    for (int a = 0; a < 2; ++a) {
        const int64_t nl = a == 0 ? ny : nx, len = a == 0 ? nx : ny;
        const int64_t *lo = a == 0 ? g->row_lo : g->col_lo, *hi = a == 0 ? g->row_hi : g->col_hi;
        const double *ga = a == 0 ? g->row_gap_lo : g->col_gap_lo, *gb = a == 0 ? g->row_gap_hi : g->col_gap_hi;
        for (int64_t l = 0; l < nl; ++l) {
            if (lo[l] > hi[l]) continue;
            const std::string who = std::string(a == 0 ? "row " : "column ") + std::to_string(l) + ": ";
            if (lo[l] < 0 || hi[l] >= len) return efail(nullptr, MOL_EINVAL, who + "interior nodes outside the grid");
            if (hi[l] - lo[l] + 1 > kObjMaxM)
                return efail(nullptr, MOL_EINVAL, who + "more than " + std::to_string(kObjMaxM) + " interior nodes");
            if (!(ga[l] > 0) || !(gb[l] > 0) || !std::isfinite(ga[l]) || !std::isfinite(gb[l]))
                return efail(nullptr, MOL_EINVAL, who + "gaps must be positive and finite");
            for (int64_t k = lo[l]; k <= hi[l]; ++k) seen[(size_t)(a == 0 ? l * nx + k : k * nx + l)] |= 1 << a;
            maxm = std::max<int64_t>(maxm, hi[l] - lo[l] + 1);
        }
    }
    for (int v : seen)
        if (v == 1 || v == 2)
            return efail(nullptr, MOL_EINVAL, "rows and columns disagree on which nodes are interior");

    mol_embed_ctx *e = new mol_embed_ctx();
    e->nx = nx;
    e->ny = ny;
    e->N = nx * ny;
    e->hx = g->hx;
    e->hy = g->hy;
    e->P = P;
    e->prec = prec;
    e->beta = beta;
    e->alpha = beta / (c * dt);                          // eq. L_def
    e->tw.assign(8 * 8, 0.0);
    for (int p = 1; p <= P; ++p)
        for (int m = 1; m <= p; ++m) e->tw[p * 8 + m] = term_weight(p, m, beta);
    mol_status st = MOL_OK;
    cudaError_t ce;
    for (int a = 0; a < 2 && st == MOL_OK; ++a) {
        const double h = a == 0 ? e->hx : e->hy, alpha = e->alpha;
        ObjAxis &X = e->ax[a];
        X.stride = a == 0 ? 1 : nx;
        X.d = std::exp(-alpha * h);
        double w[3];
        const double sL[3] = {h, 0.0, -h}, sR[3] = {-h, 0.0, h};
        obj_cell_weights(sL, h, alpha, w);
        for (int i = 0; i < 3; ++i) X.uL[i] = w[i];
        obj_cell_weights(sR, h, alpha, w);
        for (int i = 0; i < 3; ++i) X.uR[i] = w[i];
        std::vector<double> tab(kObjMaxM + 1);
        for (int k = 0; k <= kObjMaxM; ++k) tab[k] = std::exp(-alpha * h * (double)k);
        std::vector<ObjLine> ls;
        const int64_t nl = a == 0 ? ny : nx;
        const int64_t *lo = a == 0 ? g->row_lo : g->col_lo, *hi = a == 0 ? g->row_hi : g->col_hi;
        const double *ga = a == 0 ? g->row_gap_lo : g->col_gap_lo, *gb = a == 0 ? g->row_gap_hi : g->col_gap_hi;
        for (int64_t l = 0; l < nl; ++l) {
            if (lo[l] > hi[l]) continue;
            const long long base = a == 0 ? l * nx + lo[l] : lo[l] * nx + l;   // first interior node
            ls.push_back(make_line(base, (int)(hi[l] - lo[l] + 1), h, ga[l], gb[l], alpha));
        }
        e->nlines[a] = (int)ls.size();
        if ((st = ealloc(e, (void **)&e->dpow[a], sizeof(double) * tab.size())) != MOL_OK) break;
        if ((ce = cudaMemcpy(e->dpow[a], tab.data(), sizeof(double) * tab.size(), cudaMemcpyHostToDevice)) != cudaSuccess) {
            st = efail(e, MOL_ECUDA, "table upload");
            break;
        }
        X.dpow = e->dpow[a];
        if (!ls.empty()) {
            if ((st = ealloc(e, (void **)&e->lines[a], sizeof(ObjLine) * ls.size())) != MOL_OK) break;
            if ((ce = cudaMemcpy(e->lines[a], ls.data(), sizeof(ObjLine) * ls.size(), cudaMemcpyHostToDevice)) !=
                cudaSuccess) {
                st = efail(e, MOL_ECUDA, "line table upload");
                break;
            }
        }
        if (prec == MOL_MIXED) {
            // float32 constants of the difference form
            ObjAxisF &Y = e->ax32[a];
            Y.stride = X.stride;
            Y.d = (float)X.d;
            Y.c = (float)(-std::expm1(-2.0 * alpha * h));
            uniform_rows32(h, alpha, Y.gc, Y.ge);
            std::vector<float> tab32(tab.begin(), tab.end());
            std::vector<ObjLineF> ls32;
            for (int64_t l = 0; l < nl; ++l) {
                if (lo[l] > hi[l]) continue;
                const long long base = a == 0 ? l * nx + lo[l] : lo[l] * nx + l;
                ls32.push_back(make_line32(base, (int)(hi[l] - lo[l] + 1), h, ga[l], gb[l], alpha));
            }
            if ((st = ealloc(e, (void **)&e->dpow32[a], sizeof(float) * tab32.size())) != MOL_OK) break;
            if ((ce = cudaMemcpy(e->dpow32[a], tab32.data(), sizeof(float) * tab32.size(), cudaMemcpyHostToDevice)) !=
                cudaSuccess) {
                st = efail(e, MOL_ECUDA, "table upload");
                break;
            }
            Y.dpow = e->dpow32[a];
            if (!ls32.empty()) {
                if ((st = ealloc(e, (void **)&e->lines32[a], sizeof(ObjLineF) * ls32.size())) != MOL_OK) break;
                if ((ce = cudaMemcpy(e->lines32[a], ls32.data(), sizeof(ObjLineF) * ls32.size(),
                                     cudaMemcpyHostToDevice)) != cudaSuccess) {
                    st = efail(e, MOL_ECUDA, "line table upload");
                    break;
                }
            }
        }
    }
    // work fields; every sweep writes only interior nodes, so they start at zero
    std::vector<std::pair<void **, size_t>> work;
    const size_t plane = sizeof(double) * (size_t)e->N, plane32 = sizeof(float) * (size_t)e->N;
    if (prec == MOL_FP64) {
        for (double **b : {&e->tmp, &e->t1, &e->lev, &e->Fb}) work.push_back({(void **)b, plane});
        for (int k = 1; k <= P; ++k) work.push_back({(void **)&e->V[k], plane});
    } else {
        for (float **b : {&e->tmp32, &e->t132, &e->t232, &e->t332, &e->Fb32}) work.push_back({(void **)b, plane32});
        for (int k = 1; k <= P; ++k) work.push_back({(void **)&e->V32[k], plane32});
        for (int k = 0; k < 3; ++k) {
            work.push_back({(void **)&e->lh[k], plane32});
            work.push_back({(void **)&e->ll[k], plane32});
        }
    }
    for (auto &w : work) {
        if (st != MOL_OK) break;
        if ((st = ealloc(e, w.first, w.second)) != MOL_OK) break;
        if ((ce = cudaMemset(*w.first, 0, w.second)) != cudaSuccess) st = efail(e, MOL_ECUDA, "memset");
    }
    if (st == MOL_OK) {
        // line arrays sized for the longest line (even, for 16-byte alignment)
        e->slot = (int)((maxm + 2 + 1) & ~(int64_t)1);
        // float64: two line arrays of doubles per warp; float32: four arrays of
        // floats per line
        int dev = 0, sms = 152, per_sm = 1;
        if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (prec == MOL_FP64) {
            e->smem = (int)(sizeof(double) * 2 * (size_t)e->slot * kObjWarps);
            if ((ce = cudaFuncSetAttribute(k_obj_sweep, cudaFuncAttributeMaxDynamicSharedMemorySize, e->smem)) !=
                cudaSuccess)
                st = efail(e, MOL_ECUDA, std::string("kernel attributes: ") + cudaGetErrorString(ce));
            if (st == MOL_OK && cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_obj_sweep, 32 * kObjWarps,
                                                                              e->smem) != cudaSuccess) {
                cudaGetLastError();
                per_sm = 1;
            }
        } else {
            const void *kf[2][2] = {{(const void *)k_obj_sweep32<true, 1>, (const void *)k_obj_sweep32<false, 1>},
                                    {(const void *)k_obj_sweep32<true, kObjCpb[1]>,
                                     (const void *)k_obj_sweep32<false, kObjCpb[1]>}};
            for (int a = 0; a < 2 && st == MOL_OK; ++a) {
                e->smem32[a] = (int)(sizeof(float) * 4 * (size_t)e->slot * kObjCpb[a]);
                for (int v = 0; v < 2 && st == MOL_OK; ++v)
                    if ((ce = cudaFuncSetAttribute(kf[a][v], cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                   e->smem32[a])) != cudaSuccess)
                        st = efail(e, MOL_ECUDA, std::string("kernel attributes: ") + cudaGetErrorString(ce));
                int ps = 1;
                if (st == MOL_OK && cudaOccupancyMaxActiveBlocksPerMultiprocessor(&ps, kf[a][0], kObjThreads32 *
                                                                                  kObjCpb[a], e->smem32[a]) !=
                                        cudaSuccess) {
                    cudaGetLastError();
                    ps = 1;
                }
                e->grid32[a] = std::max(1, sms) * std::max(1, ps);
            }
        }
        e->grid = std::max(1, sms) * std::max(1, per_sm);
    }
    if (st != MOL_OK) {
        set_global_error(e->err);
        efree_all(e);
        delete e;
        return st;
    }
    *out = e;
    return MOL_OK;
}

mol_status mol_embed_destroy(mol_embed e)
{
    if (!e) return MOL_OK;
    efree_all(e);
    delete e;
    return MOL_OK;
}

const char *mol_embed_last_error(mol_embed e) { return e ? e->err.c_str() : mol_last_error(nullptr); }

mol_status mol_embed_linv(mol_embed e, const double *v, double *w, int axis, void *stream)
{
    if (!e) return efail(nullptr, MOL_EINVAL, "handle is NULL");
    EST(check_dev(e, v, "v"));
    EST(check_dev(e, w, "w"));
    if (axis != 0 && axis != 1) return efail(e, MOL_EINVAL, "axis must be 0 (x) or 1 (y)");
    if (v == w) return efail(e, MOL_EINVAL, "v and w must not overlap");
    cudaStream_t s = (cudaStream_t)stream;
    if (e->prec == MOL_MIXED) {
        EST(to_pair(e, v, 0, s));
        ECK(cudaMemsetAsync(e->t132, 0, sizeof(float) * (size_t)e->N, s), "memset");
        EST(sweep32(e, axis, e->lh[0], e->ll[0], e->t132, nullptr, OBJF_LINV, 0, s));
        ECK(launch_from_f32(e->t132, w, e->N, s), "conversion");
        ++e->launches;
        return MOL_OK;
    }
    ECK(cudaMemsetAsync(w, 0, sizeof(double) * (size_t)e->N, s), "memset");
    return sweep(e, axis, v, w, OBJ_LINV, 0, nullptr, s);
}

mol_status mol_embed_apply_F(mol_embed e, const double *u, double *F, void *stream)
{
    if (!e) return efail(nullptr, MOL_EINVAL, "handle is NULL");
    EST(check_dev(e, u, "u"));
    EST(check_dev(e, F, "F"));
    if (u == F) return efail(e, MOL_EINVAL, "u and F must not overlap");
    cudaStream_t s = (cudaStream_t)stream;
    if (e->prec == MOL_MIXED) {
        EST(to_pair(e, u, 0, s));
        EST(run_update32(e, e->lh[0], e->ll[0], nullptr, nullptr, nullptr, nullptr, e->t232, 0.f, 0.f, 1.f, s));
        ECK(launch_from_f32(e->t232, F, e->N, s), "conversion");
        ++e->launches;
        return MOL_OK;
    }
    return run_update(e, u, nullptr, F, 0.0, 0.0, 1.0, s);
}

mol_status mol_embed_start(mol_embed e, const double *u0, double *u1, void *stream)
{
    if (!e) return efail(nullptr, MOL_EINVAL, "handle is NULL");
    EST(check_dev(e, u0, "u0"));
    EST(check_dev(e, u1, "u1"));
    if (u0 == u1) return efail(e, MOL_EINVAL, "u0 and u1 must not overlap");
    cudaStream_t s = (cudaStream_t)stream;
    if (e->prec == MOL_MIXED) {
        EST(to_pair(e, u0, 0, s));
        EST(run_update32(e, e->lh[0], e->ll[0], nullptr, nullptr, e->lh[1], e->ll[1], nullptr, 1.f, 0.f, 0.5f, s));
        return from_pair(e, 1, u1, s);
    }
    return run_update(e, u0, nullptr, u1, 1.0, 0.0, 0.5, s);
}

mol_status mol_embed_step(mol_embed e, double *u_prev, double *u_cur, int64_t nsteps, void *stream)
{
    if (!e) return efail(nullptr, MOL_EINVAL, "handle is NULL");
    EST(check_dev(e, u_prev, "u_prev"));
    EST(check_dev(e, u_cur, "u_cur"));
    if (u_prev == u_cur) return efail(e, MOL_EINVAL, "u_prev and u_cur must not overlap");
    if (nsteps < 0) return efail(e, MOL_EINVAL, "nsteps must be >= 0");
    cudaStream_t s = (cudaStream_t)stream;
    if (e->prec == MOL_MIXED) {
        if (nsteps == 0) return MOL_OK;
        // the levels as float32 pairs for the whole call (rotating through
        // three internal pair levels), converted back at the end
        EST(to_pair(e, u_prev, 0, s));
        EST(to_pair(e, u_cur, 1, s));
        int r[3] = {0, 1, 2};
        for (int64_t k = 0; k < nsteps; ++k) {
            EST(run_update32(e, e->lh[r[1]], e->ll[r[1]], e->lh[r[0]], e->ll[r[0]], e->lh[r[2]], e->ll[r[2]], nullptr,
                             2.f, -1.f, 1.f, s));
            const int t = r[0];
            r[0] = r[1];
            r[1] = r[2];
            r[2] = t;
        }
        EST(from_pair(e, r[0], u_prev, s));
        return from_pair(e, r[1], u_cur, s);
    }
    double *b[3] = {u_prev, u_cur, e->lev};
    for (int64_t k = 0; k < nsteps; ++k) {
        EST(run_update(e, b[1], b[0], b[2], 2.0, -1.0, 1.0, s));
        double *t = b[0];
        b[0] = b[1];
        b[1] = b[2];
        b[2] = t;
    }
    // the levels back into the caller's buffers: after k steps the roles
    // (previous, current, spare) have rotated k times through (u_prev, u_cur, lev)
    const size_t bytes = sizeof(double) * (size_t)e->N;
    if (b[1] == e->lev) {                 // (u_cur, lev, u_prev)
        ECK(cudaMemcpyAsync(u_prev, u_cur, bytes, cudaMemcpyDeviceToDevice, s), "level copy");
        ECK(cudaMemcpyAsync(u_cur, e->lev, bytes, cudaMemcpyDeviceToDevice, s), "level copy");
    } else if (b[0] == e->lev) {          // (lev, u_prev, u_cur)
        ECK(cudaMemcpyAsync(u_cur, u_prev, bytes, cudaMemcpyDeviceToDevice, s), "level copy");
        ECK(cudaMemcpyAsync(u_prev, e->lev, bytes, cudaMemcpyDeviceToDevice, s), "level copy");
    }
    return MOL_OK;
}

mol_status mol_embed_solve_host(mol_embed e, const double *u0, double *u_out, int64_t nsteps, void *stream)
{
    if (!e) return efail(nullptr, MOL_EINVAL, "handle is NULL");
    if (!u0 || !u_out) return efail(e, MOL_EINVAL, "u0 and u_out must not be NULL");
    if (nsteps < 0) return efail(e, MOL_EINVAL, "nsteps must be >= 0");
    cudaStream_t s = (cudaStream_t)stream;
    const size_t bytes = sizeof(double) * (size_t)e->N;
    for (int k = 0; k < 2; ++k)
        if (!e->io[k]) EST(ealloc(e, (void **)&e->io[k], bytes));
    ECK(cudaMemcpyAsync(e->io[0], u0, bytes, cudaMemcpyHostToDevice, s), "copy in");
    if (nsteps > 0) {
        EST(mol_embed_start(e, e->io[0], e->io[1], stream));
        EST(mol_embed_step(e, e->io[0], e->io[1], nsteps - 1, stream));
        ECK(cudaMemcpyAsync(u_out, e->io[1], bytes, cudaMemcpyDeviceToHost, s), "copy out");
    } else {
        ECK(cudaMemcpyAsync(u_out, e->io[0], bytes, cudaMemcpyDeviceToHost, s), "copy out");
    }
    ECK(cudaStreamSynchronize(s), "synchronize");
    return MOL_OK;
}

mol_status mol_embed_sync(mol_embed e, void *stream)
{
    if (!e) return efail(nullptr, MOL_EINVAL, "handle is NULL");
    ECK(cudaStreamSynchronize((cudaStream_t)stream), "synchronize");
    return MOL_OK;
}

int64_t mol_embed_launch_count(mol_embed e) { return e ? e->launches : 0; }

mol_status mol_embed_set_pass_timing(mol_embed e, int enable)
{
    if (!e) return efail(nullptr, MOL_EINVAL, "handle is NULL");
    e->timing = enable != 0;
    return MOL_OK;
}

mol_status mol_embed_pass_times(mol_embed e, double total_ms[3], int64_t launches[3])
{
    if (!e) return efail(nullptr, MOL_EINVAL, "handle is NULL");
    if (!total_ms || !launches) return efail(e, MOL_EINVAL, "output arrays must not be NULL");
    for (int k = 0; k < 3; ++k) { total_ms[k] = 0.0; launches[k] = 0; }
    for (auto &r : e->recs) {
        float ms = 0.f;
        cudaError_t ce = cudaEventSynchronize(r.b);
        if (ce == cudaSuccess) ce = cudaEventElapsedTime(&ms, r.a, r.b);
        if (ce != cudaSuccess) return efail(e, MOL_ECUDA, std::string("pass timing: ") + cudaGetErrorString(ce));
        total_ms[r.kind] += ms;
        launches[r.kind] += 1;
        e->ev_pool.push_back(r.a);
        e->ev_pool.push_back(r.b);
    }
    e->recs.clear();
    return MOL_OK;
}

}  // extern "C"
