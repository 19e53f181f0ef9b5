// molt_kernels.cuh -- device code of libmolt (sm_103a).
//
// One warp owns one grid line at a time.  The line sits in shared memory in
// 32 lane segments of m = ceil(n/32) points; segment s starts at s*ms with ms
// odd, so the 32 lanes walking their segments hit 32 different banks.  A CTA
// holds W lines (W warps) and moves them between HBM and shared memory in
// cooperative, coalesced phases: rows of W neighbouring lines for an axis with
// a stride (y, z), whole rows for the contiguous axis (x).
//
// The operator D = 1 - L^{-1} of one line (Sec. 2, eqs. L_Inverse, D_def_1d)
// is evaluated without forming L^{-1} v and subtracting it.  With the local
// increments of Sec. 2 (quadratic interpolant, weights W0, W1, R) the two
// exponential recurrences and the boundary terms give, for e = D v,
//     (1 + d^2) e_j - d (e_{j-1} + e_{j+1}) = q_j,
//     q_j = c1 s_j + c2 (s_{j-1} + s_{j+1}),  s_j = v_{j+1} - 2 v_j + v_{j-1},
//     c1 = -(K/2 + R),  c2 = R d / 2,  K = (1 - d^2)/nu,
// at every interior node, with e = 0 at Dirichlet end nodes (the corrected
// L^{-1} returns v there) and s_0 := s_1, s_{n-1} := s_{n-2} (the one-sided
// interpolants of the end cells); periodic lines wrap.  So e is a causal
// recurrence y_j = d y_{j-1} + q_j followed by an anti-causal one
// e_j = d e_{j+1} + y_j, plus the homogeneous terms A' d^j + B' d^{n-1-j} that
// zero the Dirichlet ends (or the sums over periodic images).  This is the
// same operator; it never cancels v - L^{-1}v, which is what lets the
// sweeps run in float32 (D v is much smaller than v for smooth fields).
//
// Each recurrence runs as a chunked scan: every lane reduces its segment,
// the lane carries combine in a 5-step shuffle scan with multipliers
// d^{m 2^k}, and every lane re-scans its segment from its carry.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace molt {

enum : int { BC_PERIODIC = 0, BC_DIRICHLET = 1 };

// Constants of one axis (host computes them in float64).
struct AxisDev {
    int n;          // points on a line
    int m;          // points per lane segment, ceil(n/32)
    int ms;         // segment stride in shared memory (odd)
    int ls;         // line stride in shared memory (elements)
    unsigned mmagic;// ceil(2^32 / m): j / m == __umulhi(j, mmagic) for j < 2^16
    double d;       // e^{-nu}, nu = alpha h
    double c1, c2;  // q_j = c1 s_j + c2 (s_{j-1} + s_{j+1})
    double mu;      // d^n (periodic) or d^{n-1} (Dirichlet)
    double inv;     // 1/(1-mu) (periodic) or 1/(1-mu^2) (Dirichlet)
    double dm[5];   // d^{m 2^k}, k = 0..4
    const double *dpow64;  // d^j, j = 0..n
    const float *dpow32;
    // float32 copies of the constants above (axis_mirror): float kernels read
    // these and so do no float64 arithmetic, which runs on a narrow pipe
    float fd, fc1, fc2, fmu, finv, fdm[5];

    template <class T> __host__ __device__ T cd() const { if constexpr (sizeof(T) == 4) return fd; else return d; }
    template <class T> __host__ __device__ T cc1() const { if constexpr (sizeof(T) == 4) return fc1; else return c1; }
    template <class T> __host__ __device__ T cc2() const { if constexpr (sizeof(T) == 4) return fc2; else return c2; }
    template <class T> __host__ __device__ T cmu() const { if constexpr (sizeof(T) == 4) return fmu; else return mu; }
    template <class T> __host__ __device__ T cinv() const { if constexpr (sizeof(T) == 4) return finv; else return inv; }
    template <class T> __host__ __device__ T cdm(int k) const
    {
        if constexpr (sizeof(T) == 4) return fdm[k];
        else return dm[k];
    }
};

// fills the float32 copies of an axis' constants (after any change to them)
inline void axis_mirror(AxisDev &A)
{
    A.fd = (float)A.d;
    A.fc1 = (float)A.c1;
    A.fc2 = (float)A.c2;
    A.fmu = (float)A.mu;
    A.finv = (float)A.inv;
    for (int k = 0; k < 5; ++k) A.fdm[k] = (float)A.dm[k];
}

// Where the lines of one pass live in global memory.
struct PassGeom {
    int64_t stride;  // element stride along the axis
    int64_t inner;   // product of the extents of the axes before this one
    int64_t nlines;  // number of lines
    int W;           // lines (warps) per CTA, a power of two <= 16
    int wshift;      // log2(W)
    int dps;         // 1: the d^j table is copied to shared memory; 0 (long lines whose
                     //    buffers leave no room): it is read from global memory
    int cta;         // 1: one line per CTA of kCtaLineThreads threads, each owning a segment
                     //    (A.m, A.ms, A.dm describe those segments): sweep_D_cta
};

constexpr int kCtaLineThreads = 512;   // threads (segments) of a line swept by a whole CTA

constexpr int MAXP = 6;     // P <= 5, Horner steps 0..P
constexpr int MAXG = 8;     // input fields of a Horner pass

struct PowersParams {
    int P;                   // powers 1..P
    const void *u_hi;        // T == float: hi plane; T == double: the field
    const void *u_lo;        // T == float: lo plane
    void *out[MAXG];         // out[p-1] receives D^p u (nullptr: not stored)
};

struct HornerParams {
    int P;                   // D applications per output
    int ng;                  // number of input fields g
    int nout;                // outputs
    const void *g[MAXG];
    void *out[MAXG];         // epi == 0: out[o] receives output o (type T)
    double coef[MAXP][MAXP][MAXG];  // [o][step][k]: weight of g_k in step
    double cu[MAXP][MAXP];          // [o][step]: weight of u in step (>= 1)
    int epi;                 // 0: store outputs; 1: level combination
    double ea, eb, ec;       // level: u_next = ea u + eb u_prev + ec F
    const void *u_hi, *u_lo;
    const void *up_hi, *up_lo;
    void *un_hi, *un_lo;
    // Time-dependent Dirichlet data (1D, Sec. 3.2; bcd = 1): the end values of
    // the D application of Horner step t (bgL[t], bgR[t]) and of the new level
    // (bnew); zero data is the homogeneous operator
    int bcd;
    double bgL[MAXP], bgR[MAXP];
    double bnew[2];
};

// Coefficients and fields of a pass program.
//   mode 0 (powers): out[p-1] = D^p u, p = 1..P
//   mode 1 (Horner): for each output o:
//       X = 0;  for t = P..1: X = D( sum_k coef[o][t][k] g_k + X + cu[o][t] u )
//       out_o = sum_k coef[o][0][k] g_k + X     (or the level combination)
struct ProgParams {
    int mode;             // 0 powers, 1 Horner, 2 powers of D^T, 3 Horner in D^T (adjoint step)
    int P, ng, nout;
    const void *g[MAXG];
    void *out[MAXG];
    const double *coef;   // device, [nout][P+1][ng]
    const double *cu;     // device, [nout][P+1]
    int epi;              // 1: out_0 combined into the next level
    double ea, eb, ec;    // u_next = ea u + eb u_prev + ec F
    const void *u_hi, *u_lo, *up_hi, *up_lo;
    void *un_hi, *un_lo;
    // float32 copies for the float kernels (no float64 arithmetic on their
    // paths): the tables in the kernel's parameter space, the level weights
    float coef32[MAXP * MAXP * MAXG];
    float cu32[MAXP * MAXP];
    float fea, feb, fec;
};

// Horner weights in the kernel's precision: float kernels read the copies in
// the parameter space, float64 kernels the device tables
template <class T> __device__ __forceinline__ T prog_coef(const ProgParams &p, size_t i)
{
    if constexpr (sizeof(T) == 4) return p.coef32[i];
    else return __ldg(p.coef + i);
}
template <class T> __device__ __forceinline__ T prog_cu(const ProgParams &p, size_t i)
{
    if constexpr (sizeof(T) == 4) return p.cu32[i];
    else return __ldg(p.cu + i);
}

// fills the float32 copies of a program's level weights and Horner weights
// (flattened as the device tables: [o][t][k] and [o][t])
inline void prog_mirror(ProgParams &p, const HornerParams &hp)
{
    int nc = 0, nu = 0;
    for (int o = 0; o < (hp.nout > 1 ? hp.nout : 1); ++o)
        for (int t = 0; t <= hp.P; ++t) {
            for (int k = 0; k < hp.ng; ++k) p.coef32[nc++] = (float)hp.coef[o][t][k];
            p.cu32[nu++] = (float)hp.cu[o][t];
        }
    p.fea = (float)p.ea;
    p.feb = (float)p.eb;
    p.fec = (float)p.ec;
}

struct LineSet {
    int64_t stride;   // element stride along the axis
    int64_t inner;    // product of the extents before the axis
    int64_t nlines;
    int S, K;         // strided: segments per CTA (warps) and CTAs per line
    int persist_sms;  // row-split x pass: > 0 runs persistent CTAs on this many SMs
    int rows_nb;      // row-split x pass: 1 = one neighbour exchange per sweep where exact to rounding
    int pdl;          // 1 = launched as a programmatic dependent of the previous kernel in the stream
};

// Programmatic dependent launch: a kernel launched with that attribute may be
// scheduled while its predecessor in the stream is still running; it waits
// here for the predecessor's completion (and its memory) before it touches
// global memory, and lets its own successor be scheduled once all of its CTAs
// have started.  Both are no-ops for a kernel launched without the attribute.
__device__ __forceinline__ void pdl_enter()
{
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// ---------------------------------------------------------------------------
// float32 pair ("hi + lo") arithmetic for the time levels.  The __f*_rn
// intrinsics keep the compiler from contracting or re-associating.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e)
{
    s = __fadd_rn(a, b);
    float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// second difference of a pair field: ((u+ - u0) - (u0 - u-)) for hi and lo
__device__ __forceinline__ float sdiff_pair(float hm, float h0, float hp, float lm, float l0, float lp)
{
    float dh = __fsub_rn(__fsub_rn(hp, h0), __fsub_rn(h0, hm));
    float dl = __fsub_rn(__fsub_rn(lp, l0), __fsub_rn(l0, lm));
    return __fadd_rn(dh, dl);
}

// --- level conversions (begin) ---
// float64 <-> float32 conversions by integer operations on the IEEE-754
// encodings (round to nearest, ties to even, as the standard defines it):
// GB300 runs float64 arithmetic and conversions on its narrow float64 pipe
// (about one lane-operation per SM and clock), so the pair conversions below
// take none on their common paths.  Infinities and NaNs take the hardware
// conversion.
__device__ __forceinline__ float d2f_rn_bits(double v)
{
    const unsigned long long b = (unsigned long long)__double_as_longlong(v);
    const unsigned s = (unsigned)(b >> 63) << 31;
    const int e = (int)((b >> 52) & 0x7ff);
    const unsigned long long m = b & 0xfffffffffffffull;
    if (e == 0x7ff) return __double2float_rn(v);
    const int fe = e - 896;                                  // float32 biased exponent of the value
    unsigned long long q, rem, half;
    if (fe >= 1) {
        if (fe >= 255) return __uint_as_float(s | 0x7f800000u);
        q = ((unsigned long long)fe << 23) | (m >> 29);      // exponent and 23 mantissa bits; a carry
        rem = m & ((1ull << 29) - 1);                        // from rounding moves into the exponent
        half = 1ull << 28;
    } else {
        if (e == 0) return __uint_as_float(s);               // float64 zero or subnormal -> +-0
        const int sh = 30 - fe;                              // subnormal result in units of 2^-149
        if (sh > 63) return __uint_as_float(s);
        const unsigned long long M = m | (1ull << 52);
        q = M >> sh;
        rem = M & ((1ull << sh) - 1);
        half = 1ull << (sh - 1);
    }
    if (rem > half || (rem == half && (q & 1ull))) ++q;
    return __uint_as_float(s | (unsigned)q);
}

// float64 encoding of a finite float32 encoding b: a normal value moves its
// exponent and mantissa over; a subnormal m 2^-149 with leading bit p becomes
// a normal float64 of exponent p - 149
__device__ __forceinline__ unsigned long long f2d_enc(unsigned b)
{
    const unsigned long long s = (unsigned long long)(b >> 31) << 63;
    const unsigned e = (b >> 23) & 0xffu, m = b & 0x7fffffu;
    if (e != 0u) return s | ((unsigned long long)(e + 896u) << 52) | ((unsigned long long)m << 29);
    if (m == 0u) return s;
    const int p = 31 - __clz((int)m);
    return s | ((unsigned long long)(p + 874) << 52) | (((unsigned long long)m << (52 - p)) & 0xfffffffffffffull);
}

__device__ __forceinline__ double f2d_bits(float f)
{
    const unsigned b = __float_as_uint(f);
    if (((b >> 23) & 0xffu) == 0xffu) return (double)f;
    return __longlong_as_double((long long)f2d_enc(b));
}

// The common case in 32-bit integer operations: a value whose float32
// rounding is a normal number or overflows to infinity (biased float64
// exponent 897 .. 1150); the rest takes d2f_rn_bits.  hw, lw: the high and
// low words of the encoding; the float32 mantissa is the top 23 of the 52
// mantissa bits, rounded by the 29 below them.
__device__ __forceinline__ float d2f_rn_fast(double v)
{
    const unsigned hw = (unsigned)__double2hiint(v), lw = (unsigned)__double2loint(v);
    const unsigned e = (hw >> 20) & 0x7ffu;
    if (e - 897u <= 1150u - 897u) {
        unsigned q = ((e - 896u) << 23) | ((hw & 0xfffffu) << 3) | (lw >> 29);
        const unsigned rem = lw & 0x1fffffffu;
        q += (rem > 0x10000000u || (rem == 0x10000000u && (q & 1u))) ? 1u : 0u;   // a carry moves into the exponent
        return __uint_as_float((hw & 0x80000000u) | q);
    }
    return d2f_rn_bits(v);
}

// RN32(R 2^k) for an integer 0 < R < 2^29, k = e - 1075 with e the biased
// float64 exponent of a value in the float32 normal range (897 <= e): a
// normal result takes the top 24 bits of R, rounded to nearest even by those
// below; a subnormal one the bits of R at or above 2^-149.
__device__ __forceinline__ unsigned rn32_scaled(unsigned R, unsigned e)
{
    const int nb = 32 - __clz((int)R);                  // bit length of R
    const int bl = (int)e + nb - 949;                    // biased float32 exponent of the result
    unsigned q, s;
    if (bl >= 1) {
        if (nb <= 24) return ((unsigned)(bl - 1) << 23) + (R << (24 - nb));
        s = (unsigned)(nb - 24);
        q = ((unsigned)(bl - 1) << 23) + (R >> s);       // a carry from rounding moves into the exponent
    } else {
        const int t = (int)e - 926;                      // R 2^k in units of 2^-149 is R 2^t
        if (t >= 0) return R << t;
        if (t <= -30) return 0u;                         // below half the smallest subnormal
        s = (unsigned)(-t);
        q = R >> s;
    }
    const unsigned rem = R & ((1u << s) - 1u), half = 1u << (s - 1u);
    return q + ((rem > half || (rem == half && (q & 1u))) ? 1u : 0u);
}

// v -> (h, l) = (RN32(v), RN32(v - h)), the float32 pair of a float64 value,
// in integer operations on the encoding for every |v| below 2^127 (biased
// float64 exponent e < 1150); v - h is exact in float64.
//  - h a normal float32 (897 <= e): h takes the top 23 mantissa bits rounded
//    by the 29 below them (rem), and v - h is +-R units of the last place of
//    v with R = rem (rounded down) or 2^29 - rem (rounded up, the sign of l
//    then opposite to that of v);
//  - below (e < 897): h is a subnormal or zero, |v - h| <= 2^-150 rounds to
//    a zero carrying the sign of v - h (+0 where v = h).
// Larger values, infinities and NaNs go through the float64 subtraction.
__device__ __forceinline__ void split_pair(double v, float &h, float &l)
{
    const unsigned hw = (unsigned)__double2hiint(v), lw = (unsigned)__double2loint(v);
    const unsigned e = (hw >> 20) & 0x7ffu;
    const unsigned sv = hw & 0x80000000u;
    if (e - 897u <= 1149u - 897u) {
        const unsigned q = ((e - 896u) << 23) | ((hw & 0xfffffu) << 3) | (lw >> 29);
        const unsigned rem = lw & 0x1fffffffu;
        const bool up = rem > 0x10000000u || (rem == 0x10000000u && (q & 1u));
        h = __uint_as_float(sv | (q + (up ? 1u : 0u)));
        const unsigned R = up ? 0x20000000u - rem : rem;
        l = R == 0u ? 0.0f : __uint_as_float((up ? sv ^ 0x80000000u : sv) | rn32_scaled(R, e));
        return;
    }
    if (e < 897u) {
        const unsigned long long m = ((unsigned long long)(hw & 0xfffffu) << 32) | lw;
        if (e == 0u) {                                   // float64 zero or subnormal: h = +-0
            h = __uint_as_float(sv);
            l = __uint_as_float(m == 0ull ? 0u : sv);
            return;
        }
        const unsigned sh = 926u - e;                    // >= 30: the value in units of 2^-149 is M 2^-sh
        const unsigned long long M = m | (1ull << 52);
        unsigned q = 0u;
        bool up = false, exact = false;
        if (sh <= 63u) {
            q = (unsigned)(M >> sh);
            const unsigned long long rem = M & ((1ull << sh) - 1ull), half = 1ull << (sh - 1u);
            up = rem > half || (rem == half && (q & 1u));
            exact = rem == 0ull;
        }
        h = __uint_as_float(sv | (q + (up ? 1u : 0u)));  // a carry gives the smallest normal
        l = __uint_as_float(exact ? 0u : (up ? sv ^ 0x80000000u : sv));
        return;
    }
    h = d2f_rn_fast(v);
    l = d2f_rn_fast(v - f2d_bits(h));
}

// RN64(h + l) for a float32 pair, in integer operations where
//  - l is a zero and h finite: the sum is h (a zero of sign sign(h) & sign(l)
//    where h is a zero too);
//  - h and l are normal, l no larger than h and every bit of l at or above
//    2^-32 ulp(h) (always so for a pair from split_pair of a value in the
//    float32 normal range): the sum is formed in a 64-bit integer in units of
//    2^-32 ulp(h), below 2^57, and rounded to 53 bits to nearest even.
// Other pairs go through the float64 addition.
__device__ __forceinline__ double join_pair(float h, float l)
{
    const unsigned hb = __float_as_uint(h), lb = __float_as_uint(l);
    const unsigned eh = (hb >> 23) & 0xffu, el = (lb >> 23) & 0xffu, la = lb & 0x7fffffffu;
    if (la == 0u && eh != 0xffu) {
        if ((hb & 0x7fffffffu) == 0u) return __longlong_as_double((long long)((unsigned long long)(hb & lb) << 32));
        return __longlong_as_double((long long)f2d_enc(hb));
    }
    const unsigned d = eh - el;                          // exponent gap (wraps when l is larger)
    const unsigned ml = (lb & 0x7fffffu) | 0x800000u;
    const bool fast = eh - 1u <= 253u && el - 1u <= 253u &&
                      (d <= 32u || (d < 56u && (ml & ((1u << (d - 32u)) - 1u)) == 0u));
    if (!fast) return f2d_bits(h) + f2d_bits(l);
    const unsigned long long H = (unsigned long long)((hb & 0x7fffffu) | 0x800000u) << 32;
    const unsigned long long L = d <= 32u ? (unsigned long long)ml << (32u - d) : (unsigned long long)(ml >> (d - 32u));
    unsigned long long sg = (unsigned long long)(hb >> 31) << 63, S;
    if (((hb ^ lb) >> 31) == 0u) {
        S = H + L;
    } else if (H >= L) {
        S = H - L;
    } else {
        S = L - H;
        sg ^= 1ull << 63;
    }
    if (S == 0ull) return 0.0;                           // h + (-h) = +0
    const int nb = 64 - __clzll((long long)S);           // <= 57
    const unsigned long long top = (unsigned long long)(eh + (unsigned)nb + 839u) << 52;   // biased exponent - 1
    if (nb <= 53) return __longlong_as_double((long long)(sg | (top + (S << (53 - nb)))));
    const int s = nb - 53;
    unsigned long long q = S >> s;
    const unsigned long long rem = S & ((1ull << s) - 1ull), half = 1ull << (s - 1);
    q += (rem > half || (rem == half && (q & 1ull))) ? 1ull : 0ull;
    return __longlong_as_double((long long)(sg | (top + q)));  // a carry moves into the exponent
}

// --- level conversions (end) ---

// u_next = a u + b up + c F with a, b, c in {0, +-1, 2, 0.5} (exact scalings)
__device__ __forceinline__ void level_pair(float uh, float ul, float ph, float pl, float F,
                                           float a, float b, float c, float &nh, float &nl)
{
    float s1, e1, s2, e2;
    two_sum(__fmul_rn(a, uh), __fmul_rn(b, ph), s1, e1);
    two_sum(s1, __fmul_rn(c, F), s2, e2);
    float lo = __fadd_rn(__fadd_rn(e1, e2), __fadd_rn(__fmul_rn(a, ul), __fmul_rn(b, pl)));
    two_sum(s2, lo, nh, nl);
}

template <class T> __device__ __forceinline__ const T *dpow_of(const AxisDev &A);
template <> __device__ __forceinline__ const float *dpow_of<float>(const AxisDev &A) { return A.dpow32; }
template <> __device__ __forceinline__ const double *dpow_of<double>(const AxisDev &A) { return A.dpow64; }

// point j (0 <= j < n) of a line -> shared-memory position
__device__ __forceinline__ int spos_raw(int j, int m, int ms, unsigned mmagic)
{
    int s = (int)__umulhi((unsigned)j, mmagic);
    return s * ms + (j - s * m);
}

// any j -> position, wrapping (periodic) or clamping (Dirichlet) into the line
template <int BC>
__device__ __forceinline__ int spos(int j, const AxisDev &A)
{
    const int n = A.n;
    if (BC == BC_PERIODIC) { j %= n; if (j < 0) j += n; }
    else { j = j < 0 ? 0 : (j > n - 1 ? n - 1 : j); }
    return spos_raw(j, A.m, A.ms, A.mmagic);
}

// ---------------------------------------------------------------------------
// The line sweep: buf <- D z (in place), one warp.
//   MODE 0: buf holds s already (first power of u; ends pre-duplicated).
//   MODE 1: s = second difference of buf.
//   MODE 2: s = second difference of buf + cu * r, r from rbuf.
// dp points to the d^j table (shared memory, or global memory for long lines).
// ---------------------------------------------------------------------------
// gL, gR (Dirichlet): the values D must take at the end nodes (zero for
// homogeneous data)
template <class T, int MODE, int BC>
__device__ void sweep_D(T *buf, const T *rbuf, T cu, const AxisDev &A,
                        const T *__restrict__ dp, int lane, T gL = 0, T gR = 0)
{
    const int n = A.n, m = A.m, ms = A.ms;
    const T d = A.cd<T>(), c1 = A.cc1<T>(), c2 = A.cc2<T>();
    const int a = lane * m;
    const int b = min(a + m, n);
    const int cnt = b > a ? b - a : 0;
    T *seg = buf + lane * ms;
    const T *rseg = rbuf + lane * ms;

    // ---- halo values from neighbouring segments, read before any write ----
    T h_l2 = 0, h_l1 = 0, h_r0 = 0, h_r1 = 0;
    if (cnt > 0) {
        h_l1 = buf[spos<BC>(a - 1, A)];
        h_r0 = buf[spos<BC>(b, A)];
        if (MODE != 0) {
            h_l2 = buf[spos<BC>(a - 2, A)];
            h_r1 = buf[spos<BC>(b + 1, A)];
        }
    }
    __syncwarp();

    // ---- q_j and the causal reduction of this segment ----
    T E = 0;
    if (cnt > 0) {
        // raw s at a-1 and a, and the z window (MODE 1/2)
        T sm1, s0, z0 = 0, zp1 = 0;
        if (MODE == 0) {
            sm1 = h_l1;
            s0 = seg[0];
        } else {
            T zm1 = h_l1;
            z0 = seg[0];
            zp1 = cnt > 1 ? seg[1] : h_r0;
            sm1 = (z0 - zm1) - (zm1 - h_l2);
            s0 = (zp1 - z0) - (z0 - zm1);
            if (MODE == 2) {
                sm1 += cu * rbuf[spos<BC>(a - 1, A)];
                s0 += cu * rseg[0];
            }
        }
        for (int k = 0; k < cnt; ++k) {
            const int j = a + k;
            T sp1;
            if (MODE == 0) {
                sp1 = (k + 1 < cnt) ? seg[k + 1] : h_r0;
            } else {
                T zp2 = (k + 2 < cnt) ? seg[k + 2] : (k + 2 == cnt ? h_r0 : h_r1);
                sp1 = (zp2 - zp1) - (zp1 - z0);
                if (MODE == 2) sp1 += cu * ((k + 1 < cnt) ? rseg[k + 1] : rbuf[spos<BC>(b, A)]);
                z0 = zp1;
                zp1 = zp2;
            }
            T q;
            if (BC == BC_DIRICHLET) {
                T sl = (j - 1 < 1) ? s0 : sm1;
                T sr = (j + 1 > n - 2) ? s0 : sp1;
                q = (j == 0 || j == n - 1) ? (T)0 : c1 * s0 + c2 * (sl + sr);
            } else {
                q = c1 * s0 + c2 * (sm1 + sp1);
            }
            seg[k] = q;
            E = d * E + q;
            sm1 = s0;
            s0 = sp1;
        }
    }

    // ---- causal carries: y at a-1 ----
    // reconverge the warp before the shuffles (lanes ran loops of different
    // lengths; __shfl_sync pairs lanes by mask, not by call site)
    __syncwarp();
    T x = E;
#pragma unroll
    for (int k = 0; k < 5; ++k) {
        T y = __shfl_up_sync(0xffffffffu, x, 1 << k);
        if (lane >= (1 << k)) x += A.cdm<T>(k) * y;
    }
    T excl = __shfl_up_sync(0xffffffffu, x, 1);
    if (lane == 0) excl = 0;
    const int Ld = (n - 1) / m;        // last lane holding data
    T y = excl;
    if (BC == BC_PERIODIC) {
        // zero-inflow y_{n-1}: the last lane may hold fewer than m points
        T tot = __shfl_sync(0xffffffffu, cnt > 0 ? dp[cnt] * excl + E : (T)0, Ld);
        T y_m1 = tot * A.cinv<T>();                        // y_{-1} over all images
        if (cnt > 0) y += dp[a] * y_m1;
    }

    // ---- causal scan of the segment; anti-causal reduction ----
    T ER = 0, pw = 1;
    for (int k = 0; k < cnt; ++k) {
        y = d * y + seg[k];
        seg[k] = y;
        ER += pw * y;
        pw *= d;
    }

    // ---- anti-causal carries ----
    __syncwarp();
    T xb = ER;
#pragma unroll
    for (int k = 0; k < 5; ++k) {
        T t = __shfl_down_sync(0xffffffffu, xb, 1 << k);
        if (lane + (1 << k) < 32) xb += A.cdm<T>(k) * t;
    }
    T exclb = __shfl_down_sync(0xffffffffu, xb, 1);
    if (lane == 31) exclb = 0;
    const T e00 = __shfl_sync(0xffffffffu, xb, 0);     // zero-inflow e_0
    T Z, Acoef = 0;
    if (BC == BC_DIRICHLET) {
        const T ylast = __shfl_sync(0xffffffffu, y, Ld);  // y_{n-1} = zero-inflow e_{n-1}
        const T mu = A.cmu<T>(), inv = A.cinv<T>();
        Acoef = (mu * ylast - e00) * inv + (gL - mu * gR) * inv;   // A': e_0 = gL
        Z = (mu * e00 - ylast) * inv + (gR - mu * gL) * inv;       // B': e_{n-1} = gR
    } else {
        Z = d * e00 * A.cinv<T>();                         // d * e_n, e_n = e_0 over all images
    }
    // c = d * e_b including the inflow from the right end
    T acc = d * exclb + (cnt > 0 ? dp[n - b] * Z : (T)0);
    for (int k = cnt - 1; k >= 0; --k) {
        T e = acc + seg[k];
        acc = d * e;
        if (BC == BC_DIRICHLET) e += Acoef * dp[a + k];
        seg[k] = e;
    }
    __syncwarp();
}

// The same sweep with the line split over the kCtaLineThreads threads of the
// CTA (thread t owns points t m .. t m + m - 1): the chunk carries combine
// over the lanes of a warp by shuffles, as in sweep_D, then over the warps
// through their totals in shared memory (the warps before the last one
// holding data are full, so a warp spans d^(32 m)).  Every thread of the CTA
// calls it; the line's n >= 32 m.
// scratch: 2 kCtaLineThreads / 32 + 3 elements of shared memory.
template <class T, int MODE, int BC>
__device__ void sweep_D_cta(T *buf, const T *rbuf, T cu, const AxisDev &A, const T *__restrict__ dp, T *scratch,
                            T gL = 0, T gR = 0)
{
    constexpr int NWC = kCtaLineThreads / 32;
    T *s_tc = scratch, *s_ta = scratch + NWC, *s_bc = scratch + 2 * NWC;
    const int tt = threadIdx.x, lane = tt & 31, warp = tt >> 5;
    const int n = A.n, m = A.m, ms = A.ms;
    const T d = A.cd<T>(), c1 = A.cc1<T>(), c2 = A.cc2<T>();
    const int a = tt * m;
    const int b = min(a + m, n);
    const int cnt = b > a ? b - a : 0;
    T *seg = buf + tt * ms;
    const T *rseg = rbuf + tt * ms;
    const T D32 = A.cdm<T>(4) * A.cdm<T>(4);          // d^(32 m): across one full warp

    // ---- halo values from neighbouring segments (other warps' too), read
    // before any write ----
    T h_l2 = 0, h_l1 = 0, h_r0 = 0, h_r1 = 0;
    if (cnt > 0) {
        h_l1 = buf[spos<BC>(a - 1, A)];
        h_r0 = buf[spos<BC>(b, A)];
        if (MODE != 0) {
            h_l2 = buf[spos<BC>(a - 2, A)];
            h_r1 = buf[spos<BC>(b + 1, A)];
        }
    }
    __syncthreads();

    // ---- q_j and the causal reduction of this segment (as sweep_D) ----
    T E = 0;
    if (cnt > 0) {
        T sm1, s0, z0 = 0, zp1 = 0;
        if (MODE == 0) {
            sm1 = h_l1;
            s0 = seg[0];
        } else {
            T zm1 = h_l1;
            z0 = seg[0];
            zp1 = cnt > 1 ? seg[1] : h_r0;
            sm1 = (z0 - zm1) - (zm1 - h_l2);
            s0 = (zp1 - z0) - (z0 - zm1);
            if (MODE == 2) {
                sm1 += cu * rbuf[spos<BC>(a - 1, A)];
                s0 += cu * rseg[0];
            }
        }
        for (int k = 0; k < cnt; ++k) {
            const int j = a + k;
            T sp1;
            if (MODE == 0) {
                sp1 = (k + 1 < cnt) ? seg[k + 1] : h_r0;
            } else {
                T zp2 = (k + 2 < cnt) ? seg[k + 2] : (k + 2 == cnt ? h_r0 : h_r1);
                sp1 = (zp2 - zp1) - (zp1 - z0);
                if (MODE == 2) sp1 += cu * ((k + 1 < cnt) ? rseg[k + 1] : rbuf[spos<BC>(b, A)]);
                z0 = zp1;
                zp1 = zp2;
            }
            T q;
            if (BC == BC_DIRICHLET) {
                T sl = (j - 1 < 1) ? s0 : sm1;
                T sr = (j + 1 > n - 2) ? s0 : sp1;
                q = (j == 0 || j == n - 1) ? (T)0 : c1 * s0 + c2 * (sl + sr);
            } else {
                q = c1 * s0 + c2 * (sm1 + sp1);
            }
            seg[k] = q;
            E = d * E + q;
            sm1 = s0;
            s0 = sp1;
        }
    }

    // ---- causal carries: y at a-1, over the lanes, then over the warps ----
    __syncwarp();
    T x = E;
#pragma unroll
    for (int k = 0; k < 5; ++k) {
        T y = __shfl_up_sync(0xffffffffu, x, 1 << k);
        if (lane >= (1 << k)) x += A.cdm<T>(k) * y;
    }
    T excl = __shfl_up_sync(0xffffffffu, x, 1);
    if (lane == 0) excl = 0;
    if (lane == 31) s_tc[warp] = x;
    __syncthreads();
    {
        T win = 0;                                          // y just before this warp
        for (int w = 0; w < warp; ++w) win = D32 * win + s_tc[w];
        excl += dp[lane * m] * win;
    }
    const int Ld = (n - 1) / m;        // last thread holding data
    T y = excl;
    if (BC == BC_PERIODIC) {
        if (tt == Ld) s_bc[0] = dp[cnt] * excl + E;        // zero-inflow y_{n-1}
        __syncthreads();
        const T y_m1 = s_bc[0] * A.cinv<T>();              // y_{-1} over all images
        if (cnt > 0) y += dp[a] * y_m1;
    }

    // ---- causal scan of the segment; anti-causal reduction ----
    T ER = 0, pw = 1;
    for (int k = 0; k < cnt; ++k) {
        y = d * y + seg[k];
        seg[k] = y;
        ER += pw * y;
        pw *= d;
    }

    // ---- anti-causal carries: e at b, over the lanes, then over the warps ----
    __syncwarp();
    T xb = ER;
#pragma unroll
    for (int k = 0; k < 5; ++k) {
        T t2 = __shfl_down_sync(0xffffffffu, xb, 1 << k);
        if (lane + (1 << k) < 32) xb += A.cdm<T>(k) * t2;
    }
    T exclb = __shfl_down_sync(0xffffffffu, xb, 1);
    if (lane == 31) exclb = 0;
    if (lane == 0) s_ta[warp] = xb;
    if (BC == BC_DIRICHLET && tt == Ld) s_bc[1] = y;       // y_{n-1} = zero-inflow e_{n-1}
    __syncthreads();
    T wout = 0;                                             // e at the first point after this warp
    for (int w = NWC - 1; w > warp; --w) wout = D32 * wout + s_ta[w];
    exclb += dp[(31 - lane) * m] * wout;
    if (tt == 0) s_bc[2] = xb + D32 * wout;                // zero-inflow e_0
    __syncthreads();
    const T e00 = s_bc[2];
    T Z, Acoef = 0;
    if (BC == BC_DIRICHLET) {
        const T ylast = s_bc[1];
        const T mu = A.cmu<T>(), inv = A.cinv<T>();
        Acoef = (mu * ylast - e00) * inv + (gL - mu * gR) * inv;   // A': e_0 = gL
        Z = (mu * e00 - ylast) * inv + (gR - mu * gL) * inv;       // B': e_{n-1} = gR
    } else {
        Z = d * e00 * A.cinv<T>();                         // d * e_n, e_n = e_0 over all images
    }
    T acc = d * exclb + (cnt > 0 ? dp[n - b] * Z : (T)0);
    for (int k = cnt - 1; k >= 0; --k) {
        T e = acc + seg[k];
        acc = d * e;
        if (BC == BC_DIRICHLET) e += Acoef * dp[a + k];
        seg[k] = e;
    }
    __syncthreads();
}

// ---------------------------------------------------------------------------
// CTA helpers
// ---------------------------------------------------------------------------
// Shared-memory carve-out of a pass CTA: `arrays` line buffers of W lines,
// the d^j table (n+1 values; none when dps == 0), the W line base offsets and
// the carry scratch of sweep_D_cta.
struct SmemLayout {
    size_t lines, dpow, lbase, scratch, total;
};
__host__ __device__ inline size_t round16(size_t x) { return (x + 15) & ~(size_t)15; }
__host__ __device__ inline SmemLayout smem_layout(int arrays, int W, int ls, int n, size_t tsize, int dps = 1)
{
    SmemLayout L;
    L.lines = 0;
    L.dpow = round16((size_t)arrays * W * ls * tsize);
    L.lbase = L.dpow + (dps ? round16((size_t)(n + 1) * tsize) : 0);
    L.scratch = L.lbase + round16((size_t)W * sizeof(int64_t));
    L.total = L.scratch + round16((size_t)(2 * kCtaLineThreads / 32 + 3) * tsize);
    return L;
}
__device__ __forceinline__ int64_t line_base(const PassGeom &G, int64_t L, int n)
{
    return (L % G.inner) + (L / G.inner) * G.inner * (int64_t)n;
}

// centre of the second difference used at point j (Dirichlet clamps into [1, n-2])
template <int BC>
__device__ __forceinline__ int sd_centre(int j, int n)
{
    if (BC == BC_DIRICHLET) return j < 1 ? 1 : (j > n - 2 ? n - 2 : j);
    return j;
}

template <int BC>
__device__ __forceinline__ int wrap(int j, int n)
{
    if (BC == BC_PERIODIC) { if (j < 0) j += n; else if (j >= n) j -= n; }
    return j;
}

// second difference of u along the axis at point j (accurate: from the pair
// levels for T = float, float64 for T = double)
template <class T, int BC>
__device__ __forceinline__ T u_sdiff(const void *uh, const void *ul, int64_t base, int64_t stride, int j, int n);

template <>
__device__ __forceinline__ float u_sdiff<float, BC_PERIODIC>(const void *uh, const void *ul, int64_t base, int64_t stride, int j, int n)
{
    const float *H = (const float *)uh, *Lo = (const float *)ul;
    int jm = wrap<BC_PERIODIC>(j - 1, n), jp = wrap<BC_PERIODIC>(j + 1, n);
    return sdiff_pair(H[base + jm * stride], H[base + j * stride], H[base + jp * stride],
                      Lo[base + jm * stride], Lo[base + j * stride], Lo[base + jp * stride]);
}
template <>
__device__ __forceinline__ float u_sdiff<float, BC_DIRICHLET>(const void *uh, const void *ul, int64_t base, int64_t stride, int j, int n)
{
    const float *H = (const float *)uh, *Lo = (const float *)ul;
    int c = sd_centre<BC_DIRICHLET>(j, n);
    return sdiff_pair(H[base + (c - 1) * stride], H[base + c * stride], H[base + (c + 1) * stride],
                      Lo[base + (c - 1) * stride], Lo[base + c * stride], Lo[base + (c + 1) * stride]);
}
template <>
__device__ __forceinline__ double u_sdiff<double, BC_PERIODIC>(const void *uh, const void *, int64_t base, int64_t stride, int j, int n)
{
    const double *U = (const double *)uh;
    int jm = wrap<BC_PERIODIC>(j - 1, n), jp = wrap<BC_PERIODIC>(j + 1, n);
    double u0 = U[base + j * stride];
    return (U[base + jp * stride] - u0) - (u0 - U[base + jm * stride]);
}
template <>
__device__ __forceinline__ double u_sdiff<double, BC_DIRICHLET>(const void *uh, const void *, int64_t base, int64_t stride, int j, int n)
{
    const double *U = (const double *)uh;
    int c = sd_centre<BC_DIRICHLET>(j, n);
    double u0 = U[base + c * stride];
    return (U[base + (c + 1) * stride] - u0) - (u0 - U[base + (c - 1) * stride]);
}

// Iterate over the (line, point) pairs of the CTA's block in a coalesced order:
// contiguous axis: a warp walks consecutive points of one line;
// strided axis: a warp walks W neighbouring lines of consecutive rows.
template <bool CONTIG, class F>
__device__ __forceinline__ void for_block(const PassGeom &G, int n, int nl, F &&f)
{
    const int tid = threadIdx.x, nth = blockDim.x;
    if (CONTIG) {
        for (int l = 0; l < nl; ++l)
            for (int j = tid; j < n; j += nth) f(l, j);
    } else {
        const int W = G.W;
        const int l = tid & (W - 1);
        const int rstep = nth >> G.wshift;
        if (l < nl)
            for (int j = tid >> G.wshift; j < n; j += rstep) f(l, j);
    }
}

// ---------------------------------------------------------------------------
// Powers pass: out[p-1] = D^p u along the axis, p = 1..P.
// ---------------------------------------------------------------------------
template <class T, int BC, bool CONTIG>
__global__ void __launch_bounds__(512) k_powers(AxisDev A, PassGeom G, PowersParams prm)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int n = A.n, W = G.W;
    const SmemLayout SL = smem_layout(1, W, A.ls, n, sizeof(T), G.dps);
    T *lines = reinterpret_cast<T *>(smem_raw + SL.lines);
    T *dps = reinterpret_cast<T *>(smem_raw + SL.dpow);
    int64_t *lbase = reinterpret_cast<int64_t *>(smem_raw + SL.lbase);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t L0 = (int64_t)blockIdx.x * W;
    const int64_t rem = G.nlines - L0;
    const int nl = rem < W ? (int)rem : W;

    const T *dpg = dpow_of<T>(A);
    if (G.dps)
        for (int j = threadIdx.x; j <= n; j += blockDim.x) dps[j] = dpg[j];
    const T *dp = G.dps ? dps : dpg;
    if (threadIdx.x < W) lbase[threadIdx.x] = line_base(G, L0 + ((int)threadIdx.x < nl ? (int)threadIdx.x : nl - 1), n);
    __syncthreads();

    // s = second difference of u (Dirichlet ends duplicated)
    for_block<CONTIG>(G, n, nl, [&](int l, int j) {
        lines[(size_t)l * A.ls + spos_raw(j, A.m, A.ms, A.mmagic)] =
            u_sdiff<T, BC>(prm.u_hi, prm.u_lo, lbase[l], G.stride, j, n);
    });
    __syncthreads();

    T *mine = lines + (size_t)warp * A.ls;
    for (int p = 1; p <= prm.P; ++p) {
        if (G.cta) {
            T *scr = reinterpret_cast<T *>(smem_raw + SL.scratch);
            if (p == 1) sweep_D_cta<T, 0, BC>(lines, lines, (T)0, A, dp, scr);
            else sweep_D_cta<T, 1, BC>(lines, lines, (T)0, A, dp, scr);
        } else if (warp < nl) {
            if (p == 1) sweep_D<T, 0, BC>(mine, mine, (T)0, A, dp, lane);
            else sweep_D<T, 1, BC>(mine, mine, (T)0, A, dp, lane);
        }
        if (prm.out[p - 1] != nullptr) {
            __syncthreads();
            T *o = reinterpret_cast<T *>(prm.out[p - 1]);
            for_block<CONTIG>(G, n, nl, [&](int l, int j) {
                o[lbase[l] + (int64_t)j * G.stride] = lines[(size_t)l * A.ls + spos_raw(j, A.m, A.ms, A.mmagic)];
            });
            __syncthreads();
        }
    }
}

// ---------------------------------------------------------------------------
// Horner pass: for each output o,
//   X = 0;  for t = P..1:  X = D( sum_k coef[o][t][k] g_k + cu[o][t] u + X )
//   out_o = sum_k coef[o][0][k] g_k + X
// The u term enters through its accurate second difference r (kept on chip).
// epi == 1: the single output F is combined into the next time level.
// ---------------------------------------------------------------------------
template <class T> struct LevelIO;
template <> struct LevelIO<float> {
    __device__ static void combine(const HornerParams &p, int64_t i, float F)
    {
        const float *uh = (const float *)p.u_hi, *ul = (const float *)p.u_lo;
        float ph = 0.f, pl = 0.f;
        if (p.eb != 0.0) { ph = ((const float *)p.up_hi)[i]; pl = ((const float *)p.up_lo)[i]; }
        float nh, nl;
        level_pair(uh[i], ul[i], ph, pl, F, (float)p.ea, (float)p.eb, (float)p.ec, nh, nl);
        ((float *)p.un_hi)[i] = nh;
        ((float *)p.un_lo)[i] = nl;
    }
    __device__ static void set(const HornerParams &p, int64_t i, double v)
    {
        const float h = __double2float_rn(v);
        ((float *)p.un_hi)[i] = h;
        ((float *)p.un_lo)[i] = __double2float_rn(v - (double)h);
    }
};
template <> struct LevelIO<double> {
    __device__ static void combine(const HornerParams &p, int64_t i, double F)
    {
        double v = p.ea * ((const double *)p.u_hi)[i] + p.ec * F;
        if (p.eb != 0.0) v += p.eb * ((const double *)p.up_hi)[i];
        ((double *)p.un_hi)[i] = v;
    }
    __device__ static void set(const HornerParams &p, int64_t i, double v) { ((double *)p.un_hi)[i] = v; }
};

template <class T, int BC, bool CONTIG>
__global__ void __launch_bounds__(512) k_horner(AxisDev A, PassGeom G, HornerParams prm)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int n = A.n, W = G.W;
    const SmemLayout SL = smem_layout(2, W, A.ls, n, sizeof(T), G.dps);
    T *lines = reinterpret_cast<T *>(smem_raw + SL.lines);
    T *rlines = lines + (size_t)W * A.ls;
    T *dps = reinterpret_cast<T *>(smem_raw + SL.dpow);
    int64_t *lbase = reinterpret_cast<int64_t *>(smem_raw + SL.lbase);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t L0 = (int64_t)blockIdx.x * W;
    const int64_t rem = G.nlines - L0;
    const int nl = rem < W ? (int)rem : W;

    const T *dpg = dpow_of<T>(A);
    if (G.dps)
        for (int j = threadIdx.x; j <= n; j += blockDim.x) dps[j] = dpg[j];
    const T *dp = G.dps ? dps : dpg;
    if (threadIdx.x < W) lbase[threadIdx.x] = line_base(G, L0 + ((int)threadIdx.x < nl ? (int)threadIdx.x : nl - 1), n);
    __syncthreads();

    // r = accurate second difference of u along this axis
    for_block<CONTIG>(G, n, nl, [&](int l, int j) {
        rlines[(size_t)l * A.ls + spos_raw(j, A.m, A.ms, A.mmagic)] =
            u_sdiff<T, BC>(prm.u_hi, prm.u_lo, lbase[l], G.stride, j, n);
    });

    T *mine = lines + (size_t)warp * A.ls;
    const T *rmine = rlines + (size_t)warp * A.ls;
    for (int o = 0; o < prm.nout; ++o) {
        for (int t = prm.P; t >= 0; --t) {
            // buf = (t == P ? 0 : buf) + sum_k coef g_k
            const bool first = (t == prm.P);
            for_block<CONTIG>(G, n, nl, [&](int l, int j) {
                const int64_t gi = lbase[l] + (int64_t)j * G.stride;
                const size_t si = (size_t)l * A.ls + spos_raw(j, A.m, A.ms, A.mmagic);
                T acc = first ? (T)0 : lines[si];
                for (int k = 0; k < prm.ng; ++k) {
                    const double w = prm.coef[o][t][k];
                    if (w != 0.0) acc += (T)w * reinterpret_cast<const T *>(prm.g[k])[gi];
                }
                if (t > 0) {
                    lines[si] = acc;
                } else if (prm.epi == 0) {
                    reinterpret_cast<T *>(prm.out[o])[gi] = acc;
                } else if (BC == BC_DIRICHLET && prm.bcd && (j == 0 || j == n - 1)) {
                    LevelIO<T>::set(prm, gi, prm.bnew[j == 0 ? 0 : 1]);    // the data at the end nodes
                } else {
                    LevelIO<T>::combine(prm, gi, acc);
                }
            });
            __syncthreads();
            if (t > 0 && G.cta)
                sweep_D_cta<T, 2, BC>(lines, rlines, (T)prm.cu[o][t], A, dp,
                                      reinterpret_cast<T *>(smem_raw + SL.scratch), prm.bcd ? (T)prm.bgL[t] : (T)0,
                                      prm.bcd ? (T)prm.bgR[t] : (T)0);
            else if (t > 0 && warp < nl)
                sweep_D<T, 2, BC>(mine, rmine, (T)prm.cu[o][t], A, dp, lane, prm.bcd ? (T)prm.bgL[t] : (T)0,
                                  prm.bcd ? (T)prm.bgR[t] : (T)0);
            __syncthreads();
        }
    }
}

// ---------------------------------------------------------------------------
// Level conversions (float64 <-> pair) and plain copies
// ---------------------------------------------------------------------------
__global__ void k_to_pair(const double *__restrict__ x, float *__restrict__ hi, float *__restrict__ lo, int64_t N);
__global__ void k_from_pair(const float *__restrict__ hi, const float *__restrict__ lo, double *__restrict__ x, int64_t N);
__global__ void k_from_f32(const float *__restrict__ f, double *__restrict__ x, int64_t N);

}  // namespace molt
