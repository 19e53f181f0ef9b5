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
    int64_t launches = 0;
    std::string err;
    bool timing = false;                // per-kind CUDA events (0 x sweeps, 1 y sweeps, 2 combinations)
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
        CombTerms t{};
        const bool last = p == P;
        if (p > 1) { t.c[t.n] = last ? ec : 1.0; t.x[t.n++] = e->Fb; }
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

mol_status mol_embed_create(const mol_embed_geom *g, double c, double dt, double beta, int P, mol_embed *out)
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
    }
    const size_t plane = sizeof(double) * (size_t)e->N;
    double **bufs[] = {&e->tmp, &e->t1, &e->lev, &e->Fb};
    for (double **b : bufs)
        if (st == MOL_OK) st = ealloc(e, (void **)b, plane);
    for (int k = 1; k <= P && st == MOL_OK; ++k) st = ealloc(e, (void **)&e->V[k], plane);
    if (st == MOL_OK) {
        // every sweep writes only interior nodes: the work fields start at zero
        for (void *p : e->allocs)
            if (p != e->dpow[0] && p != e->dpow[1] && p != e->lines[0] && p != e->lines[1] &&
                (ce = cudaMemset(p, 0, plane)) != cudaSuccess) {
                st = efail(e, MOL_ECUDA, "memset");
                break;
            }
    }
    if (st == MOL_OK) {
        // line arrays sized for the longest line (even, for 16-byte alignment)
        e->slot = (int)((maxm + 2 + 1) & ~(int64_t)1);
        e->smem = (int)(sizeof(double) * 2 * (size_t)e->slot * kObjWarps);
        if ((ce = cudaFuncSetAttribute(k_obj_sweep, cudaFuncAttributeMaxDynamicSharedMemorySize, e->smem)) !=
            cudaSuccess)
            st = efail(e, MOL_ECUDA, std::string("kernel attributes: ") + cudaGetErrorString(ce));
        int dev = 0, sms = 152, per_sm = 1;
        if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (st == MOL_OK &&
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_obj_sweep, 32 * kObjWarps, e->smem) != cudaSuccess) {
            cudaGetLastError();
            per_sm = 1;
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
    ECK(cudaMemsetAsync(w, 0, sizeof(double) * (size_t)e->N, s), "memset");
    return sweep(e, axis, v, w, OBJ_LINV, 0, nullptr, s);
}

mol_status mol_embed_apply_F(mol_embed e, const double *u, double *F, void *stream)
{
    if (!e) return efail(nullptr, MOL_EINVAL, "handle is NULL");
    EST(check_dev(e, u, "u"));
    EST(check_dev(e, F, "F"));
    if (u == F) return efail(e, MOL_EINVAL, "u and F must not overlap");
    return run_update(e, u, nullptr, F, 0.0, 0.0, 1.0, (cudaStream_t)stream);
}

mol_status mol_embed_start(mol_embed e, const double *u0, double *u1, void *stream)
{
    if (!e) return efail(nullptr, MOL_EINVAL, "handle is NULL");
    EST(check_dev(e, u0, "u0"));
    EST(check_dev(e, u1, "u1"));
    if (u0 == u1) return efail(e, MOL_EINVAL, "u0 and u1 must not overlap");
    return run_update(e, u0, nullptr, u1, 1.0, 0.0, 0.5, (cudaStream_t)stream);
}

mol_status mol_embed_step(mol_embed e, double *u_prev, double *u_cur, int64_t nsteps, void *stream)
{
    if (!e) return efail(nullptr, MOL_EINVAL, "handle is NULL");
    EST(check_dev(e, u_prev, "u_prev"));
    EST(check_dev(e, u_cur, "u_cur"));
    if (u_prev == u_cur) return efail(e, MOL_EINVAL, "u_prev and u_cur must not overlap");
    if (nsteps < 0) return efail(e, MOL_EINVAL, "nsteps must be >= 0");
    cudaStream_t s = (cudaStream_t)stream;
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
        EST(run_update(e, e->io[0], nullptr, e->io[1], 1.0, 0.0, 0.5, s));
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
