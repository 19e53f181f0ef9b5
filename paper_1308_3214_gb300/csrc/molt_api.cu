// molt_api.cu -- the C ABI of libmolt: constants, workspace, pass plans,
// CUDA-graph time loop.  See include/molt.h for the contract.
#include <algorithm>
#include <atomic>
#include <mutex>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "molt.h"
#include "molt_internal.h"
#include "molt_recv.cuh"

using namespace molt;

namespace {

constexpr size_t kNoallocScratchBytes = size_t(32) << 20;   // static scratch of mol_apply_F_noalloc

struct Level {
    void *hi = nullptr;   // float32 hi plane (mixed) or the float64 field
    void *lo = nullptr;   // float32 lo plane (mixed)
};

}  // namespace

struct mol_ctx {
    int ndim = 0;
    int64_t n[3] = {1, 1, 1};
    double lo[3] = {0, 0, 0}, hi[3] = {1, 1, 1};
    double c = 1, dt = 1, beta = 0, alpha = 0;
    int P = 1, bc = 0, prec = 0;
    mol_options opt{};
    int tbytes = 8;
    int64_t N = 0;
    double h[3] = {0, 0, 0}, nu[3] = {0, 0, 0};
    AxisDev ax[3]{};
    double *dpow64[3] = {nullptr, nullptr, nullptr};
    float *dpow32[3] = {nullptr, nullptr, nullptr};
    std::vector<double> f;       // expanded coefficients, (P+1)^ndim, x degree fastest
    HornerParams xtpl{}, ytpl{}; // coefficient templates of the Horner passes
    double *coef_dev = nullptr;  // the same tables on the device: x coef, x cu, y coef, y cu
    size_t off_xc = 0, off_xu = 0, off_yc = 0, off_yu = 0;
    double dmr[4][5] = {};       // d^{R 2^k} for register segments R = 8, 16, 32, 64 (per axis below)
    double dmr_ax[3][4][5] = {};
    Level lev[3];
    std::vector<void *> inter;   // intermediate planes (T)
    double *io[2] = {nullptr, nullptr};
    std::vector<void *> allocs;
    int device = 0;
    int num_sms = 152;
    size_t smem_optin = 227 * 1024;
    cudaStream_t cap_stream = nullptr;
    cudaGraphExec_t gexec[4] = {nullptr, nullptr, nullptr, nullptr};   // graphs of kGraphSteps[k] steps
    int64_t launches = 0;
    // launch choices (mol_autotune): warps per CTA of the resident x pass,
    // strided segment length (0 = default) and segments per CTA at most
    int tune_res_warps = 2, tune_strided_rpt = 0, tune_strided_warps = 8;
    int tune_rows_warps = 0;                   // > 0: the x pass splits each row over this many warps
    int tune_rows_persist = 0;                 // row-split x pass: persistent CTAs with next-row L2 prefetch
    int tune_rows_nb = 1;                      // row-split x pass: one neighbour exchange per sweep where
                                               // exact to rounding (two warps per row)
    int tune_strided_nb = 1;                   // float32 strided passes: one neighbour exchange per sweep
                                               // where that is exact to rounding (2: the Horner pass
                                               // also stages its input fields in shared memory)
    int tune_strided_stage = 2;                // ... its tiles: 0 direct, 1 TMA loads, 2 TMA stores, 3 both
    int tune_pdl = 0;                          // register pass kernels as programmatic dependent launches
                                               // (measured slower on the 2D and 3D steps: off)
    double tune_ms = 0.0;                      // step time of the chosen configuration
    // 2D Dirichlet grids (n <= 1024 per axis) whose lines the register
    // kernels cannot split into whole segments run on the batched kernels
    // (ragged lines) as a batch of one problem
    mol_batch batch = nullptr;
    mol_batch adj = nullptr;                   // one-problem batch for the adjoint entry points
    long long *irec = nullptr;                 // receivers (molt_recv.cuh layout), capacity irec_cap
    int nrec = 0, irec_cap = 0, nnode = 0;
    double *srcbuf = nullptr;                  // mol_solve_source: C[g] and two temporaries (3 N)
    float *src32 = nullptr;                    //   float32 copies of g and C[g] (mixed, 2 N)
    double *norm_acc = nullptr;                // mol_field_norm: one double of device scratch
    bool timing = false;                       // per-pass events (benchmarks)
    std::vector<cudaEvent_t> ev_pool;          // reusable events
    std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>> ev_used;  // (axis, (start, stop))
    std::string err;
};

namespace {

thread_local std::string g_err;

// NVTX range for the lifetime of a scope (shows in Nsight timelines; no cost
// without a tool attached)
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};

constexpr int kGraphSteps[4] = {1, 2, 3, 9};

void drop_graphs(mol_ctx *h)
{
    for (cudaGraphExec_t &g : h->gexec) {
        if (g) cudaGraphExecDestroy(g);
        g = nullptr;
    }
}

mol_status fail(mol_ctx *h, mol_status st, const std::string &msg)
{
    if (h) h->err = msg; else g_err = msg;
    return st;
}

mol_status cuda_fail(mol_ctx *h, cudaError_t e, const char *what)
{
    std::string m = std::string(what) + ": " + cudaGetErrorString(e);
    return fail(h, MOL_ECUDA, m);
}

#define CK(expr, what)                                   \
    do {                                                 \
        cudaError_t e_ = (expr);                         \
        if (e_ != cudaSuccess) return cuda_fail(h, e_, what); \
    } while (0)

int ilog2(int W)
{
    int s = 0;
    while ((1 << s) < W) ++s;
    return s;
}

// ---------------------------------------------------------------------------
// Workspace
// ---------------------------------------------------------------------------
mol_status dev_alloc(mol_ctx *h, void **p, size_t bytes)
{
    if (alloc_injected_failure())
        return fail(h, MOL_ENOMEM, "device allocation of " + std::to_string(bytes) + " bytes failed (injected)");
    cudaError_t e = cudaMalloc(p, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(h, MOL_ENOMEM, std::string("device allocation of ") + std::to_string(bytes) +
                                       " bytes failed: " + cudaGetErrorString(e));
    }
    h->allocs.push_back(*p);
    return MOL_OK;
}

void free_all(mol_ctx *h)
{
    if (h->batch) { mol_batch_destroy(h->batch); h->batch = nullptr; }
    if (h->adj) { mol_batch_destroy(h->adj); h->adj = nullptr; }
    for (auto &u : h->ev_used) { h->ev_pool.push_back(u.second.first); h->ev_pool.push_back(u.second.second); }
    h->ev_used.clear();
    for (cudaEvent_t e : h->ev_pool) cudaEventDestroy(e);
    h->ev_pool.clear();
    drop_graphs(h);
    if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
    h->cap_stream = nullptr;
    for (void *p : h->allocs) cudaFree(p);
    h->allocs.clear();
}

// ---------------------------------------------------------------------------
// Passes
// ---------------------------------------------------------------------------
PassGeom geom_of(const mol_ctx *h, int axis)
{
    PassGeom G{};
    int64_t stride = 1;
    for (int a = 0; a < axis; ++a) stride *= h->n[a];
    G.stride = stride;
    G.inner = stride;
    G.nlines = h->N / h->n[axis];
    return G;
}

int choose_W(const mol_ctx *h, int axis, bool horner)
{
    const PassGeom G = geom_of(h, axis);
    const bool contig = (axis == 0);
    int W;
    if (h->opt.lines_per_block > 0) {
        W = h->opt.lines_per_block;
    } else if (contig) {
        W = horner ? (h->tbytes == 4 ? 8 : 4) : 8;
    } else {
        W = h->tbytes == 4 ? 16 : 8;
    }
    const AxisDev &A = h->ax[axis];
    while (W > 1 && pass_smem_bytes(horner, h->tbytes, W, line_stride(A.ms, W, h->tbytes), A.n) > h->smem_optin) W >>= 1;
    if (h->opt.lines_per_block <= 0) {
        // keep at least one CTA per SM; the strided axis keeps >= 8 lines per
        // row access when it can
        const int floorW = contig ? 1 : (h->tbytes == 4 ? 8 : 4);
        while (W > floorW && (G.nlines + W - 1) / W < h->num_sms) W >>= 1;
        while (W > 1 && W > G.nlines) W >>= 1;
    }
    return W;
}

cudaEvent_t take_event(mol_ctx *h)
{
    if (!h->ev_pool.empty()) {
        cudaEvent_t e = h->ev_pool.back();
        h->ev_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    return e;
}

mol_status timing_begin(mol_ctx *h, cudaStream_t s, cudaEvent_t *e0, cudaEvent_t *e1)
{
    if (!h->timing) return MOL_OK;
    *e0 = take_event(h);
    *e1 = take_event(h);
    if (!*e0 || !*e1) return fail(h, MOL_ECUDA, "event creation failed");
    CK(cudaEventRecord(*e0, s), "event record");
    return MOL_OK;
}

mol_status timing_end(mol_ctx *h, cudaStream_t s, int axis, cudaEvent_t e0, cudaEvent_t e1)
{
    if (!h->timing) return MOL_OK;
    CK(cudaEventRecord(e1, s), "event record");
    h->ev_used.push_back({axis, {e0, e1}});
    return MOL_OK;
}

int rpt_index(int rpt) { return rpt == 8 ? 0 : rpt == 16 ? 1 : rpt == 32 ? 2 : 3; }

AxisDev regs_axis(const mol_ctx *h, int axis, int rpt)
{
    AxisDev A = h->ax[axis];
    for (int k = 0; k < 5; ++k) A.dm[k] = h->dmr_ax[axis][rpt_index(rpt)][k];
    axis_mirror(A);
    return A;
}

LineSet lineset_of(const mol_ctx *h, int axis)
{
    const PassGeom G = geom_of(h, axis);
    LineSet L{};
    L.stride = G.stride;
    L.inner = G.inner;
    L.nlines = G.nlines;
    L.S = L.K = 1;
    L.pdl = h->tune_pdl;
    return L;
}

// Launch shape of a shared-memory pass: W lines per CTA, one warp each; a
// single long contiguous line (1D) is swept by the whole CTA instead,
// kCtaLineThreads segments of m points (their constants replace the warp's).
void smem_pass_geom(const mol_ctx *h, int axis, bool horner, PassGeom &G, AxisDev &A)
{
    const int n = (int)h->n[axis];
    G = geom_of(h, axis);
    G.W = choose_W(h, axis, horner);
    G.wshift = ilog2(G.W);
    A = h->ax[axis];
    A.ls = line_stride(A.ms, G.W, h->tbytes);
    if (axis == 0 && G.nlines == 1 && n >= 1024) {
        G.W = 1;
        G.wshift = 0;
        G.cta = 1;
        A.m = (n + kCtaLineThreads - 1) / kCtaLineThreads;
        A.ms = (A.m % 2 == 0) ? A.m + 1 : A.m;
        A.mmagic = (unsigned)(((1ull << 32) + (unsigned long long)A.m - 1) / (unsigned long long)A.m);
        const double nu = -std::log(A.d);
        for (int k = 0; k < 5; ++k) A.dm[k] = std::exp(-nu * (double)A.m * (double)(1 << k));
        axis_mirror(A);
        A.ls = kCtaLineThreads * A.ms;
    }
    G.dps = pass_smem_bytes(horner, h->tbytes, G.W, A.ls, A.n, 1) <= h->smem_optin ? 1 : 0;
}

// Launch one pass program: the register-resident kernel when the line length
// and boundary condition allow it, else the shared-memory kernels.
mol_status run_program(mol_ctx *h, int axis, const ProgParams &pr, const PowersParams *pp, const HornerParams *hp,
                       cudaStream_t s)
{
    static const char *const kPassNames[3] = {"pass x", "pass y", "pass z"};
    NvtxRange nvtx_(kPassNames[axis < 0 || axis > 2 ? 0 : axis]);
    const int n = (int)h->n[axis];
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    mol_status st = timing_begin(h, s, &e0, &e1);
    if (st != MOL_OK) return st;
    int rpt = 0, S = 0, K = 0;
    cudaError_t e;
    const bool bcd = hp != nullptr && hp->bcd;      // boundary data: the shared-memory kernels carry it
    if (bcd) {
        PassGeom G;
        AxisDev A;
        smem_pass_geom(h, axis, true, G, A);
        e = launch_horner(h->tbytes, h->bc, axis == 0, A, G, *hp, s);
    } else if (pr.mode == 2 || pr.mode == 3) {
        // the transposed passes of the adjoint step (register kernels only;
        // single_adjoint checks that the grid has both plans)
        int W = 0;
        if (pr.mode == 3) {
            for (int w : {h->tune_rows_warps, 4, 2, 8})
                if (w > 0 && regs_rows_plan(h->tbytes, n, pr.ng, w, &rpt)) { W = w; break; }
            if (W == 0) return fail(h, MOL_EINVAL, "no register plan for the transposed x pass");
            LineSet L = lineset_of(h, 0);
            L.persist_sms = h->tune_rows_persist ? h->num_sms : 0;
            L.rows_nb = 0;                                      // the transposed pass keeps the full carries
            e = launch_rows(h->bc, rpt, pr.ng, W, regs_axis(h, 0, rpt), L, pr, s);
        } else {
            if (!regs_strided_plan(h->tbytes, h->bc, n, &rpt, &S, &K, h->tune_strided_rpt, h->tune_strided_warps))
                return fail(h, MOL_EINVAL, "no register plan for the transposed y pass");
            LineSet L = lineset_of(h, axis);
            L.S = S;
            L.K = K;
            const AxisDev A = regs_axis(h, axis, rpt);
            if (h->tbytes == 4 && h->tune_strided_nb && regs_strided_nb_plan(A.d, n, rpt))
                e = launch_strided_nb_T(rpt, A, L, pr, s);
            else
                e = launch_strided(h->tbytes, h->bc, rpt, A, L, pr, s);
        }
    } else if (axis == 0 && pr.mode == 1 && pr.nout == 1 && h->tune_rows_warps > 0 &&
        regs_rows_plan(h->tbytes, n, pr.ng, h->tune_rows_warps, &rpt)) {
        LineSet L = lineset_of(h, 0);
        L.persist_sms = h->tune_rows_persist ? h->num_sms : 0;
        L.rows_nb = h->tune_rows_nb;
        e = launch_rows(h->bc, rpt, pr.ng, h->tune_rows_warps, regs_axis(h, 0, rpt), L, pr, s);
    } else if (axis == 0 && pr.mode == 1 && pr.nout == 1 && regs_res_plan(h->tbytes, n, pr.ng, &rpt)) {
        e = launch_res(h->bc, rpt, pr.ng, h->tune_res_warps, regs_axis(h, 0, rpt), lineset_of(h, 0), pr, s);
    } else if (axis == 0 && regs_contig_plan(h->tbytes, h->bc, n, &rpt)) {
        e = launch_contig(h->tbytes, h->bc, rpt, regs_axis(h, 0, rpt), lineset_of(h, 0), pr, s);
    } else if (axis > 0 && regs_strided_plan(h->tbytes, h->bc, n, &rpt, &S, &K, h->tune_strided_rpt,
                                             h->tune_strided_warps)) {
        LineSet L = lineset_of(h, axis);
        L.S = S;
        L.K = K;
        const AxisDev A = regs_axis(h, axis, rpt);
        if (h->tbytes == 4 && pr.mode == 0 && h->tune_strided_nb && regs_strided_nb_plan(A.d, n, rpt))
            e = launch_strided_nb(h->bc, rpt, A, L, pr, s, h->tune_strided_stage);
        else if (h->tbytes == 4 && pr.mode == 1 && h->tune_strided_nb && regs_strided_nb_plan(A.d, n, rpt))
            e = launch_strided_nb_h(h->bc, rpt, A, L, pr, s, h->tune_strided_nb == 2);
        else
            e = launch_strided(h->tbytes, h->bc, rpt, A, L, pr, s);
    } else {
        PassGeom G;
        AxisDev A;
        smem_pass_geom(h, axis, hp != nullptr, G, A);
        e = hp ? launch_horner(h->tbytes, h->bc, axis == 0, A, G, *hp, s)
               : launch_powers(h->tbytes, h->bc, axis == 0, A, G, *pp, s);
    }
    if (e != cudaSuccess) return cuda_fail(h, e, "pass launch");
    h->launches++;
    return timing_end(h, s, axis, e0, e1);
}

mol_status run_powers(mol_ctx *h, int axis, const Level &u, int P, void *const *outs, cudaStream_t s)
{
    PowersParams p{};
    p.P = P;
    p.u_hi = u.hi;
    p.u_lo = u.lo;
    ProgParams pr{};
    pr.mode = 0;
    pr.P = P;
    pr.u_hi = u.hi;
    pr.u_lo = u.lo;
    for (int k = 0; k < P && k < MAXG; ++k) p.out[k] = pr.out[k] = outs[k];
    return run_program(h, axis, pr, &p, nullptr, s);
}

// hp carries the fields; dcoef / dcu are the device copies of its tables
mol_status run_horner(mol_ctx *h, int axis, HornerParams &hp, const double *dcoef, const double *dcu, cudaStream_t s)
{
    ProgParams pr{};
    pr.mode = 1;
    pr.P = hp.P;
    pr.ng = hp.ng;
    pr.nout = hp.nout;
    for (int k = 0; k < MAXG; ++k) { pr.g[k] = hp.g[k]; pr.out[k] = hp.out[k]; }
    pr.coef = dcoef;
    pr.cu = dcu;
    pr.epi = hp.epi;
    pr.ea = hp.ea; pr.eb = hp.eb; pr.ec = hp.ec;
    prog_mirror(pr, hp);
    pr.u_hi = hp.u_hi; pr.u_lo = hp.u_lo; pr.up_hi = hp.up_hi; pr.up_lo = hp.up_lo;
    pr.un_hi = hp.un_hi; pr.un_lo = hp.un_lo;
    return run_program(h, axis, pr, nullptr, &hp, s);
}

double fco(const mol_ctx *h, int i, int j, int k)
{
    const int D = h->P + 1;
    return h->f[(size_t)i + D * ((size_t)j + D * (size_t)k)];
}

// Coefficient tables of the Horner passes (Sec. 4, eq. Full_2D expanded in
// the per-axis D_gamma):
//   1D x pass:  F = sum_t D_x^t (f_t u)                       (cu only)
//   2D x pass:  F = sum_t D_x^t (sum_j f_tj D_y^j u)           g_k = D_y^{k+1} u
//   3D y pass:  G_o = sum_t D_y^t (sum_k f_otk D_z^k u), (t,k) != (0,0)
//   3D x pass:  F = sum_t D_x^t (f_t00 u + G_t)
template <class Fco>
void fill_tables(int ndim, int P, Fco fco, HornerParams &x, HornerParams &y)
{
    x = HornerParams{};
    x.P = P;
    x.nout = 1;
    x.epi = 1;
    if (ndim == 1) {
        x.ng = 0;
        for (int t = 1; t <= P; ++t) x.cu[0][t] = fco(t, 0, 0);
    } else if (ndim == 2) {
        x.ng = P;
        for (int t = 0; t <= P; ++t) {
            for (int k = 0; k < P; ++k) x.coef[0][t][k] = fco(t, k + 1, 0);
            x.cu[0][t] = fco(t, 0, 0);
        }
    } else {
        x.ng = P + 1;
        for (int t = 0; t <= P; ++t) {
            for (int k = 0; k <= P; ++k) x.coef[0][t][k] = (k == t) ? 1.0 : 0.0;
            x.cu[0][t] = fco(t, 0, 0);
        }
        y = HornerParams{};
        y.P = P;
        y.epi = 0;
        y.ng = P;
        y.nout = P + 1;
        for (int o = 0; o <= P; ++o)
            for (int t = 0; t <= P; ++t) {
                for (int k = 0; k < P; ++k) y.coef[o][t][k] = fco(o, t, k + 1);
                y.cu[o][t] = fco(o, t, 0);
            }
    }
}

void build_tables(mol_ctx *h)
{
    fill_tables(h->ndim, h->P, [h](int i, int j, int k) { return fco(h, i, j, k); }, h->xtpl, h->ytpl);
}

void flatten(const HornerParams &hp, std::vector<double> &coef, std::vector<double> &cu)
{
    coef.clear();
    cu.clear();
    for (int o = 0; o < std::max(hp.nout, 1); ++o)
        for (int t = 0; t <= hp.P; ++t) {
            for (int k = 0; k < hp.ng; ++k) coef.push_back(hp.coef[o][t][k]);
            cu.push_back(hp.cu[o][t]);
        }
    if (coef.empty()) coef.push_back(0.0);
}

// un = ea*u + eb*up + ec*F[u]  (the full pass plan of one step).  inter:
// the intermediate planes; xc/xu/yc/yu: device copies of the Horner tables.
mol_status run_update_with(mol_ctx *h, void *const *inter, const double *xc, const double *xu, const double *yc,
                           const double *yu, const Level &u, const Level &up, const Level &un, double ea, double eb,
                           double ec, cudaStream_t s)
{
    const int P = h->P;
    HornerParams hp = h->xtpl;
    hp.ea = ea; hp.eb = eb; hp.ec = ec;
    hp.u_hi = u.hi; hp.u_lo = u.lo;
    hp.up_hi = up.hi; hp.up_lo = up.lo;
    hp.un_hi = un.hi; hp.un_lo = un.lo;
    mol_status st;
    if (h->ndim == 1) return run_horner(h, 0, hp, xc, xu, s);
    if (h->ndim == 2) {
        if ((st = run_powers(h, 1, u, P, inter, s)) != MOL_OK) return st;
        for (int k = 0; k < P; ++k) hp.g[k] = inter[k];
        return run_horner(h, 0, hp, xc, xu, s);
    }
    if ((st = run_powers(h, 2, u, P, inter, s)) != MOL_OK) return st;
    HornerParams yp = h->ytpl;
    yp.u_hi = u.hi; yp.u_lo = u.lo;
    for (int k = 0; k < P; ++k) yp.g[k] = inter[k];
    for (int o = 0; o <= P; ++o) yp.out[o] = inter[P + o];
    if ((st = run_horner(h, 1, yp, yc, yu, s)) != MOL_OK) return st;
    for (int k = 0; k <= P; ++k) hp.g[k] = inter[P + k];
    return run_horner(h, 0, hp, xc, xu, s);
}

mol_status run_update(mol_ctx *h, const Level &u, const Level &up, const Level &un,
                      double ea, double eb, double ec, cudaStream_t s)
{
    const double *b = h->coef_dev;
    return run_update_with(h, h->inter.data(), b + h->off_xc, b + h->off_xu, b + h->off_yc, b + h->off_yu, u, up,
                           un, ea, eb, ec, s);
}

// 2D Dirichlet handles of float32-pair levels whose x rows split over warps
// and whose y lines split into strided segments run the adjoint step on the
// register kernels (transposed modes); others go through a one-problem batch
bool single_adjoint(const mol_ctx *h)
{
    if (h->batch || h->ndim != 2 || h->bc != MOL_BC_DIRICHLET || h->prec != MOL_MIXED) return false;
    int r = 0, S = 0, K = 0;
    bool rows = false;
    for (int w : {2, 4, 8}) rows = rows || regs_rows_plan(h->tbytes, (int)h->n[0], h->xtpl.ng, w, &r);
    return rows && regs_strided_plan(h->tbytes, h->bc, (int)h->n[1], &r, &S, &K, h->tune_strided_rpt,
                                     h->tune_strided_warps);
}

// un = ea u + eb up + ec F^T[u]: powers of D_y^T into the intermediate
// planes, then the Horner pass in D_x^T with the same coefficients (F^T is
// the same polynomial in the transposed one-axis operators, which commute)
mol_status run_update_T(mol_ctx *h, const Level &u, const Level &up, const Level &un, double ea, double eb,
                        double ec, cudaStream_t s)
{
    const int P = h->P;
    ProgParams y{};
    y.mode = 2;
    y.P = P;
    y.u_hi = u.hi;
    y.u_lo = u.lo;
    for (int k = 0; k < P && k < MAXG; ++k) y.out[k] = h->inter[k];
    mol_status st = run_program(h, 1, y, nullptr, nullptr, s);
    if (st != MOL_OK) return st;
    HornerParams hp = h->xtpl;
    hp.ea = ea; hp.eb = eb; hp.ec = ec;
    hp.u_hi = u.hi; hp.u_lo = u.lo;
    hp.up_hi = up.hi; hp.up_lo = up.lo;
    hp.un_hi = un.hi; hp.un_lo = un.lo;
    for (int k = 0; k < P; ++k) hp.g[k] = h->inter[k];
    ProgParams x{};
    x.mode = 3;
    x.P = hp.P;
    x.ng = hp.ng;
    x.nout = hp.nout;
    for (int k = 0; k < MAXG; ++k) { x.g[k] = hp.g[k]; x.out[k] = hp.out[k]; }
    x.coef = h->coef_dev + h->off_xc;
    x.cu = h->coef_dev + h->off_xu;
    x.epi = hp.epi;
    x.ea = ea; x.eb = eb; x.ec = ec;
    x.u_hi = u.hi; x.u_lo = u.lo; x.up_hi = up.hi; x.up_lo = up.lo; x.un_hi = un.hi; x.un_lo = un.lo;
    prog_mirror(x, hp);
    return run_program(h, 0, x, nullptr, &hp, s);
}

// receivers: flat indices of the field (the levels' own layout)
mol_status set_receivers(mol_ctx *h, int nrec, const int64_t *rec, cudaStream_t s)
{
    if (nrec < 1 || !rec) return fail(h, MOL_EINVAL, "need nrec >= 1 receiver indices");
    std::vector<long long> ir(nrec);
    for (int r = 0; r < nrec; ++r) {
        if (rec[r] < 0 || rec[r] >= h->N) return fail(h, MOL_EINVAL, "receiver index out of range");
        ir[r] = rec[r];
    }
    std::vector<long long> buf;
    const int nn = receiver_layout(ir, buf);
    CK(cudaStreamSynchronize(s), "stream synchronize");         // earlier calls may still read the buffer
    if (nrec > h->irec_cap) {
        if (h->irec) {
            cudaFree(h->irec);
            h->allocs.erase(std::find(h->allocs.begin(), h->allocs.end(), (void *)h->irec));
            h->irec = nullptr;
            h->irec_cap = 0;
        }
        mol_status st = dev_alloc(h, (void **)&h->irec, sizeof(long long) * buf.size());
        if (st != MOL_OK) return st;
        h->irec_cap = nrec;
    }
    CK(cudaMemcpy(h->irec, buf.data(), sizeof(long long) * buf.size(), cudaMemcpyHostToDevice), "receiver upload");
    h->nrec = nrec;
    h->nnode = nn;
    return MOL_OK;
}

mol_status gather(mol_ctx *h, const Level &L, double *out, cudaStream_t s)
{
    const int blocks = (h->nrec + 255) / 256;
    k_recv_gather<float><<<blocks, 256, 0, s>>>((const float *)L.hi, (const float *)L.lo, h->irec, h->nrec, out);
    CK(cudaGetLastError(), "receiver gather");
    h->launches++;
    return MOL_OK;
}

mol_status inject(mol_ctx *h, const Level &L, const double *vals, cudaStream_t s)
{
    const long long *node = h->irec + h->nrec, *start = node + h->nrec, *order = start + h->nrec + 1;
    k_recv_inject<float><<<(h->nnode + 127) / 128, 128, 0, s>>>((float *)L.hi, (float *)L.lo, node, start, order,
                                                                h->nnode, vals);
    CK(cudaGetLastError(), "receiver injection");
    h->launches++;
    return MOL_OK;
}

mol_status zero_level(mol_ctx *h, const Level &L, cudaStream_t s)
{
    CK(cudaMemsetAsync(L.hi, 0, (size_t)h->tbytes * h->N, s), "level clear");
    if (L.lo) CK(cudaMemsetAsync(L.lo, 0, (size_t)h->tbytes * h->N, s), "level clear");
    return MOL_OK;
}

mol_status load_level(mol_ctx *h, const double *x, const Level &L, cudaStream_t s)
{
    if (h->prec == MOL_MIXED) {
        CK(launch_to_pair(x, (float *)L.hi, (float *)L.lo, h->N, s), "level conversion");
        h->launches++;
    } else {
        CK(cudaMemcpyAsync(L.hi, x, sizeof(double) * h->N, cudaMemcpyDeviceToDevice, s), "level copy");
    }
    return MOL_OK;
}

mol_status store_level(mol_ctx *h, const Level &L, double *x, cudaStream_t s)
{
    if (h->prec == MOL_MIXED) {
        CK(launch_from_pair((const float *)L.hi, (const float *)L.lo, x, h->N, s), "level conversion");
        h->launches++;
    } else {
        CK(cudaMemcpyAsync(x, L.hi, sizeof(double) * h->N, cudaMemcpyDeviceToDevice, s), "level copy");
    }
    return MOL_OK;
}

// the two levels of a time-stepping call, in and out: one launch each way
// on the mixed path (two when a field is not 16-byte aligned)
mol_status load_levels(mol_ctx *h, const double *x0, const Level &L0, const double *x1, const Level &L1,
                       cudaStream_t s)
{
    if (h->prec != MOL_MIXED) {
        mol_status st = load_level(h, x0, L0, s);
        return st != MOL_OK ? st : load_level(h, x1, L1, s);
    }
    CK(launch_to_pair2(x0, (float *)L0.hi, (float *)L0.lo, x1, (float *)L1.hi, (float *)L1.lo, h->N, s),
       "level conversion");
    h->launches += (((uintptr_t)x0 | (uintptr_t)L0.hi | (uintptr_t)L0.lo | (uintptr_t)x1 | (uintptr_t)L1.hi |
                     (uintptr_t)L1.lo) & 15) ? 2 : 1;
    return MOL_OK;
}

mol_status store_levels(mol_ctx *h, const Level &L0, double *x0, const Level &L1, double *x1, cudaStream_t s)
{
    if (h->prec != MOL_MIXED) {
        mol_status st = store_level(h, L0, x0, s);
        return st != MOL_OK ? st : store_level(h, L1, x1, s);
    }
    CK(launch_from_pair2((const float *)L0.hi, (const float *)L0.lo, x0, (const float *)L1.hi, (const float *)L1.lo,
                         x1, h->N, s), "level conversion");
    h->launches += (((uintptr_t)x0 | (uintptr_t)L0.hi | (uintptr_t)L0.lo | (uintptr_t)x1 | (uintptr_t)L1.hi |
                     (uintptr_t)L1.lo) & 15) ? 2 : 1;
    return MOL_OK;
}

int passes_per_step(const mol_ctx *h) { return h->ndim; }

// Capture three steps (one full rotation of the three level buffers) as a graph.
// Graph k holds kGraphSteps[k] time steps from the first level buffer
// rotation (lev[0] = u^{n-1}, lev[1] = u^n); 3 and 9 steps return to it, 1 and
// 2 end a call's run.  Captured lazily, dropped whenever a launch choice
// changes.
mol_status build_graph(mol_ctx *h, int k)
{
    if (h->gexec[k]) return MOL_OK;
    if (!h->cap_stream) CK(cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking), "stream create");
    cudaGraph_t g = nullptr;
    CK(cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeThreadLocal), "graph capture begin");
    const int64_t before = h->launches;
    mol_status st = MOL_OK;
    for (int j = 0; j < kGraphSteps[k] && st == MOL_OK; ++j)
        st = run_update(h, h->lev[(j + 1) % 3], h->lev[j % 3], h->lev[(j + 2) % 3], 2.0, -1.0, 1.0, h->cap_stream);
    cudaError_t e = cudaStreamEndCapture(h->cap_stream, &g);
    h->launches = before;
    if (st != MOL_OK) { if (g) cudaGraphDestroy(g); return st; }
    if (e != cudaSuccess) return cuda_fail(h, e, "graph capture end");
    e = cudaGraphInstantiate(&h->gexec[k], g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) { h->gexec[k] = nullptr; return cuda_fail(h, e, "graph instantiate"); }
    return MOL_OK;
}

mol_status check_ptr(mol_ctx *h, const void *p, const char *name)
{
    if (!p) return fail(h, MOL_EINVAL, std::string(name) + " is NULL");
    cudaPointerAttributes at{};
    cudaError_t e = cudaPointerGetAttributes(&at, p);
    if (e != cudaSuccess) { cudaGetLastError(); return fail(h, MOL_EINVAL, std::string(name) + ": not a CUDA pointer"); }
    if (at.type != cudaMemoryTypeDevice && at.type != cudaMemoryTypeManaged)
        return fail(h, MOL_EINVAL, std::string(name) + " must be device memory");
    return MOL_OK;
}

// Rows split over two warps where the row length allows it (faster than one
// warp per row on every measured grid; mol_autotune may still choose
// otherwise).  Needs h->xtpl filled.
void default_rows_split(mol_ctx *h)
{
    int r = 0;
    if (h->ndim >= 2 && regs_rows_plan(h->tbytes, (int)h->n[0], h->xtpl.ng, 2, &r)) h->tune_rows_warps = 2;
}

}  // namespace

void molt::set_global_error(const std::string &msg) { g_err = msg; }

// ===========================================================================
// C ABI
// ===========================================================================
extern "C" {

void mol_default_options(mol_options *opt)
{
    if (!opt) return;
    opt->quad_order = 2;
    opt->lines_per_block = 0;
    opt->use_graphs = 1;
}

double mol_beta_max(int P) { return beta_max_of(P); }

int64_t mol_max_line(mol_prec) { return kMaxLine; }

const char *mol_last_error(mol_handle h)
{
    if (!h) return g_err.c_str();
    return h->err.c_str();
}

mol_status mol_create(const mol_grid *grid, double c, double dt, double beta, int P, mol_bc bc,
                      mol_prec prec, const mol_options *opt, mol_handle *out)
{
    mol_ctx *h = nullptr;
    if (!out) return fail(nullptr, MOL_EINVAL, "out is NULL");
    *out = nullptr;
    if (!grid) return fail(nullptr, MOL_EINVAL, "grid is NULL");
    if (grid->ndim < 1 || grid->ndim > 3) return fail(nullptr, MOL_EINVAL, "ndim must be 1, 2 or 3");
    if (P < 1 || P > kMaxP) return fail(nullptr, MOL_EINVAL, "P must be in 1..5");
    if (!(c > 0) || !(dt > 0) || !std::isfinite(c) || !std::isfinite(dt)) return fail(nullptr, MOL_EINVAL, "c and dt must be positive");
    if (bc != MOL_BC_PERIODIC && bc != MOL_BC_DIRICHLET) return fail(nullptr, MOL_EINVAL, "unknown boundary condition");
    if (prec != MOL_FP64 && prec != MOL_MIXED) return fail(nullptr, MOL_EINVAL, "unknown precision");
    mol_options o;
    mol_default_options(&o);
    if (opt) o = *opt;
    if (o.quad_order != 1 && o.quad_order != 2) return fail(nullptr, MOL_EINVAL, "quad_order must be 1 or 2");
    if (o.lines_per_block != 0 && (o.lines_per_block < 1 || o.lines_per_block > 16 ||
                                   (o.lines_per_block & (o.lines_per_block - 1))))
        return fail(nullptr, MOL_EINVAL, "lines_per_block must be 0 or a power of two <= 16");
    for (int a = 0; a < grid->ndim; ++a) {
        if (grid->n[a] < 3 || grid->n[a] > kMaxLine)
            return fail(nullptr, MOL_EINVAL, "every axis needs 3 <= n <= " + std::to_string(kMaxLine));
        if (!(grid->hi[a] > grid->lo[a])) return fail(nullptr, MOL_EINVAL, "hi must exceed lo on every axis");
    }
    const double bmax = beta_max_of(P);
    if (beta <= 0) beta = bmax;
    if (beta > bmax * (1.0 + 1e-12) && !unstable_allowed())
        return fail(nullptr, MOL_EUNSTABLE, "beta above beta_max(P): the scheme is not A-stable");

    h = new mol_ctx();
    h->ndim = grid->ndim;
    h->N = 1;
    for (int a = 0; a < 3; ++a) {
        h->n[a] = a < grid->ndim ? grid->n[a] : 1;
        h->lo[a] = grid->lo[a];
        h->hi[a] = grid->hi[a];
        h->N *= h->n[a];
    }
    h->c = c; h->dt = dt; h->beta = beta; h->P = P; h->bc = bc; h->prec = prec; h->opt = o;
    h->alpha = beta / (c * dt);                        // eq. L_def
    h->tbytes = (prec == MOL_MIXED) ? 4 : 8;
    mol_status st;
    cudaError_t e;
    if ((e = cudaGetDevice(&h->device)) != cudaSuccess) { st = cuda_fail(h, e, "cudaGetDevice"); goto bad; }
    {
        int v = 0;
        if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, h->device) == cudaSuccess && v > 0) h->num_sms = v;
        if (cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, h->device) == cudaSuccess && v > 0)
            h->smem_optin = (size_t)v;
    }
    if ((e = configure_kernels()) != cudaSuccess) { st = cuda_fail(h, e, "kernel attributes"); goto bad; }
    if ((e = configure_regs_kernels()) != cudaSuccess) { st = cuda_fail(h, e, "kernel attributes"); goto bad; }
    if (!expand_coefficients(h->ndim, P, beta, h->f)) { st = fail(h, MOL_EINVAL, "coefficient expansion failed"); goto bad; }

    for (int a = 0; a < h->ndim; ++a) {
        const int64_t n = h->n[a];
        h->h[a] = (h->hi[a] - h->lo[a]) / (double)(bc == MOL_BC_DIRICHLET ? n - 1 : n);
        h->nu[a] = h->alpha * h->h[a];
        axis_constants(h->nu[a], n, bc, o.quad_order, h->ax[a]);
        std::vector<double> t64(n + 1);
        std::vector<float> t32(n + 1);
        for (int64_t j = 0; j <= n; ++j) {
            t64[j] = std::exp(-h->nu[a] * (double)j);
            t32[j] = (float)t64[j];
        }
        if ((st = dev_alloc(h, (void **)&h->dpow64[a], sizeof(double) * (n + 1))) != MOL_OK) goto bad;
        if ((st = dev_alloc(h, (void **)&h->dpow32[a], sizeof(float) * (n + 1))) != MOL_OK) goto bad;
        if ((e = cudaMemcpy(h->dpow64[a], t64.data(), sizeof(double) * (n + 1), cudaMemcpyHostToDevice)) != cudaSuccess ||
            (e = cudaMemcpy(h->dpow32[a], t32.data(), sizeof(float) * (n + 1), cudaMemcpyHostToDevice)) != cudaSuccess) {
            st = cuda_fail(h, e, "constant upload");
            goto bad;
        }
        h->ax[a].dpow64 = h->dpow64[a];
        h->ax[a].dpow32 = h->dpow32[a];
        for (int r = 0; r < 4; ++r)
            for (int k = 0; k < 5; ++k)
                h->dmr_ax[a][r][k] = std::exp(-h->nu[a] * (double)(8 << r) * (double)(1 << k));
    }
    {
        build_tables(h);
        std::vector<double> xc, xu, yc, yu, all;
        flatten(h->xtpl, xc, xu);
        if (h->ndim == 3) flatten(h->ytpl, yc, yu);
        else { yc.assign(1, 0.0); yu.assign(1, 0.0); }
        h->off_xc = 0;
        h->off_xu = xc.size();
        h->off_yc = h->off_xu + xu.size();
        h->off_yu = h->off_yc + yc.size();
        all = xc;
        all.insert(all.end(), xu.begin(), xu.end());
        all.insert(all.end(), yc.begin(), yc.end());
        all.insert(all.end(), yu.begin(), yu.end());
        if ((st = dev_alloc(h, (void **)&h->coef_dev, sizeof(double) * all.size())) != MOL_OK) goto bad;
        if ((e = cudaMemcpy(h->coef_dev, all.data(), sizeof(double) * all.size(), cudaMemcpyHostToDevice)) != cudaSuccess) {
            st = cuda_fail(h, e, "coefficient upload");
            goto bad;
        }
    }
    // levels: three rotating buffers
    for (int k = 0; k < 3; ++k) {
        if (prec == MOL_MIXED) {
            if ((st = dev_alloc(h, &h->lev[k].hi, sizeof(float) * h->N)) != MOL_OK) goto bad;
            if ((st = dev_alloc(h, &h->lev[k].lo, sizeof(float) * h->N)) != MOL_OK) goto bad;
        } else {
            if ((st = dev_alloc(h, &h->lev[k].hi, sizeof(double) * h->N)) != MOL_OK) goto bad;
        }
    }
    {
        // intermediate planes: 2D P (powers of D_y), 3D P + (P+1); at least one
        // for mol_apply_D
        int ninter = h->ndim == 2 ? P : (h->ndim == 3 ? 2 * P + 1 : 0);
        if (ninter < 1) ninter = 1;
        h->inter.assign(MAXG * 2, nullptr);
        for (int k = 0; k < ninter; ++k)
            if ((st = dev_alloc(h, &h->inter[k], (size_t)h->tbytes * h->N)) != MOL_OK) goto bad;
    }
    default_rows_split(h);
    if (h->ndim == 2 && bc == MOL_BC_DIRICHLET && h->n[0] <= 1024 && h->n[1] <= 1024) {
        int r = 0, S = 0, K = 0;
        const bool xreg = regs_res_plan(h->tbytes, (int)h->n[0], h->xtpl.ng, &r) ||
                          regs_contig_plan(h->tbytes, h->bc, (int)h->n[0], &r);
        const bool yreg = regs_strided_plan(h->tbytes, h->bc, (int)h->n[1], &r, &S, &K);
        if (!xreg || !yreg) {
            if ((st = mol_batch_create(1, grid, &c, &dt, &beta, &P, bc, prec, &o, &h->batch)) != MOL_OK) {
                h->err = mol_last_error(nullptr);
                goto bad;
            }
        }
    }
    *out = h;
    return MOL_OK;
bad:
    g_err = h->err;
    free_all(h);
    delete h;
    return st;
}

mol_status mol_destroy(mol_handle h)
{
    if (!h) return fail(nullptr, MOL_EINVAL, "handle is NULL");
    cudaDeviceSynchronize();
    free_all(h);
    delete h;
    return MOL_OK;
}

mol_status mol_get_params(mol_handle h, double out[8])
{
    if (!h || !out) return fail(h, MOL_EINVAL, "NULL argument");
    out[0] = h->alpha;
    out[1] = h->beta;
    for (int a = 0; a < 3; ++a) {
        out[2 + a] = a < h->ndim ? h->nu[a] : 0.0;
        out[5 + a] = a < h->ndim ? h->ax[a].d : 0.0;
    }
    return MOL_OK;
}

mol_status mol_apply_D(mol_handle h, const double *v, double *outp, int axis, int power, void *stream)
{
    NvtxRange nvtx_("mol_apply_D");
    if (!h) return fail(nullptr, MOL_EINVAL, "handle is NULL");
    if (axis < 0 || axis >= h->ndim) return fail(h, MOL_EINVAL, "axis out of range");
    if (power < 1 || power > MAXG) return fail(h, MOL_EINVAL, "power must be in 1..8");
    mol_status st;
    if ((st = check_ptr(h, v, "v")) != MOL_OK || (st = check_ptr(h, outp, "out")) != MOL_OK) return st;
    if (v == outp) return fail(h, MOL_EINVAL, "v and out must not overlap");
    cudaStream_t s = (cudaStream_t)stream;
    void *outs[MAXG] = {nullptr};
    if (h->prec == MOL_MIXED) {
        if ((st = load_level(h, v, h->lev[0], s)) != MOL_OK) return st;
        outs[power - 1] = h->inter[0];
        if ((st = run_powers(h, axis, h->lev[0], power, outs, s)) != MOL_OK) return st;
        CK(launch_from_f32((const float *)h->inter[0], outp, h->N, s), "output conversion");
        h->launches++;
    } else {
        Level L;
        L.hi = (void *)v;
        outs[power - 1] = outp;
        if ((st = run_powers(h, axis, L, power, outs, s)) != MOL_OK) return st;
    }
    return MOL_OK;
}

mol_status mol_apply_F(mol_handle h, const double *u, double *F, void *stream)
{
    NvtxRange nvtx_("mol_apply_F");
    if (!h) return fail(nullptr, MOL_EINVAL, "handle is NULL");
    if (h->batch) {
        const mol_status st0 = mol_batch_apply_F(h->batch, u, F, stream);
        if (st0 != MOL_OK) h->err = mol_batch_last_error(h->batch);
        return st0;
    }
    mol_status st;
    if ((st = check_ptr(h, u, "u")) != MOL_OK || (st = check_ptr(h, F, "F")) != MOL_OK) return st;
    if (u == F) return fail(h, MOL_EINVAL, "u and F must not overlap");
    cudaStream_t s = (cudaStream_t)stream;
    if (h->prec == MOL_MIXED) {
        if ((st = load_level(h, u, h->lev[0], s)) != MOL_OK) return st;
        if ((st = run_update(h, h->lev[0], h->lev[0], h->lev[1], 0.0, 0.0, 1.0, s)) != MOL_OK) return st;
        return store_level(h, h->lev[1], F, s);
    }
    Level U, O;
    U.hi = (void *)u;
    O.hi = F;
    return run_update(h, U, U, O, 0.0, 0.0, 1.0, s);
}

mol_status mol_start(mol_handle h, const double *u0, double *u1, void *stream)
{
    NvtxRange nvtx_("mol_start");
    if (!h) return fail(nullptr, MOL_EINVAL, "handle is NULL");
    if (h->batch) {
        const mol_status st0 = mol_batch_start(h->batch, u0, u1, stream);
        if (st0 != MOL_OK) h->err = mol_batch_last_error(h->batch);
        return st0;
    }
    mol_status st;
    if ((st = check_ptr(h, u0, "u0")) != MOL_OK || (st = check_ptr(h, u1, "u1")) != MOL_OK) return st;
    if (u0 == u1) return fail(h, MOL_EINVAL, "u0 and u1 must not overlap");
    cudaStream_t s = (cudaStream_t)stream;
    if (h->prec == MOL_MIXED) {
        if ((st = load_level(h, u0, h->lev[0], s)) != MOL_OK) return st;
        if ((st = run_update(h, h->lev[0], h->lev[0], h->lev[1], 1.0, 0.0, 0.5, s)) != MOL_OK) return st;
        return store_level(h, h->lev[1], u1, s);
    }
    Level U, O;
    U.hi = (void *)u0;
    O.hi = u1;
    return run_update(h, U, U, O, 1.0, 0.0, 0.5, s);
}

mol_status mol_step(mol_handle h, double *u_prev, double *u_cur, int64_t nsteps, void *stream)
{
    NvtxRange nvtx_("mol_step");
    if (!h) return fail(nullptr, MOL_EINVAL, "handle is NULL");
    if (h->batch) {
        const mol_status st0 = mol_batch_step(h->batch, u_prev, u_cur, nsteps, stream);
        if (st0 != MOL_OK) h->err = mol_batch_last_error(h->batch);
        return st0;
    }
    if (nsteps < 0) return fail(h, MOL_EINVAL, "nsteps must be >= 0");
    mol_status st;
    if ((st = check_ptr(h, u_prev, "u_prev")) != MOL_OK || (st = check_ptr(h, u_cur, "u_cur")) != MOL_OK) return st;
    if (u_prev == u_cur) return fail(h, MOL_EINVAL, "u_prev and u_cur must not overlap");
    if (nsteps == 0) return MOL_OK;
    cudaStream_t s = (cudaStream_t)stream;
    if ((st = load_levels(h, u_prev, h->lev[0], u_cur, h->lev[1], s)) != MOL_OK) return st;
    int64_t done = 0;
    if (h->opt.use_graphs && !h->timing) {
        // whole rotations by graphs of 9 and 3 steps, the rest by a graph of 1 or 2
        while (done < nsteps) {
            const int64_t left = nsteps - done;
            const int k = left >= 9 ? 3 : (left >= 3 ? 2 : (int)left - 1);
            if ((st = build_graph(h, k)) != MOL_OK) return st;
            CK(cudaGraphLaunch(h->gexec[k], s), "graph launch");
            h->launches += kGraphSteps[k] * passes_per_step(h);
            done += kGraphSteps[k];
        }
    }
    for (; done < nsteps; ++done) {
        const int k = (int)(done % 3);
        if ((st = run_update(h, h->lev[(k + 1) % 3], h->lev[k], h->lev[(k + 2) % 3], 2.0, -1.0, 1.0, s)) != MOL_OK)
            return st;
    }
    const int k = (int)(nsteps % 3);
    return store_levels(h, h->lev[k], u_prev, h->lev[(k + 1) % 3], u_cur, s);
}

mol_status mol_solve_host(mol_handle h, const double *u0, double *u_out, int64_t nsteps, void *stream)
{
    NvtxRange nvtx_("mol_solve_host");
    if (!h) return fail(nullptr, MOL_EINVAL, "handle is NULL");
    if (h->batch) {
        const mol_status st0 = mol_batch_solve_host(h->batch, u0, u_out, nsteps, stream);
        if (st0 != MOL_OK) h->err = mol_batch_last_error(h->batch);
        return st0;
    }
    if (!u0 || !u_out) return fail(h, MOL_EINVAL, "NULL host buffer");
    if (nsteps < 1) return fail(h, MOL_EINVAL, "nsteps must be >= 1");
    mol_status st;
    for (int k = 0; k < 2; ++k)
        if (!h->io[k] && (st = dev_alloc(h, (void **)&h->io[k], sizeof(double) * h->N)) != MOL_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    CK(cudaMemcpyAsync(h->io[0], u0, sizeof(double) * h->N, cudaMemcpyHostToDevice, s), "host to device copy");
    if ((st = mol_start(h, h->io[0], h->io[1], stream)) != MOL_OK) return st;
    if ((st = mol_step(h, h->io[0], h->io[1], nsteps - 1, stream)) != MOL_OK) return st;
    CK(cudaMemcpyAsync(u_out, h->io[1], sizeof(double) * h->N, cudaMemcpyDeviceToHost, s), "device to host copy");
    CK(cudaStreamSynchronize(s), "solve");
    return MOL_OK;
}

mol_status mol_autotune(mol_handle h, void *stream)
{
    NvtxRange nvtx_("mol_autotune");
    if (!h) return fail(nullptr, MOL_EINVAL, "handle is NULL");
    if (h->batch) {
        const mol_status st0 = mol_batch_autotune(h->batch, stream);
        double ms[2] = {0.0, 0.0};
        if (st0 == MOL_OK) {
            int out[3];
            mol_batch_get_tuning(h->batch, out, ms);
            h->tune_ms = ms[0] + ms[1];
        }
        return st0;
    }
    cudaStream_t s = (cudaStream_t)stream;
    // candidates that change something for this grid
    int dummy = 0, r0 = 0, S0 = 0, K0 = 0;
    const bool res = h->ndim >= 2 && regs_res_plan(h->tbytes, (int)h->n[0], h->xtpl.ng, &dummy);
    bool strided = false;
    for (int a = 1; a < h->ndim; ++a) strided |= regs_strided_plan(h->tbytes, h->bc, (int)h->n[a], &r0, &S0, &K0);
    // x variants: one warp per row with 1, 2 or 4 warps per CTA (code 1, 2, 4),
    // or each row split over 2, 4 or 8 warps, one CTA per row (code -2, -4,
    // -8) or persistent CTAs (code -102, -104, -108)
    std::vector<int> warps_c = res ? std::vector<int>{1, 2, 4} : std::vector<int>{h->tune_res_warps};
    if (h->ndim >= 2) {
        for (int W : {2, 4, 8})
            if (regs_rows_plan(h->tbytes, (int)h->n[0], h->xtpl.ng, W, &dummy)) {
                warps_c.push_back(-W);
                warps_c.push_back(-100 - W);
                if (rows_nb_plan(h->ax[0].d, (int)h->n[0], dummy, W)) warps_c.push_back(-200 - W);
            }
    }
    // strided variants: segment length code, segments per CTA at most, and
    // (float32) the neighbour-exchange kernel where it applies (code + 100)
    std::vector<std::pair<int, int>> str_c = {
        {h->tune_strided_rpt + 100 * h->tune_strided_nb + 1000 * h->tune_strided_stage, h->tune_strided_warps}};
    if (strided) {
        std::vector<std::pair<int, int>> base = {{0, 8}, {0, 4}};
        if (h->tbytes == 4) { base.push_back({32, 8}); base.push_back({32, 4}); }
        str_c.clear();
        for (auto &b : base) {
            bool nb = false;
            for (int a = 1; a < h->ndim && h->tbytes == 4; ++a) {
                int rr = 0, SS = 0, KK = 0;
                if (regs_strided_plan(h->tbytes, h->bc, (int)h->n[a], &rr, &SS, &KK, b.first, b.second))
                    nb |= regs_strided_nb_plan(h->ax[a].d, (int)h->n[a], rr);
            }
            if (nb)
                for (int stg = 0; stg < 4; ++stg) str_c.push_back({b.first + 100 + 1000 * stg, b.second});
            if (nb && h->ndim == 3)               // the y Horner pass with its fields staged
                for (int stg : {0, 2}) str_c.push_back({b.first + 200 + 1000 * stg, b.second});
            str_c.push_back(b);
        }
    }
    for (int k = 0; k < 3; ++k) {
        const size_t bytes = (size_t)h->tbytes * h->N;
        if (h->lev[k].hi) CK(cudaMemsetAsync(h->lev[k].hi, 0, bytes, s), "memset");
        if (h->lev[k].lo) CK(cudaMemsetAsync(h->lev[k].lo, 0, bytes, s), "memset");
    }
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    CK(cudaEventCreate(&e0), "event create");
    if (cudaEventCreate(&e1) != cudaSuccess) { cudaEventDestroy(e0); return fail(h, MOL_ECUDA, "event create"); }
    const bool was_timing = h->timing;
    h->timing = false;
    const int64_t launches0 = h->launches;
    double best = 1e30;
    int bw = h->tune_res_warps, br = h->tune_strided_rpt, bsw = h->tune_strided_warps, brw = h->tune_rows_warps;
    int bpe = h->tune_rows_persist, bnb = h->tune_strided_nb, bst = h->tune_strided_stage, brn = h->tune_rows_nb;
    mol_status st = MOL_OK;
    for (int w : warps_c) {
        for (auto &sc : str_c) {
            int rr = 0, SS = 0, KK = 0;
            bool ok = true;
            for (int a = 1; a < h->ndim && strided; ++a)
                ok &= regs_strided_plan(h->tbytes, h->bc, (int)h->n[a], &rr, &SS, &KK, sc.first % 100, sc.second);
            if (!ok) continue;
            h->tune_res_warps = w > 0 ? w : h->tune_res_warps;
            h->tune_rows_warps = w < 0 ? (-w) % 100 : 0;
            h->tune_rows_persist = (w < -100 && w > -200) ? 1 : 0;
            h->tune_rows_nb = w < -200 ? 1 : 0;
            h->tune_strided_rpt = sc.first % 100;
            h->tune_strided_nb = (sc.first / 100) % 10;
            h->tune_strided_stage = sc.first / 1000;
            h->tune_strided_warps = sc.second;
            // 2 warm-up steps, then the minimum of 3 timings of 3 steps
            double t = 1e30;
            for (int rep = 0; rep < 4 && st == MOL_OK; ++rep) {
                if (rep > 0 && cudaEventRecord(e0, s) != cudaSuccess) { st = fail(h, MOL_ECUDA, "event record"); break; }
                for (int k = 0; k < (rep == 0 ? 2 : 3) && st == MOL_OK; ++k)
                    st = run_update(h, h->lev[(k + 1) % 3], h->lev[k % 3], h->lev[(k + 2) % 3], 2.0, -1.0, 1.0, s);
                if (st != MOL_OK) break;
                if (rep > 0) {
                    float ms = 0.f;
                    if (cudaEventRecord(e1, s) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
                        cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
                        st = fail(h, MOL_ECUDA, "tuning timer");
                        break;
                    }
                    t = std::min(t, (double)ms / 3.0);
                }
            }
            if (st != MOL_OK) break;
            if (t < best) {
                best = t;
                bw = h->tune_res_warps;
                brw = h->tune_rows_warps;
                bpe = h->tune_rows_persist;
                brn = h->tune_rows_nb;
                bnb = h->tune_strided_nb;
                bst = h->tune_strided_stage;
                br = sc.first % 100;
                bsw = sc.second;
            }
        }
        if (st != MOL_OK) break;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    h->timing = was_timing;
    h->launches = launches0;
    h->tune_res_warps = bw;
    h->tune_rows_warps = brw;
    h->tune_rows_persist = bpe;
    h->tune_rows_nb = brn;
    h->tune_strided_nb = bnb;
    h->tune_strided_stage = bst;
    h->tune_strided_rpt = br;
    h->tune_strided_warps = bsw;
    h->tune_ms = best < 1e30 ? best : 0.0;
    drop_graphs(h);                                      // rebuilt with the choice
    return st;
}

mol_status mol_set_tuning(mol_handle h, int res_warps, int strided_rpt, int strided_warps, int rows_warps)
{
    if (!h) return fail(nullptr, MOL_EINVAL, "handle is NULL");
    if (res_warps != 1 && res_warps != 2 && res_warps != 4) return fail(h, MOL_EINVAL, "res_warps must be 1, 2 or 4");
    if (rows_warps != 0 && rows_warps != 2 && rows_warps != 4 && rows_warps != 8)
        return fail(h, MOL_EINVAL, "rows_warps must be 0, 2, 4 or 8");
    if (strided_rpt != 0 && strided_rpt != 32) return fail(h, MOL_EINVAL, "strided_rpt must be 0 or 32");
    if (strided_warps < 1 || strided_warps > 8) return fail(h, MOL_EINVAL, "strided_warps must be in 1..8");
    for (int a = 1; a < h->ndim; ++a) {
        int r = 0, S = 0, K = 0;
        const int n = (int)h->n[a];
        // a choice must keep every strided axis that has a register plan on one
        if (regs_strided_plan(h->tbytes, h->bc, n, &r, &S, &K) &&
            !regs_strided_plan(h->tbytes, h->bc, n, &r, &S, &K, strided_rpt, strided_warps))
            return fail(h, MOL_EINVAL, "the strided choice does not fit an axis of this grid");
    }
    h->tune_res_warps = res_warps;
    h->tune_rows_warps = rows_warps;
    h->tune_strided_rpt = strided_rpt;
    h->tune_strided_warps = strided_warps;
    drop_graphs(h);
    return MOL_OK;
}

mol_status mol_get_tuning(mol_handle h, int out[4], double *ms_per_step)
{
    if (!h || !out) return fail(h, MOL_EINVAL, "NULL argument");
    out[0] = h->tune_res_warps;
    out[1] = h->tune_strided_rpt;
    out[2] = h->tune_strided_warps;
    out[3] = h->tune_rows_warps;
    if (ms_per_step) *ms_per_step = h->tune_ms;
    return MOL_OK;
}

mol_status mol_set_tuning_ex(mol_handle h, const int *vals, int count)
{
    if (!h || !vals) return fail(h, MOL_EINVAL, "NULL argument");
    if (count < 4 || count > MOL_TUNE_COUNT)
        return fail(h, MOL_EINVAL, "count must be in 4.." + std::to_string(MOL_TUNE_COUNT));
    if (count > MOL_TUNE_ROWS_PERSIST && vals[MOL_TUNE_ROWS_PERSIST] != 0 && vals[MOL_TUNE_ROWS_PERSIST] != 1)
        return fail(h, MOL_EINVAL, "rows_persist must be 0 or 1");
    if (count > MOL_TUNE_STRIDED_NB && (vals[MOL_TUNE_STRIDED_NB] < 0 || vals[MOL_TUNE_STRIDED_NB] > 2))
        return fail(h, MOL_EINVAL, "strided_nb must be 0, 1 or 2");
    if (count > MOL_TUNE_STRIDED_STAGE && (vals[MOL_TUNE_STRIDED_STAGE] < 0 || vals[MOL_TUNE_STRIDED_STAGE] > 3))
        return fail(h, MOL_EINVAL, "strided_stage must be 0, 1, 2 or 3");
    if (count > MOL_TUNE_ROWS_NB && vals[MOL_TUNE_ROWS_NB] != 0 && vals[MOL_TUNE_ROWS_NB] != 1)
        return fail(h, MOL_EINVAL, "rows_nb must be 0 or 1");
    if (count > MOL_TUNE_PDL && vals[MOL_TUNE_PDL] != 0 && vals[MOL_TUNE_PDL] != 1)
        return fail(h, MOL_EINVAL, "pdl must be 0 or 1");
    mol_status st = mol_set_tuning(h, vals[MOL_TUNE_RES_WARPS], vals[MOL_TUNE_STRIDED_RPT],
                                   vals[MOL_TUNE_STRIDED_WARPS], vals[MOL_TUNE_ROWS_WARPS]);
    if (st != MOL_OK) return st;
    if (count > MOL_TUNE_ROWS_PERSIST) h->tune_rows_persist = vals[MOL_TUNE_ROWS_PERSIST];
    if (count > MOL_TUNE_STRIDED_NB) h->tune_strided_nb = vals[MOL_TUNE_STRIDED_NB];
    if (count > MOL_TUNE_STRIDED_STAGE) h->tune_strided_stage = vals[MOL_TUNE_STRIDED_STAGE];
    if (count > MOL_TUNE_ROWS_NB) h->tune_rows_nb = vals[MOL_TUNE_ROWS_NB];
    if (count > MOL_TUNE_PDL) h->tune_pdl = vals[MOL_TUNE_PDL];
    drop_graphs(h);
    return MOL_OK;
}

mol_status mol_get_tuning_ex(mol_handle h, int *vals, int count, double *ms_per_step)
{
    if (!h || !vals) return fail(h, MOL_EINVAL, "NULL argument");
    if (count < 1 || count > MOL_TUNE_COUNT)
        return fail(h, MOL_EINVAL, "count must be in 1.." + std::to_string(MOL_TUNE_COUNT));
    const int all[MOL_TUNE_COUNT] = {h->tune_res_warps, h->tune_strided_rpt, h->tune_strided_warps,
                                     h->tune_rows_warps, h->tune_rows_persist, h->tune_strided_nb,
                                     h->tune_strided_stage, h->tune_rows_nb, h->tune_pdl};
    for (int i = 0; i < count; ++i) vals[i] = all[i];
    if (ms_per_step) *ms_per_step = h->tune_ms;
    return MOL_OK;
}

// The adjoint runs on the batched kernels (ragged lines, transposed sweeps):
// the handle's own one-problem batch, or one made on first use.
static mol_status adjoint_batch(mol_ctx *h, mol_batch *out)
{
    if (h->batch) { *out = h->batch; return MOL_OK; }
    if (!h->adj) {
        if (h->ndim != 2 || h->bc != MOL_BC_DIRICHLET || h->n[0] > 1024 || h->n[1] > 1024)
            return fail(h, MOL_EINVAL, "the adjoint entry points take 2D Dirichlet grids of at most 1024 points per axis");
        mol_grid g{};
        g.ndim = 2;
        for (int a = 0; a < 2; ++a) { g.n[a] = h->n[a]; g.lo[a] = h->lo[a]; g.hi[a] = h->hi[a]; }
        mol_status st = mol_batch_create(1, &g, &h->c, &h->dt, &h->beta, &h->P, MOL_BC_DIRICHLET, (mol_prec)h->prec,
                                         &h->opt, &h->adj);
        if (st != MOL_OK) return fail(h, st, mol_last_error(nullptr));
    }
    *out = h->adj;
    return MOL_OK;
}

mol_status mol_apply_FT(mol_handle h, const double *w, double *out, void *stream)
{
    if (!h) return fail(nullptr, MOL_EINVAL, "handle is NULL");
    if (single_adjoint(h)) {
        mol_status st;
        if ((st = check_ptr(h, w, "w")) != MOL_OK || (st = check_ptr(h, out, "out")) != MOL_OK) return st;
        if (w == out) return fail(h, MOL_EINVAL, "w and out must not overlap");
        cudaStream_t s = (cudaStream_t)stream;
        if ((st = load_level(h, w, h->lev[0], s)) != MOL_OK) return st;
        if ((st = run_update_T(h, h->lev[0], h->lev[0], h->lev[1], 0.0, 0.0, 1.0, s)) != MOL_OK) return st;
        return store_level(h, h->lev[1], out, s);
    }
    mol_batch b = nullptr;
    mol_status st = adjoint_batch(h, &b);
    if (st != MOL_OK) return st;
    if ((st = mol_batch_apply_FT(b, w, out, stream)) != MOL_OK) h->err = mol_batch_last_error(b);
    return st;
}

mol_status mol_traces(mol_handle h, const double *u0, int nrec, const int64_t *rec, int64_t nsteps, double *traces,
                      void *stream)
{
    if (!h) return fail(nullptr, MOL_EINVAL, "handle is NULL");
    if (single_adjoint(h)) {
        if (nsteps < 1) return fail(h, MOL_EINVAL, "nsteps must be >= 1");
        mol_status st;
        if ((st = check_ptr(h, u0, "u0")) != MOL_OK || (st = check_ptr(h, traces, "traces")) != MOL_OK) return st;
        cudaStream_t s = (cudaStream_t)stream;
        if ((st = set_receivers(h, nrec, rec, s)) != MOL_OK) return st;
        // traces[n-1] = u^n at the receivers, n = 1..nsteps
        int ip = 0, ic = 1, in = 2;
        if ((st = load_level(h, u0, h->lev[ip], s)) != MOL_OK) return st;
        if ((st = run_update(h, h->lev[ip], h->lev[ip], h->lev[ic], 1.0, 0.0, 0.5, s)) != MOL_OK) return st;
        if ((st = gather(h, h->lev[ic], traces, s)) != MOL_OK) return st;
        for (int64_t n = 1; n < nsteps; ++n) {
            if ((st = run_update(h, h->lev[ic], h->lev[ip], h->lev[in], 2.0, -1.0, 1.0, s)) != MOL_OK) return st;
            if ((st = gather(h, h->lev[in], traces + n * nrec, s)) != MOL_OK) return st;
            const int t = ip; ip = ic; ic = in; in = t;
        }
        return MOL_OK;
    }
    mol_batch b = nullptr;
    mol_status st = adjoint_batch(h, &b);
    if (st != MOL_OK) return st;
    if ((st = mol_batch_traces(b, u0, nrec, rec, nsteps, traces, stream)) != MOL_OK) h->err = mol_batch_last_error(b);
    return st;
}

mol_status mol_adjoint(mol_handle h, int nrec, const int64_t *rec, int64_t nsteps, const double *tgrad, double *grad,
                       void *stream)
{
    if (!h) return fail(nullptr, MOL_EINVAL, "handle is NULL");
    if (single_adjoint(h)) {
        if (nsteps < 1) return fail(h, MOL_EINVAL, "nsteps must be >= 1");
        mol_status st;
        if ((st = check_ptr(h, tgrad, "tgrad")) != MOL_OK || (st = check_ptr(h, grad, "grad")) != MOL_OK) return st;
        cudaStream_t s = (cudaStream_t)stream;
        if ((st = set_receivers(h, nrec, rec, s)) != MOL_OK) return st;
        // the reverse recursion of the trace map: mu^N = g^N,
        // mu^n = 2 mu^{n+1} - mu^{n+2} + F^T mu^{n+1} + g^n,
        // dJ/du^0 = mu^1 + F^T mu^1 / 2 - mu^2
        int ia = 0, ib = 1, ic = 2;
        if ((st = zero_level(h, h->lev[ia], s)) != MOL_OK) return st;
        if ((st = zero_level(h, h->lev[ib], s)) != MOL_OK) return st;
        if ((st = inject(h, h->lev[ib], tgrad + (nsteps - 1) * nrec, s)) != MOL_OK) return st;
        for (int64_t n = nsteps - 1; n >= 1; --n) {
            if ((st = run_update_T(h, h->lev[ib], h->lev[ia], h->lev[ic], 2.0, -1.0, 1.0, s)) != MOL_OK) return st;
            if ((st = inject(h, h->lev[ic], tgrad + (n - 1) * nrec, s)) != MOL_OK) return st;
            const int t = ia; ia = ib; ib = ic; ic = t;
        }
        if ((st = run_update_T(h, h->lev[ib], h->lev[ia], h->lev[ic], 1.0, -1.0, 0.5, s)) != MOL_OK) return st;
        return store_level(h, h->lev[ic], grad, s);
    }
    mol_batch b = nullptr;
    mol_status st = adjoint_batch(h, &b);
    if (st != MOL_OK) return st;
    if ((st = mol_batch_adjoint(b, nrec, rec, nsteps, tgrad, grad, stream)) != MOL_OK) h->err = mol_batch_last_error(b);
    return st;
}

mol_status mol_solve_dirichlet(mol_handle h, const double *u0, int64_t nsteps, const double *data, double *u_out,
                               void *stream)
{
    if (!h) return fail(nullptr, MOL_EINVAL, "handle is NULL");
    if (h->ndim != 1 || h->bc != MOL_BC_DIRICHLET)
        return fail(h, MOL_EINVAL, "time-dependent Dirichlet data is for 1D Dirichlet handles");
    if (nsteps < 1) return fail(h, MOL_EINVAL, "nsteps must be >= 1");
    if (!data) return fail(h, MOL_EINVAL, "data is NULL");
    mol_status st;
    if ((st = check_ptr(h, u0, "u0")) != MOL_OK || (st = check_ptr(h, u_out, "u_out")) != MOL_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    const int P = h->P, Q = P + 1;
    // binomials C(j - 1, p - 1) of the boundary values of D^p u (molt.h)
    double binom[MAXP][MAXP] = {};
    for (int j = 0; j < MAXP; ++j) {
        binom[j][0] = 1.0;
        for (int k = 1; k <= j; ++k) binom[j][k] = binom[j - 1][k - 1] + (k <= j - 1 ? binom[j - 1][k] : 0.0);
    }
    const double a2 = h->alpha * h->alpha;              // the data carries (d_tt / c^2)^m
    const double *cu = h->xtpl.cu[0];
    int ip = 0, ic = 1, in = 2;
    if ((st = load_level(h, u0, h->lev[ic], s)) != MOL_OK) return st;
    for (int64_t k = 0; k < nsteps; ++k) {
        // boundary values of D^p u at t_k from the data's time derivatives
        double g[2][MAXP] = {};
        for (int side = 0; side < 2; ++side) {
            const double *dk = data + (k * 2 + side) * Q;
            for (int p = 1; p <= P; ++p) {
                double acc = 0.0, sc = 1.0;
                for (int j = 1; j <= P; ++j) {
                    sc /= a2;
                    if (j >= p) acc += binom[j - 1][p - 1] * dk[j] * sc;
                }
                g[side][p] = (p & 1) ? -acc : acc;
            }
        }
        HornerParams hp = h->xtpl;
        const bool first = k == 0;
        hp.ea = 1.0 + (first ? 0.0 : 1.0);
        hp.eb = first ? 0.0 : -1.0;
        hp.ec = first ? 0.5 : 1.0;
        hp.u_hi = h->lev[ic].hi; hp.u_lo = h->lev[ic].lo;
        hp.up_hi = h->lev[ip].hi; hp.up_lo = h->lev[ip].lo;
        hp.un_hi = h->lev[in].hi; hp.un_lo = h->lev[in].lo;
        hp.bcd = 1;
        // the D application of Horner step t returns sum_{p >= t} cu_p D^{p-t+1} u
        for (int t = 1; t <= P; ++t)
            for (int side = 0; side < 2; ++side) {
                double acc = 0.0;
                for (int p = t; p <= P; ++p) acc += cu[p] * g[side][p - t + 1];
                (side == 0 ? hp.bgL : hp.bgR)[t] = acc;
            }
        hp.bnew[0] = data[((k + 1) * 2 + 0) * Q];
        hp.bnew[1] = data[((k + 1) * 2 + 1) * Q];
        const double *b = h->coef_dev;
        if ((st = run_horner(h, 0, hp, b + h->off_xc, b + h->off_xu, s)) != MOL_OK) return st;
        const int t0 = ip; ip = ic; ic = in; in = t0;
    }
    return store_level(h, h->lev[ic], u_out, s);
}

}  // extern "C"

namespace {

// out = a x + b y (float64; the one-time C[g] of mol_solve_source)
__global__ void k_axpby(double *out, const double *x, const double *y, double a, double b, int64_t N)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = a * x[i] + b * y[i];
}

__global__ void k_to_f32(const double *x, float *y, int64_t N)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x)
        y[i] = (float)x[i];
}

// level += a g + b Cg: float32 pairs (the increment in float32, compensated
// into the pair) or float64
__global__ void k_add_source_pair(float *hi, float *lo, const float *g, const float *cg, float a, float b, int64_t N)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
        const float inc = __fadd_rn(__fmul_rn(a, g[i]), __fmul_rn(b, cg[i]));
        float sh, se, nh, nl;
        two_sum(hi[i], inc, sh, se);
        two_sum(sh, __fadd_rn(lo[i], se), nh, nl);
        hi[i] = nh;
        lo[i] = nl;
    }
}

__global__ void k_add_source_f64(double *x, const double *g, const double *cg, double a, double b, int64_t N)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x)
        x[i] += a * g[i] + b * cg[i];
}

int grid_for(const mol_ctx *h) { return (int)std::min<int64_t>((h->N + 255) / 256, 8 * (int64_t)h->num_sms); }

}  // namespace

extern "C" {

// Grids whose stepping runs on a one-problem batch (ragged 2D Dirichlet) run
// this on the handle's own shared-memory kernels.
mol_status mol_solve_source(mol_handle h, const double *u0, int64_t nsteps, const double *g, const double *f,
                            double *u_out, void *stream)
{
    if (!h) return fail(nullptr, MOL_EINVAL, "handle is NULL");
    if (h->P < 1 || h->P > 2) return fail(h, MOL_EINVAL, "source terms are defined for P = 1 and 2");
    if (nsteps < 1) return fail(h, MOL_EINVAL, "nsteps must be >= 1");
    if (!f) return fail(h, MOL_EINVAL, "f is NULL");
    mol_status st;
    if ((st = check_ptr(h, u0, "u0")) != MOL_OK || (st = check_ptr(h, g, "g")) != MOL_OK ||
        (st = check_ptr(h, u_out, "u_out")) != MOL_OK)
        return st;
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t N = h->N;
    const int nb = grid_for(h);
    if (!h->srcbuf && (st = dev_alloc(h, (void **)&h->srcbuf, sizeof(double) * 3 * (size_t)N)) != MOL_OK) return st;
    if (h->prec == MOL_MIXED && !h->src32 &&
        (st = dev_alloc(h, (void **)&h->src32, sizeof(float) * 2 * (size_t)N)) != MOL_OK)
        return st;
    double *Cg = h->srcbuf, *t1 = Cg + N, *t2 = t1 + N;
    // C[g] = sum_gamma (prod_{a != gamma} (1 - D_a)) D_gamma g (eq. C_def_ADI, L^{-1} = 1 - D)
    CK(cudaMemsetAsync(Cg, 0, sizeof(double) * (size_t)N, s), "clear");
    for (int gam = 0; gam < h->ndim; ++gam) {
        if ((st = mol_apply_D(h, g, t1, gam, 1, stream)) != MOL_OK) return st;
        for (int a = 0; a < h->ndim; ++a) {
            if (a == gam) continue;
            if ((st = mol_apply_D(h, t1, t2, a, 1, stream)) != MOL_OK) return st;
            k_axpby<<<nb, 256, 0, s>>>(t1, t1, t2, 1.0, -1.0, N);
        }
        k_axpby<<<nb, 256, 0, s>>>(Cg, Cg, t1, 1.0, 1.0, N);
    }
    CK(cudaGetLastError(), "source setup");
    float *g32 = h->src32, *cg32 = g32 ? g32 + N : nullptr;
    if (h->prec == MOL_MIXED) {
        k_to_f32<<<nb, 256, 0, s>>>(g, g32, N);
        k_to_f32<<<nb, 256, 0, s>>>(Cg, cg32, N);
        CK(cudaGetLastError(), "source setup");
    }
    const double sc = h->c * h->c * h->dt * h->dt, b2 = h->beta * h->beta;
    int ip = 0, ic = 1, in = 2;
    if ((st = load_level(h, u0, h->lev[ic], s)) != MOL_OK) return st;
    for (int64_t k = 0; k < nsteps; ++k) {
        const double fm = k > 0 ? f[k - 1] : f[1], f0 = f[k], fp = f[k + 1];
        double a = h->P == 1 ? sc * f0 : sc * (fp + 10.0 * f0 + fm) / 12.0;
        double b = h->P == 1 ? 0.0 : -b2 * sc * f0 / 12.0;
        if (k == 0) {
            if ((st = run_update(h, h->lev[ic], h->lev[ic], h->lev[in], 1.0, 0.0, 0.5, s)) != MOL_OK) return st;
            a *= 0.5;
            b *= 0.5;
        } else if ((st = run_update(h, h->lev[ic], h->lev[ip], h->lev[in], 2.0, -1.0, 1.0, s)) != MOL_OK) {
            return st;
        }
        if (h->prec == MOL_MIXED)
            k_add_source_pair<<<nb, 256, 0, s>>>((float *)h->lev[in].hi, (float *)h->lev[in].lo, g32, cg32, (float)a,
                                                 (float)b, N);
        else
            k_add_source_f64<<<nb, 256, 0, s>>>((double *)h->lev[in].hi, g, Cg, a, b, N);
        CK(cudaGetLastError(), "source term");
        h->launches++;
        const int t0 = ip; ip = ic; ic = in; in = t0;
    }
    return store_level(h, h->lev[ic], u_out, s);
}

mol_status mol_sync(mol_handle h, void *stream)
{
    if (!h) return fail(nullptr, MOL_EINVAL, "handle is NULL");
    CK(cudaStreamSynchronize((cudaStream_t)stream), "stream synchronize");
    CK(cudaGetLastError(), "device error");
    const int to = regs_timeout_take((cudaStream_t)stream);
    if (to < 0) return fail(h, MOL_ECUDA, "reading the device wait flag failed");
    if (to > 0)
        return fail(h, MOL_ETIMEOUT, "a bounded device wait (tile copy barrier) gave up; the results since the last "
                                     "mol_sync are not valid");
    return MOL_OK;
}

int64_t mol_launch_count(mol_handle h) { return h ? h->launches + (h->batch ? mol_batch_launch_count(h->batch) : 0) : 0; }

mol_status mol_set_pass_timing(mol_handle h, int enable)
{
    if (!h) return fail(nullptr, MOL_EINVAL, "handle is NULL");
    if (h->batch) return mol_batch_set_pass_timing(h->batch, enable);
    for (auto &u : h->ev_used) { h->ev_pool.push_back(u.second.first); h->ev_pool.push_back(u.second.second); }
    h->ev_used.clear();
    h->timing = enable != 0;
    return MOL_OK;
}

mol_status mol_pass_times(mol_handle h, double total_ms[3], int64_t launches[3])
{
    if (!h || !total_ms || !launches) return fail(h, MOL_EINVAL, "NULL argument");
    if (h->batch) return mol_batch_pass_times(h->batch, total_ms, launches);
    for (int a = 0; a < 3; ++a) { total_ms[a] = 0.0; launches[a] = 0; }
    for (auto &u : h->ev_used) {
        CK(cudaEventSynchronize(u.second.second), "event synchronize");
        float ms = 0.f;
        CK(cudaEventElapsedTime(&ms, u.second.first, u.second.second), "event elapsed time");
        total_ms[u.first] += ms;
        launches[u.first] += 1;
    }
    return MOL_OK;
}

}  // extern "C"

// ===========================================================================
// F[u] without allocation (float64)
// ===========================================================================
// Callers that cannot allocate device memory at the point where they need
// F[u]: a process whose caching allocator (PyTorch's, for one) already holds
// nearly all of the device, so that cudaMalloc fails or forces the cache to
// be emptied; and loops that cannot afford cudaFree, which synchronises the
// whole device.  mol_apply_F_noalloc serves them.  Every buffer it needs
// besides u and F -- the intermediate planes of the pass plan, the tables
// d^j and the Horner coefficients -- lives in the fixed array below, so the
// array's size bounds the grids it accepts.
static __device__ __align__(256) double g_noalloc_scratch[kNoallocScratchBytes / sizeof(double)];

namespace {

constexpr int kNoallocMaxDevices = 64;
constexpr int kNoallocCoefCap = 512;   // doubles reserved for the Horner tables
constexpr int kNoallocCoefMax = 288;   // >= the 258 table entries of 3D, P = 5; keeps the
                                       // parameter block of k_noalloc_tables under 4 KB
std::atomic<double *> g_noalloc_ptr[kNoallocMaxDevices];
int g_noalloc_sms[kNoallocMaxDevices];
int g_noalloc_smem[kNoallocMaxDevices];
std::mutex g_noalloc_setup_mutex;      // first calls on one device from several host threads

// Resolve the array's device address once per device (with that device
// current) and give the pass kernels their shared-memory limits.  The
// per-device values are written under the mutex and published by the
// release store of the pointer; later calls only read them.
mol_status noalloc_setup(int dev, double **out)
{
    if (dev < 0 || dev >= kNoallocMaxDevices) return fail(nullptr, MOL_EINVAL, "device ordinal out of range");
    double *p = g_noalloc_ptr[dev].load(std::memory_order_acquire);
    if (!p) {
        std::lock_guard<std::mutex> lock(g_noalloc_setup_mutex);
        p = g_noalloc_ptr[dev].load(std::memory_order_acquire);
    }
    if (!p) {
        void *q = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&q, g_noalloc_scratch);
        if (e != cudaSuccess) return cuda_fail(nullptr, e, "cudaGetSymbolAddress of the static scratch");
        if ((e = configure_kernels()) != cudaSuccess) return cuda_fail(nullptr, e, "kernel attributes");
        if ((e = configure_regs_kernels()) != cudaSuccess) return cuda_fail(nullptr, e, "kernel attributes");
        int v = 0;
        g_noalloc_sms[dev] = (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess && v > 0)
                                 ? v : 152;
        g_noalloc_smem[dev] = (cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) == cudaSuccess &&
                               v > 0) ? v : 227 * 1024;
        p = (double *)q;
        g_noalloc_ptr[dev].store(p, std::memory_order_release);
    }
    *out = p;
    return MOL_OK;
}

// Coefficient expansion of F with fixed-capacity polynomials: the same
// products, in the same order, as expand_coefficients (index i + 6 (j + 6 k)).
constexpr int kFS = kMaxP + 1;
struct FPoly {
    double c[kFS * kFS * kFS];
};

int fidx(int i, int j, int k) { return i + kFS * (j + kFS * k); }

void fset(FPoly &r, const FPoly &a, const FPoly &b, double sb)   // r = a + sb b
{
    for (int i = 0; i < kFS * kFS * kFS; ++i) r.c[i] = a.c[i] + sb * b.c[i];
}

bool fmul(const FPoly &a, const FPoly &b, int P, FPoly &r)
{
    for (double &x : r.c) x = 0.0;
    for (int k1 = 0; k1 <= P; ++k1) for (int j1 = 0; j1 <= P; ++j1) for (int i1 = 0; i1 <= P; ++i1) {
        const double x = a.c[fidx(i1, j1, k1)];
        if (x == 0.0) continue;
        for (int k2 = 0; k2 <= P; ++k2) for (int j2 = 0; j2 <= P; ++j2) for (int i2 = 0; i2 <= P; ++i2) {
            const double y = b.c[fidx(i2, j2, k2)];
            if (y == 0.0) continue;
            if (i1 + i2 > P || j1 + j2 > P || k1 + k2 > P) return false;
            r.c[fidx(i1 + i2, j1 + j2, k1 + k2)] += x * y;
        }
    }
    return true;
}

bool expand_fixed(int ndim, int P, double beta, FPoly &F)
{
    FPoly one{}, zero{}, Dg[3]{}, Lg[3]{}, prodL{}, Dop{}, C{}, t{}, tmp{}, Cp[kFS]{}, Dp[kFS]{};
    one.c[0] = 1.0;
    for (int a = 0; a < ndim; ++a) {
        int e[3] = {0, 0, 0};
        e[a] = 1;
        Dg[a].c[fidx(e[0], e[1], e[2])] = 1.0;
        fset(Lg[a], one, Dg[a], -1.0);
    }
    prodL = one;
    for (int a = 0; a < ndim; ++a) { if (!fmul(prodL, Lg[a], P, tmp)) return false; prodL = tmp; }
    fset(Dop, one, prodL, -1.0);
    for (int g = 0; g < ndim; ++g) {
        t = Dg[g];
        for (int a = 0; a < ndim; ++a) if (a != g) { if (!fmul(t, Lg[a], P, tmp)) return false; t = tmp; }
        fset(C, C, t, 1.0);
    }
    Cp[0] = Dp[0] = one;
    for (int k = 1; k <= P; ++k) {
        if (!fmul(Cp[k - 1], C, P, Cp[k])) return false;
        if (!fmul(Dp[k - 1], Dop, P, Dp[k])) return false;
    }
    F = zero;
    for (int p = 1; p <= P; ++p)
        for (int m = 1; m <= p; ++m) {
            if (!fmul(Cp[m], Dp[p - m], P, tmp)) return false;
            fset(F, F, tmp, term_weight(p, m, beta));
        }
    return true;
}

// Constants written into the scratch by one small kernel at the start of
// every call (they travel as the kernel's parameters, so no host copy).
struct NoallocTables {
    double *coef_dst;
    int ncoef;
    double coef[kNoallocCoefMax];
    double *dpow[3];
    int n[3];
    double nu[3];
};

__global__ void k_noalloc_tables(const NoallocTables t)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < t.ncoef) t.coef_dst[i] = t.coef[i];
    for (int a = 0; a < 3; ++a)
        if (t.dpow[a] && i <= t.n[a]) t.dpow[a][i] = exp(-t.nu[a] * (double)i);
}

size_t round_up32(size_t x) { return (x + 31) & ~(size_t)31; }   // doubles -> 256-byte alignment

}  // namespace

extern "C" mol_status mol_apply_F_noalloc(const mol_grid *grid, double c, double dt, double beta, int P, mol_bc bc,
                                          int quad_order, const double *u, double *F, void *stream)
{
    if (!grid) return fail(nullptr, MOL_EINVAL, "grid is NULL");
    if (grid->ndim < 1 || grid->ndim > 3) return fail(nullptr, MOL_EINVAL, "ndim must be 1, 2 or 3");
    if (P < 1 || P > kMaxP) return fail(nullptr, MOL_EINVAL, "P must be in 1..5");
    if (!(c > 0) || !(dt > 0) || !std::isfinite(c) || !std::isfinite(dt))
        return fail(nullptr, MOL_EINVAL, "c and dt must be positive");
    if (bc != MOL_BC_PERIODIC && bc != MOL_BC_DIRICHLET) return fail(nullptr, MOL_EINVAL, "unknown boundary condition");
    if (quad_order != 1 && quad_order != 2) return fail(nullptr, MOL_EINVAL, "quad_order must be 1 or 2");
    int64_t N = 1;
    for (int a = 0; a < grid->ndim; ++a) {
        if (grid->n[a] < 3 || grid->n[a] > kMaxLine)
            return fail(nullptr, MOL_EINVAL, "every axis needs 3 <= n <= " + std::to_string(kMaxLine));
        if (!(grid->hi[a] > grid->lo[a])) return fail(nullptr, MOL_EINVAL, "hi must exceed lo on every axis");
        N *= grid->n[a];
    }
    const double bmax = beta_max_of(P);
    if (beta <= 0) beta = bmax;
    if (beta > bmax * (1.0 + 1e-12) && !unstable_allowed())
        return fail(nullptr, MOL_EUNSTABLE, "beta above beta_max(P): the scheme is not A-stable");

    // scratch layout (doubles, every part 256-byte aligned): Horner tables,
    // d^j per axis, intermediate planes (2D: D_y^k u; 3D: D_z^k u and the
    // P + 1 outputs of the y pass)
    const int ndim = grid->ndim;
    const int nplanes = ndim == 2 ? P : (ndim == 3 ? 2 * P + 1 : 0);
    size_t off_dpow[3] = {0, 0, 0};
    size_t need = kNoallocCoefCap;
    for (int a = 0; a < ndim; ++a) { off_dpow[a] = need; need += round_up32((size_t)grid->n[a] + 1); }
    const size_t off_planes = need;
    need += (size_t)nplanes * round_up32((size_t)N);
    if (need * sizeof(double) > kNoallocScratchBytes)
        return fail(nullptr, MOL_EINVAL, "the grid needs " + std::to_string(need * sizeof(double)) +
                                             " bytes of static scratch; the maximum is " +
                                             std::to_string(kNoallocScratchBytes));
    mol_status st;
    if ((st = check_ptr(nullptr, u, "u")) != MOL_OK || (st = check_ptr(nullptr, F, "F")) != MOL_OK) return st;
    {
        const uintptr_t ub = (uintptr_t)u, fb = (uintptr_t)F, nb = (uintptr_t)N * sizeof(double);
        if (ub < fb + nb && fb < ub + nb) return fail(nullptr, MOL_EINVAL, "u and F must not overlap");
    }

    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(nullptr, e, "cudaGetDevice");
    // the kernels run on the current device: both fields must live there
    for (const void *p : {(const void *)u, (const void *)F}) {
        cudaPointerAttributes at{};
        if ((e = cudaPointerGetAttributes(&at, p)) != cudaSuccess) {
            cudaGetLastError();
            return fail(nullptr, MOL_EINVAL, "u / F: not a CUDA pointer");
        }
        if (at.type == cudaMemoryTypeDevice && at.device != dev)
            return fail(nullptr, MOL_EINVAL, "u and F must be on the current device (" + std::to_string(dev) +
                                                 "); one is on device " + std::to_string(at.device));
    }
    double *scratch = nullptr;
    if ((st = noalloc_setup(dev, &scratch)) != MOL_OK) return st;

    // a context on the stack: the pass launchers read only its scalars
    mol_ctx h;
    h.ndim = ndim;
    h.N = N;
    for (int a = 0; a < 3; ++a) {
        h.n[a] = a < ndim ? grid->n[a] : 1;
        h.lo[a] = grid->lo[a];
        h.hi[a] = grid->hi[a];
    }
    h.c = c; h.dt = dt; h.beta = beta; h.P = P; h.bc = bc; h.prec = MOL_FP64;
    mol_default_options(&h.opt);
    h.opt.quad_order = quad_order;
    h.opt.use_graphs = 0;
    h.alpha = beta / (c * dt);                        // eq. L_def
    h.tbytes = 8;
    h.device = dev;
    h.num_sms = g_noalloc_sms[dev];
    h.smem_optin = (size_t)g_noalloc_smem[dev];

    NoallocTables tb{};
    int nmax = 0;
    for (int a = 0; a < ndim; ++a) {
        const int64_t n = h.n[a];
        h.h[a] = (h.hi[a] - h.lo[a]) / (double)(bc == MOL_BC_DIRICHLET ? n - 1 : n);
        h.nu[a] = h.alpha * h.h[a];
        axis_constants(h.nu[a], n, bc, quad_order, h.ax[a]);
        h.ax[a].dpow64 = scratch + off_dpow[a];
        h.ax[a].dpow32 = nullptr;                      // float64 kernels read only dpow64
        for (int r = 0; r < 4; ++r)
            for (int k = 0; k < 5; ++k)
                h.dmr_ax[a][r][k] = std::exp(-h.nu[a] * (double)(8 << r) * (double)(1 << k));
        tb.dpow[a] = scratch + off_dpow[a];
        tb.n[a] = (int)n;
        tb.nu[a] = h.nu[a];
        nmax = std::max(nmax, (int)n + 1);
    }

    FPoly f;
    if (!expand_fixed(ndim, P, beta, f)) return fail(nullptr, MOL_EINVAL, "coefficient expansion failed");
    fill_tables(ndim, P, [&f](int i, int j, int k) { return f.c[fidx(i, j, k)]; }, h.xtpl, h.ytpl);
    default_rows_split(&h);                           // as mol_create (float64: one warp per row either way)
    // flattened like flatten(): per output o and Horner term t, the ng field
    // weights, then the weights of u
    double flat[2 * kNoallocCoefMax];
    size_t off[4];
    int nc = 0;
    const HornerParams *tp[2] = {&h.xtpl, &h.ytpl};
    for (int q = 0; q < 2; ++q) {
        const HornerParams &hp = *tp[q];
        const bool used = q == 0 || ndim == 3;
        off[2 * q] = nc;
        if (used)
            for (int o = 0; o < std::max(hp.nout, 1); ++o)
                for (int t = 0; t <= hp.P; ++t)
                    for (int k = 0; k < hp.ng; ++k) flat[nc++] = hp.coef[o][t][k];
        if (nc == (int)off[2 * q]) flat[nc++] = 0.0;
        off[2 * q + 1] = nc;
        if (used)
            for (int o = 0; o < std::max(hp.nout, 1); ++o)
                for (int t = 0; t <= hp.P; ++t) flat[nc++] = hp.cu[o][t];
        if (nc == (int)off[2 * q + 1]) flat[nc++] = 0.0;
    }
    if (nc > kNoallocCoefMax) return fail(nullptr, MOL_EINVAL, "coefficient tables exceed their reserved space");
    for (int i = 0; i < nc; ++i) tb.coef[i] = flat[i];
    tb.coef_dst = scratch;
    tb.ncoef = nc;

    cudaStream_t s = (cudaStream_t)stream;
    const int nthr = 256, nblk = (std::max(nmax, nc) + nthr - 1) / nthr;
    k_noalloc_tables<<<nblk, nthr, 0, s>>>(tb);
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(nullptr, e, "table kernel launch");

    void *inter[2 * MAXG] = {nullptr};
    for (int k = 0; k < nplanes; ++k) inter[k] = scratch + off_planes + (size_t)k * round_up32((size_t)N);
    Level U, O;
    U.hi = (void *)u;
    O.hi = F;
    st = run_update_with(&h, inter, scratch + off[0], scratch + off[1], scratch + off[2], scratch + off[3], U, U, O,
                         0.0, 0.0, 1.0, s);
    if (st != MOL_OK) g_err = h.err;
    return st;
}

// ===========================================================================
// Robustness: field norm and checked stepping, checkpoint files, the device
// wait self-test (no counterpart in the paper)
// ===========================================================================
namespace {

// sum of squares of x[0..N) into *acc (block partial sums, one atomic add
// per block); NaN and Inf propagate into the sum
__global__ void k_sumsq(const double *x, int64_t N, double *acc)
{
    double s = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x)
        s += x[i] * x[i];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    __shared__ double part[32];
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x < 32) {
        s = threadIdx.x < (blockDim.x >> 5) ? part[threadIdx.x] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
        if (threadIdx.x == 0) atomicAdd(acc, s);
    }
}

mol_status field_norm(mol_ctx *h, const double *u, double *norm, cudaStream_t s)
{
    if (!h->norm_acc) {
        mol_status st = dev_alloc(h, (void **)&h->norm_acc, sizeof(double));
        if (st != MOL_OK) return st;
    }
    CK(cudaMemsetAsync(h->norm_acc, 0, sizeof(double), s), "memset");
    const int64_t blocks = std::min<int64_t>((h->N + 255) / 256, 4 * (int64_t)h->num_sms);
    k_sumsq<<<(unsigned)blocks, 256, 0, s>>>(u, h->N, h->norm_acc);
    CK(cudaGetLastError(), "norm launch");
    double ss = 0.0;
    CK(cudaMemcpyAsync(&ss, h->norm_acc, sizeof(double), cudaMemcpyDeviceToHost, s), "norm copy");
    CK(cudaStreamSynchronize(s), "stream synchronize");
    double vol = 1.0;
    for (int a = 0; a < h->ndim; ++a) vol *= h->h[a];
    *norm = std::sqrt(vol * ss);
    return MOL_OK;
}

// Checkpoint file: a fixed header that names the problem, the step index,
// then u^{n-1} and u^n (float64, x fastest) and an FNV-1a hash of them.
constexpr char kCkpMagic[8] = {'M', 'O', 'L', 'T', 'C', 'K', 'P', '1'};
struct CkpHeader {
    char magic[8];
    int32_t ndim, P, bc, prec, quad;
    int32_t pad;
    int64_t n[3];
    double lo[3], hi[3], c, dt, beta;
    int64_t step;
};

uint64_t fnv1a(const void *p, size_t bytes, uint64_t h = 1469598103934665603ull)
{
    const unsigned char *b = static_cast<const unsigned char *>(p);
    for (size_t i = 0; i < bytes; ++i) { h ^= b[i]; h *= 1099511628211ull; }
    return h;
}

CkpHeader header_of(const mol_ctx *h, int64_t step)
{
    CkpHeader hd{};
    std::memcpy(hd.magic, kCkpMagic, 8);
    hd.ndim = h->ndim;
    hd.P = h->P;
    hd.bc = (int32_t)h->bc;
    hd.prec = (int32_t)h->prec;
    hd.quad = h->opt.quad_order;
    for (int a = 0; a < 3; ++a) { hd.n[a] = h->n[a]; hd.lo[a] = h->lo[a]; hd.hi[a] = h->hi[a]; }
    hd.c = h->c;
    hd.dt = h->dt;
    hd.beta = h->beta;
    hd.step = step;
    return hd;
}

}  // namespace

extern "C" {

mol_status mol_field_norm(mol_handle h, const double *u, double *norm, void *stream)
{
    if (!h || !norm) return fail(h, MOL_EINVAL, "NULL argument");
    mol_status st = check_ptr(h, u, "u");
    if (st != MOL_OK) return st;
    NvtxRange r("mol_field_norm");
    return field_norm(h, u, norm, (cudaStream_t)stream);
}

mol_status mol_pair_split(const double *x, float *hi, float *lo, int64_t n, void *stream)
{
    if (!x || !hi || !lo || n < 0) return fail(nullptr, MOL_EINVAL, "NULL pointer or n < 0");
    if (n == 0) return MOL_OK;
    const cudaError_t e = launch_to_pair(x, hi, lo, n, (cudaStream_t)stream);
    return e == cudaSuccess ? MOL_OK : cuda_fail(nullptr, e, "pair split");
}

mol_status mol_pair_join(const float *hi, const float *lo, double *x, int64_t n, void *stream)
{
    if (!x || !hi || !lo || n < 0) return fail(nullptr, MOL_EINVAL, "NULL pointer or n < 0");
    if (n == 0) return MOL_OK;
    const cudaError_t e = launch_from_pair(hi, lo, x, n, (cudaStream_t)stream);
    return e == cudaSuccess ? MOL_OK : cuda_fail(nullptr, e, "pair join");
}

mol_status mol_step_checked(mol_handle h, double *u_prev, double *u_cur, int64_t nsteps, double growth_limit,
                            void *stream)
{
    if (!h) return fail(nullptr, MOL_EINVAL, "handle is NULL");
    if (!(growth_limit > 0) || !std::isfinite(growth_limit)) return fail(h, MOL_EINVAL, "growth_limit must be > 0");
    mol_status st;
    if ((st = check_ptr(h, u_cur, "u_cur")) != MOL_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    double n0 = 0.0, n1 = 0.0;
    if ((st = field_norm(h, u_cur, &n0, s)) != MOL_OK) return st;
    if ((st = mol_step(h, u_prev, u_cur, nsteps, stream)) != MOL_OK) return st;
    if ((st = field_norm(h, u_cur, &n1, s)) != MOL_OK) return st;
    if (!std::isfinite(n1))
        return fail(h, MOL_EUNSTABLE, "the field is no longer finite after " + std::to_string(nsteps) + " steps");
    if (n1 > growth_limit * std::max(n0, 1e-300))
        return fail(h, MOL_EUNSTABLE, "the field norm grew from " + std::to_string(n0) + " to " + std::to_string(n1) +
                                          " in " + std::to_string(nsteps) + " steps (limit x" +
                                          std::to_string(growth_limit) + ")");
    return MOL_OK;
}

mol_status mol_checkpoint_write(mol_handle h, const char *path, const double *u_prev, const double *u_cur, int64_t step,
                                void *stream)
{
    if (!h || !path) return fail(h, MOL_EINVAL, "NULL argument");
    mol_status st;
    if ((st = check_ptr(h, u_prev, "u_prev")) != MOL_OK || (st = check_ptr(h, u_cur, "u_cur")) != MOL_OK) return st;
    NvtxRange r("mol_checkpoint_write");
    cudaStream_t s = (cudaStream_t)stream;
    std::vector<double> buf(2 * (size_t)h->N);
    CK(cudaMemcpyAsync(buf.data(), u_prev, sizeof(double) * h->N, cudaMemcpyDeviceToHost, s), "copy u_prev");
    CK(cudaMemcpyAsync(buf.data() + h->N, u_cur, sizeof(double) * h->N, cudaMemcpyDeviceToHost, s), "copy u_cur");
    CK(cudaStreamSynchronize(s), "stream synchronize");
    const CkpHeader hd = header_of(h, step);
    const uint64_t sum = fnv1a(buf.data(), sizeof(double) * buf.size());
    FILE *f = std::fopen(path, "wb");
    if (!f) return fail(h, MOL_EINVAL, std::string("cannot open ") + path + " for writing");
    bool ok = std::fwrite(&hd, sizeof hd, 1, f) == 1 && std::fwrite(buf.data(), sizeof(double), buf.size(), f) == buf.size() &&
              std::fwrite(&sum, sizeof sum, 1, f) == 1;
    ok = (std::fclose(f) == 0) && ok;
    return ok ? MOL_OK : fail(h, MOL_EINVAL, std::string("writing ") + path + " failed");
}

mol_status mol_checkpoint_read(mol_handle h, const char *path, double *u_prev, double *u_cur, int64_t *step,
                               void *stream)
{
    if (!h || !path || !step) return fail(h, MOL_EINVAL, "NULL argument");
    mol_status st;
    if ((st = check_ptr(h, u_prev, "u_prev")) != MOL_OK || (st = check_ptr(h, u_cur, "u_cur")) != MOL_OK) return st;
    NvtxRange r("mol_checkpoint_read");
    FILE *f = std::fopen(path, "rb");
    if (!f) return fail(h, MOL_EINVAL, std::string("cannot open ") + path);
    CkpHeader hd{};
    std::vector<double> buf(2 * (size_t)h->N);
    uint64_t sum = 0;
    const bool ok = std::fread(&hd, sizeof hd, 1, f) == 1 && std::fread(buf.data(), sizeof(double), buf.size(), f) == buf.size() &&
                    std::fread(&sum, sizeof sum, 1, f) == 1;
    std::fclose(f);
    if (!ok) return fail(h, MOL_EINVAL, std::string(path) + ": truncated or not a checkpoint of this grid");
    CkpHeader want = header_of(h, hd.step);
    if (std::memcmp(&hd, &want, sizeof hd) != 0)
        return fail(h, MOL_EINVAL, std::string(path) + ": written for another problem (grid, c, dt, beta, P, boundary, "
                                                       "precision or quadrature differ)");
    if (fnv1a(buf.data(), sizeof(double) * buf.size()) != sum)
        return fail(h, MOL_EINVAL, std::string(path) + ": the field data do not match their checksum");
    cudaStream_t s = (cudaStream_t)stream;
    CK(cudaMemcpyAsync(u_prev, buf.data(), sizeof(double) * h->N, cudaMemcpyHostToDevice, s), "copy u_prev");
    CK(cudaMemcpyAsync(u_cur, buf.data() + h->N, sizeof(double) * h->N, cudaMemcpyHostToDevice, s), "copy u_cur");
    CK(cudaStreamSynchronize(s), "stream synchronize");
    *step = hd.step;
    return MOL_OK;
}

mol_status mol_wait_selftest(int64_t limit_cycles, void *stream)
{
    if (limit_cycles < 1 || limit_cycles > (int64_t)1 << 40)
        return fail(nullptr, MOL_EINVAL, "limit_cycles must be in 1..2^40");
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = launch_wait_selftest((long long)limit_cycles, s);
    if (e != cudaSuccess) return cuda_fail(nullptr, e, "self-test launch");
    if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return cuda_fail(nullptr, e, "stream synchronize");
    const int to = regs_timeout_take(s);
    if (to < 0) return fail(nullptr, MOL_ECUDA, "reading the device wait flag failed");
    if (to > 0) return fail(nullptr, MOL_ETIMEOUT, "the bounded device wait gave up, as it must");
    return MOL_OK;
}

}  // extern "C"

// ===========================================================================
// History gradient (checkpoint-and-recompute) on a single-problem handle
// ===========================================================================
namespace {

mol_status hist_fail(void *c, mol_status st, const char *msg) { return fail((mol_ctx *)c, st, msg); }

mol_status hist_start(void *c, const double *u0, double *u1, cudaStream_t s)
{
    return mol_start((mol_ctx *)c, u0, u1, (void *)s);
}

mol_status hist_step(void *c, double *prev, double *cur, int64_t n, cudaStream_t s)
{
    return mol_step((mol_ctx *)c, prev, cur, n, (void *)s);
}

// m steps on the handle's levels, each new level written out once
mol_status hist_step_emit(void *c, const double *prev, const double *cur, int64_t m, double *states, cudaStream_t s)
{
    mol_ctx *h = (mol_ctx *)c;
    mol_status st;
    if ((st = load_levels(h, prev, h->lev[0], cur, h->lev[1], s)) != MOL_OK) return st;
    for (int64_t j = 0; j < m; ++j) {
        const int k = (int)(j % 3);
        if ((st = run_update(h, h->lev[(k + 1) % 3], h->lev[k], h->lev[(k + 2) % 3], 2.0, -1.0, 1.0, s)) != MOL_OK)
            return st;
        if ((st = store_level(h, h->lev[(k + 2) % 3], states + (size_t)j * h->N, s)) != MOL_OK) return st;
    }
    return MOL_OK;
}

mol_status hist_update_T(void *c, const double *u, const double *up, double *un, double ea, double eb, double ec,
                         const double *add, cudaStream_t s)
{
    mol_ctx *h = (mol_ctx *)c;
    mol_status st;
    if ((st = load_levels(h, u, h->lev[0], up, h->lev[1], s)) != MOL_OK) return st;
    if ((st = run_update_T(h, h->lev[0], h->lev[1], h->lev[2], ea, eb, ec, s)) != MOL_OK) return st;
    if ((st = store_level(h, h->lev[2], un, s)) != MOL_OK) return st;
    if (add) {
        const int nb = grid_for(h);
        k_axpby<<<nb, 256, 0, s>>>(un, un, add, 1.0, 1.0, h->N);
        CK(cudaGetLastError(), "gradient injection");
        h->launches++;
    }
    return MOL_OK;
}

}  // namespace

extern "C" mol_status mol_adjoint_history(mol_handle h, const double *u0, int64_t nsteps, int64_t checkpoint_every,
                                          mol_grad_fn grad_fn, void *user, double *grad, void *stream)
{
    if (!h) return fail(nullptr, MOL_EINVAL, "handle is NULL");
    NvtxRange nvtx_("mol_adjoint_history");
    if (!single_adjoint(h)) {
        mol_batch b = nullptr;
        mol_status st = adjoint_batch(h, &b);
        if (st != MOL_OK) return st;
        st = mol_batch_adjoint_history(b, u0, nsteps, checkpoint_every, grad_fn, user, grad, stream);
        if (st != MOL_OK) h->err = mol_batch_last_error(b);
        return st;
    }
    mol_status st;
    if ((st = check_ptr(h, u0, "u0")) != MOL_OK || (st = check_ptr(h, grad, "grad")) != MOL_OK) return st;
    HistoryOps o{h, h->N, hist_start, hist_step, hist_step_emit, hist_update_T, hist_fail};
    return history_gradient_run(o, u0, nsteps, checkpoint_every, grad_fn, user, grad, (cudaStream_t)stream);
}
