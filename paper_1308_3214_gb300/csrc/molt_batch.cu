// molt_batch.cu -- the batched C ABI (mol_batch_* in include/molt.h): many
// independent 2D Dirichlet problems of uneven size stepped together, a few
// concurrent launches per pass over flat work lists, the time loop captured
// in a CUDA graph.
#include <algorithm>
#include <cmath>
#include <string>
#include <utility>
#include <vector>

#include "molt.h"
#include "molt_internal.h"
#include "molt_batch.cuh"

using namespace molt;

namespace {

struct BLevel {
    void *hi = nullptr;
    void *lo = nullptr;
};

}  // namespace

struct mol_batch_ctx {
    int nprob = 0, prec = 0, tbytes = 8, Pmax = 1, quad = 2, use_graphs = 1;
    int64_t nrows = 0, total_int = 0;
    int64_t rows_small = 0;             // rows are ordered by length class: <= 256 points first,
    int64_t rows_mid = 0;               //   then 257..512 (up to rows_mid), then 513..1024
    int nitems_y = 0;
    std::vector<int64_t> uoff;          // packed user layout: nprob + 1 prefix sums
    std::vector<BatchProb> hp;          // host copy of the problem table
    BatchProb *probs = nullptr;
    int *row_prob = nullptr;
    int2 *items = nullptr;
    long long *uoff_dev = nullptr;
    double *dp64 = nullptr;
    float *dp32 = nullptr;
    BLevel lev[3];
    double *io[2] = {nullptr, nullptr};  // packed float64 fields of mol_batch_solve_host
    long long *irec = nullptr;           // receivers in the internal layout, then their distinct
    int nrec = 0, irec_cap = 0;          //   nodes, the node groups' starts and the receivers by node
    int nnode = 0;
    void *inter[BMAXP] = {nullptr, nullptr, nullptr, nullptr, nullptr};
    int xW[2] = {8, 8}, xgrid[2] = {1, 1}, nbuf = 1, cgrid = 1;
    int ycls_begin[4] = {0, 0, 0, 0};   // y work list: the items of clusters of 1, 2, 4, 8 CTAs
    int ycls_count[4] = {0, 0, 0, 0};
    size_t xsmem[2] = {0, 0}, ysmem = 0;
    int num_sms = 152;
    std::vector<void *> allocs;
    cudaStream_t cap_stream = nullptr;
    cudaStream_t ys[3] = {nullptr, nullptr, nullptr};   // y pass: side streams of the cluster-size classes
    cudaEvent_t yev[4] = {nullptr, nullptr, nullptr, nullptr};   // their fork and joins
    cudaEvent_t xev[3] = {nullptr, nullptr, nullptr};            // x pass: fork and joins of its classes
    cudaGraphExec_t gexec = nullptr;
    int64_t launches = 0;
    bool timing = false;
    std::vector<cudaEvent_t> ev_pool;
    std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>> ev_used;
    std::string err;
    int64_t one_warp_end() const { return xmid ? rows_small : rows_mid; }
    int y_launches() const
    {
        int n = 0;
        for (int k = 0; k < 4; ++k) n += ycls_count[k] > 0 ? 1 : 0;
        return n;
    }
    int x_launches() const
    {
        return (one_warp_end() > 0 ? 1 : 0) + ((xmid && rows_mid > rows_small) ? 1 : 0) + (nrows > rows_mid ? 1 : 0);
    }
    int smem_sm = 228 * 1024, smem_blk = 227 * 1024;
    int ymode = 0;                      // y rule: bit 0: 0 the fewest CTAs per column group, 1 twice as
                                        // many (shorter segments); bit 1: full carries even where the
                                        // neighbour exchange is exact
    int xsplit = 1;                     // rows of > 512 points: 1 one CTA of two warps per row, 0 one warp
    size_t xs_smem = 0;                 // shared memory of the split-row kernel
    int xmid = 1;                       // rows of 257..512 points: 1 one CTA of two warps per row (8-point
    size_t xs8_smem = 0;                //   segments), 0 the one-warp kernel; its shared memory
    double tune_ms[2] = {0.0, 0.0};     // tuned x / y pass times
    int chains = 1;                     // graphs: the y / x launch pairs as independent chains where
                                        // they pair up (chain_plan)
};

namespace {

mol_status bfail(mol_batch_ctx *b, mol_status st, const std::string &msg)
{
    if (b) b->err = msg;
    else set_global_error(msg);
    return st;
}

mol_status bcuda(mol_batch_ctx *b, cudaError_t e, const char *what)
{
    return bfail(b, MOL_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

#define BCK(expr, what)                                      \
    do {                                                     \
        cudaError_t e_ = (expr);                             \
        if (e_ != cudaSuccess) return bcuda(b, e_, what);    \
    } while (0)

mol_status balloc(mol_batch_ctx *b, void **p, size_t bytes)
{
    if (alloc_injected_failure())
        return bfail(b, MOL_ENOMEM, "device allocation of " + std::to_string(bytes) + " bytes failed (injected)");
    cudaError_t e = cudaMalloc(p, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return bfail(b, MOL_ENOMEM, "device allocation of " + std::to_string(bytes) + " bytes failed: " +
                                        cudaGetErrorString(e));
    }
    b->allocs.push_back(*p);
    return MOL_OK;
}

void bfree_all(mol_batch_ctx *b)
{
    for (auto &u : b->ev_used) { b->ev_pool.push_back(u.second.first); b->ev_pool.push_back(u.second.second); }
    b->ev_used.clear();
    for (cudaEvent_t e : b->ev_pool) cudaEventDestroy(e);
    b->ev_pool.clear();
    if (b->gexec) cudaGraphExecDestroy(b->gexec);
    b->gexec = nullptr;
    if (b->cap_stream) cudaStreamDestroy(b->cap_stream);
    b->cap_stream = nullptr;
    for (int k = 0; k < 3; ++k) {
        if (b->ys[k]) cudaStreamDestroy(b->ys[k]);
        b->ys[k] = nullptr;
    }
    for (int k = 0; k < 4; ++k) {
        if (b->yev[k]) cudaEventDestroy(b->yev[k]);
        b->yev[k] = nullptr;
    }
    for (int k = 0; k < 3; ++k) {
        if (b->xev[k]) cudaEventDestroy(b->xev[k]);
        b->xev[k] = nullptr;
    }
    for (void *p : b->allocs) cudaFree(p);
    b->allocs.clear();
}

// segment lengths: x pass 32 lanes x rpt >= nx (pick_y below for the y pass)
int pick_rpt_x(int n)
{
    int r = 4;
    while (32 * r < n) r *= 2;
    return r;
}
// y pass of a column of n points: K CTAs of kBatchYSeg warps (K a power of
// two, the fewest whose segments of at most 64 (float32) / 32 (float64)
// points cover the column; mode bit 0: twice as many, up to 8) and the
// segment length R (a power of two >= 4 with kBatchYSeg K R >= n)
void pick_y(int n, int mode, int tbytes, int &K, int &R)
{
    const int rmax = tbytes == 4 ? 64 : 32;
    K = 1;
    while (kBatchYSeg * K * rmax < n) K *= 2;
    if ((mode & 1) && K < 8) K *= 2;
    R = 4;
    while (kBatchYSeg * K * R < n) R *= 2;
}

// The neighbour-exchange y pass of one problem (batch_cols_nb): on where the
// decay over a segment is below float32 rounding, d^(RPT-1) <= 2^-30, and the
// column has more than two segments; the constants of its segment length and
// of its ragged last segment.
void set_y_nb(BatchProb &pb, bool allow)
{
    const int R = pb.rpt_y, n = pb.ay.n;
    const double d = pb.ay.d;
    pb.ynb = (allow && R >= 4 && (n + R - 1) / R > 2 && std::pow(d, (double)(R - 1)) <= std::ldexp(1.0, -30)) ? 1 : 0;
    pb.nby = strided_nb_consts(d, R);
    const int kl = (n - 1) % R;
    double gl = 0.0, g1l = 0.0;
    for (int k = 0; k <= kl; ++k) {
        gl += std::pow(d, 2.0 * k + 1.0);
        if (k >= 1) g1l += std::pow(d, 2.0 * k);
    }
    pb.nbGL = (float)gl;
    pb.nbG1L = (float)g1l;
    pb.nbdk = (float)std::pow(d, (double)kl);
    pb.nbdk1 = kl >= 1 ? (float)std::pow(d, (double)(kl - 1)) : 0.f;
    pb.nbdkp = (float)std::pow(d, (double)(kl + 1));
}

// length class of a row: 0 (<= 256 points), 1 (257..512), 2 (513..1024)
int row_class(int nx) { return nx <= 256 ? 0 : (nx <= 512 ? 1 : 2); }

// The y-pass work list: one item (problem, first column) per group of 32
// columns, grouped by the cluster size of its problem (one launch per size),
// and within a group by decreasing cost (the segment length times the P + 1
// phases of a column group: loads and P sweeps), so that the long items
// start first.  Items are independent, so the order changes no result.
std::vector<int2> y_work_list(mol_batch_ctx *b)
{
    std::vector<int2> out;
    out.reserve(b->nitems_y);
    for (int k = 0; k < 4; ++k) {
        std::vector<std::pair<int, int2>> cls;
        for (int i = 0; i < b->nprob; ++i) {
            const BatchProb &pb = b->hp[i];
            if (pb.ky != (1 << k)) continue;
            for (int c0 = 0; c0 < pb.ax.n; c0 += 32) cls.push_back({pb.rpt_y * (pb.P + 1), make_int2(i, c0)});
        }
        std::stable_sort(cls.begin(), cls.end(), [](const std::pair<int, int2> &a, const std::pair<int, int2> &c) {
            return a.first > c.first;
        });
        b->ycls_begin[k] = (int)out.size();
        b->ycls_count[k] = (int)cls.size();
        for (auto &c : cls) out.push_back(c.second);
    }
    return out;
}

// the problem table to the device, with its float32 copies refreshed
cudaError_t upload_table(mol_batch_ctx *b)
{
    for (BatchProb &pb : b->hp) batch_mirror(pb);
    return cudaMemcpy(b->probs, b->hp.data(), sizeof(BatchProb) * b->nprob, cudaMemcpyHostToDevice);
}

// per-problem x-pass segment constants of the long rows for the current
// choice: 16-point segments over two warps (split) or 32-point segments
// over one warp
void set_x_segments(mol_batch_ctx *b)
{
    for (BatchProb &pb : b->hp) {
        const int cls = row_class(pb.ax.n);
        if (cls == 0) continue;
        pb.rpt_x = cls == 2 ? (b->xsplit ? 16 : 32) : (b->xmid ? 8 : 16);
        const double nux = -std::log(pb.ax.d);
        for (int k = 0; k < 5; ++k) pb.ax.dm[k] = std::exp(-nux * (double)pb.rpt_x * (double)(1 << k));
    }
}

// per-problem y-pass segment constants for the current rule
void set_y_problems(mol_batch_ctx *b)
{
    for (BatchProb &pb : b->hp) {
        pick_y(pb.ay.n, b->ymode, b->tbytes, pb.ky, pb.rpt_y);
        const double nuy = -std::log(pb.ay.d);
        for (int k = 0; k < 5; ++k) pb.ay.dm[k] = std::exp(-nuy * (double)pb.rpt_y * (double)(1 << k));
        set_y_nb(pb, b->tbytes == 4 && !(b->ymode & 2));
    }
}

// ... and the work list grouped by the new cluster sizes (synchronous)
cudaError_t set_y_segments(mol_batch_ctx *b)
{
    set_y_problems(b);
    const std::vector<int2> it = y_work_list(b);
    cudaError_t e = cudaDeviceSynchronize();
    if (e == cudaSuccess) e = cudaMemcpy(b->items, it.data(), sizeof(int2) * it.size(), cudaMemcpyHostToDevice);
    return e;
}

// x-pass launch shape L (0: rows of <= 512 points, 1: longer rows) for W warps per CTA
bool set_x_shape(mol_batch_ctx *b, int L, int W)
{
    const int ctas = L == 0 ? 2 : 1;
    const size_t bytes = batch_x_smem((size_t)b->tbytes, W, b->nbuf, L == 1);
    if (W < 1 || W > 8 || bytes > (size_t)b->smem_blk || ctas * (bytes + 1024) > (size_t)b->smem_sm) return false;
    b->xW[L] = W;
    b->xsmem[L] = bytes;
    const int64_t nr = L == 0 ? b->one_warp_end() : b->nrows - b->rows_mid;
    b->xgrid[L] = (int)std::max<int64_t>(1, std::min<int64_t>((nr + W - 1) / W, ctas * (int64_t)b->num_sms));
    return true;
}

cudaEvent_t btake_event(mol_batch_ctx *b)
{
    if (!b->ev_pool.empty()) {
        cudaEvent_t e = b->ev_pool.back();
        b->ev_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    return e;
}

template <class T, bool ADJ>
cudaError_t launch_y_class(const mol_batch_ctx *b, BatchPass bp, int k, cudaStream_t s)
{
    const unsigned K = 1u << k;
    bp.items += b->ycls_begin[k];
    bp.nitems = b->ycls_count[k];
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3((unsigned)b->ycls_count[k], K, 1);
    cfg.blockDim = dim3(32 * kBatchYSeg, 1, 1);
    cfg.dynamicSmemBytes = b->ysmem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = 1;
    attr[0].val.clusterDim.y = K;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = K > 1 ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, k_batch_y<T, ADJ>, bp);
}

// One launch per cluster size (a cluster of K CTAs per item of that size).
// The classes are independent: the one with the most CTAs runs on s, the
// others on side streams forked from s and joined back into it, so that the
// few long-latency CTAs of the short-column classes overlap the large class
// instead of running after it.
template <class T, bool ADJ>
cudaError_t launch_pass_y(mol_batch_ctx *b, const BatchPass &bp, cudaStream_t s)
{
    int main_k = -1, nside = 0;
    for (int k = 0; k < 4; ++k)
        if (b->ycls_count[k] > 0 && (main_k < 0 || (int64_t)b->ycls_count[k] << k >
                                                       (int64_t)b->ycls_count[main_k] << main_k))
            main_k = k;
    if (main_k < 0) return cudaSuccess;
    cudaError_t e = cudaSuccess;
    for (int k = 0; k < 4; ++k) nside += (k != main_k && b->ycls_count[k] > 0) ? 1 : 0;
    if (nside > 0) {
        for (int j = 0; j < 3 && e == cudaSuccess; ++j)
            if (!b->ys[j]) e = cudaStreamCreateWithFlags(&b->ys[j], cudaStreamNonBlocking);
        for (int j = 0; j < 4 && e == cudaSuccess; ++j)
            if (!b->yev[j]) e = cudaEventCreateWithFlags(&b->yev[j], cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventRecord(b->yev[0], s);
        int j = 0;
        for (int k = 0; k < 4 && e == cudaSuccess; ++k) {
            if (k == main_k || b->ycls_count[k] == 0) continue;
            e = cudaStreamWaitEvent(b->ys[j], b->yev[0], 0);
            if (e == cudaSuccess) e = launch_y_class<T, ADJ>(b, bp, k, b->ys[j]);
            if (e == cudaSuccess) e = cudaEventRecord(b->yev[1 + j], b->ys[j]);
            ++j;
        }
        if (e != cudaSuccess) return e;
    }
    e = launch_y_class<T, ADJ>(b, bp, main_k, s);
    for (int j = 0; j < nside && e == cudaSuccess; ++j) e = cudaStreamWaitEvent(s, b->yev[1 + j], 0);
    return e;
}

// One launch of the x pass per row group: g = 0 the rows of short lines
// (one warp per row, persistent), 1 rows of 257..512 points (one CTA of two
// warps per row, when their buffers fit), 2 longer rows (one CTA per row, or
// persistent warps).
template <class T, bool ADJ>
cudaError_t launch_x_group(const mol_batch_ctx *b, BatchPass bp, int g, cudaStream_t s)
{
    if (g == 0) {
        bp.row_begin = 0;
        bp.nitems = (int)b->one_warp_end();
        k_batch_x<T, false, ADJ><<<b->xgrid[0], 32 * b->xW[0], b->xsmem[0], s>>>(bp, b->nbuf);
    } else if (g == 1) {
        bp.row_begin = (int)b->rows_small;
        bp.nitems = (int)b->rows_mid;
        k_batch_xs<T, 8, 2, ADJ><<<(unsigned)(b->rows_mid - b->rows_small), 64, b->xs8_smem, s>>>(bp);
    } else {
        bp.row_begin = (int)b->rows_mid;
        bp.nitems = (int)b->nrows;
        if (b->xsplit)
            k_batch_xs<T, 16, 2, ADJ><<<(unsigned)(b->nrows - b->rows_mid), 64, b->xs_smem, s>>>(bp);
        else
            k_batch_x<T, true, ADJ><<<b->xgrid[1], 32 * b->xW[1], b->xsmem[1], s>>>(bp, b->nbuf);
    }
    return cudaGetLastError();
}

// the row groups present
void x_groups(const mol_batch_ctx *b, bool c[3])
{
    c[0] = b->one_warp_end() > 0;
    c[1] = b->xmid && b->rows_mid > b->rows_small;
    c[2] = b->nrows > b->rows_mid;
}

// The x pass: one launch per row group.  The groups are independent: the
// long rows (most of the work) run on s, the others on side streams forked
// from s and joined back into it, so that their launches overlap instead of
// queueing.
template <class T, bool ADJ>
cudaError_t launch_pass_x(mol_batch_ctx *b, BatchPass bp, cudaStream_t s)
{
    bool c[3];
    x_groups(b, c);
    const int nside = (c[0] ? 1 : 0) + (c[1] ? 1 : 0);
    cudaError_t e = cudaSuccess;
    cudaStream_t side[2] = {s, s};
    if (c[2] && nside > 0) {
        for (int j = 0; j < 2 && e == cudaSuccess; ++j)
            if (!b->ys[j]) e = cudaStreamCreateWithFlags(&b->ys[j], cudaStreamNonBlocking);
        for (int j = 0; j < 3 && e == cudaSuccess; ++j)
            if (!b->xev[j]) e = cudaEventCreateWithFlags(&b->xev[j], cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventRecord(b->xev[0], s);
        for (int j = 0; j < 2 && e == cudaSuccess; ++j) {
            e = cudaStreamWaitEvent(b->ys[j], b->xev[0], 0);
            side[j] = b->ys[j];
        }
        if (e != cudaSuccess) return e;
    }
    for (int g = 0; g < 3 && e == cudaSuccess; ++g)
        if (c[g]) e = launch_x_group<T, ADJ>(b, bp, g, g == 2 ? s : side[g]);
    if (e == cudaSuccess && c[2] && nside > 0) {
        for (int j = 0; j < 2 && e == cudaSuccess; ++j) e = cudaEventRecord(b->xev[1 + j], side[j]);
        for (int j = 0; j < 2 && e == cudaSuccess; ++j) e = cudaStreamWaitEvent(s, b->xev[1 + j], 0);
    }
    return e;
}

template <class T>
cudaError_t set_kernel_smem(const mol_batch_ctx *b)
{
    cudaError_t e = cudaSuccess;
    const void *xk[2][2] = {{(const void *)k_batch_x<T, false, false>, (const void *)k_batch_x<T, true, false>},
                            {(const void *)k_batch_x<T, false, true>, (const void *)k_batch_x<T, true, true>}};
    const void *yk[2] = {(const void *)k_batch_y<T, false>, (const void *)k_batch_y<T, true>};
    for (int adj = 0; adj < 2 && e == cudaSuccess; ++adj) {
        for (int L = 0; L < 2 && e == cudaSuccess; ++L)
            e = cudaFuncSetAttribute(xk[adj][L], cudaFuncAttributeMaxDynamicSharedMemorySize, (int)b->xsmem[L]);
        if (e == cudaSuccess) e = cudaFuncSetAttribute(yk[adj], cudaFuncAttributeMaxDynamicSharedMemorySize, (int)b->ysmem);
    }
    const void *sk[2] = {(const void *)k_batch_xs<T, 16, 2, false>, (const void *)k_batch_xs<T, 16, 2, true>};
    for (int adj = 0; adj < 2 && e == cudaSuccess; ++adj)
        e = cudaFuncSetAttribute(sk[adj], cudaFuncAttributeMaxDynamicSharedMemorySize, (int)b->xs_smem);
    const void *mk[2] = {(const void *)k_batch_xs<T, 8, 2, false>, (const void *)k_batch_xs<T, 8, 2, true>};
    for (int adj = 0; adj < 2 && e == cudaSuccess; ++adj)
        e = cudaFuncSetAttribute(mk[adj], cudaFuncAttributeMaxDynamicSharedMemorySize, (int)b->xs8_smem);
    return e;
}

// one pass, timed when pass timing is on (axis 0 = x, 1 = y); adj: the
// transposed operators
mol_status run_pass(mol_batch_ctx *b, int axis, const BatchPass &bp, cudaStream_t s, bool adj = false)
{
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (b->timing) {
        e0 = btake_event(b);
        e1 = btake_event(b);
        if (!e0 || !e1) return bfail(b, MOL_ECUDA, "event creation failed");
        BCK(cudaEventRecord(e0, s), "event record");
    }
    cudaError_t e;
    if (axis == 1) {
        if (adj) e = b->tbytes == 4 ? launch_pass_y<float, true>(b, bp, s) : launch_pass_y<double, true>(b, bp, s);
        else e = b->tbytes == 4 ? launch_pass_y<float, false>(b, bp, s) : launch_pass_y<double, false>(b, bp, s);
    } else {
        if (adj) e = b->tbytes == 4 ? launch_pass_x<float, true>(b, bp, s) : launch_pass_x<double, true>(b, bp, s);
        else e = b->tbytes == 4 ? launch_pass_x<float, false>(b, bp, s) : launch_pass_x<double, false>(b, bp, s);
    }
    if (e != cudaSuccess) return bcuda(b, e, "batched pass launch");
    b->launches += (axis == 1) ? b->y_launches() : b->x_launches();
    if (b->timing) {
        BCK(cudaEventRecord(e1, s), "event record");
        b->ev_used.push_back({axis, {e0, e1}});
    }
    return MOL_OK;
}

// the two passes of un = ea u + eb up + ec F[u]
void update_passes(const mol_batch_ctx *b, const BLevel &u, const BLevel &up, const BLevel &un, double ea, double eb,
                   double ec, BatchPass &y, BatchPass &x)
{
    y = BatchPass{};
    y.probs = b->probs;
    y.row_prob = b->row_prob;
    y.items = b->items;
    y.nitems = b->nitems_y;
    y.pr.u_hi = u.hi;
    y.pr.u_lo = u.lo;
    for (int k = 0; k < b->Pmax; ++k) y.pr.out[k] = b->inter[k];
    x = y;
    x.nitems = (int)b->nrows;
    for (int k = 0; k < b->Pmax; ++k) { x.pr.g[k] = b->inter[k]; x.pr.out[k] = nullptr; }
    x.pr.up_hi = up.hi;
    x.pr.up_lo = up.lo;
    x.pr.un_hi = un.hi;
    x.pr.un_lo = un.lo;
    x.pr.ea = ea;
    x.pr.eb = eb;
    x.pr.ec = ec;
    x.pr.fea = (float)ea;
    x.pr.feb = (float)eb;
    x.pr.fec = (float)ec;
}

// un = ea u + eb up + ec F[u] (adj: F^T[u]) for every problem: y pass, then x pass
mol_status run_update(mol_batch_ctx *b, const BLevel &u, const BLevel &up, const BLevel &un, double ea, double eb,
                      double ec, cudaStream_t s, bool adj = false)
{
    BatchPass y, x;
    update_passes(b, u, up, un, ea, eb, ec, y, x);
    mol_status st = run_pass(b, 1, y, s, adj);
    if (st != MOL_OK) return st;
    return run_pass(b, 0, x, s, adj);
}

mol_status pack(mol_batch_ctx *b, const double *x, const BLevel &L, cudaStream_t s)
{
    if (b->tbytes == 4)
        k_batch_pack<float><<<b->cgrid, 256, 0, s>>>(b->probs, b->row_prob, b->uoff_dev, (int)b->nrows, x,
                                                     (float *)L.hi, (float *)L.lo);
    else
        k_batch_pack<double><<<b->cgrid, 256, 0, s>>>(b->probs, b->row_prob, b->uoff_dev, (int)b->nrows, x,
                                                      (double *)L.hi, nullptr);
    BCK(cudaGetLastError(), "batched level conversion");
    b->launches++;
    return MOL_OK;
}

mol_status unpack(mol_batch_ctx *b, const BLevel &L, double *x, cudaStream_t s, const double *add = nullptr)
{
    if (b->tbytes == 4)
        k_batch_unpack<float><<<b->cgrid, 256, 0, s>>>(b->probs, b->row_prob, b->uoff_dev, (int)b->nrows,
                                                       (const float *)L.hi, (const float *)L.lo, x, add);
    else
        k_batch_unpack<double><<<b->cgrid, 256, 0, s>>>(b->probs, b->row_prob, b->uoff_dev, (int)b->nrows,
                                                        (const double *)L.hi, nullptr, x, add);
    BCK(cudaGetLastError(), "batched level conversion");
    b->launches++;
    return MOL_OK;
}

// receivers: packed user indices (host) -> internal-layout indices (device).
// Waits for the stream first: kernels of an earlier call may still read them.
mol_status set_receivers(mol_batch_ctx *b, int nrec, const int64_t *rec, cudaStream_t s)
{
    if (nrec < 1 || !rec) return bfail(b, MOL_EINVAL, "need nrec >= 1 receiver indices");
    std::vector<long long> ir(nrec);
    const int64_t total = b->uoff[b->nprob];
    for (int r = 0; r < nrec; ++r) {
        const int64_t g = rec[r];
        if (g < 0 || g >= total) return bfail(b, MOL_EINVAL, "receiver index out of range");
        const int p = (int)(std::upper_bound(b->uoff.begin(), b->uoff.end(), g) - b->uoff.begin()) - 1;
        const BatchProb &pb = b->hp[p];
        const int64_t loc = g - b->uoff[p];
        ir[r] = pb.off + (loc / pb.ax.n) * pb.pitch + loc % pb.ax.n;
    }
    // receivers grouped by node, so that the injection runs one thread per
    // distinct node (molt_recv.cuh)
    std::vector<long long> buf;
    const int nn = receiver_layout(ir, buf);
    BCK(cudaStreamSynchronize(s), "stream synchronize");
    if (nrec > b->irec_cap) {
        if (b->irec) {
            cudaFree(b->irec);
            b->allocs.erase(std::find(b->allocs.begin(), b->allocs.end(), (void *)b->irec));
            b->irec = nullptr;
            b->irec_cap = 0;
        }
        mol_status st = balloc(b, (void **)&b->irec, sizeof(long long) * (4 * (size_t)nrec + 1));
        if (st != MOL_OK) return st;
        b->irec_cap = nrec;
    }
    BCK(cudaMemcpy(b->irec, buf.data(), sizeof(long long) * buf.size(), cudaMemcpyHostToDevice), "receiver upload");
    b->nrec = nrec;
    b->nnode = nn;
    return MOL_OK;
}

mol_status gather(mol_batch_ctx *b, const BLevel &L, double *out, cudaStream_t s)
{
    const int blocks = (b->nrec + 255) / 256;
    if (b->tbytes == 4) k_recv_gather<float><<<blocks, 256, 0, s>>>((const float *)L.hi, (const float *)L.lo, b->irec, b->nrec, out);
    else k_recv_gather<double><<<blocks, 256, 0, s>>>((const double *)L.hi, nullptr, b->irec, b->nrec, out);
    BCK(cudaGetLastError(), "receiver gather");
    b->launches++;
    return MOL_OK;
}

mol_status inject(mol_batch_ctx *b, const BLevel &L, const double *vals, cudaStream_t s)
{
    // layout of the receiver buffer: see set_receivers
    const long long *node = b->irec + b->nrec, *start = node + b->nrec, *order = start + b->nrec + 1;
    const int blocks = (b->nnode + 127) / 128;
    if (b->tbytes == 4)
        k_recv_inject<float><<<blocks, 128, 0, s>>>((float *)L.hi, (float *)L.lo, node, start, order, b->nnode, vals);
    else
        k_recv_inject<double><<<blocks, 128, 0, s>>>((double *)L.hi, nullptr, node, start, order, b->nnode, vals);
    BCK(cudaGetLastError(), "receiver injection");
    b->launches++;
    return MOL_OK;
}

mol_status zero_level(mol_batch_ctx *b, const BLevel &L, cudaStream_t s)
{
    const size_t plane = (size_t)b->tbytes * b->total_int;
    BCK(cudaMemsetAsync(L.hi, 0, plane, s), "level clear");
    if (L.lo) BCK(cudaMemsetAsync(L.lo, 0, plane, s), "level clear");
    return MOL_OK;
}

// Chains of the time loop.  A problem's y pass runs in the launch of its
// cluster size and its x pass in the launch of its row group; where these
// pair up one to one (every problem of a y launch in the same x launch and
// back; so for square problems), each pair (y launch, then x launch, step
// after step) touches only its own problems' fields and runs as a chain of
// its own, joined with the others only at the end of the graph: the short
// problems' launches fill the ramps and tails of the long ones' instead of
// waiting at every pass.  ych / xch: the pairs; false where they do not
// pair up or there is only one.
bool chain_plan(const mol_batch_ctx *b, int ych[3], int xch[3], int &nch)
{
    int x2y[3] = {-1, -1, -1}, y2x[4] = {-1, -1, -1, -1};
    for (const BatchProb &pb : b->hp) {
        int xg = row_class(pb.ax.n);
        if (xg == 1 && !b->xmid) xg = 0;
        int yk = 0;
        while ((1 << yk) < pb.ky) ++yk;
        if (yk > 3 || (1 << yk) != pb.ky) return false;
        if (x2y[xg] < 0) x2y[xg] = yk;
        else if (x2y[xg] != yk) return false;
        if (y2x[yk] < 0) y2x[yk] = xg;
        else if (y2x[yk] != xg) return false;
    }
    nch = 0;
    for (int g = 0; g < 3; ++g)
        if (x2y[g] >= 0) {
            ych[nch] = x2y[g];
            xch[nch] = g;
            ++nch;
        }
    return nch > 1;
}

// three time steps captured as chains (see chain_plan)
template <class T>
mol_status capture_chains(mol_batch_ctx *b, const int ych[3], const int xch[3], int nch)
{
    cudaStream_t cs[3] = {b->cap_stream, nullptr, nullptr};
    for (int c = 1; c < nch; ++c) {
        if (!b->ys[c - 1]) BCK(cudaStreamCreateWithFlags(&b->ys[c - 1], cudaStreamNonBlocking), "stream create");
        cs[c] = b->ys[c - 1];
    }
    for (int j = 0; j < 4; ++j)
        if (!b->yev[j]) BCK(cudaEventCreateWithFlags(&b->yev[j], cudaEventDisableTiming), "event create");
    BCK(cudaEventRecord(b->yev[0], cs[0]), "event record");
    for (int c = 1; c < nch; ++c) BCK(cudaStreamWaitEvent(cs[c], b->yev[0], 0), "stream wait");
    for (int k = 0; k < 3; ++k) {
        BatchPass y, x;
        update_passes(b, b->lev[(k + 1) % 3], b->lev[k % 3], b->lev[(k + 2) % 3], 2.0, -1.0, 1.0, y, x);
        for (int c = 0; c < nch; ++c) {
            BCK((launch_y_class<T, false>(b, y, ych[c], cs[c])), "batched pass launch");
            BCK((launch_x_group<T, false>(b, x, xch[c], cs[c])), "batched pass launch");
        }
    }
    for (int c = 1; c < nch; ++c) {
        BCK(cudaEventRecord(b->yev[c], cs[c]), "event record");
        BCK(cudaStreamWaitEvent(cs[0], b->yev[c], 0), "stream wait");
    }
    return MOL_OK;
}

mol_status build_graph(mol_batch_ctx *b)
{
    if (b->gexec) return MOL_OK;
    if (!b->cap_stream) BCK(cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking), "stream create");
    int ych[3], xch[3], nch = 0;
    const bool chains = b->chains && chain_plan(b, ych, xch, nch);
    cudaGraph_t g = nullptr;
    BCK(cudaStreamBeginCapture(b->cap_stream, cudaStreamCaptureModeThreadLocal), "graph capture begin");
    const int64_t before = b->launches;
    mol_status st = MOL_OK;
    if (chains) {
        st = b->tbytes == 4 ? capture_chains<float>(b, ych, xch, nch) : capture_chains<double>(b, ych, xch, nch);
    } else {
        for (int k = 0; k < 3 && st == MOL_OK; ++k)
            st = run_update(b, b->lev[(k + 1) % 3], b->lev[k % 3], b->lev[(k + 2) % 3], 2.0, -1.0, 1.0, b->cap_stream);
    }
    cudaError_t e = cudaStreamEndCapture(b->cap_stream, &g);
    b->launches = before;
    if (st != MOL_OK) { if (g) cudaGraphDestroy(g); return st; }
    if (e != cudaSuccess) return bcuda(b, e, "graph capture end");
    e = cudaGraphInstantiate(&b->gexec, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) { b->gexec = nullptr; return bcuda(b, e, "graph instantiate"); }
    return MOL_OK;
}

mol_status bcheck_ptr(mol_batch_ctx *b, const void *p, const char *name)
{
    if (!p) return bfail(b, MOL_EINVAL, std::string(name) + " is NULL");
    cudaPointerAttributes at{};
    cudaError_t e = cudaPointerGetAttributes(&at, p);
    if (e != cudaSuccess) { cudaGetLastError(); return bfail(b, MOL_EINVAL, std::string(name) + ": not a CUDA pointer"); }
    if (at.type != cudaMemoryTypeDevice && at.type != cudaMemoryTypeManaged)
        return bfail(b, MOL_EINVAL, std::string(name) + " must be device memory");
    return MOL_OK;
}

// host-side validation and constants of every problem (no device work)
mol_status plan_batch(mol_batch_ctx *b, int nprob, const mol_grid *grids, const double *c, const double *dt,
                      const double *beta, const int *P, int quad)
{
    b->hp.assign(nprob, BatchProb{});
    b->uoff.assign(nprob + 1, 0);
    int64_t off = 0, rows = 0, items = 0;
    b->rows_small = 0;
    b->rows_mid = 0;
    for (int i = 0; i < nprob; ++i) {
        const mol_grid &g = grids[i];
        const std::string who = "problem " + std::to_string(i) + ": ";
        if (g.ndim != 2) return bfail(nullptr, MOL_EINVAL, who + "batched problems are 2D (ndim = 2)");
        for (int a = 0; a < 2; ++a) {
            if (g.n[a] < 3 || g.n[a] > kBatchMaxN)
                return bfail(nullptr, MOL_EINVAL, who + "every axis needs 3 <= n <= " + std::to_string(kBatchMaxN));
            if (!(g.hi[a] > g.lo[a])) return bfail(nullptr, MOL_EINVAL, who + "hi must exceed lo on every axis");
        }
        if (P[i] < 1 || P[i] > BMAXP) return bfail(nullptr, MOL_EINVAL, who + "P must be in 1..5");
        if (!(c[i] > 0) || !(dt[i] > 0) || !std::isfinite(c[i]) || !std::isfinite(dt[i]))
            return bfail(nullptr, MOL_EINVAL, who + "c and dt must be positive");
        const double bmax = beta_max_of(P[i]);
        double bt = beta ? beta[i] : 0.0;
        if (bt <= 0) bt = bmax;
        if (bt > bmax * (1.0 + 1e-12))
            return bfail(nullptr, MOL_EUNSTABLE, who + "beta above beta_max(P): the scheme is not A-stable");

        BatchProb &pb = b->hp[i];
        const int nx = (int)g.n[0], ny = (int)g.n[1];
        const double alpha = bt / (c[i] * dt[i]);                       // eq. L_def
        const double nux = alpha * (g.hi[0] - g.lo[0]) / (double)(nx - 1);
        const double nuy = alpha * (g.hi[1] - g.lo[1]) / (double)(ny - 1);
        axis_constants(nux, nx, BC_DIRICHLET, quad, pb.ax);
        axis_constants(nuy, ny, BC_DIRICHLET, quad, pb.ay);
        pb.rpt_x = pick_rpt_x(nx);
        pick_y(ny, 0, b->tbytes, pb.ky, pb.rpt_y);
        for (int k = 0; k < 5; ++k) {
            pb.ax.dm[k] = std::exp(-nux * (double)pb.rpt_x * (double)(1 << k));
            pb.ay.dm[k] = std::exp(-nuy * (double)pb.rpt_y * (double)(1 << k));
        }
        set_y_nb(pb, b->tbytes == 4);
        pb.P = P[i];
        pb.pitch = (nx + 3) & ~3;
        items += (nx + 31) / 32;
        std::vector<double> f;
        if (!expand_coefficients(2, P[i], bt, f)) return bfail(nullptr, MOL_EINVAL, who + "coefficient expansion failed");
        const int D = P[i] + 1;
        for (int t = 0; t <= P[i]; ++t) {
            pb.cu[t] = f[t];
            for (int k = 0; k < P[i]; ++k) pb.coef[t][k] = f[t + D * (k + 1)];
        }
        b->Pmax = std::max(b->Pmax, P[i]);
        b->uoff[i + 1] = b->uoff[i] + (int64_t)nx * ny;
    }
    // internal order: problems by the length class of their rows, so that each
    // x-pass kernel takes one contiguous range of rows
    for (int pass = 0; pass < 3; ++pass) {
        for (int i = 0; i < nprob; ++i) {
            BatchProb &pb = b->hp[i];
            if (row_class(pb.ax.n) != pass) continue;
            pb.off = off;
            pb.row0 = (int)rows;
            off += ((int64_t)pb.ay.n * pb.pitch + 63) & ~(int64_t)63;
            rows += pb.ay.n;
        }
        if (pass == 0) b->rows_small = rows;
        if (pass == 1) b->rows_mid = rows;
    }
    if (rows > (1ll << 30) || items > (1ll << 30)) return bfail(nullptr, MOL_EINVAL, "batch too large");
    b->total_int = off;
    b->nrows = rows;
    b->nitems_y = (int)items;
    b->xs_smem = batch_xs_smem((size_t)b->tbytes, 16, 2, b->Pmax);
    b->xsplit = b->xs_smem <= (size_t)b->smem_blk ? 1 : 0;
    b->xs8_smem = batch_xs_smem((size_t)b->tbytes, 8, 2, b->Pmax);
    b->xmid = b->xs8_smem <= (size_t)b->smem_blk ? 1 : 0;
    set_x_segments(b);
    return MOL_OK;
}

}  // namespace

extern "C" {

mol_status mol_batch_create(int nprob, const mol_grid *grids, const double *c, const double *dt, const double *beta,
                            const int *P, mol_bc bc, mol_prec prec, const mol_options *opt, mol_batch *out)
{
    if (!out) return bfail(nullptr, MOL_EINVAL, "out is NULL");
    *out = nullptr;
    if (nprob < 1) return bfail(nullptr, MOL_EINVAL, "nprob must be >= 1");
    if (!grids || !c || !dt || !P) return bfail(nullptr, MOL_EINVAL, "grids, c, dt and P must not be NULL");
    if (bc != MOL_BC_DIRICHLET) return bfail(nullptr, MOL_EINVAL, "batched problems take homogeneous Dirichlet conditions");
    if (prec != MOL_FP64 && prec != MOL_MIXED) return bfail(nullptr, MOL_EINVAL, "unknown precision");
    mol_options o;
    mol_default_options(&o);
    if (opt) o = *opt;
    if (o.quad_order != 1 && o.quad_order != 2) return bfail(nullptr, MOL_EINVAL, "quad_order must be 1 or 2");

    mol_batch_ctx *b = new mol_batch_ctx();
    b->nprob = nprob;
    b->prec = prec;
    b->tbytes = prec == MOL_MIXED ? 4 : 8;
    b->quad = o.quad_order;
    b->use_graphs = o.use_graphs ? 1 : 0;
    b->chains = o.use_graphs == 1 ? 1 : 0;
    mol_status st = plan_batch(b, nprob, grids, c, dt, beta, P, o.quad_order);
    if (st != MOL_OK) { delete b; return st; }

    int dev = 0, smem_sm = 228 * 1024, smem_blk = 227 * 1024, v = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) { st = bcuda(b, e, "cudaGetDevice"); goto bad; }
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess && v > 0) b->num_sms = v;
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev) == cudaSuccess && v > 0) smem_sm = v;
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) == cudaSuccess && v > 0) smem_blk = v;
    {
        // tables d^j per problem and axis (n + 1 + kBatchDpowPad entries)
        std::vector<int64_t> tofs(2 * nprob + 1, 0);
        for (int i = 0; i < nprob; ++i) {
            tofs[2 * i + 1] = tofs[2 * i] + b->hp[i].ax.n + 1 + kBatchDpowPad;
            tofs[2 * i + 2] = tofs[2 * i + 1] + b->hp[i].ay.n + 1 + kBatchDpowPad;
        }
        const int64_t nt = tofs[2 * nprob];
        std::vector<double> t64(nt);
        std::vector<float> t32(nt);
        for (int i = 0; i < nprob; ++i)
            for (int a = 0; a < 2; ++a) {
                const AxisDev &A = a == 0 ? b->hp[i].ax : b->hp[i].ay;
                const double nu = -std::log(A.d);
                for (int64_t j = 0; j < tofs[2 * i + a + 1] - tofs[2 * i + a]; ++j) {
                    t64[tofs[2 * i + a] + j] = std::exp(-nu * (double)j);
                    t32[tofs[2 * i + a] + j] = (float)t64[tofs[2 * i + a] + j];
                }
            }
        if ((st = balloc(b, (void **)&b->dp64, sizeof(double) * nt)) != MOL_OK) goto bad;
        if ((st = balloc(b, (void **)&b->dp32, sizeof(float) * nt)) != MOL_OK) goto bad;
        if ((e = cudaMemcpy(b->dp64, t64.data(), sizeof(double) * nt, cudaMemcpyHostToDevice)) != cudaSuccess ||
            (e = cudaMemcpy(b->dp32, t32.data(), sizeof(float) * nt, cudaMemcpyHostToDevice)) != cudaSuccess) {
            st = bcuda(b, e, "constant upload");
            goto bad;
        }
        for (int i = 0; i < nprob; ++i) {
            b->hp[i].ax.dpow64 = b->dp64 + tofs[2 * i];
            b->hp[i].ax.dpow32 = b->dp32 + tofs[2 * i];
            b->hp[i].ay.dpow64 = b->dp64 + tofs[2 * i + 1];
            b->hp[i].ay.dpow32 = b->dp32 + tofs[2 * i + 1];
        }
    }
    {
        std::vector<int> rp(b->nrows);
        std::vector<long long> uo(nprob + 1);
        for (int i = 0; i < nprob; ++i) {
            const BatchProb &pb = b->hp[i];
            for (int r = 0; r < pb.ay.n; ++r) rp[pb.row0 + r] = i;
        }
        const std::vector<int2> it = y_work_list(b);
        for (int i = 0; i <= nprob; ++i) uo[i] = b->uoff[i];
        if ((st = balloc(b, (void **)&b->probs, sizeof(BatchProb) * nprob)) != MOL_OK) goto bad;
        if ((st = balloc(b, (void **)&b->row_prob, sizeof(int) * rp.size())) != MOL_OK) goto bad;
        if ((st = balloc(b, (void **)&b->items, sizeof(int2) * it.size())) != MOL_OK) goto bad;
        if ((st = balloc(b, (void **)&b->uoff_dev, sizeof(long long) * uo.size())) != MOL_OK) goto bad;
        if ((e = upload_table(b)) != cudaSuccess ||
            (e = cudaMemcpy(b->row_prob, rp.data(), sizeof(int) * rp.size(), cudaMemcpyHostToDevice)) != cudaSuccess ||
            (e = cudaMemcpy(b->items, it.data(), sizeof(int2) * it.size(), cudaMemcpyHostToDevice)) != cudaSuccess ||
            (e = cudaMemcpy(b->uoff_dev, uo.data(), sizeof(long long) * uo.size(), cudaMemcpyHostToDevice)) !=
                cudaSuccess) {
            st = bcuda(b, e, "work list upload");
            goto bad;
        }
    }
    {
        const size_t plane = (size_t)b->tbytes * b->total_int;
        for (int k = 0; k < 3; ++k) {
            if ((st = balloc(b, &b->lev[k].hi, plane)) != MOL_OK) goto bad;
            if ((e = cudaMemset(b->lev[k].hi, 0, plane)) != cudaSuccess) { st = bcuda(b, e, "memset"); goto bad; }
            if (b->tbytes == 4) {
                if ((st = balloc(b, &b->lev[k].lo, plane)) != MOL_OK) goto bad;
                if ((e = cudaMemset(b->lev[k].lo, 0, plane)) != cudaSuccess) { st = bcuda(b, e, "memset"); goto bad; }
            }
        }
        for (int k = 0; k < b->Pmax; ++k) {
            if ((st = balloc(b, &b->inter[k], plane)) != MOL_OK) goto bad;
            if ((e = cudaMemset(b->inter[k], 0, plane)) != cudaSuccess) { st = bcuda(b, e, "memset"); goto bad; }
        }
    }
    {
        // launch shapes: x pass W warps per CTA with two CTAs per SM when the
        // field buffers allow it; y pass clusters of 4-warp CTAs per column group
        b->nbuf = b->Pmax;
        b->smem_sm = smem_sm;
        b->smem_blk = smem_blk;
        for (int L = 0; L < 2; ++L) {
            int W = 8;                             // the most warps per CTA that fit
            while (W > 1 && !set_x_shape(b, L, W)) --W;
            if (!set_x_shape(b, L, W)) { st = bfail(b, MOL_EINVAL, "x-pass buffers exceed shared memory"); goto bad; }
        }
        b->ysmem = batch_y_smem((size_t)b->tbytes);
        b->cgrid = (int)std::min<int64_t>((b->nrows + 7) / 8, 8 * (int64_t)b->num_sms);
        e = b->tbytes == 4 ? set_kernel_smem<float>(b) : set_kernel_smem<double>(b);
        if (e != cudaSuccess) { st = bcuda(b, e, "kernel attributes"); goto bad; }
    }
    *out = b;
    return MOL_OK;
bad:
    set_global_error(b->err);
    bfree_all(b);
    delete b;
    return st;
}

mol_status mol_batch_destroy(mol_batch b)
{
    if (!b) return bfail(nullptr, MOL_EINVAL, "handle is NULL");
    cudaDeviceSynchronize();
    bfree_all(b);
    delete b;
    return MOL_OK;
}

const char *mol_batch_last_error(mol_batch b) { return b ? b->err.c_str() : mol_last_error(nullptr); }

mol_status mol_batch_offsets(mol_batch b, int64_t *offsets)
{
    if (!b || !offsets) return bfail(b, MOL_EINVAL, "NULL argument");
    for (int i = 0; i <= b->nprob; ++i) offsets[i] = b->uoff[i];
    return MOL_OK;
}

mol_status mol_batch_apply_F(mol_batch b, const double *u, double *F, void *stream)
{
    if (!b) return bfail(nullptr, MOL_EINVAL, "handle is NULL");
    mol_status st;
    if ((st = bcheck_ptr(b, u, "u")) != MOL_OK || (st = bcheck_ptr(b, F, "F")) != MOL_OK) return st;
    if (u == F) return bfail(b, MOL_EINVAL, "u and F must not overlap");
    cudaStream_t s = (cudaStream_t)stream;
    if ((st = pack(b, u, b->lev[0], s)) != MOL_OK) return st;
    if ((st = run_update(b, b->lev[0], b->lev[0], b->lev[1], 0.0, 0.0, 1.0, s)) != MOL_OK) return st;
    return unpack(b, b->lev[1], F, s);
}

mol_status mol_batch_start(mol_batch b, const double *u0, double *u1, void *stream)
{
    if (!b) return bfail(nullptr, MOL_EINVAL, "handle is NULL");
    mol_status st;
    if ((st = bcheck_ptr(b, u0, "u0")) != MOL_OK || (st = bcheck_ptr(b, u1, "u1")) != MOL_OK) return st;
    if (u0 == u1) return bfail(b, MOL_EINVAL, "u0 and u1 must not overlap");
    cudaStream_t s = (cudaStream_t)stream;
    if ((st = pack(b, u0, b->lev[0], s)) != MOL_OK) return st;
    if ((st = run_update(b, b->lev[0], b->lev[0], b->lev[1], 1.0, 0.0, 0.5, s)) != MOL_OK) return st;
    return unpack(b, b->lev[1], u1, s);
}

mol_status mol_batch_step(mol_batch b, double *u_prev, double *u_cur, int64_t nsteps, void *stream)
{
    if (!b) return bfail(nullptr, MOL_EINVAL, "handle is NULL");
    if (nsteps < 0) return bfail(b, MOL_EINVAL, "nsteps must be >= 0");
    mol_status st;
    if ((st = bcheck_ptr(b, u_prev, "u_prev")) != MOL_OK || (st = bcheck_ptr(b, u_cur, "u_cur")) != MOL_OK) return st;
    if (u_prev == u_cur) return bfail(b, MOL_EINVAL, "u_prev and u_cur must not overlap");
    if (nsteps == 0) return MOL_OK;
    cudaStream_t s = (cudaStream_t)stream;
    if ((st = pack(b, u_prev, b->lev[0], s)) != MOL_OK) return st;
    if ((st = pack(b, u_cur, b->lev[1], s)) != MOL_OK) return st;
    int64_t done = 0;
    if (b->use_graphs && !b->timing && nsteps >= 3) {
        if ((st = build_graph(b)) != MOL_OK) return st;
        for (; done + 3 <= nsteps; done += 3) {
            BCK(cudaGraphLaunch(b->gexec, s), "graph launch");
            b->launches += 3 * (b->y_launches() + b->x_launches());
        }
    }
    for (; done < nsteps; ++done) {
        const int k = (int)(done % 3);
        if ((st = run_update(b, b->lev[(k + 1) % 3], b->lev[k], b->lev[(k + 2) % 3], 2.0, -1.0, 1.0, s)) != MOL_OK)
            return st;
    }
    const int k = (int)(nsteps % 3);
    if ((st = unpack(b, b->lev[k], u_prev, s)) != MOL_OK) return st;
    return unpack(b, b->lev[(k + 1) % 3], u_cur, s);
}

mol_status mol_batch_solve_host(mol_batch b, const double *u0, double *u_out, int64_t nsteps, void *stream)
{
    if (!b) return bfail(nullptr, MOL_EINVAL, "handle is NULL");
    if (!u0 || !u_out) return bfail(b, MOL_EINVAL, "NULL host buffer");
    if (nsteps < 1) return bfail(b, MOL_EINVAL, "nsteps must be >= 1");
    mol_status st;
    const size_t bytes = sizeof(double) * (size_t)b->uoff[b->nprob];
    for (int k = 0; k < 2; ++k)
        if (!b->io[k] && (st = balloc(b, (void **)&b->io[k], bytes)) != MOL_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    BCK(cudaMemcpyAsync(b->io[0], u0, bytes, cudaMemcpyHostToDevice, s), "host to device copy");
    if ((st = mol_batch_start(b, b->io[0], b->io[1], stream)) != MOL_OK) return st;
    if ((st = mol_batch_step(b, b->io[0], b->io[1], nsteps - 1, stream)) != MOL_OK) return st;
    BCK(cudaMemcpyAsync(u_out, b->io[1], bytes, cudaMemcpyDeviceToHost, s), "device to host copy");
    BCK(cudaStreamSynchronize(s), "solve");
    return MOL_OK;
}

mol_status mol_batch_apply_FT(mol_batch b, const double *w, double *out, void *stream)
{
    if (!b) return bfail(nullptr, MOL_EINVAL, "handle is NULL");
    mol_status st;
    if ((st = bcheck_ptr(b, w, "w")) != MOL_OK || (st = bcheck_ptr(b, out, "out")) != MOL_OK) return st;
    if (w == out) return bfail(b, MOL_EINVAL, "w and out must not overlap");
    cudaStream_t s = (cudaStream_t)stream;
    if ((st = pack(b, w, b->lev[0], s)) != MOL_OK) return st;
    if ((st = run_update(b, b->lev[0], b->lev[0], b->lev[1], 0.0, 0.0, 1.0, s, true)) != MOL_OK) return st;
    return unpack(b, b->lev[1], out, s);
}

mol_status mol_batch_update(mol_batch b, const double *u, const double *up, double *un, double ea, double eb,
                            double ec, int transpose, const double *add, void *stream)
{
    if (!b) return bfail(nullptr, MOL_EINVAL, "handle is NULL");
    mol_status st;
    if ((st = bcheck_ptr(b, u, "u")) != MOL_OK || (st = bcheck_ptr(b, un, "un")) != MOL_OK) return st;
    if (eb != 0.0 && (st = bcheck_ptr(b, up, "up")) != MOL_OK) return st;
    if (add && (st = bcheck_ptr(b, add, "add")) != MOL_OK) return st;
    if (un == u || (eb != 0.0 && un == up)) return bfail(b, MOL_EINVAL, "un must not overlap u or up");
    cudaStream_t s = (cudaStream_t)stream;
    if ((st = pack(b, u, b->lev[0], s)) != MOL_OK) return st;
    if (eb != 0.0 && (st = pack(b, up, b->lev[1], s)) != MOL_OK) return st;
    if ((st = run_update(b, b->lev[0], eb != 0.0 ? b->lev[1] : b->lev[0], b->lev[2], ea, eb, ec, s, transpose != 0)) !=
        MOL_OK)
        return st;
    return unpack(b, b->lev[2], un, s, add);
}

mol_status mol_batch_traces(mol_batch b, const double *u0, int nrec, const int64_t *rec, int64_t nsteps,
                            double *traces, void *stream)
{
    if (!b) return bfail(nullptr, MOL_EINVAL, "handle is NULL");
    if (nsteps < 1) return bfail(b, MOL_EINVAL, "nsteps must be >= 1");
    mol_status st;
    if ((st = bcheck_ptr(b, u0, "u0")) != MOL_OK || (st = bcheck_ptr(b, traces, "traces")) != MOL_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    if ((st = set_receivers(b, nrec, rec, s)) != MOL_OK) return st;
    int ip = 0, ic = 1, in = 2;
    if ((st = pack(b, u0, b->lev[ip], s)) != MOL_OK) return st;
    if ((st = run_update(b, b->lev[ip], b->lev[ip], b->lev[ic], 1.0, 0.0, 0.5, s)) != MOL_OK) return st;
    if ((st = gather(b, b->lev[ic], traces, s)) != MOL_OK) return st;
    for (int64_t n = 1; n < nsteps; ++n) {
        if ((st = run_update(b, b->lev[ic], b->lev[ip], b->lev[in], 2.0, -1.0, 1.0, s)) != MOL_OK) return st;
        if ((st = gather(b, b->lev[in], traces + n * nrec, s)) != MOL_OK) return st;
        const int t = ip; ip = ic; ic = in; in = t;
    }
    return MOL_OK;
}

mol_status mol_batch_adjoint(mol_batch b, int nrec, const int64_t *rec, int64_t nsteps, const double *tgrad,
                             double *grad, void *stream)
{
    if (!b) return bfail(nullptr, MOL_EINVAL, "handle is NULL");
    if (nsteps < 1) return bfail(b, MOL_EINVAL, "nsteps must be >= 1");
    mol_status st;
    if ((st = bcheck_ptr(b, tgrad, "tgrad")) != MOL_OK || (st = bcheck_ptr(b, grad, "grad")) != MOL_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    if ((st = set_receivers(b, nrec, rec, s)) != MOL_OK) return st;
    // mu^{N+1} = 0 in ia, mu^N = g^N in ib
    int ia = 0, ib = 1, ic = 2;
    if ((st = zero_level(b, b->lev[ia], s)) != MOL_OK) return st;
    if ((st = zero_level(b, b->lev[ib], s)) != MOL_OK) return st;
    if ((st = inject(b, b->lev[ib], tgrad + (nsteps - 1) * nrec, s)) != MOL_OK) return st;
    for (int64_t n = nsteps - 1; n >= 1; --n) {
        // mu^n = 2 mu^{n+1} - mu^{n+2} + F^T mu^{n+1} + g^n
        if ((st = run_update(b, b->lev[ib], b->lev[ia], b->lev[ic], 2.0, -1.0, 1.0, s, true)) != MOL_OK) return st;
        if ((st = inject(b, b->lev[ic], tgrad + (n - 1) * nrec, s)) != MOL_OK) return st;
        const int t = ia; ia = ib; ib = ic; ic = t;
    }
    // dJ/du^0 = mu^1 + F^T mu^1 / 2 - mu^2
    if ((st = run_update(b, b->lev[ib], b->lev[ia], b->lev[ic], 1.0, -1.0, 0.5, s, true)) != MOL_OK) return st;
    return unpack(b, b->lev[ic], grad, s);
}

mol_status mol_batch_sync(mol_batch b, void *stream)
{
    if (!b) return bfail(nullptr, MOL_EINVAL, "handle is NULL");
    BCK(cudaStreamSynchronize((cudaStream_t)stream), "stream synchronize");
    BCK(cudaGetLastError(), "device error");
    return MOL_OK;
}

int64_t mol_batch_launch_count(mol_batch b) { return b ? b->launches : 0; }

// x and y pass times (ms per launch, minimum over 3 steps) with the current choices
static mol_status batch_pass_ms(mol_batch b, cudaStream_t s, double out[2])
{
    const bool was = b->timing;
    for (auto &u : b->ev_used) { b->ev_pool.push_back(u.second.first); b->ev_pool.push_back(u.second.second); }
    b->ev_used.clear();
    b->timing = true;
    mol_status st = MOL_OK;
    for (int k = 0; k < 4 && st == MOL_OK; ++k)
        st = run_update(b, b->lev[(k + 1) % 3], b->lev[k % 3], b->lev[(k + 2) % 3], 2.0, -1.0, 1.0, s);
    out[0] = out[1] = 1e30;
    if (st == MOL_OK) {
        int idx = 0;
        for (auto &u : b->ev_used) {
            float ms = 0.f;
            if (cudaEventSynchronize(u.second.second) != cudaSuccess ||
                cudaEventElapsedTime(&ms, u.second.first, u.second.second) != cudaSuccess) {
                st = bfail(b, MOL_ECUDA, "tuning timer");
                break;
            }
            if (idx++ >= 2) out[u.first] = std::min(out[u.first], (double)ms);   // the first step warms up
        }
    }
    for (auto &u : b->ev_used) { b->ev_pool.push_back(u.second.first); b->ev_pool.push_back(u.second.second); }
    b->ev_used.clear();
    b->timing = was;
    return st;
}

mol_status mol_batch_autotune(mol_batch b, void *stream)
{
    if (!b) return bfail(nullptr, MOL_EINVAL, "handle is NULL");
    cudaStream_t s = (cudaStream_t)stream;
    mol_status st;
    for (int k = 0; k < 3; ++k)
        if ((st = zero_level(b, b->lev[k], s)) != MOL_OK) return st;
    const int64_t launches0 = b->launches;
    double t[2];
    // warps per CTA of each x launch (the other held; long rows also split
    // over two warps, W = 0 below), then the y segment rule
    auto upload = [&]() {
        return upload_table(b);
    };
    for (int L = 0; L < 2; ++L) {
        if ((L == 0 && b->one_warp_end() == 0) || (L == 1 && b->nrows == b->rows_mid)) continue;
        int bestW = b->xW[L], bestSplit = b->xsplit;
        double best = 1e30;
        for (int W : {0, 2, 4, 8}) {
            if (W == 0 && (L == 0 || b->xs_smem > (size_t)b->smem_blk)) continue;
            if (L == 1) {
                b->xsplit = W == 0 ? 1 : 0;
                set_x_segments(b);
                BCK(upload(), "table upload");
            }
            if (W > 0 && !set_x_shape(b, L, W)) continue;
            if ((st = batch_pass_ms(b, s, t)) != MOL_OK) return st;
            if (t[0] < best) { best = t[0]; bestW = W > 0 ? W : bestW; bestSplit = W == 0; }
        }
        if (L == 1) {
            b->xsplit = bestSplit;
            set_x_segments(b);
            BCK(upload(), "table upload");
        }
        set_x_shape(b, L, bestW);
        b->tune_ms[0] = best;
    }
    int bestY = b->ymode;
    double besty = 1e30;
    for (int mode : {0, 1, 2}) {
        b->ymode = mode;
        BCK(set_y_segments(b), "y work list upload");
        BCK(upload(), "table upload");
        if ((st = batch_pass_ms(b, s, t)) != MOL_OK) return st;
        if (t[1] < besty) { besty = t[1]; bestY = mode; }
    }
    b->ymode = bestY;
    BCK(set_y_segments(b), "y work list upload");
    BCK(upload(), "table upload");
    b->tune_ms[1] = besty;
    b->launches = launches0;
    if (b->gexec) { cudaGraphExecDestroy(b->gexec); b->gexec = nullptr; }
    return MOL_OK;
}

mol_status mol_batch_set_tuning(mol_batch b, int x_warps_short, int x_warps_long, int y_rule)
{
    if (!b) return bfail(nullptr, MOL_EINVAL, "handle is NULL");
    auto okW = [](int W) { return W == 2 || W == 4 || W == 8; };
    if (!okW(x_warps_short) || !(okW(x_warps_long) || x_warps_long == 0) || y_rule < 0 || y_rule > 3)
        return bfail(b, MOL_EINVAL, "x warps must be 2, 4 or 8 (0: split long rows) and the y rule 0..3");
    if (x_warps_long == 0 && b->xs_smem > (size_t)b->smem_blk)
        return bfail(b, MOL_EINVAL, "split-row buffers exceed shared memory");
    const int oldW[2] = {b->xW[0], b->xW[1]};
    if (!set_x_shape(b, 0, x_warps_short) || (x_warps_long > 0 && !set_x_shape(b, 1, x_warps_long))) {
        set_x_shape(b, 0, oldW[0]);
        set_x_shape(b, 1, oldW[1]);
        return bfail(b, MOL_EINVAL, "x-pass buffers exceed shared memory");
    }
    b->xsplit = x_warps_long == 0 ? 1 : 0;
    b->ymode = y_rule;
    set_x_segments(b);
    BCK(set_y_segments(b), "y work list upload");
    BCK(cudaDeviceSynchronize(), "synchronise before the table upload");
    BCK(upload_table(b), "table upload");
    if (b->gexec) { cudaGraphExecDestroy(b->gexec); b->gexec = nullptr; }
    return MOL_OK;
}

mol_status mol_batch_get_tuning(mol_batch b, int out[3], double ms[2])
{
    if (!b || !out) return bfail(b, MOL_EINVAL, "NULL argument");
    out[0] = b->xW[0];
    out[1] = b->xsplit ? 0 : b->xW[1];
    out[2] = b->ymode;
    if (ms) { ms[0] = b->tune_ms[0]; ms[1] = b->tune_ms[1]; }
    return MOL_OK;
}

mol_status mol_batch_set_pass_timing(mol_batch b, int enable)
{
    if (!b) return bfail(nullptr, MOL_EINVAL, "handle is NULL");
    for (auto &u : b->ev_used) { b->ev_pool.push_back(u.second.first); b->ev_pool.push_back(u.second.second); }
    b->ev_used.clear();
    b->timing = enable != 0;
    return MOL_OK;
}

mol_status mol_batch_pass_times(mol_batch b, double total_ms[3], int64_t launches[3])
{
    if (!b || !total_ms || !launches) return bfail(b, MOL_EINVAL, "NULL argument");
    for (int a = 0; a < 3; ++a) { total_ms[a] = 0.0; launches[a] = 0; }
    for (auto &u : b->ev_used) {
        BCK(cudaEventSynchronize(u.second.second), "event synchronize");
        float ms = 0.f;
        BCK(cudaEventElapsedTime(&ms, u.second.first, u.second.second), "event elapsed time");
        total_ms[u.first] += ms;
        launches[u.first] += 1;
    }
    return MOL_OK;
}


// history gradient (checkpoint-and-recompute) over the batch's packed fields
namespace {

mol_status bh_fail(void *c, mol_status st, const char *msg) { return bfail((mol_batch_ctx *)c, st, msg); }

mol_status bh_start(void *c, const double *u0, double *u1, cudaStream_t s)
{
    return mol_batch_start((mol_batch_ctx *)c, u0, u1, (void *)s);
}

mol_status bh_step(void *c, double *prev, double *cur, int64_t n, cudaStream_t s)
{
    return mol_batch_step((mol_batch_ctx *)c, prev, cur, n, (void *)s);
}

mol_status bh_step_emit(void *c, const double *prev, const double *cur, int64_t m, double *states, cudaStream_t s)
{
    mol_batch_ctx *b = (mol_batch_ctx *)c;
    mol_status st;
    if ((st = pack(b, prev, b->lev[0], s)) != MOL_OK) return st;
    if ((st = pack(b, cur, b->lev[1], s)) != MOL_OK) return st;
    const int64_t N = b->uoff[b->nprob];
    for (int64_t j = 0; j < m; ++j) {
        const int k = (int)(j % 3);
        if ((st = run_update(b, b->lev[(k + 1) % 3], b->lev[k], b->lev[(k + 2) % 3], 2.0, -1.0, 1.0, s)) != MOL_OK)
            return st;
        if ((st = unpack(b, b->lev[(k + 2) % 3], states + (size_t)j * N, s)) != MOL_OK) return st;
    }
    return MOL_OK;
}

mol_status bh_update_T(void *c, const double *u, const double *up, double *un, double ea, double eb, double ec,
                       const double *add, cudaStream_t s)
{
    return mol_batch_update((mol_batch_ctx *)c, u, up, un, ea, eb, ec, 1, add, (void *)s);
}

}  // namespace

mol_status mol_batch_adjoint_history(mol_batch b, const double *u0, int64_t nsteps, int64_t checkpoint_every,
                                     mol_grad_fn grad_fn, void *user, double *grad, void *stream)
{
    if (!b) return bfail(nullptr, MOL_EINVAL, "handle is NULL");
    mol_status st;
    if ((st = bcheck_ptr(b, u0, "u0")) != MOL_OK || (st = bcheck_ptr(b, grad, "grad")) != MOL_OK) return st;
    HistoryOps o{b, b->uoff[b->nprob], bh_start, bh_step, bh_step_emit, bh_update_T, bh_fail};
    return history_gradient_run(o, u0, nsteps, checkpoint_every, grad_fn, user, grad, (cudaStream_t)stream);
}

}  // extern "C"
