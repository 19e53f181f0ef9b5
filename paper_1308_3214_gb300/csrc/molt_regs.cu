// molt_regs.cu -- instantiation and launch of the register-resident pass kernels.
#include <algorithm>
#include <cmath>
#include <utility>
#include "molt_internal.h"
#include "molt_regs.cuh"
#include "molt_strided_nb.cuh"

namespace molt {

namespace {

// Launch with the launch attributes of a pass: a cluster of cluster_y CTAs
// along y (> 1), and (L.pdl) programmatic dependent launch, under which the
// kernel's CTAs may be scheduled while the previous kernel in the stream
// finishes (every pass kernel waits for it in pdl_enter before touching
// global memory).
template <class... KArgs, class... Args>
cudaError_t launch_pass(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                        const LineSet &L, int cluster_y, Args &&...args)
{
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[2];
    int na = 0;
    if (cluster_y > 1) {
        attr[na].id = cudaLaunchAttributeClusterDimension;
        attr[na].val.clusterDim.x = 1;
        attr[na].val.clusterDim.y = (unsigned)cluster_y;
        attr[na].val.clusterDim.z = 1;
        ++na;
    }
    if (L.pdl) {
        attr[na].id = cudaLaunchAttributeProgrammaticStreamSerialization;
        attr[na].val.programmaticStreamSerializationAllowed = 1;
        ++na;
    }
    cfg.attrs = attr;
    cfg.numAttrs = na;
    return cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

constexpr int kContigWarps = 4;
constexpr int kResWarpsMax = 4;

template <int RPT, int NB>
size_t res_smem(int warps) { return (size_t)warps * NB * ContigStage<float, RPT>::LINE * sizeof(float); }

template <int BC, int RPT, int NB>
cudaError_t run_res(int warps, const AxisDev &A, const LineSet &L, const ProgParams &p, cudaStream_t s)
{
    const int64_t grid = (L.nlines + warps - 1) / warps;
    return launch_pass(k_contig_res<BC, RPT, NB>, dim3((unsigned)grid), dim3(32 * warps), res_smem<RPT, NB>(warps), s, L,
                       1, A, L, p);
}

template <int BC, int RPT, int NB>
cudaError_t attr_res()
{
    return cudaFuncSetAttribute(k_contig_res<BC, RPT, NB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)res_smem<RPT, NB>(kResWarpsMax));
}

template <int RPT, int NB, int W>
size_t rows_smem() { return row_slots_bytes<float, W>() + (size_t)NB * 32 * W * ContigStage<float, RPT>::SST * sizeof(float); }

// Grid of the row-split pass: one CTA per row, or as many persistent CTAs as
// fit on L.persist_sms SMs (occupancy of the kernel, looked up once).
template <class K>
unsigned rows_grid(K kernel, int W, size_t smem, const LineSet &L, int &occ_cache)
{
    if (L.persist_sms <= 0) return (unsigned)L.nlines;
    if (occ_cache <= 0) {
        int occ = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kernel, 32 * W, smem) != cudaSuccess || occ < 1) {
            cudaGetLastError();
            occ = 1;
        }
        occ_cache = occ;
    }
    return (unsigned)std::min<int64_t>(L.nlines, (int64_t)occ_cache * L.persist_sms);
}

// Dynamic shared memory of a one-CTA-per-row launch: the row's buffers,
// padded where one CTA per SM fewer than the kernel's occupancy occ leaves
// fuller waves.  With k CTAs per SM the nrows CTAs take nrows / (SMs k)
// waves, the last one partly empty; k = occ - 1 is taken where it raises the
// filled fraction of the waves by more than 0.05 (2048 rows of two warps on
// 152 SMs: 8 per SM fill 84 % of two waves, 7 fill 96 %), and the padding
// leaves no room for a (k+1)-th CTA: (k+1) (smem + reserved) > the SM's
// shared memory.
template <class K>
size_t rows_launch_smem(K kernel, int W, size_t base, int64_t nrows, int &occ_cache)
{
    static int dev_c = -1, sms = 0, smem_sm = 0, resv = 0;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) { cudaGetLastError(); return base; }
    if (dev != dev_c) {
        if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&resv, cudaDevAttrReservedSharedMemoryPerBlock, dev) != cudaSuccess) {
            cudaGetLastError();
            return base;
        }
        dev_c = dev;
    }
    if (occ_cache <= 0) {
        int occ = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kernel, 32 * W, base) != cudaSuccess || occ < 1) {
            cudaGetLastError();
            occ = 1;
        }
        occ_cache = occ;
    }
    const int occ = occ_cache;
    if (occ < 2 || sms < 1) return base;
    auto fill = [&](int k) {
        const double w = (double)nrows / ((double)sms * (double)k);
        return w / std::ceil(w);
    };
    if (fill(occ - 1) <= fill(occ) + 0.05) return base;
    const size_t pad = ((size_t)smem_sm / (size_t)occ - (size_t)resv + 16 + 15) & ~(size_t)15;
    return pad > base ? pad : base;
}

template <int BC, int RPT, int NB, int W>
cudaError_t run_rows(const AxisDev &A, const LineSet &L, const ProgParams &p, cudaStream_t s)
{
    const size_t smem = rows_smem<RPT, NB, W>();
    const NbConsts nc = strided_nb_consts(A.d, RPT);
    if constexpr (BC == BC_DIRICHLET) {
        if (p.mode == 3) {                            // the transposed Horner pass
            static int occ_adj = 0;
            const unsigned g = rows_grid(k_contig_rows<BC, RPT, NB, W, true>, W, smem, L, occ_adj);
            return launch_pass(k_contig_rows<BC, RPT, NB, W, true>, dim3(g), dim3(32 * W), smem, s, L, 1, A, L, p, nc);
        }
    }
    if constexpr (W == 2 || W == 4) {
        if (L.rows_nb && rows_nb_plan(A.d, A.n, RPT, W)) {   // one neighbour exchange per sweep
            static int occ_nb = 0, occ_nb_pad = 0;
            const unsigned g = rows_grid(k_contig_rows<BC, RPT, NB, W, false, true>, W, smem, L, occ_nb);
            const size_t sm = L.persist_sms > 0 ? smem
                                                : rows_launch_smem(k_contig_rows<BC, RPT, NB, W, false, true>, W, smem,
                                                                   L.nlines, occ_nb_pad);
            return launch_pass(k_contig_rows<BC, RPT, NB, W, false, true>, dim3(g), dim3(32 * W), sm, s, L, 1, A, L,
                               p, nc);
        }
    }
    static int occ = 0, occ_pad = 0;
    const unsigned g = rows_grid(k_contig_rows<BC, RPT, NB, W>, W, smem, L, occ);
    const size_t sm = L.persist_sms > 0 ? smem : rows_launch_smem(k_contig_rows<BC, RPT, NB, W>, W, smem, L.nlines, occ_pad);
    return launch_pass(k_contig_rows<BC, RPT, NB, W>, dim3(g), dim3(32 * W), sm, s, L, 1, A, L, p, nc);
}

template <int BC, int RPT, int NB, int W>
cudaError_t attr_rows()
{
    // the largest shared-memory carveout: the CTAs per SM are then limited
    // by registers and the row's buffers, not by the default split with L1
    // (up to the per-CTA maximum: a launch may pad its buffers, rows_launch_smem)
    cudaError_t e = cudaFuncSetAttribute(k_contig_rows<BC, RPT, NB, W>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         227 * 1024);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_contig_rows<BC, RPT, NB, W>, cudaFuncAttributePreferredSharedMemoryCarveout,
                                 (int)cudaSharedmemCarveoutMaxShared);
    if constexpr (BC == BC_DIRICHLET) {
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(k_contig_rows<BC, RPT, NB, W, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)rows_smem<RPT, NB, W>());
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(k_contig_rows<BC, RPT, NB, W, true>,
                                     cudaFuncAttributePreferredSharedMemoryCarveout, (int)cudaSharedmemCarveoutMaxShared);
    }
    if constexpr (W == 2 || W == 4) {
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(k_contig_rows<BC, RPT, NB, W, false, true>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(k_contig_rows<BC, RPT, NB, W, false, true>,
                                     cudaFuncAttributePreferredSharedMemoryCarveout, (int)cudaSharedmemCarveoutMaxShared);
    }
    return e;
}

template <class T, int RPT>
size_t contig_smem() { return (size_t)kContigWarps * 2 * ContigStage<T, RPT>::LINE * sizeof(T); }

template <class T, int BC, int RPT>
cudaError_t run_contig(const AxisDev &A, const LineSet &L, const ProgParams &p, cudaStream_t s)
{
    const int64_t grid = (L.nlines + kContigWarps - 1) / kContigWarps;
    return launch_pass(k_contig<T, BC, RPT, kContigWarps>, dim3((unsigned)grid), dim3(32 * kContigWarps),
                       contig_smem<T, RPT>(), s, L, 1, A, L, p);
}

template <class T, int BC, int RPT>
cudaError_t run_strided(const AxisDev &A, const LineSet &L, const ProgParams &p, cudaStream_t s)
{
    size_t smem = strided_slot_bytes(L.S, sizeof(T));
    if (p.mode == 1) smem += (size_t)L.S * RPT * 32 * sizeof(T);
    const dim3 grid((unsigned)((L.nlines + 31) / 32), (unsigned)L.K, 1), block(32 * L.S, 1, 1);
    if (p.mode == 1) return launch_pass(k_strided<T, BC, RPT, 1>, grid, block, smem, s, L, L.K, A, L, p);
    if constexpr (BC == BC_DIRICHLET)
        if (p.mode == 2) return launch_pass(k_strided<T, BC, RPT, 2>, grid, block, smem, s, L, L.K, A, L, p);
    return launch_pass(k_strided<T, BC, RPT, 0>, grid, block, smem, s, L, L.K, A, L, p);
}

// cuTensorMapEncodeTiled from the driver (through the runtime, so that the
// library links no driver stub)
using EncodeTiledFn = CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                   const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_tiled_fn()
{
    static EncodeTiledFn fn = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        void *f = nullptr;
        cudaDriverEntryPointQueryResult q{};
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(f);
        else
            cudaGetLastError();
    }
    return fn;
}

// 3D view {inner, n, outer} of a float32 field (the strided axis is the
// middle one), boxes of {32, box_rows, 1}; zeros outside the field.
bool encode_field_map(CUtensorMap *m, const void *ptr, const LineSet &L, int n, int box_rows)
{
    EncodeTiledFn fn = encode_tiled_fn();
    if (!fn || ptr == nullptr || ((uintptr_t)ptr & 15) != 0 || L.inner % 32 != 0 || box_rows < 1 || box_rows > 256)
        return false;
    const cuuint64_t inner = (cuuint64_t)L.inner, outer = (cuuint64_t)(L.nlines / L.inner);
    const cuuint64_t dims[3] = {inner, (cuuint64_t)n, outer};
    const cuuint64_t strides[2] = {inner * 4, inner * (cuuint64_t)n * 4};
    const cuuint32_t box[3] = {32, (cuuint32_t)box_rows, 1};
    const cuuint32_t es[3] = {1, 1, 1};
    return fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<void *>(ptr), dims, strides, box, es,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <int BC, int RPT, int STAGE>
cudaError_t launch_nb_stage(const AxisDev &A, const LineSet &L, const ProgParams &p, const TmaMaps &tm, size_t smem,
                            cudaStream_t s)
{
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(k_strided_nb<BC, RPT, STAGE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             200 * 1024);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    return launch_pass(k_strided_nb<BC, RPT, STAGE>, dim3((unsigned)((L.nlines + 31) / 32), (unsigned)L.K, 1),
                       dim3(32 * L.S, 1, 1), smem, s, L, L.K, A, L, p, strided_nb_consts(A.d, RPT), tm);
}

template <int BC, int RPT>
cudaError_t run_strided_nb(const AxisDev &A, const LineSet &L, const ProgParams &p, cudaStream_t s, int stage)
{
    TmaMaps tm{};
    if (stage != 0) {
        // tensor maps of this launch's fields; any that cannot be made (a
        // grid whose line groups straddle an outer slice, an unaligned
        // pointer, no driver entry point) fall back to direct loads / stores
        const int in_rows = L.S * RPT + 4;
        tm.nbox = (in_rows + 255) / 256;
        tm.box_rows = (in_rows + tm.nbox - 1) / tm.nbox;
        const int out_box = L.S * RPT > 256 ? 256 : L.S * RPT;
        bool ok = true;
        if (stage & 1)
            ok = encode_field_map(&tm.in_hi, p.u_hi, L, A.n, tm.box_rows) &&
                 encode_field_map(&tm.in_lo, p.u_lo, L, A.n, tm.box_rows);
        if ((stage & 2) && ok) {
            if (p.P > kMaxTmaOut) ok = false;
            for (int k = 0; k < p.P && ok; ++k)
                if (p.out[k] != nullptr) ok = encode_field_map(&tm.out[k], p.out[k], L, A.n, out_box);
        }
        if (!ok) stage = 0;
    }
    const size_t smem = strided_nb_smem(L.S, RPT, stage, tm.nbox, tm.box_rows);
    switch (stage) {
    case 1: return launch_nb_stage<BC, RPT, 1>(A, L, p, tm, smem, s);
    case 2: return launch_nb_stage<BC, RPT, 2>(A, L, p, tm, smem, s);
    case 3: return launch_nb_stage<BC, RPT, 3>(A, L, p, tm, smem, s);
    default: return launch_nb_stage<BC, RPT, 0>(A, L, p, tm, smem, s);
    }
}

template <int BC, int RPT, bool GT>
cudaError_t run_strided_nb_h(const AxisDev &A, const LineSet &L, const ProgParams &p, const TmaGMaps &tg, size_t smem,
                             cudaStream_t s)
{
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(k_strided_nb_h<BC, RPT, GT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             200 * 1024);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    return launch_pass(k_strided_nb_h<BC, RPT, GT>, dim3((unsigned)((L.nlines + 31) / 32), (unsigned)L.K, 1),
                       dim3(32 * L.S, 1, 1), smem, s, L, L.K, A, L, p, strided_nb_consts(A.d, RPT), tg);
}

template <int BC, int RPT>
cudaError_t run_strided_nb_h_any(const AxisDev &A, const LineSet &L, const ProgParams &p, cudaStream_t s, bool gt)
{
    TmaGMaps tg{};
    if (gt) {
        // the staged tiles only with a tensor map for every field and while
        // two CTAs per SM still fit; else the fields are read from global
        const int in_rows = L.S * RPT + 4;
        tg.nbox = (in_rows + 255) / 256;
        tg.box_rows = (in_rows + tg.nbox - 1) / tg.nbox;
        const size_t smem = strided_nb_h_smem(L.S, RPT, p.ng, true, tg.nbox * tg.box_rows);
        bool ok = p.ng >= 1 && p.ng <= kMaxTmaG && smem <= 110 * 1024;
        for (int q = 0; q < p.ng && ok; ++q) ok = encode_field_map(&tg.g[q], p.g[q], L, A.n, tg.box_rows);
        if (ok) return run_strided_nb_h<BC, RPT, true>(A, L, p, tg, smem, s);
        tg = TmaGMaps{};
    }
    return run_strided_nb_h<BC, RPT, false>(A, L, p, tg, strided_nb_h_smem(L.S, RPT, p.ng, false), s);
}

template <class T, int BC, int RPT>
cudaError_t attr_contig()
{
    return cudaFuncSetAttribute(k_contig<T, BC, RPT, kContigWarps>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)contig_smem<T, RPT>());
}

template <class T, int BC, int RPT>
cudaError_t attr_strided()
{
    cudaError_t e = cudaFuncSetAttribute(k_strided<T, BC, RPT, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    if (e != cudaSuccess) return e;
    if constexpr (BC == BC_DIRICHLET) {
        e = cudaFuncSetAttribute(k_strided<T, BC, RPT, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
        if (e != cudaSuccess) return e;
    }
    return cudaFuncSetAttribute(k_strided<T, BC, RPT, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
}

}  // namespace

// Segment lengths: contiguous lines use the smallest RPT with 32*RPT >= n;
// strided lines use 64 (float) / 32 (double) points per thread by default,
// or 32 (float) as an alternative the tuner may pick.
constexpr int kStridedRptF = 64, kStridedRptF2 = 32, kStridedRptD = 32;

// Register kernels need whole segments: n a multiple of RPT (both boundary
// conditions keep the line ends at fixed register positions).
bool regs_contig_plan(int tbytes, int, int n, int *rpt)
{
    const int maxr = tbytes == 4 ? 64 : 32;
    for (int r = 8; r <= maxr; r *= 2) {
        if (32 * r < n) continue;
        if (n % r != 0) return false;
        *rpt = r;
        return true;
    }
    return false;
}

bool regs_strided_plan(int tbytes, int, int n, int *rpt, int *S, int *K, int pref_rpt, int max_warps)
{
    int r = tbytes == 4 ? kStridedRptF : kStridedRptD;
    if (tbytes == 4 && pref_rpt == kStridedRptF2) r = kStridedRptF2;
    if (n % r != 0) return false;
    const int mw = (max_warps >= 1 && max_warps <= 8) ? max_warps : 8;
    const int G = n / r;
    const int k = (G + mw - 1) / mw;  // at most mw warps per CTA
    if (k > 8) return false;          // portable cluster size
    *rpt = r;
    *S = (G + k - 1) / k;
    *K = k;
    return true;
}

bool rows_nb_plan(double d, int n, int rpt, int W)
{
    if (n != 32 * W * rpt || rpt < 16) return false;
    if (W == 2) return std::pow(d, (double)(rpt - 1)) <= std::ldexp(1.0, -27);          // one hop
    if (W == 4) return std::pow(d, (double)(2 * rpt - 1)) <= std::ldexp(1.0, -27);      // two hops
    return false;
}

bool regs_strided_nb_plan(double d, int n, int rpt)
{
    return (rpt == kStridedRptF || rpt == kStridedRptF2) && strided_nb_exact(d, n, rpt);
}

cudaError_t launch_strided_nb(int bc, int rpt, const AxisDev &A, const LineSet &L, const ProgParams &p, cudaStream_t s,
                              int stage)
{
    if (p.mode != 0 || !regs_strided_nb_plan(A.d, A.n, rpt) || stage < 0 || stage > 3) return cudaErrorInvalidValue;
    if (rpt == kStridedRptF)
        return bc == BC_PERIODIC ? run_strided_nb<BC_PERIODIC, kStridedRptF>(A, L, p, s, stage)
                                 : run_strided_nb<BC_DIRICHLET, kStridedRptF>(A, L, p, s, stage);
    return bc == BC_PERIODIC ? run_strided_nb<BC_PERIODIC, kStridedRptF2>(A, L, p, s, stage)
                             : run_strided_nb<BC_DIRICHLET, kStridedRptF2>(A, L, p, s, stage);
}

cudaError_t launch_strided_nb_T(int rpt, const AxisDev &A, const LineSet &L, const ProgParams &p, cudaStream_t s)
{
    if (p.mode != 2 || p.P < 1 || !regs_strided_nb_plan(A.d, A.n, rpt)) return cudaErrorInvalidValue;
    auto run = [&](auto kernel, int R) -> cudaError_t {
        static bool attr[2] = {false, false};
        bool &done = attr[R == kStridedRptF ? 0 : 1];
        if (!done) {
            const cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
            if (e != cudaSuccess) return e;
            done = true;
        }
        return launch_pass(kernel, dim3((unsigned)((L.nlines + 31) / 32), (unsigned)L.K, 1), dim3(32 * L.S, 1, 1),
                           strided_nb_slot_bytes(L.S), s, L, L.K, A, L, p, strided_nb_consts(A.d, R));
    };
    if (rpt == kStridedRptF) return run(k_strided_nb_T<kStridedRptF>, kStridedRptF);
    return run(k_strided_nb_T<kStridedRptF2>, kStridedRptF2);
}

cudaError_t launch_strided_nb_h(int bc, int rpt, const AxisDev &A, const LineSet &L, const ProgParams &p,
                                cudaStream_t s, bool gtile)
{
    if (p.mode != 1 || p.ng < 0 || p.ng > MAXG || p.nout < 1 || p.nout > MAXG || p.P < 1 ||
        !regs_strided_nb_plan(A.d, A.n, rpt))
        return cudaErrorInvalidValue;
    if (rpt == kStridedRptF)
        return bc == BC_PERIODIC ? run_strided_nb_h_any<BC_PERIODIC, kStridedRptF>(A, L, p, s, gtile)
                                 : run_strided_nb_h_any<BC_DIRICHLET, kStridedRptF>(A, L, p, s, gtile);
    return bc == BC_PERIODIC ? run_strided_nb_h_any<BC_PERIODIC, kStridedRptF2>(A, L, p, s, gtile)
                             : run_strided_nb_h_any<BC_DIRICHLET, kStridedRptF2>(A, L, p, s, gtile);
}

// One CTA waits on a barrier that is never completed (two arrivals expected,
// one made), bounded by `limit` cycles: the timeout path of every bounded
// wait, without a copy in flight.
__global__ void k_wait_selftest(long long limit)
{
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) mbar_init(&bar, 2);
    __syncthreads();
    if (threadIdx.x == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(&bar)) : "memory");
    __syncthreads();
    if (!mbar_wait_bounded(&bar, 0, limit) && threadIdx.x == 0) atomicExch(&g_molt_timeout, 1);
}

cudaError_t launch_wait_selftest(long long limit_cycles, cudaStream_t s)
{
    k_wait_selftest<<<1, 32, 0, s>>>(limit_cycles);
    return cudaGetLastError();
}

int regs_timeout_take(cudaStream_t s)
{
    int v = 0, zero = 0;
    if (cudaMemcpyFromSymbolAsync(&v, g_molt_timeout, sizeof(int), 0, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return -1;
    if (v != 0 && cudaMemcpyToSymbolAsync(g_molt_timeout, &zero, sizeof(int), 0, cudaMemcpyHostToDevice, s) != cudaSuccess)
        return -1;
    if (v != 0) cudaStreamSynchronize(s);
    return v;
}

size_t regs_strided_smem(int tbytes, int S, int rpt, bool horner)
{
    size_t b = strided_slot_bytes(S, (size_t)tbytes);
    if (horner) b += (size_t)S * rpt * 32 * tbytes;
    return b;
}

#define MOLT_CONTIG_R(T, BC)                                                             \
    switch (rpt) {                                                                       \
    case 8: return run_contig<T, BC, 8>(A, L, p, s);                                     \
    case 16: return run_contig<T, BC, 16>(A, L, p, s);                                   \
    case 32: return run_contig<T, BC, 32>(A, L, p, s);                                   \
    default: break;                                                                      \
    }

cudaError_t launch_contig(int tbytes, int bc, int rpt, const AxisDev &A, const LineSet &L, const ProgParams &p,
                          cudaStream_t s)
{
    if (tbytes == 4) {
        if (bc == BC_PERIODIC) {
            MOLT_CONTIG_R(float, BC_PERIODIC)
            if (rpt == 64) return run_contig<float, BC_PERIODIC, 64>(A, L, p, s);
        } else {
            MOLT_CONTIG_R(float, BC_DIRICHLET)
            if (rpt == 64) return run_contig<float, BC_DIRICHLET, 64>(A, L, p, s);
        }
    } else {
        if (bc == BC_PERIODIC) { MOLT_CONTIG_R(double, BC_PERIODIC) }
        else { MOLT_CONTIG_R(double, BC_DIRICHLET) }
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_strided(int tbytes, int bc, int rpt, const AxisDev &A, const LineSet &L, const ProgParams &p,
                           cudaStream_t s)
{
    if (tbytes == 4 && rpt == kStridedRptF)
        return bc == BC_PERIODIC ? run_strided<float, BC_PERIODIC, kStridedRptF>(A, L, p, s)
                                 : run_strided<float, BC_DIRICHLET, kStridedRptF>(A, L, p, s);
    if (tbytes == 4 && rpt == kStridedRptF2)
        return bc == BC_PERIODIC ? run_strided<float, BC_PERIODIC, kStridedRptF2>(A, L, p, s)
                                 : run_strided<float, BC_DIRICHLET, kStridedRptF2>(A, L, p, s);
    if (tbytes == 8 && rpt == kStridedRptD)
        return bc == BC_PERIODIC ? run_strided<double, BC_PERIODIC, kStridedRptD>(A, L, p, s)
                                 : run_strided<double, BC_DIRICHLET, kStridedRptD>(A, L, p, s);
    return cudaErrorInvalidValue;
}

// float32 Horner pass with the fields resident: up to 3 fields
bool regs_res_plan(int tbytes, int n, int ng, int *rpt)
{
    if (tbytes != 4 || ng > 3) return false;
    for (int r = 8; r <= 64; r *= 2) {
        if (32 * r < n) continue;
        if (n % r != 0) return false;
        *rpt = r;
        return true;
    }
    return false;
}

cudaError_t launch_res(int bc, int rpt, int ng, int warps, const AxisDev &A, const LineSet &L, const ProgParams &p,
                       cudaStream_t s)
{
    if (warps < 1 || warps > kResWarpsMax) warps = 2;
#define MOLT_RES(BC)                                                                      \
    switch (rpt * 10 + (ng < 1 ? 1 : ng)) {                                               \
    case 81: return run_res<BC, 8, 1>(warps, A, L, p, s);                                 \
    case 82: return run_res<BC, 8, 2>(warps, A, L, p, s);                                 \
    case 83: return run_res<BC, 8, 3>(warps, A, L, p, s);                                 \
    case 161: return run_res<BC, 16, 1>(warps, A, L, p, s);                               \
    case 162: return run_res<BC, 16, 2>(warps, A, L, p, s);                               \
    case 163: return run_res<BC, 16, 3>(warps, A, L, p, s);                               \
    case 321: return run_res<BC, 32, 1>(warps, A, L, p, s);                               \
    case 322: return run_res<BC, 32, 2>(warps, A, L, p, s);                               \
    case 323: return run_res<BC, 32, 3>(warps, A, L, p, s);                               \
    case 641: return run_res<BC, 64, 1>(warps, A, L, p, s);                               \
    case 642: return run_res<BC, 64, 2>(warps, A, L, p, s);                               \
    case 643: return run_res<BC, 64, 3>(warps, A, L, p, s);                               \
    default: break;                                                                       \
    }
    if (bc == BC_PERIODIC) { MOLT_RES(BC_PERIODIC) }
    else { MOLT_RES(BC_DIRICHLET) }
#undef MOLT_RES
    return cudaErrorInvalidValue;
}

// float32 Horner pass with W warps per row: n = 32 W RPT exactly, RPT 16 or 32
bool regs_rows_plan(int tbytes, int n, int ng, int W, int *rpt)
{
    if (tbytes != 4 || ng > 3 || (W != 2 && W != 4 && W != 8) || n % (32 * W) != 0) return false;
    const int r = n / (32 * W);
    if (W == 8 ? (r != 8 && r != 16) : (r != 16 && r != 32)) return false;
    *rpt = r;
    return true;
}

cudaError_t launch_rows(int bc, int rpt, int ng, int W, const AxisDev &A, const LineSet &L, const ProgParams &p,
                        cudaStream_t s)
{
#define MOLT_ROWS(BC, WW, R1, R2)                                                         \
    switch (rpt * 10 + (ng < 1 ? 1 : ng)) {                                               \
    case R1 * 10 + 1: return run_rows<BC, R1, 1, WW>(A, L, p, s);                         \
    case R1 * 10 + 2: return run_rows<BC, R1, 2, WW>(A, L, p, s);                         \
    case R1 * 10 + 3: return run_rows<BC, R1, 3, WW>(A, L, p, s);                         \
    case R2 * 10 + 1: return run_rows<BC, R2, 1, WW>(A, L, p, s);                         \
    case R2 * 10 + 2: return run_rows<BC, R2, 2, WW>(A, L, p, s);                         \
    case R2 * 10 + 3: return run_rows<BC, R2, 3, WW>(A, L, p, s);                         \
    default: break;                                                                       \
    }
    if (W == 2) {
        if (bc == BC_PERIODIC) { MOLT_ROWS(BC_PERIODIC, 2, 16, 32) } else { MOLT_ROWS(BC_DIRICHLET, 2, 16, 32) }
    } else if (W == 4) {
        if (bc == BC_PERIODIC) { MOLT_ROWS(BC_PERIODIC, 4, 16, 32) } else { MOLT_ROWS(BC_DIRICHLET, 4, 16, 32) }
    } else if (W == 8) {
        if (bc == BC_PERIODIC) { MOLT_ROWS(BC_PERIODIC, 8, 8, 16) } else { MOLT_ROWS(BC_DIRICHLET, 8, 8, 16) }
    }
#undef MOLT_ROWS
    return cudaErrorInvalidValue;
}

cudaError_t configure_regs_kernels()
{
    cudaError_t e;
#define MOLT_A(x) if ((e = (x)) != cudaSuccess) return e;
#define MOLT_ROWA(BC, WW, R1, R2) MOLT_A((attr_rows<BC, R1, 1, WW>())) MOLT_A((attr_rows<BC, R1, 2, WW>())) \
    MOLT_A((attr_rows<BC, R1, 3, WW>())) MOLT_A((attr_rows<BC, R2, 1, WW>())) MOLT_A((attr_rows<BC, R2, 2, WW>())) \
    MOLT_A((attr_rows<BC, R2, 3, WW>()))
    MOLT_ROWA(BC_PERIODIC, 2, 16, 32) MOLT_ROWA(BC_DIRICHLET, 2, 16, 32) MOLT_ROWA(BC_PERIODIC, 4, 16, 32)
    MOLT_ROWA(BC_DIRICHLET, 4, 16, 32) MOLT_ROWA(BC_PERIODIC, 8, 8, 16) MOLT_ROWA(BC_DIRICHLET, 8, 8, 16)
#undef MOLT_ROWA
#define MOLT_RA(BC) MOLT_A((attr_res<BC, 8, 1>())) MOLT_A((attr_res<BC, 8, 2>())) MOLT_A((attr_res<BC, 8, 3>())) \
    MOLT_A((attr_res<BC, 16, 1>())) MOLT_A((attr_res<BC, 16, 2>())) MOLT_A((attr_res<BC, 16, 3>()))             \
    MOLT_A((attr_res<BC, 32, 1>())) MOLT_A((attr_res<BC, 32, 2>())) MOLT_A((attr_res<BC, 32, 3>()))             \
    MOLT_A((attr_res<BC, 64, 1>())) MOLT_A((attr_res<BC, 64, 2>())) MOLT_A((attr_res<BC, 64, 3>()))
    MOLT_RA(BC_PERIODIC) MOLT_RA(BC_DIRICHLET)
#undef MOLT_RA
    MOLT_A((attr_contig<float, BC_PERIODIC, 8>())) MOLT_A((attr_contig<float, BC_PERIODIC, 16>()))
    MOLT_A((attr_contig<float, BC_PERIODIC, 32>())) MOLT_A((attr_contig<float, BC_PERIODIC, 64>()))
    MOLT_A((attr_contig<float, BC_DIRICHLET, 8>())) MOLT_A((attr_contig<float, BC_DIRICHLET, 16>()))
    MOLT_A((attr_contig<float, BC_DIRICHLET, 32>())) MOLT_A((attr_contig<float, BC_DIRICHLET, 64>()))
    MOLT_A((attr_contig<double, BC_PERIODIC, 8>())) MOLT_A((attr_contig<double, BC_PERIODIC, 16>()))
    MOLT_A((attr_contig<double, BC_PERIODIC, 32>()))
    MOLT_A((attr_contig<double, BC_DIRICHLET, 8>())) MOLT_A((attr_contig<double, BC_DIRICHLET, 16>()))
    MOLT_A((attr_contig<double, BC_DIRICHLET, 32>()))
    MOLT_A((attr_strided<float, BC_PERIODIC, kStridedRptF>())) MOLT_A((attr_strided<float, BC_DIRICHLET, kStridedRptF>()))
    MOLT_A((attr_strided<float, BC_PERIODIC, kStridedRptF2>())) MOLT_A((attr_strided<float, BC_DIRICHLET, kStridedRptF2>()))
    MOLT_A((attr_strided<double, BC_PERIODIC, kStridedRptD>())) MOLT_A((attr_strided<double, BC_DIRICHLET, kStridedRptD>()))
#undef MOLT_A
    return cudaSuccess;
}

}  // namespace molt
