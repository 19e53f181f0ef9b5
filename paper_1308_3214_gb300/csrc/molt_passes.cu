// molt_passes.cu -- instantiation and launch of the pass kernels.
#include "molt_internal.h"

namespace molt {

__global__ void k_to_pair(const double *__restrict__ x, float *__restrict__ hi, float *__restrict__ lo, int64_t N)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
        float h, l;
        split_pair(x[i], h, l);
        hi[i] = h;
        lo[i] = l;
    }
}

__global__ void k_from_pair(const float *__restrict__ hi, const float *__restrict__ lo, double *__restrict__ x, int64_t N)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x)
        x[i] = join_pair(hi[i], lo[i]);
}

__global__ void k_from_f32(const float *__restrict__ f, double *__restrict__ x, int64_t N)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x)
        x[i] = (double)f[i];
}

// The same conversions four points per thread (two 16-byte float64 loads or
// stores, one 16-byte float32 store or load per plane), for 16-byte aligned
// fields; the last N % 4 points by the scalar form.
__device__ __forceinline__ void to_pair4(const double *__restrict__ x, float *__restrict__ hi, float *__restrict__ lo,
                                         int64_t N)
{
    const int64_t n4 = N >> 2;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n4; i += (int64_t)gridDim.x * blockDim.x) {
        const double2 a = reinterpret_cast<const double2 *>(x)[2 * i];
        const double2 b = reinterpret_cast<const double2 *>(x)[2 * i + 1];
        float4 h, l;
        split_pair(a.x, h.x, l.x);
        split_pair(a.y, h.y, l.y);
        split_pair(b.x, h.z, l.z);
        split_pair(b.y, h.w, l.w);
        reinterpret_cast<float4 *>(hi)[i] = h;
        reinterpret_cast<float4 *>(lo)[i] = l;
    }
    const int64_t t = 4 * n4 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t < N) {
        float h, l;
        split_pair(x[t], h, l);
        hi[t] = h;
        lo[t] = l;
    }
}

__device__ __forceinline__ void from_pair4(const float *__restrict__ hi, const float *__restrict__ lo,
                                           double *__restrict__ x, int64_t N)
{
    const int64_t n4 = N >> 2;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n4; i += (int64_t)gridDim.x * blockDim.x) {
        const float4 h = reinterpret_cast<const float4 *>(hi)[i];
        const float4 l = reinterpret_cast<const float4 *>(lo)[i];
        reinterpret_cast<double2 *>(x)[2 * i] =
            make_double2(join_pair(h.x, l.x), join_pair(h.y, l.y));
        reinterpret_cast<double2 *>(x)[2 * i + 1] =
            make_double2(join_pair(h.z, l.z), join_pair(h.w, l.w));
    }
    const int64_t t = 4 * n4 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t < N) x[t] = join_pair(hi[t], lo[t]);
}

__global__ void k_to_pair4(const double *__restrict__ x, float *__restrict__ hi, float *__restrict__ lo, int64_t N)
{
    to_pair4(x, hi, lo, N);
}

__global__ void k_from_pair4(const float *__restrict__ hi, const float *__restrict__ lo, double *__restrict__ x, int64_t N)
{
    from_pair4(hi, lo, x, N);
}

// Two levels in one launch (blockIdx.y = the level): the two conversions at
// each end of a time-stepping call share one launch's ramp and tail.
struct PairFields2 {
    const double *x[2];
    double *xo[2];
    float *hi[2];
    float *lo[2];
};

__global__ void k_to_pair4_2(const PairFields2 f, int64_t N)
{
    const bool k = blockIdx.y != 0;                // selects, so that f stays in the parameter space
    to_pair4(k ? f.x[1] : f.x[0], k ? f.hi[1] : f.hi[0], k ? f.lo[1] : f.lo[0], N);
}

__global__ void k_from_pair4_2(const PairFields2 f, int64_t N)
{
    const bool k = blockIdx.y != 0;
    from_pair4(k ? f.hi[1] : f.hi[0], k ? f.lo[1] : f.lo[0], k ? f.xo[1] : f.xo[0], N);
}

static int elementwise_grid(int64_t N)
{
    int64_t g = (N + 255) / 256;
    return (int)(g < 152 * 16 ? (g < 1 ? 1 : g) : 152 * 16);
}

static bool aligned16(const void *a, const void *b, const void *c)
{
    return (((uintptr_t)a | (uintptr_t)b | (uintptr_t)c) & 15) == 0;
}

cudaError_t launch_to_pair(const double *x, float *hi, float *lo, int64_t N, cudaStream_t s)
{
    if (aligned16(x, hi, lo)) k_to_pair4<<<elementwise_grid((N + 3) / 4), 256, 0, s>>>(x, hi, lo, N);
    else k_to_pair<<<elementwise_grid(N), 256, 0, s>>>(x, hi, lo, N);
    return cudaGetLastError();
}
cudaError_t launch_from_pair(const float *hi, const float *lo, double *x, int64_t N, cudaStream_t s)
{
    if (aligned16(x, hi, lo)) k_from_pair4<<<elementwise_grid((N + 3) / 4), 256, 0, s>>>(hi, lo, x, N);
    else k_from_pair<<<elementwise_grid(N), 256, 0, s>>>(hi, lo, x, N);
    return cudaGetLastError();
}
cudaError_t launch_to_pair2(const double *x0, float *hi0, float *lo0, const double *x1, float *hi1, float *lo1,
                            int64_t N, cudaStream_t s)
{
    if (!(aligned16(x0, hi0, lo0) && aligned16(x1, hi1, lo1))) {
        cudaError_t e = launch_to_pair(x0, hi0, lo0, N, s);
        return e != cudaSuccess ? e : launch_to_pair(x1, hi1, lo1, N, s);
    }
    const PairFields2 f = {{x0, x1}, {nullptr, nullptr}, {hi0, hi1}, {lo0, lo1}};
    k_to_pair4_2<<<dim3(elementwise_grid((N + 3) / 4), 2), 256, 0, s>>>(f, N);
    return cudaGetLastError();
}

cudaError_t launch_from_pair2(const float *hi0, const float *lo0, double *x0, const float *hi1, const float *lo1,
                              double *x1, int64_t N, cudaStream_t s)
{
    if (!(aligned16(x0, hi0, lo0) && aligned16(x1, hi1, lo1))) {
        cudaError_t e = launch_from_pair(hi0, lo0, x0, N, s);
        return e != cudaSuccess ? e : launch_from_pair(hi1, lo1, x1, N, s);
    }
    const PairFields2 f = {{nullptr, nullptr}, {x0, x1}, {const_cast<float *>(hi0), const_cast<float *>(hi1)},
                           {const_cast<float *>(lo0), const_cast<float *>(lo1)}};
    k_from_pair4_2<<<dim3(elementwise_grid((N + 3) / 4), 2), 256, 0, s>>>(f, N);
    return cudaGetLastError();
}

cudaError_t launch_from_f32(const float *f, double *x, int64_t N, cudaStream_t s)
{
    k_from_f32<<<elementwise_grid(N), 256, 0, s>>>(f, x, N);
    return cudaGetLastError();
}

int line_stride(int ms, int W, int tbytes)
{
    // bank-conflict-free transposing stores: ls == 32/W (mod 32) for 4-byte
    // words, ls == 16/W (mod 16) in 8-byte words
    int base = 32 * ms;
    if (tbytes == 4) return base + (W <= 32 ? 32 / W : 1);
    return base + (W <= 16 ? 16 / W : 1);
}

size_t pass_smem_bytes(bool horner, int tbytes, int W, int ls, int n, int dps)
{
    return smem_layout(horner ? 2 : 1, W, ls, n, (size_t)tbytes, dps).total;
}

template <class T, int BC, bool CONTIG>
static cudaError_t set_attr()
{
    cudaError_t e = cudaFuncSetAttribute(k_powers<T, BC, CONTIG>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(k_horner<T, BC, CONTIG>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
}

cudaError_t configure_kernels()
{
    cudaError_t e;
#define MOLT_SET(T, BC, C) if ((e = set_attr<T, BC, C>()) != cudaSuccess) return e;
    MOLT_SET(float, BC_PERIODIC, true) MOLT_SET(float, BC_PERIODIC, false)
    MOLT_SET(float, BC_DIRICHLET, true) MOLT_SET(float, BC_DIRICHLET, false)
    MOLT_SET(double, BC_PERIODIC, true) MOLT_SET(double, BC_PERIODIC, false)
    MOLT_SET(double, BC_DIRICHLET, true) MOLT_SET(double, BC_DIRICHLET, false)
#undef MOLT_SET
    return cudaSuccess;
}

// Threads of a shared-memory pass CTA: one warp per line for the sweeps; a
// contiguous-axis grid of one CTA (a single line or a few) takes 512 threads,
// so that its loads, stores and per-point phases run over 16 warps while the
// sweeps stay on the lines' own warps.
template <bool CONTIG>
static int pass_threads(const PassGeom &G)
{
    return (G.cta || (CONTIG && G.nlines <= G.W && G.W < 16)) ? kCtaLineThreads : 32 * G.W;
}

template <class T, int BC, bool CONTIG>
static cudaError_t run_powers(const AxisDev &A, const PassGeom &G, const PowersParams &p, cudaStream_t s)
{
    const size_t smem = pass_smem_bytes(false, sizeof(T), G.W, A.ls, A.n, G.dps);
    const int64_t grid = (G.nlines + G.W - 1) / G.W;
    k_powers<T, BC, CONTIG><<<(unsigned)grid, pass_threads<CONTIG>(G), smem, s>>>(A, G, p);
    return cudaGetLastError();
}

template <class T, int BC, bool CONTIG>
static cudaError_t run_horner(const AxisDev &A, const PassGeom &G, const HornerParams &p, cudaStream_t s)
{
    const size_t smem = pass_smem_bytes(true, sizeof(T), G.W, A.ls, A.n, G.dps);
    const int64_t grid = (G.nlines + G.W - 1) / G.W;
    k_horner<T, BC, CONTIG><<<(unsigned)grid, pass_threads<CONTIG>(G), smem, s>>>(A, G, p);
    return cudaGetLastError();
}

#define MOLT_DISPATCH(FN, ...)                                                                   \
    do {                                                                                         \
        if (tbytes == 4) {                                                                       \
            if (bc == BC_PERIODIC) return contig ? FN<float, BC_PERIODIC, true>(__VA_ARGS__)     \
                                                 : FN<float, BC_PERIODIC, false>(__VA_ARGS__);   \
            return contig ? FN<float, BC_DIRICHLET, true>(__VA_ARGS__)                           \
                          : FN<float, BC_DIRICHLET, false>(__VA_ARGS__);                         \
        }                                                                                        \
        if (bc == BC_PERIODIC) return contig ? FN<double, BC_PERIODIC, true>(__VA_ARGS__)        \
                                             : FN<double, BC_PERIODIC, false>(__VA_ARGS__);      \
        return contig ? FN<double, BC_DIRICHLET, true>(__VA_ARGS__)                              \
                      : FN<double, BC_DIRICHLET, false>(__VA_ARGS__);                            \
    } while (0)

cudaError_t launch_powers(int tbytes, int bc, bool contig, const AxisDev &A, const PassGeom &G,
                          const PowersParams &p, cudaStream_t s)
{
    MOLT_DISPATCH(run_powers, A, G, p, s);
}

cudaError_t launch_horner(int tbytes, int bc, bool contig, const AxisDev &A, const PassGeom &G,
                          const HornerParams &p, cudaStream_t s)
{
    MOLT_DISPATCH(run_horner, A, G, p, s);
}

}  // namespace molt
