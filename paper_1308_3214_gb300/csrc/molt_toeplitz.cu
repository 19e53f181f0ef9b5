// molt_toeplitz.cu -- measurement of a design alternative for the strided
// sweeps (sm_103a); the paper has no counterpart.
//
// A sweep's causal recurrence, taken chunk by chunk with zero inflow,
// y_i = d y_{i-1} + q_i on 32 consecutive points, is the product y = T q with
// the 32 x 32 lower-triangular Toeplitz matrix T_ij = d^(i-j) (Sec. 2: the
// recursive form of the convolution with the kernel e^{-alpha|x - y|}).  The
// carries between chunks and the anti-causal half are the same in either
// form, so this file times only the part a tensor core could take over:
//   variant 0: the in-register scan the pass kernels use (lane = column, each
//              thread 32 points, the two halves as two chains);
//   variant 1: 32 x 32 tiles (32 points of 32 neighbouring columns) times T on
//              the tensor cores with mma.sync m16n8k8 TF32; every operand is
//              split into a TF32 head and tail and the three products
//              A_h B_h + A_h B_t + A_t B_h keep float32 accuracy.
// Both read q and write y once (8 bytes per point) over a row-major field of
// nrows x ncols float32 values, chunks along the rows.
#include <cmath>
#include <cstdint>
#include <cstring>
#include <string>

#include "molt.h"
#include "molt_internal.h"

namespace molt {
namespace {

constexpr int kTileStride = 36;   // shared-memory row stride: the B fragments' banks 4 tig + g are distinct

__device__ __forceinline__ uint32_t to_tf32(float x)
{
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return r;
}

__device__ __forceinline__ void mma_tf32(float (&c)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1)
{
    asm volatile(
        "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, "
        "{%0, %1, %2, %3};"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// one warp per 32 x 32 chunk; warp w: column group w % groups, chunk w / groups
__global__ void __launch_bounds__(128) k_chunk_scan(const float *__restrict__ q, float *__restrict__ y, int nrows,
                                                    int ncols, float d)
{
    const int warp = blockIdx.x * 4 + (threadIdx.x >> 5), lane = threadIdx.x & 31;
    const int groups = ncols / 32;
    if (warp >= groups * (nrows / 32)) return;
    const size_t base = (size_t)(warp / groups) * 32 * ncols + (size_t)(warp % groups) * 32 + lane;
    float v[32];
#pragma unroll
    for (int k = 0; k < 32; ++k) v[k] = q[base + (size_t)k * ncols];
    float a = 0.f, b = 0.f;
#pragma unroll
    for (int k = 0; k < 16; ++k) {
        a = d * a + v[k];
        b = d * b + v[16 + k];
        v[k] = a;
        v[16 + k] = b;
    }
    float p = d;                                     // the second half's inflow: a (= y_15) times d^(k+1)
#pragma unroll
    for (int k = 0; k < 16; ++k) {
        v[16 + k] += a * p;
        p *= d;
    }
#pragma unroll
    for (int k = 0; k < 32; ++k) y[base + (size_t)k * ncols] = v[k];
}

__global__ void __launch_bounds__(128) k_chunk_toeplitz(const float *__restrict__ q, float *__restrict__ y, int nrows,
                                                        int ncols, float d)
{
    __shared__ float tile[4][32 * kTileStride];
    const int warp = blockIdx.x * 4 + (threadIdx.x >> 5), lane = threadIdx.x & 31;
    const int groups = ncols / 32;
    if (warp >= groups * (nrows / 32)) return;
    float *t = tile[threadIdx.x >> 5];
    const size_t base = (size_t)(warp / groups) * 32 * ncols + (size_t)(warp % groups) * 32 + lane;
#pragma unroll
    for (int k = 0; k < 32; ++k) t[k * kTileStride + lane] = q[base + (size_t)k * ncols];
    __syncwarp();

    const int gid = lane >> 2, tig = lane & 3;
    // powers d^0 .. d^31 for the A fragments of T (rows 16 mb + gid (+8), columns 8 kb + tig (+4))
    float dp[32];
    dp[0] = 1.f;
#pragma unroll
    for (int k = 1; k < 32; ++k) dp[k] = dp[k - 1] * d;
    auto tval = [&](int i, int j) { return i >= j ? dp[i - j] : 0.f; };

    float acc[2][4][4];
#pragma unroll
    for (int mb = 0; mb < 2; ++mb)
#pragma unroll
        for (int nb = 0; nb < 4; ++nb)
#pragma unroll
            for (int r = 0; r < 4; ++r) acc[mb][nb][r] = 0.f;

#pragma unroll
    for (int kb = 0; kb < 4; ++kb) {
        uint32_t bh[4][2], bt[4][2];
#pragma unroll
        for (int nb = 0; nb < 4; ++nb) {
            const float b0 = t[(8 * kb + tig) * kTileStride + 8 * nb + gid];
            const float b1 = t[(8 * kb + tig + 4) * kTileStride + 8 * nb + gid];
            bh[nb][0] = to_tf32(b0);
            bh[nb][1] = to_tf32(b1);
            bt[nb][0] = to_tf32(b0 - __uint_as_float(bh[nb][0]));
            bt[nb][1] = to_tf32(b1 - __uint_as_float(bh[nb][1]));
        }
#pragma unroll
        for (int mb = 0; mb < 2; ++mb) {
            if (8 * kb > 16 * mb + 15) continue;      // block above the diagonal: zero
            const int r0 = 16 * mb + gid, c0 = 8 * kb + tig;
            const float av[4] = {tval(r0, c0), tval(r0 + 8, c0), tval(r0, c0 + 4), tval(r0 + 8, c0 + 4)};
            uint32_t ah[4], at[4];
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                ah[r] = to_tf32(av[r]);
                at[r] = to_tf32(av[r] - __uint_as_float(ah[r]));
            }
#pragma unroll
            for (int nb = 0; nb < 4; ++nb) {
                mma_tf32(acc[mb][nb], at, bh[nb][0], bh[nb][1]);
                mma_tf32(acc[mb][nb], ah, bt[nb][0], bt[nb][1]);
                mma_tf32(acc[mb][nb], ah, bh[nb][0], bh[nb][1]);
            }
        }
    }
    __syncwarp();
#pragma unroll
    for (int mb = 0; mb < 2; ++mb)
#pragma unroll
        for (int nb = 0; nb < 4; ++nb) {
            const int r0 = 16 * mb + gid, c0 = 8 * nb + 2 * tig;
            t[r0 * kTileStride + c0] = acc[mb][nb][0];
            t[r0 * kTileStride + c0 + 1] = acc[mb][nb][1];
            t[(r0 + 8) * kTileStride + c0] = acc[mb][nb][2];
            t[(r0 + 8) * kTileStride + c0 + 1] = acc[mb][nb][3];
        }
    __syncwarp();
#pragma unroll
    for (int k = 0; k < 32; ++k) y[base + (size_t)k * ncols] = t[k * kTileStride + lane];
}

__global__ void k_fill_uniform(float *x, int64_t n, uint64_t seed)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        uint64_t z = seed + 0x9E3779B97F4A7C15ull * (uint64_t)(i + 1);     // splitmix64
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        z ^= z >> 31;
        x[i] = (float)((double)(z >> 11) * (1.0 / 9007199254740992.0)) * 2.f - 1.f;
    }
}

__global__ void k_max_rel_diff(const float *a, const float *b, int64_t n, unsigned *diff_bits, unsigned *max_bits)
{
    float dm = 0.f, am = 0.f;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        dm = fmaxf(dm, fabsf(a[i] - b[i]));
        am = fmaxf(am, fabsf(a[i]));
    }
    atomicMax(diff_bits, __float_as_uint(dm));      // non-negative floats order as their bit patterns
    atomicMax(max_bits, __float_as_uint(am));
}

}  // namespace
}  // namespace molt

using namespace molt;

extern "C" mol_status mol_toeplitz_experiment(int nrows, int ncols, double d, int reps, double ms_per_launch[2],
                                              double *max_rel_diff, void *stream)
{
    if (nrows < 32 || ncols < 32 || nrows % 32 || ncols % 32 || !(d > 0.0 && d < 1.0) || reps < 1 || !ms_per_launch ||
        !max_rel_diff) {
        set_global_error("need nrows, ncols multiples of 32, 0 < d < 1, reps >= 1, output pointers");
        return MOL_EINVAL;
    }
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t n = (int64_t)nrows * ncols;
    float *q = nullptr, *y0 = nullptr, *y1 = nullptr;
    unsigned *bits = nullptr;
    mol_status st = MOL_OK;
    auto ck = [&](cudaError_t e, const char *what) {
        if (e == cudaSuccess || st != MOL_OK) return;
        cudaGetLastError();
        set_global_error(std::string(what) + ": " + cudaGetErrorString(e));
        st = (e == cudaErrorMemoryAllocation) ? MOL_ENOMEM : MOL_ECUDA;
    };
    ck(cudaMalloc(&q, sizeof(float) * n), "allocation");
    ck(cudaMalloc(&y0, sizeof(float) * n), "allocation");
    ck(cudaMalloc(&y1, sizeof(float) * n), "allocation");
    ck(cudaMalloc(&bits, 2 * sizeof(unsigned)), "allocation");
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    ck(cudaEventCreate(&e0), "event");
    ck(cudaEventCreate(&e1), "event");
    const int warps = (ncols / 32) * (nrows / 32), blocks = (warps + 3) / 4;
    const float fd = (float)d;
    if (st == MOL_OK) {
        k_fill_uniform<<<1024, 256, 0, s>>>(q, n, 0x5eedull);
        ck(cudaGetLastError(), "fill");
        for (int v = 0; v < 2 && st == MOL_OK; ++v) {
            auto launch = [&]() {
                if (v == 0) k_chunk_scan<<<blocks, 128, 0, s>>>(q, y0, nrows, ncols, fd);
                else k_chunk_toeplitz<<<blocks, 128, 0, s>>>(q, y1, nrows, ncols, fd);
            };
            for (int w = 0; w < 3; ++w) launch();
            ck(cudaEventRecord(e0, s), "event");
            for (int r = 0; r < reps; ++r) launch();
            ck(cudaEventRecord(e1, s), "event");
            ck(cudaEventSynchronize(e1), "synchronize");
            float ms = 0.f;
            ck(cudaEventElapsedTime(&ms, e0, e1), "elapsed");
            ms_per_launch[v] = (double)ms / reps;
        }
        ck(cudaMemsetAsync(bits, 0, 2 * sizeof(unsigned), s), "memset");
        k_max_rel_diff<<<1024, 256, 0, s>>>(y1, y0, n, bits, bits + 1);
        ck(cudaGetLastError(), "compare");
        unsigned hb[2] = {0, 0};
        ck(cudaMemcpyAsync(hb, bits, sizeof hb, cudaMemcpyDeviceToHost, s), "copy");
        ck(cudaStreamSynchronize(s), "synchronize");
        float df, am;
        std::memcpy(&df, &hb[0], 4);
        std::memcpy(&am, &hb[1], 4);
        *max_rel_diff = am > 0.f ? (double)df / (double)am : 0.0;
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(q);
    cudaFree(y0);
    cudaFree(y1);
    cudaFree(bits);
    return st;
}
