// molt_tma.cuh -- tensor-memory-access (TMA) tiles and mbarriers for the
// strided passes (sm_103a): tiled bulk-tensor copies between global memory
// and shared memory, their completion barriers, and a bounded wait that
// reports through a device flag instead of spinning forever.
#pragma once
#include <cuda.h>
#include <cstdint>

namespace molt {

// Set (to 1) by any kernel of this translation unit whose bounded wait gave
// up; read and cleared by the host (regs_timeout_take, molt_regs.cu).  A wait
// that gives up lets the kernel run on to its normal end (every CTA of a
// cluster still reaches every cluster barrier), so the results of that launch
// are garbage and the call reports MOL_ETIMEOUT.
static __device__ int g_molt_timeout;

// ~2 s at the GB300's 2 GHz SM clock: far beyond any tile copy of a healthy GPU
constexpr long long kTmaWaitCycles = 4000000000LL;

__device__ __forceinline__ uint32_t smem_addr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n"
        ".reg .pred p;\n"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        "selp.u32 %0, 1, 0, p;\n"
        "}\n"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Wait for phase `parity` of the barrier for at most `limit` cycles.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity, long long limit = kTmaWaitCycles)
{
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity))
        if (clock64() - t0 > limit) return false;
    return true;
}

// Wait, and on a timeout raise the flag and wait once more (bounded) for the
// copies still in flight, so that the CTA's shared memory is not released
// under them.
__device__ __forceinline__ void mbar_wait_or_flag(uint64_t *bar, uint32_t parity)
{
    if (mbar_wait_bounded(bar, parity)) return;
    atomicExch(&g_molt_timeout, 1);
    mbar_wait_bounded(bar, parity);
}

// 3D tiled load global -> this CTA's shared memory, completing on `bar`.
__device__ __forceinline__ void tma_load_3d(void *dst, const CUtensorMap *map, int x, int y, int z, uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];"
        ::"r"(smem_addr(dst)), "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(smem_addr(bar))
        : "memory");
}

// 3D tiled store shared memory -> global (bulk group of the issuing thread).
__device__ __forceinline__ void tma_store_3d(const CUtensorMap *map, int x, int y, int z, const void *src)
{
    asm volatile("cp.async.bulk.tensor.3d.global.shared::cta.bulk_group [%0, {%1, %2, %3}], [%4];"
                 ::"l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(smem_addr(src))
                 : "memory");
}

__device__ __forceinline__ void tma_store_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
// the issuing thread's stores have finished reading shared memory
__device__ __forceinline__ void tma_store_wait_read() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }
// ... and have completed
__device__ __forceinline__ void tma_store_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }
// generic-proxy writes to shared memory become visible to the TMA unit
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// Tensor maps of one strided pass: the pair level (inputs) and up to kMaxTmaOut
// outputs, a 3D view {inner, n, outer} of each float32 field with boxes of
// {32 lines, box_rows points, 1}.
constexpr int kMaxTmaOut = 5;
struct TmaMaps {
    CUtensorMap in_hi, in_lo;
    CUtensorMap out[kMaxTmaOut];
    int box_rows;   // rows of one box
    int nbox;       // boxes per tile
};

// Tensor maps of the input fields of a strided Horner pass (the same 3D view
// and boxes), for its tiles staged in shared memory.
constexpr int kMaxTmaG = 5;
struct TmaGMaps {
    CUtensorMap g[kMaxTmaG];
    int box_rows;   // rows of one box
    int nbox;       // boxes per field
};

}  // namespace molt
