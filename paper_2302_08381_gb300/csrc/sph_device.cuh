// Device helpers: bulk (TMA) copies between shared and global memory,
// mbarriers with bounded waits, proxy fences, output conversions.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace sph {

// Device status bits (OR-ed into the per-device status word).
constexpr uint32_t kStatusLoadTimeout = 1u;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// Make this thread's generic-proxy shared-memory writes visible to the async
// proxy (bulk copies) -- every writing thread runs it before the issuing sync.
__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// Bulk copy shared -> global (TMA, no tensor map). Both addresses 16-byte
// aligned, size a multiple of 16. Completion tracked by bulk groups of the
// issuing thread.
__device__ __forceinline__ void bulk_store(void* gdst, const void* ssrc, uint32_t bytes) {
    asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;"
                 :
                 : "l"(gdst), "r"(smem_u32(ssrc)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
// Wait until all committed bulk stores of this thread have finished READING
// shared memory (the buffer may then be overwritten).
__device__ __forceinline__ void bulk_wait_read_all() {
    asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
}
// Wait until all committed bulk stores of this thread are complete.
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }

// ---------------------------------------------------------------- mbarrier
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_inval(uint64_t* bar) {
    asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}
// Bulk copy global -> shared completing `bytes` of transaction on `bar`.
__device__ __forceinline__ void bulk_load(void* sdst, const void* gsrc, uint32_t bytes, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
        :
        : "r"(smem_u32(sdst)), "l"(gsrc), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}
// Hint: bring `bytes` of global memory at `gsrc` into L2 (16-byte aligned
// address, size a multiple of 16; no completion to wait for).
__device__ __forceinline__ void bulk_prefetch_l2(const void* gsrc, uint32_t bytes) {
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(gsrc), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// Bounded wait on phase `parity`: gives up after `limit` polls (each poll may
// suspend the thread for a hardware-defined interval). Returns false on
// timeout so the caller can flag it and skip the dependent work.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, uint32_t limit) {
    for (uint32_t i = 0; i < limit; ++i) {
        if (mbar_try_wait(bar, parity)) return true;
    }
    return false;
}

// ------------------------------------------------------------- conversions
template <typename TO>
struct OutConv;
template <>
struct OutConv<float> {
    template <typename T>
    __device__ __forceinline__ static float cv(T v) { return static_cast<float>(v); }
};
template <>
struct OutConv<double> {
    template <typename T>
    __device__ __forceinline__ static double cv(T v) { return static_cast<double>(v); }
};
template <>
struct OutConv<__nv_bfloat16> {
    template <typename T>
    __device__ __forceinline__ static __nv_bfloat16 cv(T v) { return __float2bfloat16_rn(static_cast<float>(v)); }
};

// Warp-cooperative element copy shared -> global for ragged tails and
// unaligned destinations (coalesced plain stores).
template <typename TO>
__device__ __forceinline__ void warp_copy_out(TO* gdst, const TO* ssrc, int64_t count, int lane) {
    for (int64_t i = lane; i < count; i += 32) gdst[i] = ssrc[i];
}
template <typename TI>
__device__ __forceinline__ void warp_copy_in(TI* sdst, const TI* gsrc, int64_t count, int lane) {
    for (int64_t i = lane; i < count; i += 32) sdst[i] = gsrc[i];
}

}  // namespace sph
