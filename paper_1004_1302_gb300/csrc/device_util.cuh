// Small device helpers shared by the kernel files.
#pragma once

#include <cstdint>
#include <cuda_fp16.h>
#include <cuda_bf16.h>

namespace spl {

__device__ __forceinline__ uint32_t lanemask_lt() {
    uint32_t m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

__device__ __forceinline__ uint32_t lane_id() { return threadIdx.x & 31u; }

// Order-preserving map of a finite float onto uint32 (for atomicMin/atomicMax).
__device__ __forceinline__ uint32_t float_to_ordered(float f) {
    uint32_t b = __float_as_uint(f);
    return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}
__host__ __device__ __forceinline__ float ordered_to_float(uint32_t e) {
    uint32_t b = (e & 0x80000000u) ? (e & 0x7FFFFFFFu) : ~e;
#ifdef __CUDA_ARCH__
    return __uint_as_float(b);
#else
    float f;
    __builtin_memcpy(&f, &b, 4);
    return f;
#endif
}

// Inclusive warp scan (add) of a uint32.
__device__ __forceinline__ uint32_t warp_inclusive_scan(uint32_t v) {
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        uint32_t t = __shfl_up_sync(0xFFFFFFFFu, v, d);
        if (lane_id() >= (uint32_t)d) v += t;
    }
    return v;
}

__device__ __forceinline__ unsigned long long warp_inclusive_scan64(unsigned long long v) {
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        unsigned long long t = __shfl_up_sync(0xFFFFFFFFu, v, d);
        if (lane_id() >= (uint32_t)d) v += t;
    }
    return v;
}

// Exclusive block scan of one uint32 per thread; `warp_sums` holds blockDim/32
// entries of shared memory.  Returns the exclusive prefix; *total gets the sum.
template <int kThreads>
__device__ __forceinline__ uint32_t block_exclusive_scan(uint32_t v, uint32_t *warp_sums, uint32_t *total) {
    constexpr int kWarps = kThreads / 32;
    const uint32_t lane = lane_id(), warp = threadIdx.x >> 5;
    uint32_t inc = warp_inclusive_scan(v);
    if (lane == 31) warp_sums[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        uint32_t s = lane < (uint32_t)kWarps ? warp_sums[lane] : 0u;
        uint32_t si = warp_inclusive_scan(s);
        if (lane < (uint32_t)kWarps) warp_sums[lane] = si - s;
        if (lane == (uint32_t)kWarps - 1) warp_sums[kWarps] = si;
    }
    __syncthreads();
    uint32_t r = warp_sums[warp] + inc - v;
    *total = warp_sums[kWarps];
    __syncthreads();
    return r;
}

template <int kThreads>
__device__ __forceinline__ unsigned long long block_exclusive_scan64(unsigned long long v, unsigned long long *warp_sums,
                                                                     unsigned long long *total) {
    constexpr int kWarps = kThreads / 32;
    const uint32_t lane = lane_id(), warp = threadIdx.x >> 5;
    unsigned long long inc = warp_inclusive_scan64(v);
    if (lane == 31) warp_sums[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        unsigned long long s = lane < (uint32_t)kWarps ? warp_sums[lane] : 0ull;
        unsigned long long si = warp_inclusive_scan64(s);
        if (lane < (uint32_t)kWarps) warp_sums[lane] = si - s;
        if (lane == (uint32_t)kWarps - 1) warp_sums[kWarps] = si;
    }
    __syncthreads();
    unsigned long long r = warp_sums[warp] + inc - v;
    *total = warp_sums[kWarps];
    __syncthreads();
    return r;
}

// Intensity widened to float (exact for half and bfloat16).
__device__ __forceinline__ float load_value(const void *v, int dtype, uint64_t i) {
    if (dtype == 1) return __half2float(static_cast<const __half *>(v)[i]);
    if (dtype == 2) return __bfloat162float(static_cast<const __nv_bfloat16 *>(v)[i]);
    return static_cast<const float *>(v)[i];
}

// --- asynchronous copies into shared memory -----------------------------------

__device__ __forceinline__ uint32_t smem_addr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// An mbarrier that completes a phase after one arrival and the expected bytes.
__device__ __forceinline__ void mbar_init(unsigned long long *bar) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(smem_addr(bar)) : "memory");
}

// The single arrival of a phase, announcing `bytes` of copies that complete on it.
__device__ __forceinline__ void mbar_arrive_expect_tx(unsigned long long *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" :: "r"(smem_addr(bar)), "r"(bytes) : "memory");
}

// Bulk asynchronous copy of `bytes` (a multiple of 16; both addresses 16-byte
// aligned) from global to shared memory, completing on `bar`.
__device__ __forceinline__ void bulk_copy_g2s(void *dst, const void *src, uint32_t bytes, unsigned long long *bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 :: "r"(smem_addr(dst)), "l"(src), "r"(bytes), "r"(smem_addr(bar)) : "memory");
}

// Wait for phase `parity` of an mbarrier, at most `limit` polls; false if
// the limit ran out.  kAsyncWaitPolls: each try_wait blocks a while, so
// this bound lies far beyond any copy's time.
constexpr uint32_t kAsyncWaitPolls = 1u << 22;
__device__ __forceinline__ bool mbar_wait(unsigned long long *bar, uint32_t parity, uint32_t limit) {
    for (uint32_t it = 0; it < limit; ++it) {
        uint32_t done;
        asm volatile(
            "{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2; selp.u32 %0, 1, 0, p; }"
            : "=r"(done) : "r"(smem_addr(bar)), "r"(parity) : "memory");
        if (done) return true;
    }
    return false;
}

// Orders this thread's earlier generic accesses to shared memory before
// later asynchronous (bulk copy) writes to it.
__device__ __forceinline__ void fence_proxy_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// --- programmatic dependent launch --------------------------------------------
// A kernel launched with programmatic stream serialization (launch_pdl) may
// be scheduled while the kernel before it on the stream finishes; it waits
// here, before its first global memory access, until that kernel has
// completed and its writes are visible, then lets the next kernel be
// scheduled as its own CTAs drain.  Launched the ordinary way, both are
// no-ops.
__device__ __forceinline__ void pdl_enter() {
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

}  // namespace spl
