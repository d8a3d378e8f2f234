// Test kernels for the library's bounded mbarrier wait (device_util.cuh): a
// phase that nothing completes must make the wait give up after its poll
// limit and report it, and a completed phase must be seen at once.  No copy
// is issued, so nothing is in flight when a CTA leaves.
#include <cuda_runtime.h>

#include "device_util.cuh"

__global__ void k_wait(int arrive, unsigned polls, int *out) {
    __shared__ unsigned long long bar;
    if (threadIdx.x == 0) {
        spl::mbar_init(&bar);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        // the one arrival the phase needs, with no bytes expected
        if (arrive) spl::mbar_arrive_expect_tx(&bar, 0u);
    }
    __syncthreads();
    const bool done = spl::mbar_wait(&bar, 0u, polls);
    if (threadIdx.x == 0) out[0] = done ? 1 : 0;
}

// Runs one CTA; *result = 1 if the wait saw the phase complete, 0 if it gave up.
extern "C" int run_bounded_wait(int arrive, unsigned polls, int *result) {
    int *d = nullptr;
    if (cudaMalloc(&d, sizeof(int)) != cudaSuccess) return -1;
    cudaMemset(d, 0xFF, sizeof(int));
    k_wait<<<1, 64>>>(arrive, polls, d);
    cudaError_t e = cudaDeviceSynchronize();
    if (e == cudaSuccess) e = cudaMemcpy(result, d, sizeof(int), cudaMemcpyDeviceToHost);
    cudaFree(d);
    return e == cudaSuccess ? 0 : -2;
}
