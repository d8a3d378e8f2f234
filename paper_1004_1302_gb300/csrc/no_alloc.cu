// Depth sort for callers that cannot allocate device memory.
//
// Some callers may not call cudaMalloc at all while they run: a renderer
// embedded in a host application that hands out device memory only from its
// own fixed pool, or a real-time loop in which an allocation (which can
// synchronise the device) is not allowed after start-up.  Such a caller can
// still hold its input keys and output buffers, but cannot give this library
// the sort's scratch.  This entry point therefore keeps its scratch in one
// file-scope device array of fixed size, which every GPU that loads the
// library holds until the process exits.
#include "internal.h"
#include "device_util.cuh"

namespace spl {

namespace {

constexpr uint32_t kNaMax = SPLOTCH_NO_ALLOC_MAX_KEYS;
constexpr uint32_t kNaCtas = (kNaMax + kSortTile - 1) / kSortTile;

// Scratch layout: header, two key and two value ping-pong buffers, the
// per-CTA digit-count table and the digit totals.
constexpr uint64_t kNaHdr = 0;
constexpr uint64_t kNaKeys0 = kHeaderBytes;
constexpr uint64_t kNaBuf = (uint64_t)kNaMax * 4;
constexpr uint64_t kNaKeys1 = kNaKeys0 + kNaBuf;
constexpr uint64_t kNaVals0 = kNaKeys1 + kNaBuf;
constexpr uint64_t kNaVals1 = kNaVals0 + kNaBuf;
constexpr uint64_t kNaHist = kNaVals1 + kNaBuf;
constexpr uint64_t kNaHtot = kNaHist + (uint64_t)kRadix * kNaCtas * 4;
constexpr uint64_t kNaBytes = kNaHtot + (uint64_t)kRadix * 4;

}  // namespace

static __device__ __align__(256) unsigned char g_no_alloc_scratch[kNaBytes];

// Clears the counters this sort accumulates into (the array keeps the last
// call's contents).
__global__ void k_na_init(Header *hdr) {
    if (threadIdx.x != 0) return;
    hdr->magic = kMagic;
    hdr->status = SPLOTCH_OK;
    hdr->visible = 0;
    hdr->key_min = kInvalidKey;
    hdr->key_max = 0;
    hdr->sorted_buf = 0;
    hdr->check_line = 0;
}

__global__ void __launch_bounds__(256) k_na_stats(const uint32_t *key, uint32_t n, Header *hdr) {
    uint32_t nvis = 0, kmin = kInvalidKey, kmax = 0;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const uint32_t k = key[i];
        if (k != kInvalidKey) {
            nvis += 1;
            kmin = min(kmin, k);
            kmax = max(kmax, k);
        }
    }
    nvis = __reduce_add_sync(0xFFFFFFFFu, nvis);
    kmin = __reduce_min_sync(0xFFFFFFFFu, kmin);
    kmax = __reduce_max_sync(0xFFFFFFFFu, kmax);
    if (lane_id() == 0 && nvis) {
        atomicAdd(&hdr->visible, nvis);
        atomicMin(&hdr->key_min, kmin);
        atomicMax(&hdr->key_max, kmax);
    }
}

// Copies the sorted indices out.  A failed device index check (libraries
// built with device checks only) writes no order and sets *count to
// 0xFFFFFFFF, so the caller sees it.
__global__ void __launch_bounds__(256) k_na_copy_out(const Header *hdr, const uint32_t *vals0, const uint32_t *vals1,
                                                     uint32_t *order, uint32_t *count) {
    if (hdr->status != SPLOTCH_OK) {
        if (blockIdx.x == 0 && threadIdx.x == 0) *count = 0xFFFFFFFFu;
        return;
    }
    const uint32_t v = hdr->visible;
    const uint32_t *src = hdr->sorted_buf ? vals1 : vals0;
    for (uint32_t k = blockIdx.x * blockDim.x + threadIdx.x; k < v; k += gridDim.x * blockDim.x) order[k] = src[k];
    if (blockIdx.x == 0 && threadIdx.x == 0) *count = v;
}

// Device address of the scratch array on the current device.  In host code
// the array's name stands for a host-side shadow, so the address the kernels
// get is asked for on every call (a host-side query, cheap next to the
// launches); a cached address could outlive a device reset.
static int na_scratch(unsigned char **out) {
    void *p = nullptr;
    if (cudaGetSymbolAddress(&p, g_no_alloc_scratch) != cudaSuccess || !p) return SPLOTCH_ERR_CUDA;
    *out = static_cast<unsigned char *>(p);
    return SPLOTCH_OK;
}

}  // namespace spl

using namespace spl;

extern "C" int splotch_sort_keys_no_alloc(const uint32_t *key, uint32_t n, uint32_t *order, uint32_t *count,
                                          void *stream) {
    if (n > kNaMax) return SPLOTCH_ERR_ARG;
    if ((n && (!key || !order)) || !count) return SPLOTCH_ERR_ARG;
    // the first pass reads the keys four at a time (16-byte vector loads)
    if (reinterpret_cast<uintptr_t>(key) & 15u) return SPLOTCH_ERR_ARG;
    if ((reinterpret_cast<uintptr_t>(order) | reinterpret_cast<uintptr_t>(count)) & 3u) return SPLOTCH_ERR_ARG;
    unsigned char *base = nullptr;
    int s = na_scratch(&base);
    if (s) return s;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    Header *hdr = reinterpret_cast<Header *>(base + kNaHdr);
    uint32_t *keys[2] = {reinterpret_cast<uint32_t *>(base + kNaKeys0), reinterpret_cast<uint32_t *>(base + kNaKeys1)};
    uint32_t *vals[2] = {reinterpret_cast<uint32_t *>(base + kNaVals0), reinterpret_cast<uint32_t *>(base + kNaVals1)};
    k_na_init<<<1, 32, 0, st>>>(hdr);
    count_launches(1);
    if (n) {
        k_na_stats<<<(n + 255) / 256 < 1024 ? (n + 255) / 256 : 1024, 256, 0, st>>>(key, n, hdr);
        count_launches(1);
        RadixPass p{};
        p.hist = reinterpret_cast<uint32_t *>(base + kNaHist);
        p.hist_stride = kNaCtas;
        p.htot = reinterpret_cast<uint32_t *>(base + kNaHtot);
        p.hdr = hdr;
        p.ctas = (n + kSortTile - 1) / kSortTile;
        p.key_in = key;
        p.val_in = nullptr;
        p.key_out = keys[0];
        p.val_out = vals[0];
        p.n_dev = nullptr;
        p.n_host = n;
        p.shift = 0;
        p.mask = 0xFFu;
        p.depth_pass = 0;
        p.skip_invalid = 1;
        if (launch_radix_pass(p, st) != cudaSuccess) return SPLOTCH_ERR_CUDA;
        for (int pass = 1; pass < 4; ++pass) {
            RadixPass q = p;
            q.key_in = keys[(pass - 1) & 1];
            q.val_in = vals[(pass - 1) & 1];
            q.key_out = keys[pass & 1];
            q.val_out = vals[pass & 1];
            q.n_dev = &hdr->visible;
            q.shift = 8u * pass;
            q.depth_pass = pass;
            q.skip_invalid = 0;
            if (launch_radix_pass(q, st) != cudaSuccess) return SPLOTCH_ERR_CUDA;
        }
    }
    if (launch_sort_finish(hdr, st) != cudaSuccess) return SPLOTCH_ERR_CUDA;
    const uint32_t grid = n ? ((n + 255) / 256 < 1024 ? (n + 255) / 256 : 1024) : 1;
    k_na_copy_out<<<grid, 256, 0, st>>>(hdr, vals[0], vals[1], order, count);
    count_launches(1);
    return cudaGetLastError() == cudaSuccess ? SPLOTCH_OK : SPLOTCH_ERR_CUDA;
}
