// Stable LSD radix sort of (uint32 key, uint32 value) pairs, 8-bit digits,
// reduce-then-scan: per-CTA digit counts (upsweep), a scan of the count
// table, then a scatter (downsweep) that ranks each 4096-item tile in shared
// memory and writes digit runs out in order.  Used for the depth sort of
// the visible particles (ascending key, ties keep ascending index because
// the first pass reads particles in index order) and for the stable
// tile-id sort of the tile entries.
#include "internal.h"
#include "device_util.cuh"

namespace spl {

__device__ __forceinline__ bool pass_skipped(const RadixPass &P) {
    if (P.depth_pass <= 0) return false;
    const Header *h = P.hdr;
    if (h->visible == 0) return true;
    return ((h->key_max - h->key_min) >> P.shift) == 0u;
}

__device__ __forceinline__ uint32_t item_count(const RadixPass &P) { return P.n_dev ? *P.n_dev : P.n_host; }

__device__ __forceinline__ void cta_range(const RadixPass &P, uint32_t n, uint64_t *beg, uint64_t *end) {
    const uint64_t tiles = (n + (uint64_t)kSortTile - 1) / kSortTile;
    const uint64_t tpc = (tiles + P.ctas - 1) / P.ctas;
    *beg = (uint64_t)blockIdx.x * tpc * kSortTile;
    uint64_t e = *beg + tpc * kSortTile;
    *end = e < n ? e : n;
    if (*beg > *end) *beg = *end;
}

__global__ void __launch_bounds__(kSortThreads) k_radix_upsweep(RadixPass P) {
    __shared__ uint32_t cnt[kRadix];
    for (int d = threadIdx.x; d < kRadix; d += blockDim.x) cnt[d] = 0;
    __syncthreads();
    if (pass_skipped(P)) return;
    const uint32_t n = item_count(P);
    const uint32_t kmin = P.depth_pass >= 0 ? P.hdr->key_min : 0u;
    uint64_t beg, end;
    cta_range(P, n, &beg, &end);
    for (uint64_t base = beg; base < end; base += 4 * kSortThreads) {
        const uint64_t i = base + 4 * threadIdx.x;
        uint32_t k[4];
        if (i + 4 <= end) {
            uint4 v = *reinterpret_cast<const uint4 *>(P.key_in + i);
            k[0] = v.x; k[1] = v.y; k[2] = v.z; k[3] = v.w;
        } else {
#pragma unroll
            for (int q = 0; q < 4; ++q) k[q] = i + q < end ? P.key_in[i + q] : kInvalidKey;
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            uint32_t d = kRadix;
            if (i + q < end && !(P.skip_invalid && k[q] == kInvalidKey)) d = ((k[q] - kmin) >> P.shift) & P.mask;
            const uint32_t peers = __match_any_sync(0xFFFFFFFFu, d);
            if (d < (uint32_t)kRadix && (peers & lanemask_lt()) == 0) atomicAdd(&cnt[d], __popc(peers));
        }
    }
    __syncthreads();
    for (int d = threadIdx.x; d < kRadix; d += blockDim.x) P.hist[(uint64_t)d * P.hist_stride + blockIdx.x] = cnt[d];
}

// One block per digit: exclusive scan of that digit's per-CTA counts and the
// digit total.
__global__ void __launch_bounds__(1024) k_radix_scan(RadixPass P) {
    __shared__ uint32_t warp_sums[33];
    if (pass_skipped(P)) return;
    const uint32_t d = blockIdx.x;
    uint32_t *row = P.hist + (uint64_t)d * P.hist_stride;
    constexpr int kPer = (kMaxSortCtas + 1023) / 1024;
    uint32_t v[kPer], sum = 0;
#pragma unroll
    for (int q = 0; q < kPer; ++q) {
        const uint32_t j = threadIdx.x * kPer + q;
        v[q] = j < P.ctas ? row[j] : 0u;
        sum += v[q];
    }
    uint32_t total;
    uint32_t run = block_exclusive_scan<1024>(sum, warp_sums, &total);
#pragma unroll
    for (int q = 0; q < kPer; ++q) {
        const uint32_t j = threadIdx.x * kPer + q;
        if (j < P.ctas) row[j] = run;
        run += v[q];
    }
    if (threadIdx.x == 0) P.htot[d] = total;
}

__global__ void __launch_bounds__(kSortThreads) k_radix_downsweep(RadixPass P) {
    __shared__ uint32_t skey[kSortTile];
    __shared__ uint32_t sval[kSortTile];
    __shared__ uint32_t wcnt[kRadix][kSortThreads / 32];
    __shared__ uint32_t base[kRadix];
    __shared__ uint32_t lstart[kRadix + 1];
    __shared__ uint32_t ltot[kRadix];
    __shared__ uint32_t scratch[kSortThreads / 32 + 1];
    constexpr int kWarps = kSortThreads / 32;
    if (pass_skipped(P)) return;
    const uint32_t n = item_count(P);
    const uint32_t kmin = P.depth_pass >= 0 ? P.hdr->key_min : 0u;
    const uint32_t lane = lane_id(), warp = threadIdx.x >> 5;
    uint64_t beg, end;
    cta_range(P, n, &beg, &end);
    {
        const uint32_t d = threadIdx.x;  // kSortThreads == kRadix
        uint32_t tot;
        uint32_t pre = block_exclusive_scan<kSortThreads>(P.htot[d], scratch, &tot);
        base[d] = pre + P.hist[(uint64_t)d * P.hist_stride + blockIdx.x];
    }
    __syncthreads();
    const uint32_t lt = lanemask_lt();
    for (uint64_t tile = beg; tile < end; tile += kSortTile) {
        for (int q = threadIdx.x; q < kRadix * kWarps; q += kSortThreads) (&wcnt[0][0])[q] = 0;
        __syncthreads();
        uint32_t key[kSortItems], val[kSortItems], dig[kSortItems], rnk[kSortItems];
        const uint64_t wbase = tile + (uint64_t)warp * (kSortItems * 32);
#pragma unroll
        for (int r = 0; r < kSortItems; ++r) {
            const uint64_t i = wbase + r * 32 + lane;
            key[r] = i < end ? P.key_in[i] : kInvalidKey;
            val[r] = i < end ? (P.val_in ? P.val_in[i] : (uint32_t)i) : 0u;
        }
#pragma unroll
        for (int r = 0; r < kSortItems; ++r) {
            const uint64_t i = wbase + r * 32 + lane;
            uint32_t d = kRadix;
            if (i < end && !(P.skip_invalid && key[r] == kInvalidKey)) d = ((key[r] - kmin) >> P.shift) & P.mask;
            const uint32_t peers = __match_any_sync(0xFFFFFFFFu, d);
            uint32_t c = 0;
            if (d < (uint32_t)kRadix) c = wcnt[d][warp];
            __syncwarp();
            if (d < (uint32_t)kRadix && (peers & lt) == 0) wcnt[d][warp] = c + __popc(peers);
            __syncwarp();
            dig[r] = d;
            rnk[r] = c + __popc(peers & lt);
        }
        __syncthreads();
        {
            const uint32_t d = threadIdx.x;
            uint32_t s = 0;
#pragma unroll
            for (int w = 0; w < kWarps; ++w) s += wcnt[d][w];
            ltot[d] = s;
            uint32_t tot;
            uint32_t pre = block_exclusive_scan<kSortThreads>(s, scratch, &tot);
            lstart[d] = pre;
            if (d == 0) lstart[kRadix] = tot;
            uint32_t run = pre;
#pragma unroll
            for (int w = 0; w < kWarps; ++w) {
                const uint32_t c = wcnt[d][w];
                wcnt[d][w] = run;
                run += c;
            }
        }
        __syncthreads();
#pragma unroll
        for (int r = 0; r < kSortItems; ++r) {
            if (dig[r] < (uint32_t)kRadix) {
                const uint32_t pos = wcnt[dig[r]][warp] + rnk[r];
                skey[pos] = key[r];
                sval[pos] = val[r];
            }
        }
        __syncthreads();
        const uint32_t nvalid = lstart[kRadix];
        for (uint32_t j = threadIdx.x; j < nvalid; j += kSortThreads) {
            const uint32_t k = skey[j];
            const uint32_t d = ((k - kmin) >> P.shift) & P.mask;
            const uint32_t pos = base[d] + (j - lstart[d]);
            P.key_out[pos] = k;
            P.val_out[pos] = sval[j];
        }
        __syncthreads();
        base[threadIdx.x] += ltot[threadIdx.x];
        __syncthreads();
    }
}

cudaError_t launch_radix_pass(const RadixPass &p, cudaStream_t st) {
    k_radix_upsweep<<<p.ctas, kSortThreads, 0, st>>>(p);
    k_radix_scan<<<kRadix, 1024, 0, st>>>(p);
    k_radix_downsweep<<<p.ctas, kSortThreads, 0, st>>>(p);
    count_launches(3);
    return cudaGetLastError();
}

// Which ping-pong buffer holds the ordered visible list after the depth sort.
__global__ void k_sort_finish(Header *hdr, int absorptive) {
    if (threadIdx.x != 0) return;
    uint32_t passes = 1;
    if (absorptive && hdr->visible) {
        const uint32_t range = hdr->key_max - hdr->key_min;
        for (int p = 1; p < 4; ++p)
            if ((range >> (8 * p)) != 0u) passes = p + 1;
    }
    hdr->sorted_buf = (passes - 1) & 1u;
}

cudaError_t launch_sort_finish(Header *hdr, cudaStream_t st) {
    k_sort_finish<<<1, 32, 0, st>>>(hdr, 1);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_sort(void *ws, const Layout &L, int mode, cudaStream_t st) {
    Header *hdr = header(ws);
    const bool absorptive = mode == SPLOTCH_ABSORPTIVE;
    RadixPass p{};
    p.hist = at<uint32_t>(ws, L.off_hist);
    p.hist_stride = L.hist_ctas;
    p.htot = at<uint32_t>(ws, L.off_htot);
    p.hdr = hdr;
    p.ctas = L.sort_ctas;
    // Pass 0 reads every particle's key in index order, drops culled ones and
    // carries the particle index as the value (emission: one bucket, a stable
    // compaction).
    p.key_in = at<uint32_t>(ws, L.off_key);
    p.val_in = nullptr;
    p.key_out = at<uint32_t>(ws, L.off_sk[0]);
    p.val_out = at<uint32_t>(ws, L.off_sv[0]);
    p.n_dev = nullptr;
    p.n_host = (uint32_t)L.n;
    p.shift = 0;
    p.mask = absorptive ? 0xFFu : 0u;
    p.depth_pass = absorptive ? 0 : -1;
    p.skip_invalid = 1;
    cudaError_t e = L.n ? launch_radix_pass(p, st) : cudaSuccess;
    if (e != cudaSuccess) return e;
    if (absorptive) {
        for (int pass = 1; pass < 4 && L.n; ++pass) {
            RadixPass q = p;
            q.key_in = at<uint32_t>(ws, L.off_sk[(pass - 1) & 1]);
            q.val_in = at<uint32_t>(ws, L.off_sv[(pass - 1) & 1]);
            q.key_out = at<uint32_t>(ws, L.off_sk[pass & 1]);
            q.val_out = at<uint32_t>(ws, L.off_sv[pass & 1]);
            q.n_dev = &hdr->visible;
            q.shift = 8u * pass;
            q.mask = 0xFFu;
            q.depth_pass = pass;
            q.skip_invalid = 0;
            e = launch_radix_pass(q, st);
            if (e != cudaSuccess) return e;
        }
    }
    k_sort_finish<<<1, 32, 0, st>>>(hdr, absorptive ? 1 : 0);
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace spl
