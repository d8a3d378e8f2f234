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

// Lanes of the warp whose 9-bit value equals this lane's (8 digit bits and
// an "invalid" bit), from nine ballots.
__device__ __forceinline__ uint32_t same_digit_lanes(uint32_t v) {
    uint32_t m = 0xFFFFFFFFu;
#pragma unroll
    for (int b = 0; b < 9; ++b) {
        const uint32_t bit = (v >> b) & 1u;
        const uint32_t x = __ballot_sync(0xFFFFFFFFu, bit);
        m &= bit ? x : ~x;
    }
    return m;
}

__global__ void __launch_bounds__(kSortThreads) k_radix_upsweep(RadixPass P) {
    constexpr int kWarps = kSortThreads / 32;
    __shared__ uint32_t cnt[kWarps][kRadix];
    for (int q = threadIdx.x; q < kWarps * kRadix; q += blockDim.x) (&cnt[0][0])[q] = 0;
    __syncthreads();
    if (pass_skipped(P)) return;
    const uint32_t n = item_count(P);
    const uint32_t kmin = P.depth_pass >= 0 ? P.hdr->key_min : 0u;
    const uint32_t warp = threadIdx.x >> 5;
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
            const uint32_t d0 = __shfl_sync(0xFFFFFFFFu, d, 0);
            if (__all_sync(0xFFFFFFFFu, d == d0)) {
                if (lane_id() == 0 && d0 < (uint32_t)kRadix) cnt[warp][d0] += 32;
            } else if (d < (uint32_t)kRadix) {
                atomicAdd(&cnt[warp][d], 1u);
            }
        }
    }
    __syncthreads();
    for (int d = threadIdx.x; d < kRadix; d += blockDim.x) {
        uint32_t c = 0;
#pragma unroll
        for (int w = 0; w < kWarps; ++w) c += cnt[w][d];
        P.hist[(uint64_t)d * P.hist_stride + blockIdx.x] = c;
    }
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

// Scatter of one pass: each CTA ranks its 4096-item tiles in shared memory
// (per-warp digit counters, ranks from ballots) and writes each digit's run
// to its global position.
constexpr int kDsThreads = 512;
// Four CTAs per SM (32 registers, a few spilled): the ranking waits on
// barriers, and more resident CTAs hide them better than the registers save
// (depth sort 0.315 -> 0.306 ms and the grouping pass 8 us faster at 10M
// particles than with 62 registers and 2 CTAs; 3 CTAs: 0.319 ms).  The
// variant carrying a payload keeps two CTAs (its third shared array and
// registers; forced to four it spilled more and the 1.07e9-particle sort
// took 43.6 instead of 35.0 ms).
constexpr int kDsMinBlocks = 4;
constexpr int kDsMinBlocksPay = 2;
constexpr int kDsWarps = kDsThreads / 32;
constexpr int kDsItems = kSortTile / kDsThreads;

template <bool PAY>
__global__ void __launch_bounds__(kDsThreads, PAY ? kDsMinBlocksPay : kDsMinBlocks) k_radix_downsweep(RadixPass P) {
    __shared__ uint32_t skey[kSortTile];
    __shared__ uint32_t sval[kSortTile];
    __shared__ uint32_t spay[PAY ? kSortTile : 1];
    __shared__ uint16_t wcnt[kDsWarps][kRadix];   // per-warp digit counters (digit-contiguous: no bank conflicts)
    __shared__ uint32_t base[kRadix];
    __shared__ uint32_t lstart[kRadix + 1];
    __shared__ uint32_t ltot[kRadix];
    __shared__ uint32_t scratch[kDsWarps + 1];
    if (pass_skipped(P)) return;
    const uint32_t n = item_count(P);
    const uint32_t kmin = P.depth_pass >= 0 ? P.hdr->key_min : 0u;
    const uint32_t lane = lane_id(), warp = threadIdx.x >> 5;
    const bool owns_digit = threadIdx.x < (uint32_t)kRadix;
    uint64_t beg, end;
    cta_range(P, n, &beg, &end);
    {
        uint32_t tot;
        const uint32_t pre = block_exclusive_scan<kDsThreads>(owns_digit ? P.htot[threadIdx.x] : 0u, scratch, &tot);
        if (owns_digit) base[threadIdx.x] = pre + P.hist[(uint64_t)threadIdx.x * P.hist_stride + blockIdx.x];
    }
    __syncthreads();
    const uint32_t lt = lanemask_lt();
    for (uint64_t tile = beg; tile < end; tile += kSortTile) {
        for (int q = threadIdx.x; q < kRadix * kDsWarps / 2; q += kDsThreads)
            reinterpret_cast<uint32_t *>(&wcnt[0][0])[q] = 0;
        __syncthreads();
        uint32_t key[kDsItems], val[kDsItems], dr[kDsItems];   // dr = rank << 9 | digit
        uint32_t pay[PAY ? kDsItems : 1];
        const uint64_t wbase = tile + (uint64_t)warp * (kDsItems * 32);
#pragma unroll
        for (int r = 0; r < kDsItems; ++r) {
            const uint64_t i = wbase + r * 32 + lane;
            key[r] = i < end ? P.key_in[i] : kInvalidKey;
            val[r] = i < end ? (P.val_in ? P.val_in[i] : (uint32_t)i) : 0u;
            if (PAY) pay[r] = i < end ? P.pay_in[i] : 0u;   // the first pass reads the transform's packed tile boxes
        }
#pragma unroll
        for (int r = 0; r < kDsItems; ++r) {
            const uint64_t i = wbase + r * 32 + lane;
            uint32_t d = kRadix;
            if (i < end && !(P.skip_invalid && key[r] == kInvalidKey)) d = ((key[r] - kmin) >> P.shift) & P.mask;
            const uint32_t peers = same_digit_lanes(d);
            uint32_t c = 0;
            if (d < (uint32_t)kRadix) c = wcnt[warp][d];
            __syncwarp();
            if (d < (uint32_t)kRadix && (peers & lt) == 0) wcnt[warp][d] = (uint16_t)(c + __popc(peers));
            __syncwarp();
            dr[r] = ((c + __popc(peers & lt)) << 9) | d;
        }
        __syncthreads();
        {
            uint32_t s = 0;
            if (owns_digit) {
#pragma unroll
                for (int w = 0; w < kDsWarps; ++w) s += wcnt[w][threadIdx.x];
                ltot[threadIdx.x] = s;
            }
            uint32_t tot;
            const uint32_t pre = block_exclusive_scan<kDsThreads>(s, scratch, &tot);
            if (owns_digit) {
                lstart[threadIdx.x] = pre;
                uint32_t run = pre;
#pragma unroll
                for (int w = 0; w < kDsWarps; ++w) {
                    const uint32_t c = wcnt[w][threadIdx.x];
                    wcnt[w][threadIdx.x] = (uint16_t)run;
                    run += c;
                }
            }
            if (threadIdx.x == 0) lstart[kRadix] = tot;
        }
        __syncthreads();
#pragma unroll
        for (int r = 0; r < kDsItems; ++r) {
            const uint32_t d = dr[r] & 511u;
            if (d < (uint32_t)kRadix) {
                const uint32_t pos = wcnt[warp][d] + (dr[r] >> 9);
                skey[pos] = key[r];
                sval[pos] = val[r];
                if (PAY) spay[pos] = pay[r];
            }
        }
        __syncthreads();
        const uint32_t nvalid = lstart[kRadix];
        for (uint32_t j = threadIdx.x; j < nvalid; j += kDsThreads) {
            const uint32_t k = skey[j];
            const uint32_t d = ((k - kmin) >> P.shift) & P.mask;
            const uint32_t pos = base[d] + (j - lstart[d]);
            if (SPL_CHECK(P.hdr, pos < n)) {
                P.key_out[pos] = k;
                P.val_out[pos] = sval[j];
                if (PAY) P.pay_out[pos] = spay[j];
            }
        }
        __syncthreads();
        if (owns_digit) base[threadIdx.x] += ltot[threadIdx.x];
        __syncthreads();
    }
}

cudaError_t launch_radix_pass(const RadixPass &p, cudaStream_t st) {
    k_radix_upsweep<<<p.ctas, kSortThreads, 0, st>>>(p);
    k_radix_scan<<<kRadix, 1024, 0, st>>>(p);
    if (p.pay_out) k_radix_downsweep<true><<<p.ctas, kDsThreads, 0, st>>>(p);
    else k_radix_downsweep<false><<<p.ctas, kDsThreads, 0, st>>>(p);
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
    // the tile box of each visible particle travels with it, so binning reads
    // it in render order instead of gathering it by index
    const bool pay = tile_payload(L);
    if (pay) {
        p.pay_in = at<uint32_t>(ws, L.off_tbox);
        p.pay_out = at<uint32_t>(ws, L.off_pay[0]);
    }
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
            if (pay) {
                q.pay_in = at<uint32_t>(ws, L.off_pay[(pass - 1) & 1]);
                q.pay_out = at<uint32_t>(ws, L.off_pay[pass & 1]);
            }
            e = launch_radix_pass(q, st);
            if (e != cudaSuccess) return e;
        }
    }
    k_sort_finish<<<1, 32, 0, st>>>(hdr, absorptive ? 1 : 0);
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace spl
