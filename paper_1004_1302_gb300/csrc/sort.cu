// Stable LSD radix sort of (uint32 key, uint32 value) pairs, 8-bit digits,
// reduce-then-scan: per-CTA digit counts (upsweep), a scan of the count
// table, then a scatter (downsweep) that ranks each 4096-item tile in shared
// memory and writes digit runs out in order.  Used for the depth sort of
// the visible particles (ascending key, ties keep ascending index because
// the first pass reads particles in index order) and for the stable
// tile-id sort of the tile entries.
#include <atomic>

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
// an "invalid" bit), from nine ballots: per bit, the lanes that share it are
// the ballot or its complement, picked by the bit's sign-extension (0 or ~0),
// so a bit costs an extract, a ballot and one three-input logic operation
// (the select form was 3-5% slower on the 10M-particle depth sort).
// MATCH: the warp's match instruction instead (fewer instructions, lower
// throughput).
template <bool MATCH = false>
__device__ __forceinline__ uint32_t same_digit_lanes(uint32_t v) {
    if constexpr (MATCH) return __match_any_sync(0xFFFFFFFFu, v);
    uint32_t m = 0xFFFFFFFFu;
#pragma unroll
    for (int b = 0; b < 9; ++b) {
        int sel;
        asm("bfe.s32 %0, %1, %2, 1;" : "=r"(sel) : "r"(v), "r"(b));
        const uint32_t x = __ballot_sync(0xFFFFFFFFu, sel != 0);
        m &= ~(x ^ (uint32_t)sel);
    }
    return m;
}

__global__ void __launch_bounds__(kSortThreads) k_radix_upsweep(RadixPass P) {
    pdl_enter();
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
    // a tile of kSortTile keys per step: every thread's four 16-byte loads are
    // in flight together (one load per step left the pass waiting on latency)
    constexpr int kLoads = kSortTile / (4 * kSortThreads);
    for (uint64_t base = beg; base < end; base += kSortTile) {
        uint32_t k[kLoads][4];
#pragma unroll
        for (int l = 0; l < kLoads; ++l) {
            const uint64_t i = base + 4 * ((uint64_t)l * kSortThreads + threadIdx.x);
            if (i + 4 <= end) {
                const uint4 v = *reinterpret_cast<const uint4 *>(P.key_in + i);
                k[l][0] = v.x; k[l][1] = v.y; k[l][2] = v.z; k[l][3] = v.w;
            } else {
#pragma unroll
                for (int q = 0; q < 4; ++q) k[l][q] = i + q < end ? P.key_in[i + q] : kInvalidKey;
            }
        }
#pragma unroll
        for (int l = 0; l < kLoads; ++l) {
            const uint64_t i = base + 4 * ((uint64_t)l * kSortThreads + threadIdx.x);
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                uint32_t d = kRadix;
                if (i + q < end && !(P.skip_invalid && k[l][q] == kInvalidKey)) d = ((k[l][q] - kmin) >> P.shift) & P.mask;
                const uint32_t d0 = __shfl_sync(0xFFFFFFFFu, d, 0);
                if (__all_sync(0xFFFFFFFFu, d == d0)) {
                    if (lane_id() == 0 && d0 < (uint32_t)kRadix) cnt[warp][d0] += 32;
                } else if (d < (uint32_t)kRadix) {
                    atomicAdd(&cnt[warp][d], 1u);
                }
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
    pdl_enter();
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
// to its global position.  A tile's items reach shared memory by bulk
// asynchronous copies (cp.async.bulk, completing on an mbarrier) issued one
// tile ahead, so the next tile's reads overlap this tile's ranking and
// writes.  Two buffer sets alternate: the set that brought a tile in then
// stages its output, and after that takes the copies of the tile two ahead.
// With five barriers per tile instead of eight this took the 1.07e9-particle
// depth sort from 27.2 to 24.8 ms; at 10M particles (the data in L2) the
// time is unchanged against register loads at four CTAs per SM.
constexpr int kDsThreads = 512;
constexpr int kDsWarps = kDsThreads / 32;
constexpr int kDsItems = kSortTile / kDsThreads;

template <bool PAY> struct DsSmem {
    uint32_t key[2][kSortTile];
    uint32_t val[2][kSortTile];
    uint32_t pay[PAY ? 2 : 1][PAY ? kSortTile : 4];
    uint16_t wcnt[kDsWarps][kRadix];   // per-warp digit counters (digit-contiguous: no bank conflicts)
    uint32_t base[kRadix];
    uint16_t lstart[kRadix + 1];       // tile-local digit starts and counts (<= kSortTile)
    uint16_t ltot[kRadix];
    uint32_t scratch[kDsWarps + 1];
    unsigned long long bar[2];
    int timeout;
};
// Resident CTAs per SM: three without a payload (74 KB of shared memory
// each, 1 KB more reserved per CTA, within the SM's 228 KB), two with one
// (106 KB).
constexpr int kDsMinBlocks = 3;
constexpr int kDsMinBlocksPay = 2;

static_assert(sizeof(DsSmem<false>) + 1024 <= 228 * 1024 / kDsMinBlocks, "three downsweeps per SM");
static_assert(sizeof(DsSmem<true>) + 1024 <= 228 * 1024 / kDsMinBlocksPay, "two downsweeps per SM");

// The payload variant ranks with the match instruction: at two CTAs per SM
// it waits on memory more than on issue slots, and the fewer instructions
// win there (1.07e9-particle depth sort 24.8 -> 24.3 ms); without a payload
// the ballots are faster (10M: 0.295 against 0.356 ms).
template <bool PAY>
__global__ void __launch_bounds__(kDsThreads, PAY ? kDsMinBlocksPay : kDsMinBlocks) k_radix_downsweep(RadixPass P) {
    pdl_enter();
    constexpr bool MATCH = PAY;
    extern __shared__ __align__(128) unsigned char ds_raw[];
    DsSmem<PAY> &sm = *reinterpret_cast<DsSmem<PAY> *>(ds_raw);
    if (pass_skipped(P)) return;
    const uint32_t n = item_count(P);
    const uint32_t kmin = P.depth_pass >= 0 ? P.hdr->key_min : 0u;
    const uint32_t lane = lane_id(), warp = threadIdx.x >> 5;
    const bool owns_digit = threadIdx.x < (uint32_t)kRadix;
    uint64_t beg, end;
    cta_range(P, n, &beg, &end);
    const uint32_t ntiles = (uint32_t)((end - beg + kSortTile - 1) / kSortTile);
    // copies of the CTA's k-th tile into buffer set k & 1 (thread 0): the
    // 16-byte multiple of each array's range; the last < 4 items are read
    // directly from global memory
    auto issue = [&](uint32_t k) {
        const uint64_t t0 = beg + (uint64_t)k * kSortTile;
        const uint32_t cnt = (uint32_t)min((uint64_t)kSortTile, end - t0);
        const uint32_t bytes = (cnt & ~3u) * 4u;
        const int b = k & 1;
        mbar_arrive_expect_tx(&sm.bar[b], bytes * (1u + (P.val_in ? 1u : 0u) + (PAY ? 1u : 0u)));
        if (bytes) {
            bulk_copy_g2s(sm.key[b], P.key_in + t0, bytes, &sm.bar[b]);
            if (P.val_in) bulk_copy_g2s(sm.val[b], P.val_in + t0, bytes, &sm.bar[b]);
            if (PAY) bulk_copy_g2s(sm.pay[b], P.pay_in + t0, bytes, &sm.bar[b]);
        }
    };
    if (threadIdx.x == 0) {
        mbar_init(&sm.bar[0]);
        mbar_init(&sm.bar[1]);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        sm.timeout = 0;
        if (ntiles) issue(0);
    }
    {
        uint32_t tot;
        const uint32_t pre = block_exclusive_scan<kDsThreads>(owns_digit ? P.htot[threadIdx.x] : 0u, sm.scratch, &tot);
        if (owns_digit) sm.base[threadIdx.x] = pre + P.hist[(uint64_t)threadIdx.x * P.hist_stride + blockIdx.x];
    }
    for (int q = threadIdx.x; q < kRadix * kDsWarps / 2; q += kDsThreads)
        reinterpret_cast<uint32_t *>(&sm.wcnt[0][0])[q] = 0;
    if (threadIdx.x == 0 && ntiles && !mbar_wait(&sm.bar[0], 0u, kAsyncWaitPolls)) sm.timeout = 1;
    __syncthreads();
    // Five barriers per tile: after the ranking, after the digit totals'
    // warp sums, after the digit starts, after the staging scatter and after
    // the writes.  Tile k's copies were waited for (thread 0) before the
    // barrier that ended tile k - 1, and the counters were zeroed then.
    const uint32_t lt = lanemask_lt();
    uint32_t kstop = 0;
    for (uint32_t k = 0; k < ntiles; ++k) {
        const int b = k & 1;
        if (sm.timeout) {
            kstop = k;
            break;
        }
        const uint64_t tile = beg + (uint64_t)k * kSortTile;
        const uint32_t cnt = (uint32_t)min((uint64_t)kSortTile, end - tile), bulk = cnt & ~3u;
        // set b ^ 1 was last read by the previous tile's writes, ordered before
        // this copy by every thread's proxy fence and the barrier that ended it
        if (threadIdx.x == 0 && k + 1 < ntiles) issue(k + 1);
        uint32_t key[kDsItems], val[kDsItems], dr[kDsItems];   // dr = rank << 9 | digit
        uint32_t pay[PAY ? kDsItems : 1];
#pragma unroll
        for (int r = 0; r < kDsItems; ++r) {
            const uint32_t li = warp * (kDsItems * 32) + r * 32 + lane;
            const uint64_t i = tile + li;
            if (li < bulk) {
                key[r] = sm.key[b][li];
                val[r] = P.val_in ? sm.val[b][li] : (uint32_t)i;
                if (PAY) pay[r] = sm.pay[b][li];
            } else {
                key[r] = li < cnt ? P.key_in[i] : kInvalidKey;
                val[r] = li < cnt ? (P.val_in ? P.val_in[i] : (uint32_t)i) : 0u;
                if (PAY) pay[r] = li < cnt ? P.pay_in[i] : 0u;   // the first pass reads the transform's packed tile boxes
            }
        }
#pragma unroll
        for (int r = 0; r < kDsItems; ++r) {
            const uint32_t li = warp * (kDsItems * 32) + r * 32 + lane;
            uint32_t d = kRadix;
            if (li < cnt && !(P.skip_invalid && key[r] == kInvalidKey)) d = ((key[r] - kmin) >> P.shift) & P.mask;
            const uint32_t peers = same_digit_lanes<MATCH>(d);
            uint32_t c = 0;
            if (d < (uint32_t)kRadix) c = sm.wcnt[warp][d];
            __syncwarp();
            if (d < (uint32_t)kRadix && (peers & lt) == 0) sm.wcnt[warp][d] = (uint16_t)(c + __popc(peers));
            __syncwarp();
            dr[r] = ((c + __popc(peers & lt)) << 9) | d;
        }
        __syncthreads();
        // digit totals of the tile and their exclusive scan (the owners are warps 0 .. 7)
        uint32_t s = 0, inc = 0;
        if (owns_digit) {
#pragma unroll
            for (int w = 0; w < kDsWarps; ++w) s += sm.wcnt[w][threadIdx.x];
            sm.ltot[threadIdx.x] = (uint16_t)s;
            inc = warp_inclusive_scan(s);
            if (lane == 31) sm.scratch[warp] = inc;
        }
        __syncthreads();
        if (owns_digit) {
            uint32_t pre = inc - s;
#pragma unroll
            for (int w = 0; w < kRadix / 32; ++w)
                if ((uint32_t)w < warp) pre += sm.scratch[w];
            sm.lstart[threadIdx.x] = (uint16_t)pre;
            if (threadIdx.x == kRadix - 1) sm.lstart[kRadix] = (uint16_t)(pre + s);
            uint32_t run = pre;
#pragma unroll
            for (int w = 0; w < kDsWarps; ++w) {
                const uint32_t c = sm.wcnt[w][threadIdx.x];
                sm.wcnt[w][threadIdx.x] = (uint16_t)run;
                run += c;
            }
        }
        __syncthreads();
        // the tile's input is in registers now: set b stages the output
#pragma unroll
        for (int r = 0; r < kDsItems; ++r) {
            const uint32_t d = dr[r] & 511u;
            if (d < (uint32_t)kRadix) {
                const uint32_t pos = sm.wcnt[warp][d] + (dr[r] >> 9);
                sm.key[b][pos] = key[r];
                sm.val[b][pos] = val[r];
                if (PAY) sm.pay[b][pos] = pay[r];
            }
        }
        __syncthreads();
        // the counters are free again: zero them for the next tile
        for (int q = threadIdx.x; q < kRadix * kDsWarps / 2; q += kDsThreads)
            reinterpret_cast<uint32_t *>(&sm.wcnt[0][0])[q] = 0;
        const uint32_t nvalid = sm.lstart[kRadix];
        for (uint32_t j = threadIdx.x; j < nvalid; j += kDsThreads) {
            const uint32_t kk = sm.key[b][j];
            const uint32_t d = ((kk - kmin) >> P.shift) & P.mask;
            const uint32_t pos = sm.base[d] + (j - sm.lstart[d]);
            if (SPL_CHECK(P.hdr, pos < n)) {
                P.key_out[pos] = kk;
                P.val_out[pos] = sm.val[b][j];
                if (PAY) P.pay_out[pos] = sm.pay[b][j];
            }
        }
        fence_proxy_async_smem();
        if (threadIdx.x == 0 && k + 1 < ntiles && !mbar_wait(&sm.bar[b ^ 1], ((k + 1) >> 1) & 1u, kAsyncWaitPolls))
            sm.timeout = 1;
        __syncthreads();
        if (owns_digit) sm.base[threadIdx.x] += sm.ltot[threadIdx.x];
    }
    if (sm.timeout && threadIdx.x == 0) {
        // tile kstop's copies never completed (the next tile's were not issued):
        // report it, and give them one more bounded wait to land
        atomicExch(const_cast<int *>(&P.hdr->status), (int)SPLOTCH_ERR_TIMEOUT);
        mbar_wait(&sm.bar[kstop & 1], (kstop >> 1) & 1u, kAsyncWaitPolls);
    }
}

template <bool PAY> static cudaError_t launch_downsweep(const RadixPass &p, cudaStream_t st) {
    // the dynamic shared memory exceeds the default 48 KB: raise the limit
    // once per device
    static std::atomic<uint64_t> configured{0};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    const uint64_t bit = 1ull << (dev & 63);
    if (!(configured.load() & bit)) {
        e = cudaFuncSetAttribute(k_radix_downsweep<PAY>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)sizeof(DsSmem<PAY>));
        if (e != cudaSuccess) return e;
        configured.fetch_or(bit);
    }
    return launch_pdl(k_radix_downsweep<PAY>, dim3(p.ctas), dim3(kDsThreads), sizeof(DsSmem<PAY>), st, p);
}

cudaError_t launch_radix_pass(const RadixPass &p, cudaStream_t st) {
    // the downsweep's bulk copies need 16-byte aligned arrays
    const uintptr_t al = reinterpret_cast<uintptr_t>(p.key_in) | reinterpret_cast<uintptr_t>(p.val_in) |
                         reinterpret_cast<uintptr_t>(p.pay_in);
    if (al & 15u) return cudaErrorInvalidValue;
    launch_pdl(k_radix_upsweep, dim3(p.ctas), dim3(kSortThreads), 0, st, p);
    launch_pdl(k_radix_scan, dim3(kRadix), dim3(1024), 0, st, p);
    const cudaError_t e = p.pay_out ? launch_downsweep<true>(p, st) : launch_downsweep<false>(p, st);
    if (e != cudaSuccess) return e;
    count_launches(3);
    return cudaGetLastError();
}

// Which ping-pong buffer holds the ordered visible list after the depth sort.
__global__ void k_sort_finish(Header *hdr, int absorptive) {
    pdl_enter();
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
    launch_pdl(k_sort_finish, dim3(1), dim3(32), 0, st, hdr, 1);
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
    launch_pdl(k_sort_finish, dim3(1), dim3(32), 0, st, hdr, absorptive ? 1 : 0);
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace spl
