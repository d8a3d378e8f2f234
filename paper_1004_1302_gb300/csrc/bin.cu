// Screen-tile binning.  Every visible particle, in render order, adds one
// entry (tile id, particle) per tile its box meets.  Entry offsets come from
// an exclusive scan of the per-particle tile counts, so the entries of one
// particle sit at fixed positions whatever the thread that writes them.
// Particles touching more tiles than a threshold are split over a whole CTA
// (the "split particles" idea of Section 3.2 applied to the emission of
// work items).  A stable radix sort by tile id then yields per-tile lists in
// render order, and a boundary pass turns the sorted ids into tile offsets.
#include "internal.h"
#include "device_util.cuh"

namespace spl {

constexpr int kBinStep = 2048;   // particles per CTA step of the emission kernel

__device__ __forceinline__ uint32_t tiles_of(const ushort4 b, int tshift) {
    return (uint32_t)((b.z >> tshift) - (b.x >> tshift) + 1) * (uint32_t)((b.w >> tshift) - (b.y >> tshift) + 1);
}

__device__ __forceinline__ void bin_range(uint32_t ctas, uint32_t n, uint64_t *beg, uint64_t *end) {
    const uint64_t steps = (n + (uint64_t)kBinStep - 1) / kBinStep;
    const uint64_t spc = (steps + ctas - 1) / ctas;
    *beg = (uint64_t)blockIdx.x * spc * kBinStep;
    uint64_t e = *beg + spc * kBinStep;
    *end = e < n ? e : n;
    if (*beg > *end) *beg = *end;
}

__global__ void __launch_bounds__(256) k_bin_reduce(BinArgs a) {
    __shared__ unsigned long long ws[9];
    const uint32_t n = a.hdr->visible;
    const uint32_t *list = a.hdr->sorted_buf ? a.list[1] : a.list[0];
    uint64_t beg, end;
    bin_range(a.ctas, n, &beg, &end);
    unsigned long long sum = 0;
    for (uint64_t k = beg + threadIdx.x; k < end; k += blockDim.x) sum += tiles_of(a.box[list[k]], a.tshift);
    unsigned long long tot;
    block_exclusive_scan64<256>(sum, ws, &tot);
    if (threadIdx.x == 0) a.part[blockIdx.x] = tot;
}

__global__ void __launch_bounds__(1024) k_bin_scan(BinArgs a) {
    __shared__ unsigned long long ws[33];
    constexpr int kPer = (kMaxSortCtas + 1023) / 1024;
    unsigned long long v[kPer], sum = 0;
#pragma unroll
    for (int q = 0; q < kPer; ++q) {
        const uint32_t j = threadIdx.x * kPer + q;
        v[q] = j < a.ctas ? a.part[j] : 0ull;
        sum += v[q];
    }
    unsigned long long total;
    unsigned long long run = block_exclusive_scan64<1024>(sum, ws, &total);
#pragma unroll
    for (int q = 0; q < kPer; ++q) {
        const uint32_t j = threadIdx.x * kPer + q;
        if (j < a.ctas) a.part[j] = run;
        run += v[q];
    }
    if (threadIdx.x == 0) {
        a.hdr->tile_entries = total;
        a.hdr->tile_entries32 = (uint32_t)(total < a.cap ? total : a.cap);
        if (total > a.cap) a.hdr->status = SPLOTCH_ERR_WORKSPACE;
    }
}

// Each CTA walks its range in steps of kBinStep particles (list order).
// A particle touching at most `large_tiles` tiles is written by the thread
// that owns it; the step's larger particles are split over the CTA's warps,
// one warp per particle with its lanes across a row of tiles, so the writes
// of a row are contiguous.
__global__ void __launch_bounds__(256) k_bin_emit(BinArgs a) {
    constexpr int kPer = kBinStep / 256;
    __shared__ uint32_t s_p[kBinStep];        // particle index per item
    __shared__ uint32_t s_off[kBinStep];      // tiles per item, then its entry offset within the step
    __shared__ uint32_t s_lidx[kBinStep];     // items of the large particles, in list order
    __shared__ ushort4 s_box[kBinStep];       // tile box per item: tx0, ty0, tx1, ty1
    __shared__ uint32_t ws32[9];
    const uint32_t n = a.hdr->visible;
    const uint32_t *list = a.hdr->sorted_buf ? a.list[1] : a.list[0];
    const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint64_t beg, end;
    bin_range(a.ctas, n, &beg, &end);
    unsigned long long running = a.part[blockIdx.x];
    uint32_t nlarge_cta = 0;
    for (uint64_t step = beg; step < end; step += kBinStep) {
        const uint32_t m = (uint32_t)min((uint64_t)kBinStep, end - step);
#pragma unroll
        for (int q = 0; q < kPer; ++q) {
            const uint32_t j = threadIdx.x + 256u * q;
            uint32_t p = 0, nt = 0;
            ushort4 tb = make_ushort4(1, 1, 0, 0);
            if (j < m) {
                p = list[step + j];
                const ushort4 b = a.box[p];
                tb = make_ushort4(b.x >> a.tshift, b.y >> a.tshift, b.z >> a.tshift, b.w >> a.tshift);
                nt = (uint32_t)(tb.z - tb.x + 1) * (uint32_t)(tb.w - tb.y + 1);
            }
            s_p[j] = p;
            s_off[j] = nt;
            s_box[j] = tb;
        }
        __syncthreads();
        // blocked arrangement: thread t owns items kPer*t .. kPer*t + kPer - 1
        uint32_t nt[kPer];
        uint32_t mine = 0, mine_large = 0;
#pragma unroll
        for (int q = 0; q < kPer; ++q) {
            nt[q] = s_off[kPer * threadIdx.x + q];
            mine += nt[q];
            mine_large += nt[q] > a.large_tiles;
        }
        uint32_t tot, ltot;
        uint32_t off = block_exclusive_scan<256>(mine, ws32, &tot);
        uint32_t lpos = block_exclusive_scan<256>(mine_large, ws32, &ltot);
#pragma unroll
        for (int q = 0; q < kPer; ++q) {
            const uint32_t j = kPer * threadIdx.x + q;
            s_off[j] = off;
            if (nt[q] > a.large_tiles) s_lidx[lpos++] = j;
            off += nt[q];
        }
        __syncthreads();
        // small particles: the owner writes its entries
#pragma unroll
        for (int q = 0; q < kPer; ++q) {
            const uint32_t j = kPer * threadIdx.x + q;
            if (nt[q] == 0 || nt[q] > a.large_tiles) continue;
            const uint32_t p = s_p[j];
            const ushort4 b = s_box[j];
            unsigned long long e = running + s_off[j];
            for (int ty = b.y; ty <= b.w; ++ty)
                for (int tx = b.x; tx <= b.z; ++tx, ++e)
                    if (e < a.cap) {
                        a.ek[e] = (uint32_t)(ty * a.ntx + tx);
                        a.ev[e] = p;
                    }
        }
        // large particles: one warp per particle, lanes across a row of tiles
        for (uint32_t i = warp; i < ltot; i += 8) {
            const uint32_t j = s_lidx[i];
            const uint32_t p = s_p[j];
            const ushort4 b = s_box[j];
            const uint32_t w = (uint32_t)(b.z - b.x + 1);
            unsigned long long e0 = running + s_off[j];
            for (int ty = b.y; ty <= b.w; ++ty, e0 += w)
                for (uint32_t c = lane; c < w; c += 32) {
                    const unsigned long long e = e0 + c;
                    if (e < a.cap) {
                        a.ek[e] = (uint32_t)(ty * a.ntx + b.x) + c;
                        a.ev[e] = p;
                    }
                }
        }
        nlarge_cta += ltot;
        running += tot;
        __syncthreads();
    }
    if (threadIdx.x == 0 && nlarge_cta) atomicAdd(&a.hdr->n_large, nlarge_cta);
}

// Tile offsets from tile-sorted entry ids: offsets[t] = first entry of tile t.
__global__ void __launch_bounds__(256) k_tile_offsets(const Header *hdr, const uint32_t *ek, uint32_t *toff,
                                                      uint32_t ntiles) {
    const uint32_t D = hdr->tile_entries32;
    const uint32_t stride = gridDim.x * blockDim.x;
    if (D == 0) {
        for (uint32_t t = blockIdx.x * blockDim.x + threadIdx.x; t <= ntiles; t += stride) toff[t] = 0;
        return;
    }
    for (uint32_t e = blockIdx.x * blockDim.x + threadIdx.x; e < D; e += stride) {
        const uint32_t t = ek[e];
        const uint32_t prev = e ? ek[e - 1] + 1u : 0u;
        for (uint32_t tt = prev; tt <= t; ++tt) toff[tt] = e;
        if (e == D - 1)
            for (uint32_t tt = t + 1; tt <= ntiles; ++tt) toff[tt] = D;
    }
}

static int sm_count_bin() {
    int dev = 0, v = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
    return v > 0 ? v : 148;
}

cudaError_t launch_bin(void *ws, const Layout &L, uint32_t large_tiles, cudaStream_t st) {
    Header *hdr = header(ws);
    BinArgs a{};
    a.hdr = hdr;
    a.list[0] = at<uint32_t>(ws, L.off_sv[0]);
    a.list[1] = at<uint32_t>(ws, L.off_sv[1]);
    a.box = at<ushort4>(ws, L.off_box);
    a.part = at<uint64_t>(ws, L.off_part);
    a.ctas = L.sort_ctas;
    a.ek = at<uint32_t>(ws, L.off_ek[0]);
    a.ev = at<uint32_t>(ws, L.off_ev[0]);
    a.cap = L.cap;
    a.tile = L.tile;
    a.ntx = L.ntx;
    a.large_tiles = large_tiles;
    a.tshift = L.tile == 8 ? 3 : (L.tile == 16 ? 4 : 5);
    k_bin_reduce<<<a.ctas, 256, 0, st>>>(a);
    k_bin_scan<<<1, 1024, 0, st>>>(a);
    k_bin_emit<<<a.ctas, 256, 0, st>>>(a);
    count_launches(3);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    // Stable sort of the entries by tile id (only the bits a tile id can use).
    int bits = 0;
    while (bits < 32 && (1ull << bits) < (unsigned long long)L.ntiles) ++bits;
    const int passes = (bits + 7) / 8;
    RadixPass p{};
    p.hist = at<uint32_t>(ws, L.off_hist);
    p.hist_stride = L.hist_ctas;
    p.htot = at<uint32_t>(ws, L.off_htot);
    p.hdr = hdr;
    p.ctas = L.ent_ctas;
    p.n_dev = &hdr->tile_entries32;
    p.depth_pass = -1;
    p.skip_invalid = 0;
    for (int pass = 0; pass < passes; ++pass) {
        p.key_in = at<uint32_t>(ws, L.off_ek[pass & 1]);
        p.val_in = at<uint32_t>(ws, L.off_ev[pass & 1]);
        p.key_out = at<uint32_t>(ws, L.off_ek[(pass + 1) & 1]);
        p.val_out = at<uint32_t>(ws, L.off_ev[(pass + 1) & 1]);
        p.shift = 8u * pass;
        p.mask = 0xFFu;
        e = launch_radix_pass(p, st);
        if (e != cudaSuccess) return e;
    }
    const int sms = sm_count_bin();
    k_tile_offsets<<<sms * 32, 256, 0, st>>>(hdr, at<uint32_t>(ws, L.off_ek[passes & 1]), at<uint32_t>(ws, L.off_toff),
                                              L.ntiles);
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace spl
