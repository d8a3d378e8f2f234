// Screen-tile binning.  Every visible particle, in render order, adds one
// entry (tile id, particle) per tile its box meets.  Entry offsets come from
// an exclusive scan of the per-particle tile counts, so the entries of one
// particle sit at fixed positions whatever the thread that writes them.
// Particles touching more tiles than a threshold are written by a whole CTA
// (the "split particles" idea of Section 3.2 applied to the emission of
// work items).  A stable radix sort by tile id then yields per-tile lists in
// render order, and a boundary pass turns the sorted ids into tile offsets.
#include "internal.h"
#include "device_util.cuh"

namespace spl {

__device__ __forceinline__ uint32_t tiles_of(const ushort4 b, int T) {
    return (uint32_t)(b.z / T - b.x / T + 1) * (uint32_t)(b.w / T - b.y / T + 1);
}

__device__ __forceinline__ void bin_range(uint32_t ctas, uint32_t n, uint64_t *beg, uint64_t *end) {
    const uint64_t tiles = (n + (uint64_t)kSortTile - 1) / kSortTile;
    const uint64_t tpc = (tiles + ctas - 1) / ctas;
    *beg = (uint64_t)blockIdx.x * tpc * kSortTile;
    uint64_t e = *beg + tpc * kSortTile;
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
    for (uint64_t k = beg + threadIdx.x; k < end; k += blockDim.x) sum += tiles_of(a.box[list[k]], a.tile);
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

// Each CTA walks its range in 4096-item steps; thread t owns items
// 16t..16t+15 of a step so that a block scan gives offsets in list order.
__global__ void __launch_bounds__(256) k_bin_emit(BinArgs a) {
    __shared__ unsigned long long ws[9];
    const uint32_t n = a.hdr->visible;
    const uint32_t *list = a.hdr->sorted_buf ? a.list[1] : a.list[0];
    uint64_t beg, end;
    bin_range(a.ctas, n, &beg, &end);
    unsigned long long running = a.part[blockIdx.x];
    constexpr int kPer = kSortTile / 256;
    for (uint64_t step = beg; step < end; step += kSortTile) {
        uint32_t p[kPer], nt[kPer];
        unsigned long long mine = 0;
#pragma unroll
        for (int q = 0; q < kPer; ++q) {
            const uint64_t k = step + threadIdx.x * kPer + q;
            p[q] = k < end ? list[k] : 0u;
            nt[q] = k < end ? tiles_of(a.box[p[q]], a.tile) : 0u;
            mine += nt[q];
        }
        unsigned long long tot;
        unsigned long long off = running + block_exclusive_scan64<256>(mine, ws, &tot);
#pragma unroll
        for (int q = 0; q < kPer; ++q) {
            if (nt[q] > a.large_tiles) {
                const uint32_t slot = atomicAdd(&a.hdr->n_large, 1u);
                a.large[slot] = make_uint2((uint32_t)(off < a.cap ? off : a.cap), p[q]);
            } else if (nt[q]) {
                const ushort4 b = a.box[p[q]];
                const int tx0 = b.x / a.tile, tx1 = b.z / a.tile, ty0 = b.y / a.tile, ty1 = b.w / a.tile;
                unsigned long long e = off;
                for (int ty = ty0; ty <= ty1; ++ty)
                    for (int tx = tx0; tx <= tx1; ++tx, ++e)
                        if (e < a.cap) {
                            a.ek[e] = (uint32_t)(ty * a.ntx + tx);
                            a.ev[e] = p[q];
                        }
            }
            off += nt[q];
        }
        running += tot;
    }
}

// Cooperative emission of the large particles: one CTA per particle.
__global__ void __launch_bounds__(256) k_emit_large(BinArgs a) {
    const uint32_t nl = a.hdr->n_large;
    for (uint32_t L = blockIdx.x; L < nl; L += gridDim.x) {
        const uint2 item = a.large[L];
        const ushort4 b = a.box[item.y];
        const int tx0 = b.x / a.tile, ty0 = b.y / a.tile;
        const uint32_t w = (uint32_t)(b.z / a.tile - tx0 + 1), h = (uint32_t)(b.w / a.tile - ty0 + 1);
        const uint32_t nt = w * h;
        for (uint32_t j = threadIdx.x; j < nt; j += blockDim.x) {
            const unsigned long long e = (unsigned long long)item.x + j;
            if (e < a.cap) {
                a.ek[e] = (uint32_t)((ty0 + (int)(j / w)) * a.ntx + tx0 + (int)(j % w));
                a.ev[e] = item.y;
            }
        }
    }
}

// Tile offsets from tile-sorted entry ids: offsets[t] = first entry of tile t.
__global__ void __launch_bounds__(256) k_tile_offsets(const Header *hdr, const uint32_t *ek, uint32_t *toff,
                                                      uint32_t ntiles) {
    const uint32_t D = hdr->tile_entries32;
    if (D == 0) {
        for (uint32_t t = blockIdx.x * blockDim.x + threadIdx.x; t <= ntiles; t += gridDim.x * blockDim.x) toff[t] = 0;
        return;
    }
    for (uint32_t e = blockIdx.x * blockDim.x + threadIdx.x; e < D; e += gridDim.x * blockDim.x) {
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
    a.large = at<uint2>(ws, L.off_large);
    a.cap = L.cap;
    a.tile = L.tile;
    a.ntx = L.ntx;
    a.large_tiles = large_tiles;
    k_bin_reduce<<<a.ctas, 256, 0, st>>>(a);
    k_bin_scan<<<1, 1024, 0, st>>>(a);
    k_bin_emit<<<a.ctas, 256, 0, st>>>(a);
    const int sms = sm_count_bin();
    k_emit_large<<<sms * 4, 256, 0, st>>>(a);
    count_launches(4);
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
    k_tile_offsets<<<sms * 4, 256, 0, st>>>(hdr, at<uint32_t>(ws, L.off_ek[passes & 1]), at<uint32_t>(ws, L.off_toff),
                                             L.ntiles);
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace spl
