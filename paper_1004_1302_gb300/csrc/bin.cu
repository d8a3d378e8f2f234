// Screen-tile binning in two levels, without sorting per-tile entries.
//
// 1. Every visible particle, in render order, adds one entry (super-tile,
//    particle) per super-tile (8 x 8 screen tiles) its box meets; offsets come
//    from a scan of the per-particle counts, so entries sit at fixed places.
//    The entries of particles touching more super-tiles than a threshold are
//    shared out over the whole CTA (the "split particles" idea of Section 3.2
//    applied to the emission of work items).
// 2. One stable radix pass groups the entries by super-tile, keeping render
//    order inside each group.
// 3. Each super-tile's list is cut into units of kUnit entries.  A particle's
//    footprint inside its super-tile is a rectangle of its 8 x 8 fine tiles;
//    per unit the fine-tile counts come from a 2-D difference array, a scan
//    over units and over fine tiles gives every (unit, fine tile) its output
//    position, and one thread per fine tile then walks the unit's entries in
//    order, appending those whose rectangle holds its tile.
//    The result is, for every fine tile (row-major), the particles whose box
//    meets it in render order: bit-exact, as a stable sort by tile would give.
#include "internal.h"
#include "device_util.cuh"

namespace spl {

constexpr int kBinStep = 2048;   // particles per CTA step of the emission kernel

// Number of (super-)tiles of side 2^shift pixels that a pixel box meets.
__device__ __forceinline__ uint32_t cells_of(const ushort4 b, int shift) {
    return (uint32_t)((b.z >> shift) - (b.x >> shift) + 1) * (uint32_t)((b.w >> shift) - (b.y >> shift) + 1);
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
    for (uint64_t k = beg + threadIdx.x; k < end; k += blockDim.x) sum += cells_of(a.box[list[k]], a.sshift);
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
        a.hdr->super_entries = total;
        a.hdr->super32 = (uint32_t)(total < a.cap ? total : a.cap);
        if (total > a.cap) {
            // the fine entries are at least as many: report that lower bound
            a.hdr->status = SPLOTCH_ERR_WORKSPACE;
            a.hdr->tile_entries = total;
        }
    }
}

// Each CTA walks its range in steps of kBinStep particles (list order).  A
// particle meeting at most `large_tiles` super-tiles is written by the thread
// that owns it.  The cells of the step's larger particles are laid end to end
// and dealt to all threads of the CTA, one cell per thread per round; a thread
// finds its cell's particle by binary search over the large particles' first
// cells, so the work is balanced whatever their sizes.
__global__ void __launch_bounds__(256) k_bin_emit(BinArgs a) {
    constexpr int kPer = kBinStep / 256;
    __shared__ uint32_t s_p[kBinStep];        // particle index per item
    __shared__ uint32_t s_off[kBinStep];      // cells per item, then its entry offset within the step
    __shared__ uint32_t s_lcell[kBinStep];    // first cell of each large item among the step's large cells
    __shared__ uint16_t s_lidx[kBinStep];     // items of the large particles, in list order
    __shared__ ushort4 s_box[kBinStep];       // super-tile box per item
    __shared__ unsigned long long ws64[9];
    __shared__ uint32_t ws32[9];
    const uint32_t n = a.hdr->visible;
    const uint32_t *list = a.hdr->sorted_buf ? a.list[1] : a.list[0];
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
                tb = make_ushort4(b.x >> a.sshift, b.y >> a.sshift, b.z >> a.sshift, b.w >> a.sshift);
                nt = (uint32_t)(tb.z - tb.x + 1) * (uint32_t)(tb.w - tb.y + 1);
            }
            s_p[j] = p;
            s_off[j] = nt;
            s_box[j] = tb;
        }
        __syncthreads();
        // blocked arrangement: thread t owns items kPer*t .. kPer*t + kPer - 1
        uint32_t nt[kPer];
        uint32_t mine = 0, mine_lcells = 0, mine_large = 0;
#pragma unroll
        for (int q = 0; q < kPer; ++q) {
            nt[q] = s_off[kPer * threadIdx.x + q];
            mine += nt[q];
            if (nt[q] > a.large_tiles) {
                mine_lcells += nt[q];
                ++mine_large;
            }
        }
        unsigned long long tot2;
        const unsigned long long pre2 =
            block_exclusive_scan64<256>((unsigned long long)mine | ((unsigned long long)mine_lcells << 32), ws64, &tot2);
        uint32_t ltot;
        uint32_t lpos = block_exclusive_scan<256>(mine_large, ws32, &ltot);
        const uint32_t tot = (uint32_t)tot2, lctot = (uint32_t)(tot2 >> 32);
        uint32_t off = (uint32_t)pre2, lcell = (uint32_t)(pre2 >> 32);
#pragma unroll
        for (int q = 0; q < kPer; ++q) {
            const uint32_t j = kPer * threadIdx.x + q;
            s_off[j] = off;
            if (nt[q] > a.large_tiles) {
                s_lidx[lpos] = (uint16_t)j;
                s_lcell[lpos] = lcell;
                ++lpos;
                lcell += nt[q];
            }
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
                        a.ek[e] = (uint32_t)(ty * a.nsx + tx);
                        a.ev[e] = p;
                    }
        }
        // large particles: their cells dealt over the CTA
        for (uint32_t c = threadIdx.x; c < lctot; c += 256) {
            uint32_t lo = 0, hi = ltot;       // last i with s_lcell[i] <= c
            while (hi - lo > 1) {
                const uint32_t mid = (lo + hi) >> 1;
                if (s_lcell[mid] <= c) lo = mid;
                else hi = mid;
            }
            const uint32_t j = s_lidx[lo];
            const uint32_t k = c - s_lcell[lo];
            const ushort4 b = s_box[j];
            const uint32_t w = (uint32_t)(b.z - b.x + 1);
            const uint32_t row = k / w, col = k - row * w;
            const unsigned long long e = running + s_off[j] + k;
            if (e < a.cap) {
                a.ek[e] = (uint32_t)((b.y + row) * a.nsx + b.x + col);
                a.ev[e] = s_p[j];
            }
        }
        nlarge_cta += ltot;
        running += tot;
        __syncthreads();
    }
    if (threadIdx.x == 0 && nlarge_cta) atomicAdd(&a.hdr->n_large, nlarge_cta);
}

// Offsets of groups in a sequence sorted by group id: offsets[g] = first
// entry of group g, offsets[ngroups] = n.
__global__ void __launch_bounds__(256) k_group_offsets(const uint32_t *count, const uint32_t *ids, uint32_t *off,
                                                       uint32_t ngroups) {
    const uint32_t n = *count;
    const uint32_t stride = gridDim.x * blockDim.x;
    if (n == 0) {
        for (uint32_t t = blockIdx.x * blockDim.x + threadIdx.x; t <= ngroups; t += stride) off[t] = 0;
        return;
    }
    for (uint32_t e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += stride) {
        const uint32_t t = ids[e];
        const uint32_t prev = e ? ids[e - 1] + 1u : 0u;
        for (uint32_t tt = prev; tt <= t; ++tt) off[tt] = e;
        if (e == n - 1)
            for (uint32_t tt = t + 1; tt <= ngroups; ++tt) off[tt] = n;
    }
}

// Fine-tile rectangle (columns c0..c1, rows r0..r1, in 0..7) that a
// particle's pixel box meets inside the super-tile whose first fine tile is
// (ox, oy).
struct FineRect {
    int c0, c1, r0, r1;
};
__device__ __forceinline__ FineRect fine_rect(const ushort4 b, int tshift, int ox, int oy) {
    FineRect f;
    f.c0 = max((b.x >> tshift) - ox, 0);
    f.c1 = min((b.z >> tshift) - ox, kSuperSide - 1);
    f.r0 = max((b.y >> tshift) - oy, 0);
    f.r1 = min((b.w >> tshift) - oy, kSuperSide - 1);
    return f;
}

// The same rectangle as a 64-bit mask: bit 8 r + c.
__device__ __forceinline__ uint64_t fine_mask(const FineRect f) {
    if (f.c0 > f.c1 || f.r0 > f.r1) return 0ull;
    const uint64_t row = (0xFFull >> (kSuperSide - 1 - f.c1)) & (0xFFull << f.c0);
    const uint64_t rows = (0xFFull >> (kSuperSide - 1 - f.r1)) & (0xFFull << f.r0);
    // spread the 8 row bits to bytes (bit r -> bit 8 r), then replicate the column pattern
    uint64_t spread = 0;
#pragma unroll
    for (int r = 0; r < kSuperSide; ++r) spread |= ((rows >> r) & 1ull) << (kSuperSide * r);
    return spread * row;
}

// Cut every super-tile's list into units of at most kUnit entries.
__global__ void __launch_bounds__(1024) k_units(FineArgs a) {
    __shared__ uint32_t ws[33];
    uint32_t carry = 0;
    for (uint32_t base = 0; base < a.nsuper; base += 1024) {
        const uint32_t s = base + threadIdx.x;
        uint32_t nseg = 0, b = 0, e = 0;
        if (s < a.nsuper) {
            b = a.soff[s];
            e = a.soff[s + 1];
            nseg = (e - b + kUnit - 1) / kUnit;
        }
        uint32_t tot;
        const uint32_t pre = block_exclusive_scan<1024>(nseg, ws, &tot);
        if (s < a.nsuper) {
            const uint32_t u0 = carry + pre;
            a.ufirst[s] = u0;
            for (uint32_t k = 0; k < nseg && u0 + k < a.max_units; ++k)
                a.units[u0 + k] = make_uint4(s, b + k * kUnit, min(b + (k + 1) * kUnit, e), 0u);
        }
        carry += tot;
    }
    if (threadIdx.x == 0) {
        a.ufirst[a.nsuper] = carry;
        a.hdr->n_units = min(carry, a.max_units);
    }
}

// Per unit: how many of the unit's entries meet each of the super-tile's 64
// fine tiles, accumulated as a 2-D difference array (four updates per entry)
// and summed at the end.
__global__ void __launch_bounds__(256) k_fine_count(FineArgs a) {
    __shared__ int diff[kSuperSide + 1][kSuperSide + 1];
    const uint32_t u = blockIdx.x;
    if (u >= a.hdr->n_units) return;
    const uint4 un = a.units[u];
    const int ox = (int)(un.x % a.nsx) * kSuperSide, oy = (int)(un.x / a.nsx) * kSuperSide;
    if (threadIdx.x < (kSuperSide + 1) * (kSuperSide + 1)) (&diff[0][0])[threadIdx.x] = 0;
    __syncthreads();
    for (uint32_t i = un.y + threadIdx.x; i < un.z; i += 256) {
        const FineRect f = fine_rect(a.box[a.sval[i]], a.tshift, ox, oy);
        atomicAdd(&diff[f.r0][f.c0], 1);
        atomicAdd(&diff[f.r0][f.c1 + 1], -1);
        atomicAdd(&diff[f.r1 + 1][f.c0], -1);
        atomicAdd(&diff[f.r1 + 1][f.c1 + 1], 1);
    }
    __syncthreads();
    if (threadIdx.x < 64) {
        const int r = threadIdx.x / kSuperSide, c = threadIdx.x % kSuperSide;
        int v = 0;
        for (int rr = 0; rr <= r; ++rr)
            for (int cc = 0; cc <= c; ++cc) v += diff[rr][cc];
        a.ucnt[(size_t)u * 64 + threadIdx.x] = (uint32_t)v;
    }
}

// Per super-tile: each fine tile's running count over the super-tile's units
// (exclusive, in place) and its total, written as the fine tile's count.
__global__ void __launch_bounds__(64) k_fine_unit_scan(FineArgs a) {
    const uint32_t s = blockIdx.x, t = threadIdx.x;
    uint32_t run = 0;
    const uint32_t u1 = min(a.ufirst[s + 1], a.max_units);
    for (uint32_t u = a.ufirst[s]; u < u1; ++u) {
        const size_t q = (size_t)u * 64 + t;
        const uint32_t c = a.ucnt[q];
        a.ucnt[q] = run;
        run += c;
    }
    const uint32_t tx = (s % a.nsx) * kSuperSide + (t % kSuperSide), ty = (s / a.nsx) * kSuperSide + t / kSuperSide;
    if (tx < a.ntx && ty < a.nty) a.toff[ty * a.ntx + tx] = run;
}

// Fine-tile counts -> offsets (exclusive scan in place), total D.
__global__ void __launch_bounds__(1024) k_fine_offsets(FineArgs a) {
    __shared__ unsigned long long ws[33];
    constexpr int kPer = 8;
    unsigned long long carry = 0;
    for (uint32_t base = 0; base < a.ntiles; base += 1024 * kPer) {
        uint32_t v[kPer];
        unsigned long long sum = 0;
#pragma unroll
        for (int q = 0; q < kPer; ++q) {
            const uint32_t j = base + threadIdx.x * kPer + q;
            v[q] = j < a.ntiles ? a.toff[j] : 0u;
            sum += v[q];
        }
        unsigned long long tot;
        unsigned long long run = carry + block_exclusive_scan64<1024>(sum, ws, &tot);
#pragma unroll
        for (int q = 0; q < kPer; ++q) {
            const uint32_t j = base + threadIdx.x * kPer + q;
            if (j < a.ntiles) a.toff[j] = (uint32_t)(run < a.cap ? run : a.cap);
            run += v[q];
        }
        carry += tot;
    }
    if (threadIdx.x == 0) {
        a.toff[a.ntiles] = (uint32_t)(carry < a.cap ? carry : a.cap);
        // after an overflow of the super-tile entries the count is only a lower bound
        const bool exact = a.hdr->status == SPLOTCH_OK;
        a.hdr->tile_entries = exact || carry > a.hdr->tile_entries ? carry : a.hdr->tile_entries;
        a.hdr->tile_entries32 = (uint32_t)(carry < a.cap ? carry : a.cap);
        if (carry > a.cap) a.hdr->status = SPLOTCH_ERR_WORKSPACE;
    }
}

// Per unit, one thread per fine tile: walk the unit's entries in order
// (256 at a time: each thread stages four entries' particles and fine-tile
// masks in shared memory, read back by broadcast) and append the particle of
// every entry whose mask has the thread's tile, starting at the tile's offset
// plus the unit's offset within the tile.  Render order is kept because each
// tile's entries are appended in list order by one thread.
__global__ void __launch_bounds__(64) k_fine_emit(FineArgs a) {
    constexpr int kStage = 256;
    __shared__ uint2 sm[kStage];     // mask as two words
    __shared__ uint32_t sp[kStage];
    const uint32_t u = blockIdx.x;
    if (u >= a.hdr->n_units) return;
    const uint4 un = a.units[u];
    const uint32_t s = un.x, t = threadIdx.x;
    const int ox = (int)(s % a.nsx) * kSuperSide, oy = (int)(s / a.nsx) * kSuperSide;
    const uint32_t tx = (uint32_t)ox + (t % kSuperSide), ty = (uint32_t)oy + t / kSuperSide;
    uint64_t pos = (tx < a.ntx && ty < a.nty) ? (uint64_t)a.toff[ty * a.ntx + tx] + a.ucnt[(size_t)u * 64 + t] : 0;
    const uint32_t word = t >> 5, bit = t & 31;
    for (uint32_t i0 = un.y; i0 < un.z; i0 += kStage) {
        uint32_t pv[kStage / 64];
#pragma unroll
        for (int q = 0; q < kStage / 64; ++q) {
            const uint32_t i = i0 + q * 64 + t;
            pv[q] = i < un.z ? a.sval[i] : 0u;
        }
#pragma unroll
        for (int q = 0; q < kStage / 64; ++q) {
            const uint32_t i = i0 + q * 64 + t;
            const uint64_t m = i < un.z ? fine_mask(fine_rect(a.box[pv[q]], a.tshift, ox, oy)) : 0ull;
            sm[q * 64 + t] = make_uint2((uint32_t)m, (uint32_t)(m >> 32));
            sp[q * 64 + t] = pv[q];
        }
        __syncthreads();
        const uint32_t nb = min((uint32_t)kStage, un.z - i0);
#pragma unroll 4
        for (uint32_t k = 0; k < nb; ++k) {
            const uint2 m = sm[k];
            if ((((word ? m.y : m.x) >> bit) & 1u)) {
                if (pos < a.cap) a.list[pos] = sp[k];
                ++pos;
            }
        }
        __syncthreads();
    }
}

static int sm_count_bin() {
    int dev = 0, v = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
    return v > 0 ? v : 148;
}

int super_passes(uint32_t nsuper) {
    int bits = 0;
    while (bits < 32 && (1ull << bits) < (unsigned long long)nsuper) ++bits;
    return (bits + 7) / 8;
}

uint64_t fine_list_offset(const Layout &L) { return L.off_ek[1 - (super_passes(L.nsuper) & 1)]; }

cudaError_t launch_bin(void *ws, const Layout &L, uint32_t large_tiles, cudaStream_t st) {
    Header *hdr = header(ws);
    const int tshift = L.tile == 8 ? 3 : (L.tile == 16 ? 4 : 5);
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
    a.nsx = (int)L.nsx;
    a.sshift = tshift + 3;
    a.large_tiles = large_tiles;
    k_bin_reduce<<<a.ctas, 256, 0, st>>>(a);
    k_bin_scan<<<1, 1024, 0, st>>>(a);
    k_bin_emit<<<a.ctas, 256, 0, st>>>(a);
    count_launches(3);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    // group the entries by super-tile (stable: render order kept inside a group)
    const int passes = super_passes(L.nsuper);
    RadixPass p{};
    p.hist = at<uint32_t>(ws, L.off_hist);
    p.hist_stride = L.hist_ctas;
    p.htot = at<uint32_t>(ws, L.off_htot);
    p.hdr = hdr;
    p.ctas = L.ent_ctas;
    p.n_dev = &hdr->super32;
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
    const int f = passes & 1;
    const int sms = sm_count_bin();
    k_group_offsets<<<sms * 8, 256, 0, st>>>(&hdr->super32, at<uint32_t>(ws, L.off_ek[f]), at<uint32_t>(ws, L.off_soff),
                                             L.nsuper);
    FineArgs fa{};
    fa.hdr = hdr;
    fa.skey = at<uint32_t>(ws, L.off_ek[f]);
    fa.sval = at<uint32_t>(ws, L.off_ev[f]);
    fa.soff = at<uint32_t>(ws, L.off_soff);
    fa.ufirst = at<uint32_t>(ws, L.off_ufirst);
    fa.units = at<uint4>(ws, L.off_units);
    fa.ucnt = at<uint32_t>(ws, L.off_ucnt);
    fa.toff = at<uint32_t>(ws, L.off_toff);
    fa.list = at<uint32_t>(ws, fine_list_offset(L));
    fa.box = at<ushort4>(ws, L.off_box);
    fa.cap = L.cap;
    fa.nsuper = L.nsuper;
    fa.nsx = L.nsx;
    fa.ntx = (uint32_t)L.ntx;
    fa.nty = (uint32_t)L.nty;
    fa.ntiles = L.ntiles;
    fa.max_units = L.max_units;
    fa.tshift = tshift;
    k_units<<<1, 1024, 0, st>>>(fa);
    k_fine_count<<<L.max_units, 256, 0, st>>>(fa);
    k_fine_unit_scan<<<L.nsuper, 64, 0, st>>>(fa);
    k_fine_offsets<<<1, 1024, 0, st>>>(fa);
    k_fine_emit<<<L.max_units, 64, 0, st>>>(fa);
    count_launches(6);
    return cudaGetLastError();
}

}  // namespace spl
