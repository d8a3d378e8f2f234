// Screen-tile binning in two levels, without sorting per-tile entries.
//
// 1. Every visible particle, in render order, adds one entry (super-tile,
//    particle) per super-tile (8 x 8 screen tiles) its box meets; offsets come
//    from a scan of the per-particle counts, so entries sit at fixed places.
//    The count pass gathers each particle's box once and stores it (in tiles)
//    in list order, so the emission reads it sequentially.  The entries of
//    particles touching more super-tiles than a threshold are shared out over
//    the whole CTA (the "split particles" idea of Section 3.2 applied to the
//    emission of work items).  An entry's key holds the super-tile id and,
//    above it, the rectangle of fine tiles the particle meets there.
// 2. One stable radix pass over the id bits groups the entries by super-tile,
//    keeping render order inside each group.
// 3. Each super-tile's list is cut into units of kUnit entries.  Per unit the
//    fine-tile counts come from a 2-D difference array over the rectangles, a
//    scan over units and over fine tiles gives every (unit, fine tile) its
//    output position, and row and column ballots over each warp's entries give
//    every (entry, fine tile) its rank inside the tile.
//    The result is, for every fine tile (row-major), the particles whose box
//    meets it in render order: bit-exact, as a stable sort by tile would give.
#include "internal.h"
#include "device_util.cuh"

namespace spl {

constexpr int kBinStep = 2048;   // particles per CTA step of the emission kernel

constexpr int kSuperShift = 3;   // log2 of kSuperSide

// Fine-tile rectangle code of an entry key: columns c0..c1 and rows r0..r1 of
// the tile box t inside super-tile (sx, sy).
__device__ __forceinline__ uint32_t rect_code(const ushort4 t, int sx, int sy) {
    const int ox = sx << kSuperShift, oy = sy << kSuperShift;
    const uint32_t c0 = (uint32_t)max((int)t.x - ox, 0), c1 = (uint32_t)min((int)t.z - ox, kSuperSide - 1);
    const uint32_t r0 = (uint32_t)max((int)t.y - oy, 0), r1 = (uint32_t)min((int)t.w - oy, kSuperSide - 1);
    return c0 | (c1 << 3) | (r0 << 6) | (r1 << 9);
}

__device__ __forceinline__ uint32_t entry_key(const ushort4 t, int sx, int sy, int nsx) {
    return (uint32_t)(sy * nsx + sx) | (rect_code(t, sx, sy) << kSidBits);
}

// Number of (super-)tiles of side 2^shift units that a box meets.
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

// Tile box from the depth sort's payload (8 bits per edge).
__device__ __forceinline__ ushort4 unpack_tile_box(uint32_t v) {
    return make_ushort4((unsigned short)(v & 0xFFu), (unsigned short)((v >> 8) & 0xFFu),
                        (unsigned short)((v >> 16) & 0xFFu), (unsigned short)(v >> 24));
}

// Count pass when the tile boxes came through the depth sort in render
// order: a sequential read, four boxes per thread at a time.
__global__ void __launch_bounds__(256) k_bin_reduce_pay(BinArgs a) {
    pdl_enter();
    __shared__ unsigned long long ws[9];
    const uint32_t n = a.hdr->visible;
    const uint32_t *pay = a.hdr->sorted_buf ? a.pk[1] : a.pk[0];
    uint64_t beg, end;
    bin_range(a.ctas, n, &beg, &end);
    unsigned long long sum = 0;
    for (uint64_t k = beg + 4 * threadIdx.x; k < end; k += 4 * blockDim.x) {
        uint32_t v[4];
        if (k + 4 <= end) {
            const uint4 q = *reinterpret_cast<const uint4 *>(pay + k);
            v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
        } else {
#pragma unroll
            for (int u = 0; u < 4; ++u) v[u] = k + u < end ? pay[k + u] : 0x000000FFu;   // x0 > x1: empty
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const ushort4 t = unpack_tile_box(v[u]);
            if (t.x <= t.z) sum += cells_of(t, kSuperShift);
        }
    }
    unsigned long long tot;
    block_exclusive_scan64<256>(sum, ws, &tot);
    if (threadIdx.x == 0) a.part[blockIdx.x] = tot;
}

// PACKED: the transform's packed tile boxes (4 B) are gathered and stored
// packed; otherwise the 8 B pixel boxes are gathered and converted.
template <bool PACKED>
__global__ void __launch_bounds__(256) k_bin_reduce(BinArgs a) {
    pdl_enter();
    __shared__ unsigned long long ws[9];
    const uint32_t n = a.hdr->visible;
    const uint32_t *list = a.hdr->sorted_buf ? a.list[1] : a.list[0];
    uint64_t beg, end;
    bin_range(a.ctas, n, &beg, &end);
    unsigned long long sum = 0;
    // eight independent gathers in flight per thread (the boxes are read in
    // render order, i.e. at random)
    constexpr int kIlp = 8;
    for (uint64_t k0 = beg; k0 < end; k0 += (uint64_t)kIlp * blockDim.x) {
        uint32_t p[kIlp];
        ushort4 b[kIlp];
#pragma unroll
        for (int u = 0; u < kIlp; ++u) {
            const uint64_t k = k0 + (uint64_t)u * blockDim.x + threadIdx.x;
            p[u] = k < end ? list[k] : 0xFFFFFFFFu;
        }
#pragma unroll
        for (int u = 0; u < kIlp; ++u) {
            const bool ok = p[u] != 0xFFFFFFFFu && SPL_CHECK(a.hdr, p[u] < a.hdr->layout.n);
            if (PACKED) b[u] = unpack_tile_box(ok ? a.tbox[p[u]] : 0x000000FFu);
            else b[u] = ok ? a.box[p[u]] : make_ushort4(1, 1, 0, 0);
        }
#pragma unroll
        for (int u = 0; u < kIlp; ++u) {
            const uint64_t k = k0 + (uint64_t)u * blockDim.x + threadIdx.x;
            if (k >= end) continue;
            // the particle's box in tiles, stored in list order for the emission
            const ushort4 t = PACKED || b[u].x > b[u].z ? b[u]
                                                         : make_ushort4(b[u].x >> a.tshift, b[u].y >> a.tshift,
                                                                        b[u].z >> a.tshift, b[u].w >> a.tshift);
            if (t.x <= t.z) sum += cells_of(t, kSuperShift);
            if (PACKED) a.psbox[k] = (uint32_t)t.x | ((uint32_t)t.y << 8) | ((uint32_t)t.z << 16) | ((uint32_t)t.w << 24);
            else a.sbox[k] = t.x <= t.z ? t : make_ushort4(1, 1, 0, 0);
        }
    }
    unsigned long long tot;
    block_exclusive_scan64<256>(sum, ws, &tot);
    if (threadIdx.x == 0) a.part[blockIdx.x] = tot;
}

__global__ void __launch_bounds__(1024) k_bin_scan(BinArgs a) {
    pdl_enter();
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

// Each CTA walks its range in steps of kBinStep particles (list order); warp
// w takes the step's w-th run of 256 particles, lane l the run's particles
// 8 l .. 8 l + 7, kept in registers.  A lane sums its own particles; one warp
// scan of (cells, large cells) and one of the large count give each particle
// its first entry within the warp's run, a scan of the 8 warp totals places
// the runs.  A particle meeting at
// most `large_tiles` super-tiles is written by its own lane.  The larger ones
// go to the warp's segment of shared memory; their cells are laid end to end
// (warp by warp, list order) and dealt to all threads of the CTA, one cell per
// thread per round.  A thread finds its cell's warp from the warp totals and
// its particle by binary search over the segment's first cells, so the work
// is balanced whatever the particles' sizes.
// PACKED: the tile boxes in render order are packed (a.pk: the depth sort's
// payload or the count pass's packed copy); otherwise a.sbox.
template <bool PACKED>
__global__ void __launch_bounds__(256, 3) k_bin_emit(BinArgs a) {
    pdl_enter();
    constexpr int kRounds = kBinStep / 256;
    __shared__ uint32_t s_lp[kBinStep];       // large particles, per warp segment of 256, in list order
    __shared__ uint32_t s_loff[kBinStep];     // their first entry within the warp's run
    __shared__ uint32_t s_lcell[kBinStep];    // their first cell among the warp's large cells
    __shared__ ushort4 s_lbox[kBinStep];      // their boxes in tiles
    __shared__ uint32_t s_wtot[3][8];         // per warp: cells, large particles, large cells
    const uint32_t n = a.hdr->visible;
    const uint32_t *list = a.hdr->sorted_buf ? a.list[1] : a.list[0];
    const uint32_t *pk = a.hdr->sorted_buf ? a.pk[1] : a.pk[0];
    const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint64_t beg, end;
    bin_range(a.ctas, n, &beg, &end);
    unsigned long long running = a.part[blockIdx.x];
    uint32_t nlarge_cta = 0;
    for (uint64_t step = beg; step < end; step += kBinStep) {
        const uint32_t m = (uint32_t)min((uint64_t)kBinStep, end - step);
        uint32_t p[kRounds], off[kRounds];
        ushort4 tb[kRounds];                  // box in tiles; (1, 1, 0, 0): no entries
        // lane l owns the warp run's items 8 l .. 8 l + 7 (consecutive in list order)
        uint32_t nt[kRounds];
        uint32_t my_cells = 0, my_lcells = 0, my_nl = 0;
#pragma unroll
        for (int q = 0; q < kRounds; ++q) {
            const uint32_t j = warp * 256u + lane * kRounds + q;
            nt[q] = 0;
            p[q] = 0;
            tb[q] = make_ushort4(1, 1, 0, 0);
            if (j < m) {
                p[q] = list[step + j];
                tb[q] = PACKED ? unpack_tile_box(pk[step + j]) : a.sbox[step + j];
                if (tb[q].x <= tb[q].z) nt[q] = cells_of(tb[q], kSuperShift);
            }
            const bool big = nt[q] > a.large_tiles;
            my_cells += nt[q];
            my_lcells += big ? nt[q] : 0u;
            my_nl += big ? 1u : 0u;
        }
        // one scan of (cells, large cells) and one of the large count place the lane's items in the run
        const unsigned long long inc2 =
            warp_inclusive_scan64((unsigned long long)my_cells | ((unsigned long long)my_lcells << 32));
        const uint32_t incl = warp_inclusive_scan(my_nl);
        const unsigned long long tot2 = __shfl_sync(0xFFFFFFFFu, inc2, 31);
        const uint32_t cells = (uint32_t)tot2, lcells = (uint32_t)(tot2 >> 32);
        const uint32_t nl = __shfl_sync(0xFFFFFFFFu, incl, 31);
        uint32_t o = (uint32_t)inc2 - my_cells, lo_cell = (uint32_t)(inc2 >> 32) - my_lcells, lr = incl - my_nl;
#pragma unroll
        for (int q = 0; q < kRounds; ++q) {
            off[q] = o;
            if (nt[q] > a.large_tiles) {
                const uint32_t r = warp * 256u + lr;
                s_lp[r] = p[q];
                s_loff[r] = o;
                s_lcell[r] = lo_cell;
                s_lbox[r] = tb[q];
                tb[q] = make_ushort4(1, 1, 0, 0);    // nothing left for the lane to write
                lo_cell += nt[q];
                ++lr;
            }
            o += nt[q];
        }
        if (lane == 0) {
            s_wtot[0][warp] = cells;
            s_wtot[1][warp] = nl;
            s_wtot[2][warp] = lcells;
        }
        __syncthreads();
        uint32_t wc[8], wl[8], wlc[8];
        uint32_t tot = 0, ltot = 0, lctot = 0;
#pragma unroll
        for (int w = 0; w < 8; ++w) {
            wc[w] = tot;
            wl[w] = s_wtot[1][w];
            wlc[w] = lctot;
            tot += s_wtot[0][w];
            ltot += wl[w];
            lctot += s_wtot[2][w];
        }
        uint32_t base = 0;
#pragma unroll
        for (int w = 0; w < 8; ++w)
            if ((uint32_t)w == warp) base = wc[w];
        // small particles: the owner writes its entries
#pragma unroll
        for (int q = 0; q < kRounds; ++q) {
            const ushort4 t = tb[q];
            if (t.x > t.z) continue;
            unsigned long long e = running + base + off[q];
            for (int sy = t.y >> kSuperShift; sy <= (t.w >> kSuperShift); ++sy)
                for (int sx = t.x >> kSuperShift; sx <= (t.z >> kSuperShift); ++sx, ++e)
                    if (e < a.cap) {
                        a.ek[e] = entry_key(t, sx, sy, a.nsx);
                        a.ev[e] = p[q];
                    }
        }
        // large particles: their cells dealt over the CTA
        for (uint32_t c = threadIdx.x; c < lctot; c += 256) {
            uint32_t seg = 0, segn = wl[0], cbase = wc[0], lbase = wlc[0];
#pragma unroll
            for (int w = 1; w < 8; ++w)
                if (wlc[w] <= c) {
                    seg = w;
                    segn = wl[w];
                    cbase = wc[w];
                    lbase = wlc[w];
                }
            const uint32_t cl = c - lbase;
            const uint32_t *lc = s_lcell + seg * 256u;
            uint32_t lo = 0, hi = segn;       // last i with lc[i] <= cl
            while (hi - lo > 1) {
                const uint32_t mid = (lo + hi) >> 1;
                if (lc[mid] <= cl) lo = mid;
                else hi = mid;
            }
            const uint32_t i = seg * 256u + lo;
            const uint32_t k = cl - lc[lo];
            const ushort4 t = s_lbox[i];
            const int sx0 = t.x >> kSuperShift, sy0 = t.y >> kSuperShift;
            const uint32_t w = (uint32_t)((t.z >> kSuperShift) - sx0 + 1);
            const uint32_t row = k / w, col = k - row * w;
            const unsigned long long e = running + cbase + s_loff[i] + k;
            if (e < a.cap) {
                a.ek[e] = entry_key(t, sx0 + (int)col, sy0 + (int)row, a.nsx);
                a.ev[e] = s_lp[i];
            }
        }
        nlarge_cta += ltot;
        running += tot;
        __syncthreads();
    }
    if (threadIdx.x == 0 && nlarge_cta) atomicAdd(&a.hdr->n_large, nlarge_cta);
}

// Offsets of groups in a sequence sorted by group id (the key's low kSidBits
// bits): offsets[g] = first entry of group g, offsets[ngroups] = n.
__global__ void __launch_bounds__(256) k_group_offsets(const uint32_t *count, const uint32_t *ids, uint32_t *off,
                                                       uint32_t ngroups) {
    pdl_enter();
    const uint32_t n = *count;
    const uint32_t stride = gridDim.x * blockDim.x;
    if (n == 0) {
        for (uint32_t t = blockIdx.x * blockDim.x + threadIdx.x; t <= ngroups; t += stride) off[t] = 0;
        return;
    }
    for (uint32_t e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += stride) {
        const uint32_t t = ids[e] & kSidMask;
        const uint32_t prev = e ? (ids[e - 1] & kSidMask) + 1u : 0u;
        for (uint32_t tt = prev; tt <= t; ++tt) off[tt] = e;
        if (e == n - 1)
            for (uint32_t tt = t + 1; tt <= ngroups; ++tt) off[tt] = n;
    }
}

// Fine-tile rectangle (columns c0..c1, rows r0..r1, in 0..7) of an entry,
// from its key.
struct FineRect {
    int c0, c1, r0, r1;
};
__device__ __forceinline__ FineRect key_rect(uint32_t key) {
    const uint32_t r = key >> kSidBits;
    FineRect f;
    f.c0 = (int)(r & 7u);
    f.c1 = (int)((r >> 3) & 7u);
    f.r0 = (int)((r >> 6) & 7u);
    f.r1 = (int)((r >> 9) & 7u);
    return f;
}

// Cut every super-tile's list into units of at most kUnit entries.
__global__ void __launch_bounds__(1024) k_units(FineArgs a) {
    pdl_enter();
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
    pdl_enter();
    __shared__ int diff[kSuperSide + 1][kSuperSide + 1];
    const uint32_t u = blockIdx.x;
    if (u >= a.hdr->n_units) return;
    const uint4 un = a.units[u];
    if (threadIdx.x < (kSuperSide + 1) * (kSuperSide + 1)) (&diff[0][0])[threadIdx.x] = 0;
    __syncthreads();
    // a unit is at most kUnit = 8 x 256 entries: every thread's loads are in flight together
    static_assert(kUnit <= 8 * 256, "one load per thread and round");
    uint32_t key[8];
#pragma unroll
    for (int r = 0; r < 8; ++r) {
        const uint32_t i = un.y + threadIdx.x + 256u * r;
        key[r] = i < un.z ? a.skey[i] : 0xFFFFFFFFu;
    }
#pragma unroll
    for (int r = 0; r < 8; ++r) {
        if (un.y + threadIdx.x + 256u * r >= un.z) continue;
        const FineRect f = key_rect(key[r]);
        atomicAdd(&diff[f.r0][f.c0], 1);
        atomicAdd(&diff[f.r0][f.c1 + 1], -1);
        atomicAdd(&diff[f.r1 + 1][f.c0], -1);
        atomicAdd(&diff[f.r1 + 1][f.c1 + 1], 1);
    }
    __syncthreads();
    // the 2-D prefix sum of the difference array: along each row (shuffles in
    // groups of eight lanes), then down each column
    __shared__ int rowp[kSuperSide][kSuperSide];
    const int r = threadIdx.x / kSuperSide, c = threadIdx.x % kSuperSide;
    if (threadIdx.x < 64) {
        int v = diff[r][c];
#pragma unroll
        for (int d = 1; d < kSuperSide; d <<= 1) {
            const int o = __shfl_up_sync(0xFFFFFFFFu, v, d, kSuperSide);
            if (c >= d) v += o;
        }
        rowp[r][c] = v;
    }
    __syncthreads();
    if (threadIdx.x < 64) {
        int v = 0;
        for (int rr = 0; rr <= r; ++rr) v += rowp[rr][c];
        a.ucnt[(size_t)u * 64 + threadIdx.x] = (uint32_t)v;
    }
}

// Per super-tile: each fine tile's running count over the super-tile's units
// (exclusive, in place) and its total, written as the fine tile's count.  The
// units are cut into 16 chunks: each chunk's sum, a scan over the chunks per
// fine tile, then the running counts inside each chunk.
__global__ void __launch_bounds__(1024) k_fine_unit_scan(FineArgs a) {
    pdl_enter();
    constexpr int kChunks = 16;
    __shared__ uint32_t part[kChunks][64];
    const uint32_t s = blockIdx.x, t = threadIdx.x & 63u, g = threadIdx.x >> 6;
    const uint32_t u0 = a.ufirst[s], u1 = min(a.ufirst[s + 1], a.max_units);
    const uint32_t nu = u1 > u0 ? u1 - u0 : 0u, per = (nu + kChunks - 1) / kChunks;
    const uint32_t b = u0 + g * per, e = min(b + per, u1);
    // eight units' counts in flight at a time (a thread walks up to thousands of units)
    constexpr uint32_t kBatch = 8;
    uint32_t sum = 0;
    uint32_t u = b;
    for (; u + kBatch <= e; u += kBatch) {
        uint32_t v[kBatch];
#pragma unroll
        for (uint32_t k = 0; k < kBatch; ++k) v[k] = a.ucnt[(size_t)(u + k) * 64 + t];
#pragma unroll
        for (uint32_t k = 0; k < kBatch; ++k) sum += v[k];
    }
    for (; u < e; ++u) sum += a.ucnt[(size_t)u * 64 + t];
    part[g][t] = sum;
    __syncthreads();
    if (g == 0) {
        uint32_t run = 0;
#pragma unroll
        for (int k = 0; k < kChunks; ++k) {
            const uint32_t v = part[k][t];
            part[k][t] = run;
            run += v;
        }
        const uint32_t tx = (s % a.nsx) * kSuperSide + (t % kSuperSide), ty = (s / a.nsx) * kSuperSide + t / kSuperSide;
        if (tx < a.ntx && ty < a.nty) a.toff[ty * a.ntx + tx] = run;
    }
    __syncthreads();
    uint32_t run = part[g][t];
    u = b;
    for (; u + kBatch <= e; u += kBatch) {
        uint32_t v[kBatch];
#pragma unroll
        for (uint32_t k = 0; k < kBatch; ++k) v[k] = a.ucnt[(size_t)(u + k) * 64 + t];
#pragma unroll
        for (uint32_t k = 0; k < kBatch; ++k) {
            a.ucnt[(size_t)(u + k) * 64 + t] = run;
            run += v[k];
        }
    }
    for (; u < e; ++u) {
        const size_t q = (size_t)u * 64 + t;
        const uint32_t c = a.ucnt[q];
        a.ucnt[q] = run;
        run += c;
    }
}

// Super-tile offsets from the digit totals of a single grouping pass (the
// totals are the super-tiles' entry counts).
__global__ void __launch_bounds__(256) k_soff_from_totals(const uint32_t *htot, uint32_t *off, uint32_t nsuper) {
    pdl_enter();
    __shared__ uint32_t ws[9];
    const uint32_t t = threadIdx.x;
    uint32_t tot;
    const uint32_t pre = block_exclusive_scan<256>(t < nsuper ? htot[t] : 0u, ws, &tot);
    if (t < nsuper) off[t] = pre;
    if (t == 0) off[nsuper] = tot;
}

// Render cost class of a tile from its list length c: c itself below 4,
// else four classes per power of two (the two bits after the leading one).
constexpr int kCostClasses = 128;
__device__ __forceinline__ int cost_class(uint32_t c) {
    if (c < 4) return (int)c;
    const int e = 31 - __clz(c);
    return min(kCostClasses - 1, e * 4 + (int)((c >> (e - 2)) & 3u));
}

// Fine-tile counts -> offsets (exclusive scan in place), total D.  Also the
// render order of the tiles: longest lists first (by cost class), so that
// the tiles that take longest start first and the short ones fill the end of
// the render instead of one long tile running on alone.  The order inside a
// class is whatever the atomics give: the tiles are independent, so the
// order changes when a tile runs, never the image.
__global__ void __launch_bounds__(1024) k_fine_offsets(FineArgs a) {
    pdl_enter();
    __shared__ unsigned long long ws[33];
    __shared__ uint32_t s_class[kCostClasses];
    constexpr int kPer = 8;
    if (threadIdx.x < kCostClasses) s_class[threadIdx.x] = 0;
    __syncthreads();
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
            const unsigned long long lo = run < a.cap ? run : a.cap;
            run += v[q];
            const unsigned long long hi = run < a.cap ? run : a.cap;
            if (j < a.ntiles) {
                a.toff[j] = (uint32_t)lo;
                atomicAdd(&s_class[cost_class((uint32_t)(hi - lo))], 1u);   // the length the render will see
            }
        }
        carry += tot;
    }
    __syncthreads();   // every tile's class is counted before the class offsets are taken
    if (threadIdx.x == 0) {
        a.toff[a.ntiles] = (uint32_t)(carry < a.cap ? carry : a.cap);
        // after an overflow of the super-tile entries the count is only a lower bound
        const bool exact = a.hdr->status == SPLOTCH_OK;
        a.hdr->tile_entries = exact || carry > a.hdr->tile_entries ? carry : a.hdr->tile_entries;
        a.hdr->tile_entries32 = (uint32_t)(carry < a.cap ? carry : a.cap);
        if (carry > a.cap) a.hdr->status = SPLOTCH_ERR_WORKSPACE;
        // first position of each class, heaviest class first
        uint32_t at = 0;
        for (int k = kCostClasses - 1; k >= 0; --k) {
            const uint32_t h = s_class[k];
            s_class[k] = at;
            at += h;
        }
    }
    __syncthreads();
    for (uint32_t j = threadIdx.x; j < a.ntiles; j += 1024) {
        const uint32_t pos = atomicAdd(&s_class[cost_class(a.toff[j + 1] - a.toff[j])], 1u);
        if (SPL_CHECK(a.hdr, pos < a.ntiles) && pos < a.ntiles) a.torder[pos] = j;
    }
}

// Fine entries of one unit staged in shared memory (tile by tile) before they
// are written out; units with more go straight to global memory.
// 6144 entries (24 KB): room for seven CTAs per SM (10M binning 0.584 ->
// 0.570 ms against 8192 entries at five CTAs; a unit holds ~3K fine entries
// at 1.07e9 particles, ~7K at 10M; larger units write to global memory)
constexpr int kFineBuf = 6144;

// Per unit, 256 entries at a time, one entry per thread.  A warp's 32
// entries (list order = lane order) are described by 16 ballots: for each
// fine-tile row r, the lanes whose rectangle spans r, and for each column c,
// the lanes whose rectangle spans c; the lanes meeting fine tile (r, c) are
// the AND of the two.  A lane's place in tile (r, c) is the number of earlier
// lanes meeting it, after the earlier warps' and earlier chunks' entries
// (a scan over the 8 warps per tile).  The warp's (entry, fine tile) pairs are
// laid end to end and dealt over its lanes, so the work follows the number of
// fine entries whatever the entries' sizes, and render order is kept inside
// every tile.  The unit's
// entries of a tile form one run of the tile's list; the runs are gathered in
// shared memory and copied out whole, so the global writes are coalesced.
// Seven CTAs per SM (32 registers, no spills; 30 KB of shared memory each):
// the expansion waits on latency more than on issue (binning 0.573 -> 0.565
// ms at 10M, 33.0 -> 32.6 ms at 1.07e9 against 46 registers and 5 CTAs)
__global__ void __launch_bounds__(256, 7) k_fine_emit(FineArgs a) {
    pdl_enter();
    __shared__ uint32_t s_buf[kFineBuf];
    __shared__ __align__(16) uint32_t s_b[8][16];   // per warp: row ballots 0..7, column ballots 8..15
    __shared__ uint32_t s_wcnt[8][64];              // per warp: its entries meeting each fine tile
    __shared__ uint32_t s_pos[8][64];               // per warp: its first place in each fine tile's run
    __shared__ uint32_t s_run[64];                  // entries placed so far per fine tile
    __shared__ uint32_t s_lb[65];                   // start of each fine tile's run in s_buf
    __shared__ unsigned long long s_gbase[64];      // list position of each fine tile's run
    const uint32_t u = blockIdx.x;
    const uint32_t n_units = a.hdr->n_units;
    if (u >= n_units) return;
    const uint4 un = a.units[u];
    const uint32_t s = un.x, lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int ox = (int)(s % a.nsx) * kSuperSide, oy = (int)(s / a.nsx) * kSuperSide;
    if (warp == 0) {
        // this unit's count per fine tile: up to the next unit of the same super-tile, or the tile's total
        const bool last = u + 1 >= n_units || a.units[u + 1].x != s;
        uint32_t cnt[2];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const uint32_t t = lane + 32u * h;
            const uint32_t tx = (uint32_t)ox + (t % kSuperSide), ty = (uint32_t)oy + t / kSuperSide;
            cnt[h] = 0;
            unsigned long long g = 0;
            if (tx < a.ntx && ty < a.nty) {
                const uint32_t tile = ty * a.ntx + tx;
                const uint32_t here = a.ucnt[(size_t)u * 64 + t];
                const uint32_t next = last ? a.toff[tile + 1] - a.toff[tile] : a.ucnt[(size_t)(u + 1) * 64 + t];
                g = (unsigned long long)a.toff[tile] + here;
                cnt[h] = next > here ? next - here : 0u;
            }
            s_gbase[t] = g;
            s_run[t] = 0;
        }
        const uint32_t i0 = warp_inclusive_scan(cnt[0]);
        const uint32_t tot0 = __shfl_sync(0xFFFFFFFFu, i0, 31);
        const uint32_t i1 = warp_inclusive_scan(cnt[1]);
        s_lb[lane] = i0 - cnt[0];
        s_lb[lane + 32] = tot0 + i1 - cnt[1];
        if (lane == 31) s_lb[64] = tot0 + i1;
    }
    __syncthreads();
    const bool staged = s_lb[64] <= (uint32_t)kFineBuf;
    // each chunk's entry is loaded one chunk ahead (its key and particle), so
    // a chunk's loads are in flight while the previous chunk is placed
    uint32_t np = 0, nk = 0xFFFFFFFFu;
    if (un.y + threadIdx.x < un.z) {
        np = a.sval[un.y + threadIdx.x];
        nk = a.skey[un.y + threadIdx.x];
    }
    for (uint32_t i0 = un.y; i0 < un.z; i0 += 256) {
        const uint32_t i = i0 + threadIdx.x;
        uint32_t p = 0;
        FineRect f{1, 0, 1, 0};                      // empty
        if (i < un.z) {
            p = np;
            f = key_rect(nk);
        }
        if (i + 256 < un.z) {
            np = a.sval[i + 256];
            nk = a.skey[i + 256];
        }
        const uint32_t rows = f.r0 <= f.r1 ? (0xFFu >> (kSuperSide - 1 - f.r1)) & (0xFFu << f.r0) : 0u;
        const uint32_t cols = f.c0 <= f.c1 ? (0xFFu >> (kSuperSide - 1 - f.c1)) & (0xFFu << f.c0) : 0u;
        uint32_t b[16];
#pragma unroll
        for (int k = 0; k < kSuperSide; ++k) {
            b[k] = __ballot_sync(0xFFFFFFFFu, (rows >> k) & 1u);
            b[kSuperSide + k] = __ballot_sync(0xFFFFFFFFu, (cols >> k) & 1u);
        }
        if (lane == 0) {
            uint4 *d = reinterpret_cast<uint4 *>(s_b[warp]);
            d[0] = make_uint4(b[0], b[1], b[2], b[3]);
            d[1] = make_uint4(b[4], b[5], b[6], b[7]);
            d[2] = make_uint4(b[8], b[9], b[10], b[11]);
            d[3] = make_uint4(b[12], b[13], b[14], b[15]);
        }
        __syncwarp();
        {
            const uint32_t bc = s_b[warp][kSuperSide + (lane & 7)];
            s_wcnt[warp][lane] = __popc(s_b[warp][lane >> 3] & bc);
            s_wcnt[warp][lane + 32] = __popc(s_b[warp][(lane >> 3) + 4] & bc);
        }
        __syncthreads();
        if (threadIdx.x < 64) {
            const uint32_t t = threadIdx.x;
            uint32_t run = s_run[t];
#pragma unroll
            for (int w = 0; w < 8; ++w) {
                s_pos[w][t] = run;
                run += s_wcnt[w][t];
            }
            s_run[t] = run;
        }
        __syncthreads();
        // (entry, fine tile) pairs of the warp, entry by entry, dealt over the lanes.  The
        // entries with pairs are the warp's first lanes and begin at distinct pair indices,
        // so a pair's entry is (entries begun before the round) + (entries begun in the round
        // up to the pair) - 1, from one OR-reduction and one ballot per round.
        const uint32_t w = f.c1 - f.c0 + 1, h = f.r1 - f.r0 + 1;
        const uint32_t npair = f.c0 <= f.c1 && f.r0 <= f.r1 ? w * h : 0u;
        const uint32_t pinc = warp_inclusive_scan(npair);
        const uint32_t K = __shfl_sync(0xFFFFFFFFu, pinc, 31);
        const uint32_t start = pinc - npair;
        const uint32_t info = (uint32_t)f.c0 | ((uint32_t)f.r0 << 3) | (w << 6) | ((w ? 65536u / w + 1u : 0u) << 10);
        const uint32_t le = lanemask_lt() | (1u << lane);
        for (uint32_t q0 = 0; q0 < K; q0 += 32) {
            const bool begins = npair && start >= q0 && start < q0 + 32;
            const uint32_t H = __reduce_or_sync(0xFFFFFFFFu, begins ? 1u << (start - q0) : 0u);
            const uint32_t before = __popc(__ballot_sync(0xFFFFFFFFu, npair && start < q0));
            const uint32_t o = min(before + __popc(H & le), 32u) - 1u;   // no entry begun: lane 31 (unused)
            const uint32_t ostart = __shfl_sync(0xFFFFFFFFu, start, o);
            const uint32_t oinfo = __shfl_sync(0xFFFFFFFFu, info, o);
            const uint32_t pp = __shfl_sync(0xFFFFFFFFu, p, o);
            const uint32_t q = q0 + lane;
            if (q < K) {
                const uint32_t k = q - ostart;
                const uint32_t ow = (oinfo >> 6) & 15u;
                const uint32_t rr = (k * (oinfo >> 10)) >> 16, cc = k - rr * ow;
                const uint32_t r = (oinfo >> 3 & 7u) + rr, c = (oinfo & 7u) + cc;
                const uint32_t t = r * kSuperSide + c;
                const uint32_t kk = s_pos[warp][t] + __popc(s_b[warp][r] & s_b[warp][kSuperSide + c] & ((1u << o) - 1u));
                if (staged) {
                    const uint32_t qq = s_lb[t] + kk;
                    if (qq < (uint32_t)kFineBuf) s_buf[qq] = pp;
                } else {
                    const unsigned long long pos = s_gbase[t] + kk;
                    if (pos < a.cap) a.list[pos] = pp;
                }
            }
        }
    }
    if (!staged) return;
    __syncthreads();
    for (int t = warp; t < 64; t += 8) {
        const uint32_t b0 = s_lb[t], n = s_lb[t + 1] - b0;
        const unsigned long long g = s_gbase[t];
        for (uint32_t k = lane; k < n; k += 32)
            if (g + k < a.cap) a.list[g + k] = s_buf[b0 + k];
    }
}

static int sm_count_bin() {
    int dev = 0, v = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
    return v > 0 ? v : 148;
}

// Bits of a super-tile id (at most kSidBits) and the 8-bit passes that sort them.
static int super_bits(uint32_t nsuper) {
    int bits = 0;
    while (bits < kSidBits && (1ull << bits) < (unsigned long long)nsuper) ++bits;
    return bits;
}

int super_passes(uint32_t nsuper) { return (super_bits(nsuper) + 7) / 8; }

uint64_t fine_list_offset(const Layout &L) { return L.off_ek[1 - (super_passes(L.nsuper) & 1)]; }

cudaError_t launch_bin(void *ws, const Layout &L, uint32_t large_tiles, cudaStream_t st) {
    Header *hdr = header(ws);
    const int tshift = L.tile == 8 ? 3 : (L.tile == 16 ? 4 : 5);
    BinArgs a{};
    a.hdr = hdr;
    a.list[0] = at<uint32_t>(ws, L.off_sv[0]);
    a.list[1] = at<uint32_t>(ws, L.off_sv[1]);
    const bool pay = tile_payload(L), packed = tile_box_packs(L);
    a.tbox = packed ? at<uint32_t>(ws, L.off_tbox) : nullptr;
    a.psbox = at<uint32_t>(ws, L.off_sbox);
    if (pay) {
        a.pk[0] = at<uint32_t>(ws, L.off_pay[0]);
        a.pk[1] = at<uint32_t>(ws, L.off_pay[1]);
    } else {
        a.pk[0] = a.pk[1] = a.psbox;
    }
    a.box = at<ushort4>(ws, L.off_box);
    a.sbox = at<ushort4>(ws, L.off_sbox);
    a.tshift = tshift;
    a.part = at<uint64_t>(ws, L.off_part);
    a.ctas = L.sort_ctas;
    a.ek = at<uint32_t>(ws, L.off_ek[0]);
    a.ev = at<uint32_t>(ws, L.off_ev[0]);
    a.cap = L.cap;
    a.nsx = (int)L.nsx;
    a.large_tiles = large_tiles;
    // the depth sort carried each particle's tile box (large frames), or the count pass
    // gathers the transform's packed tile boxes (the pixel boxes when the tile counts do
    // not fit 8 bits)
    if (pay) launch_pdl(k_bin_reduce_pay, dim3(a.ctas), dim3(256), 0, st, a);
    else if (packed) launch_pdl(k_bin_reduce<true>, dim3(a.ctas), dim3(256), 0, st, a);
    else launch_pdl(k_bin_reduce<false>, dim3(a.ctas), dim3(256), 0, st, a);
    launch_pdl(k_bin_scan, dim3(1), dim3(1024), 0, st, a);
    if (packed) launch_pdl(k_bin_emit<true>, dim3(a.ctas), dim3(256), 0, st, a);
    else launch_pdl(k_bin_emit<false>, dim3(a.ctas), dim3(256), 0, st, a);
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
        // only the super-tile id bits: the rectangle code above them is payload
        const int bits = super_bits(L.nsuper) - 8 * pass;
        p.mask = bits >= 8 ? 0xFFu : (1u << bits) - 1u;
        e = launch_radix_pass(p, st);
        if (e != cudaSuccess) return e;
    }
    const int f = passes & 1;
    const int sms = sm_count_bin();
    if (passes == 1)
        launch_pdl(k_soff_from_totals, dim3(1), dim3(256), 0, st, p.htot, at<uint32_t>(ws, L.off_soff), L.nsuper);
    else
        launch_pdl(k_group_offsets, dim3(sms * 8), dim3(256), 0, st, &hdr->super32, at<uint32_t>(ws, L.off_ek[f]),
                                                 at<uint32_t>(ws, L.off_soff), L.nsuper);
    FineArgs fa{};
    fa.hdr = hdr;
    fa.skey = at<uint32_t>(ws, L.off_ek[f]);
    fa.sval = at<uint32_t>(ws, L.off_ev[f]);
    fa.soff = at<uint32_t>(ws, L.off_soff);
    fa.ufirst = at<uint32_t>(ws, L.off_ufirst);
    fa.units = at<uint4>(ws, L.off_units);
    fa.ucnt = at<uint32_t>(ws, L.off_ucnt);
    fa.toff = at<uint32_t>(ws, L.off_toff);
    fa.torder = at<uint32_t>(ws, L.off_torder);
    fa.list = at<uint32_t>(ws, fine_list_offset(L));
    fa.cap = L.cap;
    fa.nsuper = L.nsuper;
    fa.nsx = L.nsx;
    fa.ntx = (uint32_t)L.ntx;
    fa.nty = (uint32_t)L.nty;
    fa.ntiles = L.ntiles;
    fa.max_units = L.max_units;
    launch_pdl(k_units, dim3(1), dim3(1024), 0, st, fa);
    launch_pdl(k_fine_count, dim3(L.max_units), dim3(256), 0, st, fa);
    launch_pdl(k_fine_unit_scan, dim3(L.nsuper), dim3(1024), 0, st, fa);
    launch_pdl(k_fine_offsets, dim3(1), dim3(1024), 0, st, fa);
    launch_pdl(k_fine_emit, dim3(L.max_units), dim3(256), 0, st, fa);
    count_launches(6);
    return cudaGetLastError();
}

}  // namespace spl
