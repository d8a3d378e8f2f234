// Tile renderer: one CTA per screen tile.  The tile's particle list is
// staged in batches into shared memory (prefetched into registers one batch
// ahead).  Lanes work in groups, one group per 4x4 pixel quadrant: a lane
// tests one particle of the batch against every quadrant of its warp, one
// ballot per quadrant gives each group its own list of surviving particles,
// and every group walks its list in list order, one particle per step, all
// groups in the same steps (a group that is done takes a null particle that
// adds nothing, so the steps have no branch).
//   tiles of 16 and 32: a warp covers a 16x8 block as eight groups of four
//     lanes, each lane a 2x2 pixel square (the column offsets are shared by
//     its two rows); 128 pixels per warp step
//   tiles of 8: a warp covers the 8x8 tile as four groups of eight lanes,
//     each lane two horizontally adjacent pixels; 64 pixels per warp step
// Per pixel it evaluates the truncated Gaussian footprint (Section 2, first
// item) and integrates Eq. 1 (Section 2) across the particle layer:
//   emission    C += E g
//   absorptive  C += T_acc S, T_acc *= T, with T = exp(-A g),
//               S = E (1 - T)/A (E g when A = 0)
//   E = A       C += E g, then I = 1 - exp(-C)
// Packed f32x2 arithmetic does a pair of horizontally adjacent pixels in one
// instruction.  Both layouts composite each pixel with the same operations in
// the same order, so they give the same image bit for bit.
#include <cuda.h>
#include <cstring>
#include <mutex>

#include "internal.h"
#include "device_util.cuh"

namespace spl {

// --- TMA staging of particle records ------------------------------------------
// The records of a batch are named by the tile list, so they are gathered,
// not copied as one range: a 2-D tensor map over each record array (rows =
// particles, 4 floats per row) lets one cp.async.bulk.tensor tile::gather4
// bring four rows (four particles) into shared memory, completing on an
// mbarrier.  The copies need no registers and no per-thread load
// instructions; threads only convert the landed records to operand pairs.
struct TmaMaps {
    CUtensorMap geo, col;   // rows of {sx, sy, r2, k} and {Er, Eg, Eb, A}
};

// Raw staging: kTmaStages stages (batches fetched kTmaStages - 1 ahead), per
// stage and per group of four entries one 128-byte aligned block for each
// record array (a gather4 writes 64 bytes).  Two, three and four stages gave
// the same render time (4.00, 4.01, 3.97 ms on the bench frame), so two.
constexpr int kTmaStages = 2;
template <int B> struct TmaSmem {
    __align__(128) float4 g[kTmaStages][B / 4][8];
    __align__(128) float4 c[kTmaStages][B / 4][8];
    __align__(8) unsigned long long bar[kTmaStages];
};

__device__ __forceinline__ void tma_gather4(void *dst, const CUtensorMap *map, uint32_t r0, uint32_t r1, uint32_t r2,
                                            uint32_t r3, unsigned long long *bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile::gather4.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4, %5, %6}], [%7];"
        :: "r"(smem_addr(dst)), "l"(map), "r"(0), "r"(r0), "r"(r1), "r"(r2), "r"(r3), "r"(smem_addr(bar))
        : "memory");
}

__device__ __forceinline__ float ex2_approx(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__device__ __forceinline__ float2 f2(float a) { return make_float2(a, a); }

// An absorbing layer with A <= kSeriesMaxA takes its source and
// transmission from a series: with yn = -A g,
//   q = (1 - e^{-y})/y = 1 + yn/2 + yn^2/6 + yn^3/24 + ...
// truncated after yn^3 (relative error below y^4/5! < 2.1e-6 for y <= 1/8),
// S = E g q and T = 1 + yn q, with no cancellation; A = 0 gives q = 1, T = 1.
// With u = T_acc g q the update is C += E u, T_acc -= A u.  Larger A takes T
// from exp2 and S = E (1 - T)/A.
__device__ __forceinline__ float2 q_series(float2 yn) {
    float2 q = f2(1.0f / 24.0f);
    q = __ffma2_rn(q, yn, f2(1.0f / 6.0f));
    q = __ffma2_rn(q, yn, f2(0.5f));
    q = __ffma2_rn(q, yn, f2(1.0f));
    return q;
}

// A staged particle is laid out as ready-made operand pairs for the packed
// pixel-pair arithmetic, in four arrays (conflict-free stores):
// {-sx, -sx, -sy, -sy}, {k, k, -A, -A}, {Er, Er, Eg, Eg}, {Eb, Eb, r2, A}
// with k = -log2(e)/sigma_pix^2.

// Slots: the 2x2-pixel layout keeps each run of 32 entries after a slot of
// its own that holds a particle adding nothing (slot 33 r for run r, entry
// e at 33 (e / 32) + 1 + e % 32), so a step's slot is the run's base plus
// __ffs of the group's mask, with no test for an empty mask; the two-pixel
// layout keeps entries in order with that particle at slot B.
template <int B> struct RenderSmem {
    float4 s0[2][B + B / 32 + 1], s1[2][B + B / 32 + 1], s2[2][B + B / 32 + 1], s3[2][B + B / 32 + 1];
    float4 scull[2][B];   // sx, sy, r2 for the cull test
};

// Early termination of a warp (absorptive mode, a cutoff > 0): the light
// still to come through a pixel of transmittance T is at most T M_c per
// channel (M_c bounds E_c / A over all particles), so once T_max M_c <=
// cutoff C_max,c over the warp's pixels inside the image, the rest of the
// list changes none of them by more than cutoff times the channel's image
// maximum.  Pixels outside the image take no part; a warp with none is done.
__device__ __forceinline__ bool warp_converged(float tmax, float c0, float c1, float c2, const float *M, float cutoff) {
    tmax = ordered_to_float(__reduce_max_sync(0xFFFFFFFFu, float_to_ordered(tmax)));
    c0 = ordered_to_float(__reduce_max_sync(0xFFFFFFFFu, float_to_ordered(c0)));
    c1 = ordered_to_float(__reduce_max_sync(0xFFFFFFFFu, float_to_ordered(c1)));
    c2 = ordered_to_float(__reduce_max_sync(0xFFFFFFFFu, float_to_ordered(c2)));
    if (tmax == -INFINITY) return true;
    return tmax * M[0] <= cutoff * c0 && tmax * M[1] <= cutoff * c1 && tmax * M[2] <= cutoff * c2;
}

// One screen tile, rendered by the whole CTA (all threads must call it).
// SERIES: every particle's A is at most kSeriesMaxA (absorptive mode).
// ET: early termination (absorptive mode with a cutoff).  PT: partial image
// (the transmittance is written too).
template <int T, int MODE, int B, bool SERIES, bool ET, bool PT>
__device__ __forceinline__ void render_tile(const RenderArgs &a, const int tile, RenderSmem<B> &sm) {
    constexpr int kThreads = T * T / 2;
    constexpr int WX = 8, WY = 8;               // pixel block of one warp (two pixels per lane)
    constexpr int kWarpCols = T / WX;
    constexpr int kPer = (B + kThreads - 1) / kThreads;
    auto &s0 = sm.s0;
    auto &s1 = sm.s1;
    auto &s2 = sm.s2;
    auto &s3 = sm.s3;
    auto &scull = sm.scull;

    const int tx = tile % a.ntx, ty = tile / a.ntx;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int wx0 = tx * T + (warp % kWarpCols) * WX, wy0 = ty * T + (warp / kWarpCols) * WY;
    // lanes in four groups of 8, each on a 4x4 quadrant of the warp's block
    const int grp = lane >> 3, gl = lane & 7;
    const int px0 = wx0 + (grp & 1) * 4 + 2 * (gl & 1), py = wy0 + (grp >> 1) * 4 + (gl >> 1);
    const float2 cx = make_float2((float)px0 + 0.5f, (float)px0 + 1.5f);
    const float2 cy = f2((float)py + 0.5f);
    // pixel-centre boxes of the quadrants (left/right, top/bottom), for the cull test
    const float xl0 = (float)wx0 + 0.5f, xl1 = (float)wx0 + 3.5f, xr0 = (float)wx0 + 4.5f, xr1 = (float)wx0 + 7.5f;
    const float yt0 = (float)wy0 + 0.5f, yt1 = (float)wy0 + 3.5f, yb0 = (float)wy0 + 4.5f, yb1 = (float)wy0 + 7.5f;

    float2 cr = f2(0.f), cg = f2(0.f), cb = f2(0.f), tacc = f2(1.f);
    const bool in0 = px0 < a.width && py < a.height, in1 = px0 + 1 < a.width && py < a.height;
    float M[3] = {0.f, 0.f, 0.f};
    if (ET) {
        M[0] = a.hdr->eoa_max[0];
        M[1] = a.hdr->eoa_max[1];
        M[2] = a.hdr->eoa_max[2];
    }
    bool wdone = false;

    const bool ok = a.hdr->status == SPLOTCH_OK;
    const uint32_t begin = ok ? a.toff[tile] : 0u, end = ok ? a.toff[tile + 1] : 0u;

    // A batch is loaded into registers one batch ahead and written to shared
    // memory (as operand pairs) after the current batch has been composited;
    // its list indices were loaded one batch before that.
    float4 rg[kPer], rc[kPer];
    uint32_t pidx[kPer];
#pragma unroll
    for (int q = 0; q < kPer; ++q) {
        const uint32_t j = threadIdx.x + q * kThreads;
        pidx[q] = 0;
        if (begin + j < end && SPL_CHECK(a.hdr, begin + j < a.hdr->layout.cap)) pidx[q] = __ldg(&a.list[begin + j]);
    }
    auto load = [&](uint32_t base) {
        const uint32_t nb = min((uint32_t)B, end - base);
        const uint32_t base2 = base + B;
        const uint32_t nb2 = base2 < end ? min((uint32_t)B, end - base2) : 0u;
#pragma unroll
        for (int q = 0; q < kPer; ++q) {
            const uint32_t j = threadIdx.x + q * kThreads;
            if (j < nb) {
                const uint32_t p = pidx[q];
                if (SPL_CHECK(a.hdr, p < a.hdr->layout.n)) {
                    rg[q] = __ldg(&a.geo[p]);
                    rc[q] = __ldg(&a.col[p]);
                }
            }
            if (j < nb2 && SPL_CHECK(a.hdr, base2 + j < a.hdr->layout.cap)) pidx[q] = __ldg(&a.list[base2 + j]);
        }
    };
    auto store = [&](int buf, uint32_t base) {
        const uint32_t nb = min((uint32_t)B, end - base);
#pragma unroll
        for (int q = 0; q < kPer; ++q) {
            const uint32_t j = threadIdx.x + q * kThreads;
            if (j < nb) {
                const float4 g = rg[q], c = rc[q];
                s0[buf][j] = make_float4(-g.x, -g.x, -g.y, -g.y);
                s1[buf][j] = make_float4(g.w, g.w, -c.w, -c.w);
                s2[buf][j] = make_float4(c.x, c.x, c.y, c.y);
                s3[buf][j] = make_float4(c.z, c.z, g.z, c.w);
                scull[buf][j] = g;
            }
        }
    };

    // null entry: r2 = 0 fails every membership test; E = 0, A = 0, k = 0 keep all terms finite
    if (threadIdx.x < 2) {
        const float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
        s0[threadIdx.x][B] = z;
        s1[threadIdx.x][B] = z;
        s2[threadIdx.x][B] = z;
        s3[threadIdx.x][B] = z;
    }
    if (begin < end) {
        load(begin);
        store(0, begin);
    }
    int buf = 0;
    // composite one kept particle (j: index in the batch) onto both pixels
    auto apply = [&](const int j) {
        const float4 p0 = s0[buf][j], p1 = s1[buf][j];
        const float4 p2 = s2[buf][j], p3 = s3[buf][j];
        const float2 dx = __fadd2_rn(cx, make_float2(p0.x, p0.y));
        const float2 dy = __fadd2_rn(cy, make_float2(p0.z, p0.w));
        const float2 d2 = __ffma2_rn(dy, dy, __fmul2_rn(dx, dx));
        const float2 arg = __fmul2_rn(d2, make_float2(p1.x, p1.y));
        float2 w;
        w.x = d2.x < p3.z ? ex2_approx(arg.x) : 0.0f;
        w.y = d2.y < p3.z ? ex2_approx(arg.y) : 0.0f;
        if (MODE == SPLOTCH_ABSORPTIVE) {
            const float2 na = make_float2(p1.z, p1.w);
            if (SERIES || p3.w <= kSeriesMaxA) {
                const float2 q = q_series(__fmul2_rn(w, na));
                w = __fmul2_rn(tacc, __fmul2_rn(w, q));
                tacc = __ffma2_rn(na, w, tacc);
            } else {
                const float2 yl = __fmul2_rn(w, f2(-1.4426950408889634f * p3.w));
                const float2 t = make_float2(ex2_approx(yl.x), ex2_approx(yl.y));
                w = __fmul2_rn(__fadd2_rn(f2(1.0f), make_float2(-t.x, -t.y)), f2(1.0f / p3.w));
                w = __fmul2_rn(tacc, w);
                tacc = __fmul2_rn(tacc, t);
            }
        }
        cr = __ffma2_rn(w, make_float2(p2.x, p2.y), cr);
        cg = __ffma2_rn(w, make_float2(p2.z, p2.w), cg);
        cb = __ffma2_rn(w, make_float2(p3.x, p3.y), cb);
    };
    for (uint32_t base = begin; base < end; base += B, buf ^= 1) {
        const uint32_t next = base + B;
        if (next < end) load(next);
        __syncthreads();
        const uint32_t nb = min((uint32_t)B, end - base);
        for (uint32_t c = 0; c < (ET && wdone ? 0u : nb); c += 32) {
            // each lane tests particle c + lane against the four quadrants
            bool k0 = false, k1 = false, k2 = false, k3 = false;
            if (c + lane < nb) {
                const float4 g = scull[buf][c + lane];
                const float lim = g.z * 1.0001f + 0.01f;   // conservative: never culls a pixel the exact test keeps
                const float dl = g.x - fminf(fmaxf(g.x, xl0), xl1), dr = g.x - fminf(fmaxf(g.x, xr0), xr1);
                const float dt = g.y - fminf(fmaxf(g.y, yt0), yt1), db = g.y - fminf(fmaxf(g.y, yb0), yb1);
                const float dl2 = dl * dl, dr2 = dr * dr, dt2 = dt * dt, db2 = db * db;
                k0 = dl2 + dt2 <= lim;
                k1 = dr2 + dt2 <= lim;
                k2 = dl2 + db2 <= lim;
                k3 = dr2 + db2 <= lim;
            }
            const uint32_t m0 = __ballot_sync(0xFFFFFFFFu, k0), m1 = __ballot_sync(0xFFFFFFFFu, k1);
            const uint32_t m2 = __ballot_sync(0xFFFFFFFFu, k2), m3 = __ballot_sync(0xFFFFFFFFu, k3);
            uint32_t mask = grp == 0 ? m0 : grp == 1 ? m1 : grp == 2 ? m2 : m3;
            const int n_it = max(max(__popc(m0), __popc(m1)), max(__popc(m2), __popc(m3)));
            // a group whose particles are done composites the null entry meanwhile
            int it = 0;
            if (MODE != SPLOTCH_ABSORPTIVE) {
                // two steps at a time: the short emission bodies overlap (no gain when absorptive)
                for (; it + 1 < n_it; it += 2) {
                    const int j0 = mask ? (int)c + __ffs(mask) - 1 : B;
                    mask &= mask - 1;
                    const int j1 = mask ? (int)c + __ffs(mask) - 1 : B;
                    mask &= mask - 1;
                    apply(j0);
                    apply(j1);
                }
            }
            for (; it < n_it; ++it) {
                const int j = mask ? (int)c + __ffs(mask) - 1 : B;
                mask &= mask - 1;
                apply(j);
            }
        }
        if (ET) {
            if (!wdone) {
                const float ni = -INFINITY;
                wdone = warp_converged(fmaxf(in0 ? tacc.x : ni, in1 ? tacc.y : ni),
                                       fmaxf(in0 ? cr.x : ni, in1 ? cr.y : ni), fmaxf(in0 ? cg.x : ni, in1 ? cg.y : ni),
                                       fmaxf(in0 ? cb.x : ni, in1 ? cb.y : ni), M, a.cutoff);
            }
            if (__syncthreads_and(wdone)) break;
        } else {
            __syncthreads();
        }
        if (next < end) store(buf ^ 1, next);
    }

    // transmittance of a partial render (E = A: exp(-tau) before C = 1 - exp(-tau))
    float2 tr = MODE == SPLOTCH_ABSORPTIVE ? tacc : f2(1.0f);
    float2 tg = tr, tb = tr;
    if (MODE == SPLOTCH_E_EQ_A && PT) {
        tr = make_float2(expf(-cr.x), expf(-cr.y));
        tg = make_float2(expf(-cg.x), expf(-cg.y));
        tb = make_float2(expf(-cb.x), expf(-cb.y));
    }
    if (MODE == SPLOTCH_E_EQ_A) {
        cr = make_float2(-expm1f(-cr.x), -expm1f(-cr.y));
        cg = make_float2(-expm1f(-cg.x), -expm1f(-cg.y));
        cb = make_float2(-expm1f(-cb.x), -expm1f(-cb.y));
    }
    if (py < a.height) {
        float *row = a.image + (size_t)py * a.width * 3;
        if (px0 < a.width) {
            row[3 * px0 + 0] = cr.x; row[3 * px0 + 1] = cg.x; row[3 * px0 + 2] = cb.x;
        }
        if (px0 + 1 < a.width) {
            row[3 * px0 + 3] = cr.y; row[3 * px0 + 4] = cg.y; row[3 * px0 + 5] = cb.y;
        }
        if (PT) {
            float *trow = a.trans + (size_t)py * a.width * 3;
            if (px0 < a.width) {
                trow[3 * px0 + 0] = tr.x; trow[3 * px0 + 1] = tg.x; trow[3 * px0 + 2] = tb.x;
            }
            if (px0 + 1 < a.width) {
                trow[3 * px0 + 3] = tr.y; trow[3 * px0 + 4] = tg.y; trow[3 * px0 + 5] = tb.y;
            }
        }
    }
}

// Threads of the CTA that renders a T x T tile: 2 x 2 pixels per thread for
// T >= 16, 2 x 1 for T = 8.
constexpr int render_threads(int T) { return T >= 16 ? T * T / 4 : T * T / 2; }

// The same tile render with four pixels per lane (T >= 16): a warp covers a
// 16 x 8 block as eight groups of 4 lanes, one per 4 x 4 quadrant, each lane
// a 2 x 2 square (two packed pixel pairs, one per row).  A step now composites
// eight particles (one per group) on 128 pixels, and the column terms are
// shared by the two rows.
// TMA: the batches are staged by tile::gather4 copies (maps, ts) instead of
// per-thread loads through registers.
template <int T, int MODE, int B, bool SERIES, bool ET, bool PT, bool TMA = false>
__device__ __forceinline__ void render_tile4(const RenderArgs &a, const int tile, RenderSmem<B> &sm,
                                             const TmaMaps *maps = nullptr, TmaSmem<B> *ts = nullptr) {
    constexpr int kThreads = T * T / 4;
    constexpr int WX = 16, WY = 8;
    constexpr int kWarpCols = T / WX;
    constexpr int kPer = (B + kThreads - 1) / kThreads;
    auto &s0 = sm.s0;
    auto &s1 = sm.s1;
    auto &s2 = sm.s2;
    auto &s3 = sm.s3;
    auto &scull = sm.scull;

    const int tx = tile % a.ntx, ty = tile / a.ntx;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int wx0 = tx * T + (warp % kWarpCols) * WX, wy0 = ty * T + (warp / kWarpCols) * WY;
    const int grp = lane >> 2, gl = lane & 3;
    const int px0 = wx0 + (grp & 3) * 4 + 2 * (gl & 1), py0 = wy0 + (grp >> 2) * 4 + 2 * (gl >> 1);
    const float2 cx = make_float2((float)px0 + 0.5f, (float)px0 + 1.5f);
    const float2 cyA = f2((float)py0 + 0.5f), cyB = f2((float)py0 + 1.5f);
    const float bx = (float)wx0 + 0.5f, by = (float)wy0 + 0.5f;   // first pixel centre of the warp's block

    float2 crA = f2(0.f), cgA = f2(0.f), cbA = f2(0.f), tA = f2(1.f);
    float2 crB = f2(0.f), cgB = f2(0.f), cbB = f2(0.f), tB = f2(1.f);
    float M[3] = {0.f, 0.f, 0.f};
    if (ET) {
        M[0] = a.hdr->eoa_max[0];
        M[1] = a.hdr->eoa_max[1];
        M[2] = a.hdr->eoa_max[2];
    }
    bool wdone = false;

    const bool ok = a.hdr->status == SPLOTCH_OK;
    const uint32_t begin = ok ? a.toff[tile] : 0u, end = ok ? a.toff[tile + 1] : 0u;

    float4 rg[TMA ? 1 : kPer], rc[TMA ? 1 : kPer];
    // register staging: the list indices are loaded one batch ahead of the
    // records they name, so a batch's gathers start without waiting for its
    // index loads (render 3.28 -> 3.23 ms absorptive, 2.39 -> 2.34 ms emission)
    uint32_t pidx[TMA ? 1 : kPer];
#pragma unroll
    for (int q = 0; q < (TMA ? 1 : kPer); ++q) {
        const uint32_t j = threadIdx.x + q * kThreads;
        pidx[q] = 0;
        if (!TMA && begin + j < end && SPL_CHECK(a.hdr, begin + j < a.hdr->layout.cap)) pidx[q] = __ldg(&a.list[begin + j]);
    }
    // batch staging: `load` starts fetching the batch at `base`, `store` writes
    // it to the operand buffer `buf` once it has arrived (`stage`: TMA stage)
    auto load = [&](uint32_t base, int stage) {
        const uint32_t nb = min((uint32_t)B, end - base);
        if constexpr (TMA) {
            // warp 0: lane g gathers entries 4g .. 4g + 3 (rows past the batch read particle 0, unused)
            if (threadIdx.x < 32) {
                const uint32_t ng = (nb + 3) / 4;
                if (threadIdx.x == 0) {
                    mbar_arrive_expect_tx(&ts->bar[stage], ng * 128u);
                }
                __syncwarp();
                // the stage's previous records were read by generic loads before the barrier that
                // precedes this call: order them before the copies that overwrite them
                fence_proxy_async_smem();
                for (uint32_t g = threadIdx.x; g < ng; g += 32) {
                    uint32_t r[4];
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        const uint32_t j = 4 * g + k;
                        r[k] = 0;
                        if (j < nb && SPL_CHECK(a.hdr, base + j < a.hdr->layout.cap)) {
                            const uint32_t p = __ldg(&a.list[base + j]);
                            if (SPL_CHECK(a.hdr, p < a.hdr->layout.n)) r[k] = p;
                        }
                    }
                    tma_gather4(&ts->g[stage][g][0], &maps->geo, r[0], r[1], r[2], r[3], &ts->bar[stage]);
                    tma_gather4(&ts->c[stage][g][0], &maps->col, r[0], r[1], r[2], r[3], &ts->bar[stage]);
                }
            }
        } else {
            // the batch's indices were loaded one batch earlier (pidx); load the next batch's now
            const uint32_t base2 = base + B;
            const uint32_t nb2 = base2 < end ? min((uint32_t)B, end - base2) : 0u;
#pragma unroll
            for (int q = 0; q < kPer; ++q) {
                const uint32_t j = threadIdx.x + q * kThreads;
                if (j < nb) {
                    const uint32_t p = pidx[q];
                    if (SPL_CHECK(a.hdr, p < a.hdr->layout.n)) {
                        rg[q] = __ldg(&a.geo[p]);
                        rc[q] = __ldg(&a.col[p]);
                    }
                }
                if (j < nb2 && SPL_CHECK(a.hdr, base2 + j < a.hdr->layout.cap)) pidx[q] = __ldg(&a.list[base2 + j]);
            }
        }
    };
    // batch k sits in stage k % kTmaStages and is the (k / kTmaStages)-th use of that
    // stage's barrier: phase parity (k / kTmaStages) & 1
    uint32_t nstored = 0;
    auto store = [&](int buf, uint32_t base, int stage) {
        const uint32_t nb = min((uint32_t)B, end - base);
        if constexpr (TMA) {
            if (!mbar_wait(&ts->bar[stage], (nstored / kTmaStages) & 1u, kAsyncWaitPolls) && threadIdx.x == 0)
                atomicExch(const_cast<int *>(&a.hdr->status), (int)SPLOTCH_ERR_TIMEOUT);
            nstored += 1;
        }
#pragma unroll
        for (int q = 0; q < kPer; ++q) {
            const uint32_t j = threadIdx.x + q * kThreads;
            if (j < nb) {
                const float4 g = TMA ? ts->g[stage][j >> 2][j & 3] : rg[q];
                const float4 c = TMA ? ts->c[stage][j >> 2][j & 3] : rc[q];
                const uint32_t sl = (j >> 5) * 33 + 1 + (j & 31);
                s0[buf][sl] = make_float4(-g.x, -g.x, -g.y, -g.y);
                s1[buf][sl] = make_float4(g.w, g.w, -c.w, -c.w);
                s2[buf][sl] = make_float4(c.x, c.x, c.y, c.y);
                s3[buf][sl] = make_float4(c.z, c.z, g.z, c.w);
                scull[buf][j] = g;
            }
        }
    };

    if (threadIdx.x < 2 * (B / 32)) {
        const float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
        const int nbuf = threadIdx.x & 1, sl = (threadIdx.x >> 1) * 33;
        s0[nbuf][sl] = z;
        s1[nbuf][sl] = z;
        s2[nbuf][sl] = z;
        s3[nbuf][sl] = z;
    }
    if constexpr (TMA) {
        if (threadIdx.x == 0) {
            for (int k = 0; k < kTmaStages; ++k)
                mbar_init(&ts->bar[k]);
            asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        }
        __syncthreads();
    }
    if (begin < end) {
        if constexpr (TMA) {
            for (int k = 0; k < kTmaStages - 1 && begin + (uint32_t)k * B < end; ++k) load(begin + k * B, k);
        } else {
            load(begin, 0);
        }
        store(0, begin, 0);
    }
    int buf = 0;
    // one row (pixel pair) of the lane's square: weight, transfer and colour
    auto row = [&](const float2 d2, const float4 p1, const float4 p2, const float4 p3, float2 &cr, float2 &cg,
                   float2 &cb, float2 &tacc) {
        const float2 arg = __fmul2_rn(d2, make_float2(p1.x, p1.y));
        float2 w;
        w.x = d2.x < p3.z ? ex2_approx(arg.x) : 0.0f;
        w.y = d2.y < p3.z ? ex2_approx(arg.y) : 0.0f;
        if (MODE == SPLOTCH_ABSORPTIVE) {
            const float2 na = make_float2(p1.z, p1.w);
            if (SERIES || p3.w <= kSeriesMaxA) {
                const float2 q = q_series(__fmul2_rn(w, na));
                w = __fmul2_rn(tacc, __fmul2_rn(w, q));
                tacc = __ffma2_rn(na, w, tacc);
            } else {
                const float2 yl = __fmul2_rn(w, f2(-1.4426950408889634f * p3.w));
                const float2 t = make_float2(ex2_approx(yl.x), ex2_approx(yl.y));
                w = __fmul2_rn(__fadd2_rn(f2(1.0f), make_float2(-t.x, -t.y)), f2(1.0f / p3.w));
                w = __fmul2_rn(tacc, w);
                tacc = __fmul2_rn(tacc, t);
            }
        }
        cr = __ffma2_rn(w, make_float2(p2.x, p2.y), cr);
        cg = __ffma2_rn(w, make_float2(p2.z, p2.w), cg);
        cb = __ffma2_rn(w, make_float2(p3.x, p3.y), cb);
    };
    auto apply = [&](const int j) {
        const float4 p0 = s0[buf][j], p1 = s1[buf][j];
        const float4 p2 = s2[buf][j], p3 = s3[buf][j];
        const float2 dx = __fadd2_rn(cx, make_float2(p0.x, p0.y));
        const float2 dx2 = __fmul2_rn(dx, dx);
        const float2 dyA = __fadd2_rn(cyA, make_float2(p0.z, p0.w));
        const float2 dyB = __fadd2_rn(cyB, make_float2(p0.z, p0.w));
        row(__ffma2_rn(dyA, dyA, dx2), p1, p2, p3, crA, cgA, cbA, tA);
        row(__ffma2_rn(dyB, dyB, dx2), p1, p2, p3, crB, cgB, cbB, tB);
    };
    int stage = 0;   // TMA stage of the batch being composited
    for (uint32_t base = begin; base < end; base += B, buf ^= 1, stage = stage + 1 == kTmaStages ? 0 : stage + 1) {
        const uint32_t next = base + B;
        const int nstage = stage + 1 == kTmaStages ? 0 : stage + 1;
        if (!TMA && next < end) load(next, 0);
        __syncthreads();
        // after the barrier every thread has converted the current batch: the stage of the
        // batch before it is free for the batch kTmaStages - 1 ahead
        if (TMA) {
            const uint32_t ahead = base + (uint32_t)(kTmaStages - 1) * B;
            if (ahead < end) load(ahead, stage == 0 ? kTmaStages - 1 : stage - 1);
        }
        const uint32_t nb = min((uint32_t)B, end - base);
        for (uint32_t c = 0; c < (ET && wdone ? 0u : nb); c += 32) {
            // each lane tests entry c + lane against the eight quadrants (4 columns x 2 rows)
            bool k[8];
#pragma unroll
            for (int q = 0; q < 8; ++q) k[q] = false;
            if (c + lane < nb) {
                const float4 g = scull[buf][c + lane];
                const float lim = g.z * 1.0001f + 0.01f;   // conservative: never culls a pixel the exact test keeps
                float dc[4], dr[2];
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const float x0 = bx + 4.0f * q;
                    const float d = g.x - fminf(fmaxf(g.x, x0), x0 + 3.0f);
                    dc[q] = d * d;
                }
#pragma unroll
                for (int q = 0; q < 2; ++q) {
                    const float y0 = by + 4.0f * q;
                    const float d = g.y - fminf(fmaxf(g.y, y0), y0 + 3.0f);
                    dr[q] = d * d;
                }
#pragma unroll
                for (int q = 0; q < 8; ++q) k[q] = dc[q & 3] + dr[q >> 2] <= lim;
            }
            uint32_t mask = 0;
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                const uint32_t m = __ballot_sync(0xFFFFFFFFu, k[q]);
                if (grp == q) mask = m;
            }
            const int n_it = (int)__reduce_max_sync(0xFFFFFFFFu, (uint32_t)__popc(mask));
            int it = 0;
            // two steps per iteration: the second step's geometry overlaps the first's compositing
            const int cb = (int)(c >> 5) * 33;   // slot cb holds the null particle of this run of 32
            for (; it + 1 < n_it; it += 2) {
                const int j0 = cb + __ffs(mask);
                mask &= mask - 1;
                const int j1 = cb + __ffs(mask);
                mask &= mask - 1;
                apply(j0);
                apply(j1);
            }
            for (; it < n_it; ++it) {
                const int j = cb + __ffs(mask);
                mask &= mask - 1;
                apply(j);
            }
        }
        if (ET) {
            if (!wdone) {
                const float ni = -INFINITY;
                const bool x0 = px0 < a.width, x1 = px0 + 1 < a.width;
                const bool yA = py0 < a.height, yB = py0 + 1 < a.height;
                auto mx4 = [&](float2 A, float2 Bv) {
                    return fmaxf(fmaxf(x0 && yA ? A.x : ni, x1 && yA ? A.y : ni),
                                 fmaxf(x0 && yB ? Bv.x : ni, x1 && yB ? Bv.y : ni));
                };
                wdone = warp_converged(mx4(tA, tB), mx4(crA, crB), mx4(cgA, cgB), mx4(cbA, cbB), M, a.cutoff);
            }
            if (__syncthreads_and(wdone)) {
                // the next batch's copies may be in flight: let them land before leaving
                if (TMA) {
                    // wait for every batch still in flight
                    uint32_t k = nstored;
                    int st = nstage;
                    for (uint32_t b2 = next; b2 < end && b2 < base + (uint32_t)kTmaStages * B; b2 += B, ++k) {
                        mbar_wait(&ts->bar[st], (k / kTmaStages) & 1u, kAsyncWaitPolls);
                        st = st + 1 == kTmaStages ? 0 : st + 1;
                    }
                }
                break;
            }
        } else {
            __syncthreads();
        }
        if (next < end) store(buf ^ 1, next, nstage);
    }

    // transmittance of a partial render (E = A: exp(-tau) before C = 1 - exp(-tau))
    float2 trA = MODE == SPLOTCH_ABSORPTIVE ? tA : f2(1.0f), trB = MODE == SPLOTCH_ABSORPTIVE ? tB : f2(1.0f);
    float2 tgA = trA, tbA = trA, tgB = trB, tbB = trB;
    if (MODE == SPLOTCH_E_EQ_A && PT) {
        trA = make_float2(expf(-crA.x), expf(-crA.y));
        tgA = make_float2(expf(-cgA.x), expf(-cgA.y));
        tbA = make_float2(expf(-cbA.x), expf(-cbA.y));
        trB = make_float2(expf(-crB.x), expf(-crB.y));
        tgB = make_float2(expf(-cgB.x), expf(-cgB.y));
        tbB = make_float2(expf(-cbB.x), expf(-cbB.y));
    }
    if (MODE == SPLOTCH_E_EQ_A) {
        crA = make_float2(-expm1f(-crA.x), -expm1f(-crA.y));
        cgA = make_float2(-expm1f(-cgA.x), -expm1f(-cgA.y));
        cbA = make_float2(-expm1f(-cbA.x), -expm1f(-cbA.y));
        crB = make_float2(-expm1f(-crB.x), -expm1f(-crB.y));
        cgB = make_float2(-expm1f(-cgB.x), -expm1f(-cgB.y));
        cbB = make_float2(-expm1f(-cbB.x), -expm1f(-cbB.y));
    }
    auto put = [&](float *img, int py, float2 cr, float2 cg, float2 cb) {
        if (py >= a.height) return;
        float *rowp = img + (size_t)py * a.width * 3;
        if (px0 < a.width) {
            rowp[3 * px0 + 0] = cr.x; rowp[3 * px0 + 1] = cg.x; rowp[3 * px0 + 2] = cb.x;
        }
        if (px0 + 1 < a.width) {
            rowp[3 * px0 + 3] = cr.y; rowp[3 * px0 + 4] = cg.y; rowp[3 * px0 + 5] = cb.y;
        }
    };
    put(a.image, py0, crA, cgA, cbA);
    put(a.image, py0 + 1, crB, cgB, cbB);
    if (PT) {
        put(a.trans, py0, trA, tgA, tbA);
        put(a.trans, py0 + 1, trB, tgB, tbB);
    }
}

// Tile render with the layout for the tile size.
template <int T, int MODE, int B, bool SERIES, bool ET = false, bool PT = false>
__device__ __forceinline__ void render_any(const RenderArgs &a, const int tile, RenderSmem<B> &sm) {
    if constexpr (T >= 16) render_tile4<T, MODE, B, SERIES, ET, PT>(a, tile, sm);
    else render_tile<T, MODE, B, SERIES, ET, PT>(a, tile, sm);
}

// ET: absorptive early termination (a.cutoff > 0); PT: partial image (a.trans).
// One block per multiprocessor as the stated minimum leaves the register
// count to the compiler (93-94 for the bench configuration, no spills, 10
// CTAs per SM): 3.40 -> 3.36 ms against the 80 registers and small spills it
// chose without the bound; capping at 72 (14 CTAs) or unrolling four steps
// was slower (3.52 ms).
// TMA: batches staged by tile::gather4 copies (tiles of 16 and 32, plain render).
template <int T, int MODE, int B, bool ET, bool PT, bool TMA>
__global__ void __launch_bounds__(render_threads(T), 1) k_render(RenderArgs a, const __grid_constant__ TmaMaps maps) {
    pdl_enter();
    __shared__ __align__(16) RenderSmem<B> sm;
    const uint32_t tile = __ldg(&a.torder[blockIdx.x]);
    if (tile >= gridDim.x) return;   // a workspace that was never binned
    const bool series = MODE == SPLOTCH_ABSORPTIVE && a.hdr->series_only;
    if constexpr (TMA) {
        __shared__ TmaSmem<B> ts;
        if (series) render_tile4<T, MODE, B, true, ET, PT, true>(a, (int)tile, sm, &maps, &ts);
        else render_tile4<T, MODE, B, false, ET, PT, true>(a, (int)tile, sm, &maps, &ts);
    } else {
        if (series) render_any<T, MODE, B, true, ET, PT>(a, (int)tile, sm);
        else render_any<T, MODE, B, false, ET, PT>(a, (int)tile, sm);
    }
}

// Persistent render of the tiles of many frames: each CTA takes the next
// (frame, tile) task from a counter until none is left.  Frames come in the
// order of the table (the host puts the heaviest first) and a frame's tiles
// in its render order (longest lists first), so the small ones fill the tail.
template <int T, int B>
__global__ void __launch_bounds__(render_threads(T)) k_render_batch(const __grid_constant__ BatchArgs args) {
    __shared__ __align__(16) RenderSmem<B> sm;
    __shared__ uint32_t s_task;
    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) s_task = atomicAdd(args.counter, 1u);
        __syncthreads();
        const uint32_t task = s_task;
        if (task >= args.n_tasks) break;
        int lo = 0, hi = args.n_items;   // last item whose first task is <= task
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (args.item[mid].task_begin <= task) lo = mid; else hi = mid;
        }
        const RenderArgs &a = args.item[lo].args;
        const uint32_t first = args.item[lo].task_begin;
        const uint32_t last = lo + 1 < args.n_items ? args.item[lo + 1].task_begin : args.n_tasks;
        const uint32_t t = __ldg(&a.torder[task - first]);
        if (t >= last - first) continue;   // a workspace that was never binned
        const int tile = (int)t;
        if (a.mode == SPLOTCH_EMISSION) render_any<T, SPLOTCH_EMISSION, B, false>(a, tile, sm);
        else if (a.mode == SPLOTCH_ABSORPTIVE && a.hdr->series_only) render_any<T, SPLOTCH_ABSORPTIVE, B, true>(a, tile, sm);
        else if (a.mode == SPLOTCH_ABSORPTIVE) render_any<T, SPLOTCH_ABSORPTIVE, B, false>(a, tile, sm);
        else render_any<T, SPLOTCH_E_EQ_A, B, false>(a, tile, sm);
    }
}

template <int T, int MODE, bool ET, bool PT, bool TMA>
static void launch_tb(const RenderArgs &a, const TmaMaps &m, int ntiles, cudaStream_t st) {
    switch (a.batch) {
    case 64: launch_pdl(k_render<T, MODE, 64, ET, PT, TMA>, dim3(ntiles), dim3(render_threads(T)), 0, st, a, m); break;
    case 128: launch_pdl(k_render<T, MODE, 128, ET, PT, TMA>, dim3(ntiles), dim3(render_threads(T)), 0, st, a, m); break;
    default: launch_pdl(k_render<T, MODE, 256, ET, PT, TMA>, dim3(ntiles), dim3(render_threads(T)), 0, st, a, m); break;
    }
}

template <int T, int MODE, bool ET>
static void launch_tp(const RenderArgs &a, const TmaMaps &m, bool tma, int ntiles, cudaStream_t st) {
    if (a.trans) {
        launch_tb<T, MODE, ET, true, false>(a, m, ntiles, st);
    } else if constexpr (T >= 16 && !ET) {
        if (tma) launch_tb<T, MODE, ET, false, true>(a, m, ntiles, st);
        else launch_tb<T, MODE, ET, false, false>(a, m, ntiles, st);
    } else {
        launch_tb<T, MODE, ET, false, false>(a, m, ntiles, st);
    }
}

template <int T>
static void launch_t(const RenderArgs &a, const TmaMaps &m, bool tma, int ntiles, cudaStream_t st) {
    switch (a.mode) {
    case SPLOTCH_EMISSION: launch_tp<T, SPLOTCH_EMISSION, false>(a, m, tma, ntiles, st); break;
    case SPLOTCH_ABSORPTIVE:
        if (a.cutoff > 0.0f) launch_tp<T, SPLOTCH_ABSORPTIVE, true>(a, m, tma, ntiles, st);
        else launch_tp<T, SPLOTCH_ABSORPTIVE, false>(a, m, tma, ntiles, st);
        break;
    default: launch_tp<T, SPLOTCH_E_EQ_A, false>(a, m, tma, ntiles, st); break;
    }
}

// cuTensorMapEncodeTiled, found through the runtime (no link against the driver library).
typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
static EncodeTiledFn encode_tiled() {
    static EncodeTiledFn fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess && q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(p);
    });
    return fn;
}

// A tensor map over n records of 4 floats (16 B): rows of one particle, a box
// of one row (the shape a tile::gather4 copy takes).
static bool encode_records(CUtensorMap *m, const float4 *base, uint64_t n) {
    EncodeTiledFn fn = encode_tiled();
    if (!fn) return false;
    const cuuint64_t dims[2] = {4, n ? n : 1};
    const cuuint64_t strides[1] = {16};
    const cuuint32_t box[2] = {4, 1};
    const cuuint32_t estr[2] = {1, 1};
    return fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float4 *>(base), dims, strides, box, estr,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

RenderArgs make_render_args(void *ws, const Layout &L, int mode, int batch, float *image, float *trans,
                            float cutoff) {
    RenderArgs a{};
    a.hdr = header(ws);
    a.toff = at<uint32_t>(ws, L.off_toff);
    a.torder = at<uint32_t>(ws, L.off_torder);
    a.list = at<uint32_t>(ws, fine_list_offset(L));
    a.geo = at<float4>(ws, L.off_geo);
    a.col = at<float4>(ws, L.off_col);
    a.image = image;
    a.trans = trans;
    a.cutoff = mode == SPLOTCH_ABSORPTIVE ? cutoff : 0.0f;
    a.width = L.width;
    a.height = L.height;
    a.tile = L.tile;
    a.ntx = L.ntx;
    a.mode = mode;
    a.batch = batch;
    return a;
}

cudaError_t launch_render(void *ws, const Layout &L, int mode, int batch, float *image, float *trans, float cutoff,
                          int staging, cudaStream_t st) {
    const RenderArgs a = make_render_args(ws, L, mode, batch, image, trans, cutoff);
    TmaMaps m;
    std::memset(&m, 0, sizeof(m));
    const bool tma = staging == 1 && L.tile >= 16 && !trans && !(a.cutoff > 0.0f);
    if (tma && (!encode_records(&m.geo, a.geo, L.n) || !encode_records(&m.col, a.col, L.n)))
        return cudaErrorNotSupported;
    switch (L.tile) {
    case 8: launch_t<8>(a, m, false, (int)L.ntiles, st); break;
    case 32: launch_t<32>(a, m, tma, (int)L.ntiles, st); break;
    default: launch_t<16>(a, m, tma, (int)L.ntiles, st); break;
    }
    count_launches(1);
    return cudaGetLastError();
}

// Grid of the persistent batch render: as many CTAs as fit on the GPU at once.
template <int T, int B>
static cudaError_t launch_batch_tb(const BatchArgs &b, cudaStream_t st) {
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_render_batch<T, B>, render_threads(T), 0);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) per_sm = 1;
    k_render_batch<T, B><<<sms * per_sm, render_threads(T), 0, st>>>(b);
    return cudaGetLastError();
}

template <int T>
static cudaError_t launch_batch_t(const BatchArgs &b, int batch, cudaStream_t st) {
    switch (batch) {
    case 64: return launch_batch_tb<T, 64>(b, st);
    case 128: return launch_batch_tb<T, 128>(b, st);
    default: return launch_batch_tb<T, 256>(b, st);
    }
}

cudaError_t launch_render_batch(const BatchArgs &b, int tile, int batch, cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(b.counter, 0, sizeof(unsigned int), st);
    if (e != cudaSuccess) return e;
    switch (tile) {
    case 8: e = launch_batch_t<8>(b, batch, st); break;
    case 32: e = launch_batch_t<32>(b, batch, st); break;
    default: e = launch_batch_t<16>(b, batch, st); break;
    }
    count_launches(1);
    return e;
}

// Ordered composition of two partial images (front nearer the camera):
// C = C_f + T_f C_b, T = T_f T_b, each product rounded once, no contraction.
// Four values per thread with 16-byte loads; an HBM-bound stream of 16 B read
// and 8 B (4 B without T) written per value.
__global__ void __launch_bounds__(256) k_compose(const float4 *cf, const float4 *tf, const float4 *cb, const float4 *tb,
                                                 float4 *co, float4 *to, uint64_t n4) {
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n4; i += (uint64_t)gridDim.x * blockDim.x) {
        const float4 a = cf[i], t = tf[i], b = cb[i];
        float4 u;
        if (to) u = tb[i];
        co[i] = make_float4(__fadd_rn(a.x, __fmul_rn(t.x, b.x)), __fadd_rn(a.y, __fmul_rn(t.y, b.y)),
                            __fadd_rn(a.z, __fmul_rn(t.z, b.z)), __fadd_rn(a.w, __fmul_rn(t.w, b.w)));
        if (to) to[i] = make_float4(__fmul_rn(t.x, u.x), __fmul_rn(t.y, u.y), __fmul_rn(t.z, u.z), __fmul_rn(t.w, u.w));
    }
}

__global__ void k_compose_tail(const float *cf, const float *tf, const float *cb, const float *tb, float *co, float *to,
                               uint64_t i0, uint64_t n) {
    const uint64_t i = i0 + threadIdx.x;
    if (i >= n) return;
    const float a = cf[i], t = tf[i], b = cb[i];
    const float u = to ? tb[i] : 0.0f;
    co[i] = __fadd_rn(a, __fmul_rn(t, b));
    if (to) to[i] = __fmul_rn(t, u);
}

cudaError_t launch_compose(const float *cf, const float *tf, const float *cb, const float *tb, float *co, float *to,
                           uint64_t n, cudaStream_t st) {
    const uint64_t n4 = n / 4;
    if (n4) {
        int dev = 0, sms = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        const uint64_t want = (n4 + 255) / 256, cap = (uint64_t)(sms > 0 ? sms : 148) * 8;
        k_compose<<<(unsigned)(want < cap ? want : cap), 256, 0, st>>>(
            reinterpret_cast<const float4 *>(cf), reinterpret_cast<const float4 *>(tf),
            reinterpret_cast<const float4 *>(cb), reinterpret_cast<const float4 *>(tb), reinterpret_cast<float4 *>(co),
            reinterpret_cast<float4 *>(to), n4);
        count_launches(1);
    }
    if (n % 4) {
        k_compose_tail<<<1, 32, 0, st>>>(cf, tf, cb, tb, co, to, n4 * 4, n);
        count_launches(1);
    }
    return cudaGetLastError();
}

// Number of (pixel, particle) pairs that pass the membership test, summed
// over the visible particles (a measurement helper, not part of a frame).
// With the pixel boxes stored, the pixels tested are the box's; without
// them, those whose centres lie within a slightly widened radius of the
// centre, clipped to the image: a superset of the box, which holds every
// pixel that passes, so the count is the same either way.
__global__ void __launch_bounds__(256) k_count_fragments(const Header *hdr, const float4 *geo, const ushort4 *box,
                                                         const uint32_t *key, uint64_t n, int width, int height,
                                                         unsigned long long *out) {
    const bool boxes = hdr->boxes_kept != 0;
    unsigned long long cnt = 0;
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
        if (key[i] == kInvalidKey) continue;
        const float4 g = geo[i];
        int x0, x1, y0, y1;
        if (boxes) {
            const ushort4 b = box[i];
            x0 = b.x; y0 = b.y; x1 = b.z; y1 = b.w;
        } else {
            const float rr = sqrtf(g.z) * 1.001f + 0.01f;
            x0 = max(0, (int)ceilf(g.x - rr - 0.5f));
            x1 = min(width - 1, (int)floorf(g.x + rr - 0.5f));
            y0 = max(0, (int)ceilf(g.y - rr - 0.5f));
            y1 = min(height - 1, (int)floorf(g.y + rr - 0.5f));
        }
        for (int j = y0; j <= y1; ++j) {
            const float dy = __fsub_rn((float)j + 0.5f, g.y);
            for (int x = x0; x <= x1; ++x) {
                const float dx = __fsub_rn((float)x + 0.5f, g.x);
                cnt += __fmaf_rn(dy, dy, __fmul_rn(dx, dx)) < g.z;
            }
        }
    }
    cnt = __reduce_add_sync(0xFFFFFFFFu, (unsigned)(cnt & 0xFFFFFFFFu)) +
          ((unsigned long long)__reduce_add_sync(0xFFFFFFFFu, (unsigned)(cnt >> 32)) << 32);
    if ((threadIdx.x & 31) == 0) atomicAdd(out, cnt);
}

cudaError_t launch_count_fragments(void *ws, const Layout &L, uint64_t *out, cudaStream_t st) {
    cudaMemsetAsync(out, 0, sizeof(uint64_t), st);
    if (L.n) {
        k_count_fragments<<<1024, 256, 0, st>>>(header(ws), at<float4>(ws, L.off_geo), at<ushort4>(ws, L.off_box),
                                                at<uint32_t>(ws, L.off_key), L.n, L.width, L.height,
                                                reinterpret_cast<unsigned long long *>(out));
        count_launches(1);
    }
    return cudaGetLastError();
}

}  // namespace spl
