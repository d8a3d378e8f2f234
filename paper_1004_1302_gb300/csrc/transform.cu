// Transform (camera, depth key, screen footprint, tile box) and colorize
// (range pre-pass, palette lookup) kernels.  Paper: Section 3.2 "process"
// and "display"; Section 2 for the footprint and colour.
#include "internal.h"
#include "device_util.cuh"
#include "ieee754.h"

namespace spl {

__global__ void k_init_header(Header *hdr, Layout L, int n_species, int mode, uint32_t boxes_kept) {
    pdl_enter();
    if (threadIdx.x != 0) return;
    hdr->magic = kMagic;
    hdr->boxes_kept = boxes_kept;
    hdr->status = SPLOTCH_OK;
    hdr->visible = 0;
    hdr->n_large = 0;
    hdr->tile_entries = 0;
    hdr->tile_entries32 = 0;
    hdr->key_min = kInvalidKey;
    hdr->key_max = 0;
    hdr->sorted_buf = 0;
    hdr->super_entries = 0;
    hdr->super32 = 0;
    hdr->n_units = 0;
    hdr->n_species = (uint32_t)n_species;
    hdr->mode = (uint32_t)mode;
    hdr->series_only = 0;
    hdr->check_line = 0;
    for (int s = 0; s < SPLOTCH_MAX_SPECIES; ++s) {
        hdr->range_lo_enc[s] = 0xFFFFFFFFu;
        hdr->range_hi_enc[s] = 0u;
        hdr->lo[s] = 0.0f;
        hdr->hi[s] = 0.0f;
        for (int c = 0; c < 3; ++c) {
            hdr->vlo_enc[s][c] = 0xFFFFFFFFu;
            hdr->vhi_enc[s][c] = 0u;
            hdr->vlo[s][c] = 0.0f;
            hdr->vhi[s][c] = 0.0f;
        }
        hdr->qlo_enc[s] = 0xFFFFFFFFu;
        hdr->qhi_enc[s] = 0u;
        hdr->qmax[s] = 0.0f;
    }
    for (int c = 0; c < 3; ++c) hdr->eoa_max[c] = 0.0f;
    hdr->layout = L;
}

struct Footprint {
    float4 geo;      // sx, sy, r2, -log2(e)/sigma_pix^2
    uint32_t key;    // kInvalidKey when culled
    ushort4 box;     // x0, y0, x1, y1
};

// The single-precision geometry of the transform call, operation by
// operation, each rounded on its own (no contraction).
__device__ __forceinline__ Footprint footprint(const TransformArgs &a, float x, float y, float z, float h) {
    Footprint f;
    f.geo = make_float4(0.f, 0.f, 0.f, 0.f);
    f.key = kInvalidKey;
    f.box = make_ushort4(1, 1, 0, 0);
    double Z = __dsub_rn(__fma_rn(ieee::widen(z), a.fwd2, __fma_rn(ieee::widen(y), a.fwd1, __dmul_rn(ieee::widen(x), a.fwd0))),
                         a.c_fwd);
    // the depth's conversions and near-plane test on the integer units (double throughput is low)
    if (!ieee::beyond(Z, a.znear)) return f;
    float Zf = ieee::narrow_positive(Z);
    if (a.slab) {   // depth slab of a partial render: lo <= key < hi
        const uint32_t k = __float_as_uint(Zf);
        if (k < a.slab_lo || k >= a.slab_hi) return f;
    }
    float X = __fsub_rn(__fmaf_rn(z, a.r2, __fmaf_rn(y, a.r1, __fmul_rn(x, a.r0))), a.cr);
    float Y = __fsub_rn(__fmaf_rn(z, a.u2, __fmaf_rn(y, a.u1, __fmul_rn(x, a.u0))), a.cu);
    float inv = __frcp_rn(Zf);
    float px = __fadd_rn(a.half_w, __fmul_rn(__fmul_rn(a.s, X), inv));
    float py = __fsub_rn(a.half_h, __fmul_rn(__fmul_rn(a.s, Y), inv));
    float sg = __fmul_rn(__fmul_rn(a.s, __fmul_rn(a.sigma_per_h, h)), inv);
    float r = __fmul_rn(a.trunc_f, sg);
    // pixel box: the centres within r of (px, py), widened by a 1/64 px guard
    // that covers the rounding of the cut test and of these operations
    constexpr float kGuard = 0.015625f;
    float lx = ceilf(__fsub_rn(__fsub_rn(__fsub_rn(px, r), 0.5f), kGuard));
    float hx = floorf(__fadd_rn(__fsub_rn(__fadd_rn(px, r), 0.5f), kGuard));
    float ly = ceilf(__fsub_rn(__fsub_rn(__fsub_rn(py, r), 0.5f), kGuard));
    float hy = floorf(__fadd_rn(__fsub_rn(__fadd_rn(py, r), 0.5f), kGuard));
    float x0 = lx > 0.0f ? lx : 0.0f, x1 = hx < a.w_max ? hx : a.w_max;
    float y0 = ly > 0.0f ? ly : 0.0f, y1 = hy < a.h_max ? hy : a.h_max;
    if (!(lx <= hx) || !(ly <= hy) || !(x0 <= x1) || !(y0 <= y1)) return f;
    f.key = __float_as_uint(Zf);
    // k = -log2(e) / sigma_pix^2 feeds only the weight's exponent (the oracle
    // evaluates the weight in FP64 from sigma_pix), so the fast division's
    // 2 ulp are enough
    f.geo = make_float4(px, py, __fmul_rn(r, r), __fdividef(-1.4426950408889634f, __fmul_rn(sg, sg)));
    f.box = make_ushort4((unsigned short)x0, (unsigned short)y0, (unsigned short)x1, (unsigned short)y1);
    return f;
}

// A block takes kIlp x blockDim consecutive particles, thread t the particles
// t, t + blockDim, ...: every load and store instruction of a warp covers
// consecutive particles (coalesced), and the kIlp loads of each array are in
// flight together.
template <int kIlp>
__global__ void __launch_bounds__(256) k_transform(TransformArgs a, float4 *geo, uint32_t *key, ushort4 *box,
                                                     Header *hdr) {
    pdl_enter();
    uint32_t nvis = 0, kmin = kInvalidKey, kmax = 0;
    const uint64_t chunk = (uint64_t)kIlp * blockDim.x;
    for (uint64_t b = blockIdx.x * chunk; b < a.n; b += (uint64_t)gridDim.x * chunk) {
        float xs[kIlp], ys[kIlp], zs[kIlp], hs[kIlp];
#pragma unroll
        for (int k = 0; k < kIlp; ++k) {
            const uint64_t i = b + threadIdx.x + (uint64_t)k * blockDim.x;
            const uint64_t j = i < a.n ? i : a.n - 1;
            xs[k] = __ldg(a.x + j);
            ys[k] = __ldg(a.y + j);
            zs[k] = __ldg(a.z + j);
            hs[k] = __ldg(a.h + j);
        }
#pragma unroll
        for (int k = 0; k < kIlp; ++k) {
            const uint64_t i = b + threadIdx.x + (uint64_t)k * blockDim.x;
            if (i >= a.n) break;
            Footprint f = footprint(a, xs[k], ys[k], zs[k], hs[k]);
            geo[i] = f.geo;
            key[i] = f.key;
            if (box) box[i] = f.box;
            if (a.tbox) {
                // the box in tiles, 8 bits per edge (what binning reads); x0 > x1 when culled
                a.tbox[i] = f.key == kInvalidKey
                                ? 0x000000FFu
                                : (uint32_t)(f.box.x >> a.tshift) | ((uint32_t)(f.box.y >> a.tshift) << 8) |
                                      ((uint32_t)(f.box.z >> a.tshift) << 16) | ((uint32_t)(f.box.w >> a.tshift) << 24);
            }
            if (f.key != kInvalidKey) {
                nvis += 1;
                kmin = min(kmin, f.key);
                kmax = max(kmax, f.key);
            }
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

// Range pre-pass: min/max of u (log10 of the value, or the value) of one
// quantity of one species into two of the header's order-preserving slots.
// Every quantity that needs a range is one job, all jobs in one launch
// (blockIdx.y).
struct RangeJob {
    const void *v;
    uint64_t begin, end;
    uint32_t *lo_enc, *hi_enc;
    int use_log;
};
constexpr int kMaxRangeJobs = SPLOTCH_MAX_SPECIES * 5;
struct RangeJobs {
    RangeJob job[kMaxRangeJobs];
    int dtype;
};

// loads in flight per thread in the range and colour passes (8 against 4:
// transform + colour 0.1637 -> 0.1621 ms at 10M)
constexpr int kRangeIlp = 8, kColorIlp = 8;
// The values of one 16-byte vector as floats: 4 (FP32) or 8 (FP16, BF16).
template <int DT> struct Vec16;
template <> struct Vec16<0> {
    static constexpr int kN = 4;
    __device__ static void unpack(const uint4 q, float *o) {
        o[0] = __uint_as_float(q.x); o[1] = __uint_as_float(q.y); o[2] = __uint_as_float(q.z); o[3] = __uint_as_float(q.w);
    }
};
template <> struct Vec16<1> {
    static constexpr int kN = 8;
    __device__ static void unpack(const uint4 q, float *o) {
        const uint32_t w[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            o[2 * k] = __half2float(__ushort_as_half((unsigned short)(w[k] & 0xFFFFu)));
            o[2 * k + 1] = __half2float(__ushort_as_half((unsigned short)(w[k] >> 16)));
        }
    }
};
template <> struct Vec16<2> {
    static constexpr int kN = 8;
    __device__ static void unpack(const uint4 q, float *o) {
        const uint32_t w[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
        for (int k = 0; k < 4; ++k) {   // bfloat16: the upper half of a float
            o[2 * k] = __uint_as_float(w[k] << 16);
            o[2 * k + 1] = __uint_as_float(w[k] & 0xFFFF0000u);
        }
    }
};

// Extremes of one job's values: 16-byte vector loads over the aligned body
// (kRangeIlp in flight per thread), single loads for the unaligned ends.
template <int DT>
__device__ __forceinline__ void range_extremes(const RangeJob &J, int use_log, float &lo, float &hi) {
    constexpr int kN = Vec16<DT>::kN;
    auto take = [&](float w) {
        // log10 is monotonic: the range of log10(max(v, 1e-37)) is taken from the
        // extremes of max(v, 1e-37), and the logarithm applied to those two only
        if (use_log) w = fmaxf(w, 1e-37f);
        lo = fminf(lo, w);
        hi = fmaxf(hi, w);
    };
    const uint64_t begin = J.begin, end = J.end;
    const uint64_t tid = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x, nthr = (uint64_t)gridDim.x * blockDim.x;
    const bool aligned = (reinterpret_cast<uintptr_t>(J.v) & 15u) == 0;
    const uint64_t vb = aligned ? (begin + kN - 1) / kN : end, ve = aligned ? end / kN : end;   // whole vectors
    if (!aligned || vb >= ve) {
        for (uint64_t i = begin + tid; i < end; i += nthr) take(load_value(J.v, DT, i));
        return;
    }
    // the ends: elements before the first and after the last whole vector
    const uint64_t head = vb * kN - begin, tail = end - ve * kN;
    if (tid < head) take(load_value(J.v, DT, begin + tid));
    else if (tid < head + tail) take(load_value(J.v, DT, ve * kN + (tid - head)));
    const uint4 *q = reinterpret_cast<const uint4 *>(J.v);
    for (uint64_t v0 = vb + tid; v0 < ve; v0 += kRangeIlp * nthr) {
        uint4 r[kRangeIlp];
#pragma unroll
        for (int k = 0; k < kRangeIlp; ++k) {
            const uint64_t vi = v0 + k * nthr;
            if (vi < ve) r[k] = q[vi];
        }
#pragma unroll
        for (int k = 0; k < kRangeIlp; ++k) {
            if (v0 + k * nthr >= ve) continue;
            float o[kN];
            Vec16<DT>::unpack(r[k], o);
#pragma unroll
            for (int e = 0; e < kN; ++e) take(o[e]);
        }
    }
}

__global__ void __launch_bounds__(256) k_range(const __grid_constant__ RangeJobs jobs) {
    pdl_enter();
    const RangeJob &J = jobs.job[blockIdx.y];
    float lo = INFINITY, hi = -INFINITY;
    if (jobs.dtype == 1) range_extremes<1>(J, J.use_log, lo, hi);
    else if (jobs.dtype == 2) range_extremes<2>(J, J.use_log, lo, hi);
    else range_extremes<0>(J, J.use_log, lo, hi);
    uint32_t elo = __reduce_min_sync(0xFFFFFFFFu, float_to_ordered(lo));
    uint32_t ehi = __reduce_max_sync(0xFFFFFFFFu, float_to_ordered(hi));
    if (lane_id() == 0) {
        atomicMin(J.lo_enc, elo);
        atomicMax(J.hi_enc, ehi);
    }
}

__global__ void k_range_finish(Header *hdr, ColorizeArgs a) {
    pdl_enter();
    const int s = threadIdx.x;
    const bool have = s < a.n_species;
    const bool empty = !have || a.begin[s + 1] == a.begin[s];
    const bool series = empty || a.sp[s].absorption <= kSeriesMaxA;
    const bool all = __all_sync(0xFFFFFFFFu, series);
    if (s == 0) hdr->series_only = all ? 1u : 0u;
    // Bound of the light a pixel can still receive behind transmittance T:
    // each layer adds T_acc E (1 - T_p)/A <= T_acc (1 - T_p) max|E|/A, which
    // sums to at most T max|E|/A.  Per species |E_c| <= |brightness| times
    // the largest |palette| (or |fixed rgb|, or 1 for a vector quantity) of
    // channel c; the modulation scales E and A alike and cancels.
    float pmax[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        float m = 0.0f;
        for (int k = s; k < a.n_entries; k += 32) m = fmaxf(m, fabsf(a.palette[3 * k + c]));
        pmax[c] = __uint_as_float(__reduce_max_sync(0xFFFFFFFFu, __float_as_uint(m)));
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        float r = 0.0f;
        if (!empty) {
            const splotch_species &sp = a.sp[s];
            const float cm = sp.use_vector ? 1.0f : sp.use_colormap ? pmax[c] : fabsf(sp.fixed_rgb[c]);
            const float e = fabsf(sp.brightness) * cm;
            r = sp.absorption > 0.0f ? e / sp.absorption : (e > 0.0f ? INFINITY : 0.0f);
        }
        r = __uint_as_float(__reduce_max_sync(0xFFFFFFFFu, __float_as_uint(r)));
        if (s == 0) hdr->eoa_max[c] = r;
    }
    if (!have) return;
    float lo = a.sp[s].lo, hi = a.sp[s].hi;
    const bool lg = a.sp[s].use_log;
    if (isnan(lo)) lo = empty ? 0.0f : (lg ? log10f(ordered_to_float(hdr->range_lo_enc[s])) : ordered_to_float(hdr->range_lo_enc[s]));
    if (isnan(hi)) hi = empty ? 0.0f : (lg ? log10f(ordered_to_float(hdr->range_hi_enc[s])) : ordered_to_float(hdr->range_hi_enc[s]));
    hdr->lo[s] = lo;
    hdr->hi[s] = hi;
    hdr->inv_span[s] = hi > lo ? 1.0f / (hi - lo) : 0.0f;
    if (a.sp[s].use_vector && !empty)
        for (int c = 0; c < 3; ++c) {
            hdr->vlo[s][c] = ordered_to_float(hdr->vlo_enc[s][c]);
            hdr->vhi[s][c] = ordered_to_float(hdr->vhi_enc[s][c]);
        }
    if (a.sp[s].modulate && !empty) hdr->qmax[s] = ordered_to_float(hdr->qhi_enc[s]);
}

// E and A of particle i of species s; u: its intensity (unused by a vector species).
__device__ __forceinline__ float4 colorize_one(const ColorizeArgs &a, const Header *hdr, const float *pal, float kmax,
                                               int s, uint64_t i, float u) {
    const splotch_species &sp = a.sp[s];
    float r, g, b;
    if (sp.use_vector) {
        // each component normalised linearly over the species
        float t[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const float uc = load_value(a.vec[c], a.dtype, i);
            const float lo = hdr->vlo[s][c], hi = hdr->vhi[s][c];
            const float tc = hi > lo ? __fdiv_rn(uc - lo, hi - lo) : 0.0f;
            t[c] = fminf(fmaxf(tc, 0.0f), 1.0f);
        }
        r = t[0]; g = t[1]; b = t[2];
    } else if (sp.use_colormap) {
        if (sp.use_log) u = log10f(fmaxf(u, 1e-37f));
        const float lo = hdr->lo[s], hi = hdr->hi[s];
        float t = hi > lo ? (u - lo) * hdr->inv_span[s] : 0.0f;   // 1 / (hi - lo), once per species
        t = fminf(fmaxf(t, 0.0f), 1.0f);
        float w = t * kmax;
        int k = min((int)floorf(w), a.n_entries - 2);
        float fr = w - (float)k;
        r = (1.0f - fr) * pal[3 * k + 0] + fr * pal[3 * k + 3];
        g = (1.0f - fr) * pal[3 * k + 1] + fr * pal[3 * k + 4];
        b = (1.0f - fr) * pal[3 * k + 2] + fr * pal[3 * k + 5];
    } else {
        r = sp.fixed_rgb[0]; g = sp.fixed_rgb[1]; b = sp.fixed_rgb[2];
    }
    float m = 1.0f;
    if (sp.modulate) {
        // column density scaled by q / q_max of the species: E and A alike
        const float qm = hdr->qmax[s];
        m = qm > 0.0f ? __fdiv_rn(load_value(a.q, a.dtype, i), qm) : 0.0f;
        m = fminf(fmaxf(m, 0.0f), 1.0f);
    }
    return make_float4(m * (sp.brightness * r), m * (sp.brightness * g), m * (sp.brightness * b), m * sp.absorption);
}

// A block takes kIlp x blockDim consecutive particles per step, thread t the
// particles t, t + blockDim, ...: the kIlp intensity loads are in flight
// together and every store of a warp covers consecutive particles.
template <int kIlp>
__global__ void __launch_bounds__(256) k_colorize(ColorizeArgs a, const Header *hdr, float4 *col) {
    pdl_enter();
    __shared__ float pal[SPLOTCH_MAX_PALETTE * 3];
    for (int k = threadIdx.x; k < a.n_entries * 3; k += blockDim.x) pal[k] = a.palette[k];
    __syncthreads();
    const float kmax = (float)(a.n_entries - 1);
    const uint64_t chunk = (uint64_t)kIlp * blockDim.x;
    for (uint64_t b0 = blockIdx.x * chunk; b0 < a.n; b0 += (uint64_t)gridDim.x * chunk) {
        float u[kIlp];
#pragma unroll
        for (int k = 0; k < kIlp; ++k) {
            const uint64_t i = b0 + threadIdx.x + (uint64_t)k * blockDim.x;
            u[k] = i < a.n && a.v ? load_value(a.v, a.dtype, i) : 0.0f;
        }
        int s = 0;
#pragma unroll
        for (int k = 0; k < kIlp; ++k) {
            const uint64_t i = b0 + threadIdx.x + (uint64_t)k * blockDim.x;
            if (i >= a.n) break;
#pragma unroll 1
            while (s + 1 < a.n_species && i >= a.begin[s + 1]) ++s;
            col[i] = colorize_one(a, hdr, pal, kmax, s, i, u[k]);
        }
    }
}

static int sm_count() {
    static int cached[64] = {0};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64) return 148;
    if (!cached[dev]) {
        int v = 0;
        cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
        cached[dev] = v > 0 ? v : 148;
    }
    return cached[dev];
}

cudaError_t launch_init_header(void *ws, const Layout &L, int n_species, int mode, bool boxes_kept, cudaStream_t st) {
    launch_pdl(k_init_header, dim3(1), dim3(32), 0, st, header(ws), L, n_species, mode, boxes_kept ? 1u : 0u);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_transform(const TransformArgs &a, void *ws, const Layout &L, bool keep_boxes, cudaStream_t st) {
    if (a.n == 0) return cudaGetLastError();
    const int sms = sm_count();
    float4 *geo = at<float4>(ws, L.off_geo);
    uint32_t *key = at<uint32_t>(ws, L.off_key);
    // the pixel boxes are stored when binning reads them (no packed tile boxes) or when asked for
    ushort4 *box = keep_boxes || !a.tbox ? at<ushort4>(ws, L.off_box) : nullptr;
    constexpr int kIlp = 4;
    const uint64_t blocks = (a.n + kIlp * 256 - 1) / (kIlp * 256);
    const int grid = (int)(blocks < (uint64_t)sms * 8 ? blocks : (uint64_t)sms * 8);
    launch_pdl(k_transform<kIlp>, dim3(grid), dim3(256), 0, st, a, geo, key, box, header(ws));
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_colorize(const ColorizeArgs &a, void *ws, const Layout &L, cudaStream_t st) {
    const int sms = sm_count();
    static thread_local RangeJobs jobs;
    int nj = 0;
    uint64_t longest = 0;
    Header *h = header(ws);
    auto add = [&](const void *v, uint64_t b, uint64_t e, int use_log, uint32_t *lo, uint32_t *hi) {
        jobs.job[nj++] = RangeJob{v, b, e, lo, hi, use_log};
        if (e - b > longest) longest = e - b;
    };
    for (int s = 0; s < a.n_species; ++s) {
        const splotch_species &sp = a.sp[s];
        const uint64_t b = a.begin[s], e = a.begin[s + 1];
        if (e <= b) continue;
        if (isnan(sp.lo) || isnan(sp.hi)) add(a.v, b, e, sp.use_log, &h->range_lo_enc[s], &h->range_hi_enc[s]);
        if (sp.use_vector)
            for (int c = 0; c < 3; ++c) add(a.vec[c], b, e, 0, &h->vlo_enc[s][c], &h->vhi_enc[s][c]);
        if (sp.modulate) add(a.q, b, e, 0, &h->qlo_enc[s], &h->qhi_enc[s]);
    }
    if (nj) {
        jobs.dtype = a.dtype;
        // about eight CTAs per SM in all, shared by the jobs; none gets more CTAs than its
        // values fill
        const uint64_t want = (longest + kRangeIlp * 256 - 1) / (kRangeIlp * 256);
        const uint64_t share = (uint64_t)sms * 8 / (uint64_t)nj;
        const unsigned gx = (unsigned)(want < share ? want : (share ? share : 1));
        launch_pdl(k_range, dim3(gx ? gx : 1, (unsigned)nj), dim3(256), 0, st, jobs);
        count_launches(1);
    }
    launch_pdl(k_range_finish, dim3(1), dim3(32), 0, st, header(ws), a);
    count_launches(1);
    if (a.n) {
        uint64_t blocks = (a.n + kColorIlp * 256 - 1) / (kColorIlp * 256);
        int grid = (int)(blocks < (uint64_t)sms * 8 ? blocks : (uint64_t)sms * 8);
        launch_pdl(k_colorize<kColorIlp>, dim3(grid), dim3(256), 0, st, a, header(ws), at<float4>(ws, L.off_col));
        count_launches(1);
    }
    return cudaGetLastError();
}

}  // namespace spl
