// Region-of-interest cut of a resident particle set: the particles inside an
// axis-aligned box, copied in index order (a stable compaction), so that a
// request's particles depend on its box alone.
#include "internal.h"
#include "device_util.cuh"

namespace spl {

constexpr int kRoiThreads = 256;
constexpr int kRoiItems = 16;
constexpr int kRoiTile = kRoiThreads * kRoiItems;

struct RoiArgs {
    const float *x, *y, *z, *h;
    const void *v;
    int dtype;
    uint64_t n;
    float lo[3], hi[3];
    uint32_t ctas;
    unsigned long long *part;   // per-CTA counts, then exclusive offsets
    unsigned long long *count;  // total (device, caller-owned)
    float *ox, *oy, *oz, *oh;
    void *ov;
    uint64_t capacity;
};

__device__ __forceinline__ bool in_box(const RoiArgs &a, uint64_t i) {
    const float px = a.x[i], py = a.y[i], pz = a.z[i];
    return px >= a.lo[0] && px < a.hi[0] && py >= a.lo[1] && py < a.hi[1] && pz >= a.lo[2] && pz < a.hi[2];
}

__device__ __forceinline__ void roi_range(const RoiArgs &a, uint64_t *beg, uint64_t *end) {
    const uint64_t tiles = (a.n + kRoiTile - 1) / kRoiTile;
    const uint64_t tpc = (tiles + a.ctas - 1) / a.ctas;
    *beg = (uint64_t)blockIdx.x * tpc * kRoiTile;
    const uint64_t e = *beg + tpc * kRoiTile;
    *end = e < a.n ? e : a.n;
    if (*beg > *end) *beg = *end;
}

__global__ void __launch_bounds__(kRoiThreads) k_roi_count(RoiArgs a) {
    __shared__ unsigned long long ws[kRoiThreads / 32 + 1];
    uint64_t beg, end;
    roi_range(a, &beg, &end);
    unsigned long long c = 0;
    for (uint64_t i = beg + threadIdx.x; i < end; i += kRoiThreads) c += in_box(a, i);
    unsigned long long tot;
    block_exclusive_scan64<kRoiThreads>(c, ws, &tot);
    if (threadIdx.x == 0) a.part[blockIdx.x] = tot;
}

__global__ void __launch_bounds__(1024) k_roi_scan(RoiArgs a) {
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
    if (threadIdx.x == 0) *a.count = total;
}

// Scatter: thread t owns items t*kRoiItems .. of each 4096-item step, so a
// block scan gives the order-preserving output positions.
__global__ void __launch_bounds__(kRoiThreads) k_roi_scatter(RoiArgs a) {
    __shared__ unsigned long long ws[kRoiThreads / 32 + 1];
    uint64_t beg, end;
    roi_range(a, &beg, &end);
    unsigned long long base = a.part[blockIdx.x];
    const size_t vsize = a.dtype == 0 ? 4 : 2;
    for (uint64_t step = beg; step < end; step += kRoiTile) {
        uint32_t flags = 0, mine = 0;
#pragma unroll
        for (int q = 0; q < kRoiItems; ++q) {
            const uint64_t i = step + (uint64_t)threadIdx.x * kRoiItems + q;
            if (i < end && in_box(a, i)) {
                flags |= 1u << q;
                ++mine;
            }
        }
        unsigned long long tot;
        unsigned long long o = base + block_exclusive_scan64<kRoiThreads>(mine, ws, &tot);
#pragma unroll
        for (int q = 0; q < kRoiItems; ++q) {
            if (!(flags >> q & 1u)) continue;
            const uint64_t i = step + (uint64_t)threadIdx.x * kRoiItems + q;
            if (o < a.capacity) {
                a.ox[o] = a.x[i];
                a.oy[o] = a.y[i];
                a.oz[o] = a.z[i];
                a.oh[o] = a.h[i];
                if (vsize == 4)
                    static_cast<float *>(a.ov)[o] = static_cast<const float *>(a.v)[i];
                else
                    static_cast<uint16_t *>(a.ov)[o] = static_cast<const uint16_t *>(a.v)[i];
            }
            ++o;
        }
        base += tot;
    }
}

uint32_t roi_ctas(uint64_t n) {
    uint64_t tiles = (n + kRoiTile - 1) / kRoiTile;
    if (tiles == 0) tiles = 1;
    const uint64_t tpc = (tiles + kMaxSortCtas - 1) / kMaxSortCtas;
    return (uint32_t)((tiles + tpc - 1) / tpc);
}

cudaError_t launch_roi(const splotch_particles *p, const double box[6], void *scratch, uint64_t *count,
                       float *ox, float *oy, float *oz, float *oh, void *ov, uint64_t capacity, bool scatter,
                       cudaStream_t st) {
    RoiArgs a{};
    a.x = p->x; a.y = p->y; a.z = p->z; a.h = p->h;
    a.v = p->intensity;
    a.dtype = p->intensity_dtype;
    a.n = p->n;
    for (int k = 0; k < 3; ++k) {
        a.lo[k] = (float)box[k];
        a.hi[k] = (float)box[3 + k];
    }
    a.ctas = roi_ctas(p->n);
    a.part = static_cast<unsigned long long *>(scratch);
    a.count = reinterpret_cast<unsigned long long *>(count);
    a.ox = ox; a.oy = oy; a.oz = oz; a.oh = oh; a.ov = ov;
    a.capacity = capacity;
    k_roi_count<<<a.ctas, kRoiThreads, 0, st>>>(a);
    k_roi_scan<<<1, 1024, 0, st>>>(a);
    count_launches(2);
    if (scatter) {
        k_roi_scatter<<<a.ctas, kRoiThreads, 0, st>>>(a);
        count_launches(1);
    }
    return cudaGetLastError();
}

}  // namespace spl
