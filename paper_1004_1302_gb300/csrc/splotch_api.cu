// C ABI of the library: argument checks, workspace layout and the order in
// which each call enqueues its kernels.  See include/splotch.h for the
// contract of every entry point.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <numeric>
#include <vector>

#include "internal.h"

namespace spl {

static std::atomic<uint64_t> g_launches{0};
void count_launches(uint64_t k) { g_launches.fetch_add(k, std::memory_order_relaxed); }

static uint64_t align256(uint64_t v) { return (v + 255u) & ~uint64_t(255u); }

int tile_payload_override() {
    static const int v = [] {
        const char *e = std::getenv("SPLOTCH_TILE_PAYLOAD");
        if (!e || !*e) return -1;
        return e[0] == '1' ? 1 : (e[0] == '0' ? 0 : -1);
    }();
    return v;
}

uint64_t device_l2_bytes() {
    static std::atomic<uint64_t> cached[64];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 0;
    uint64_t v = cached[dev].load(std::memory_order_relaxed);
    if (!v) {
        int b = 0;
        cudaDeviceGetAttribute(&b, cudaDevAttrL2CacheSize, dev);
        v = b > 0 ? (uint64_t)b : 1;
        cached[dev].store(v, std::memory_order_relaxed);
    }
    return v;
}

static uint32_t balanced_ctas(uint64_t items) {
    uint64_t tiles = (items + kSortTile - 1) / kSortTile;
    if (tiles == 0) tiles = 1;
    const uint64_t tpc = (tiles + kMaxSortCtas - 1) / kMaxSortCtas;
    return (uint32_t)((tiles + tpc - 1) / tpc);
}

int compute_layout(uint64_t n, int width, int height, int tile, uint64_t cap, Layout *out) {
    if (n >= (1ull << 32) || width < 1 || height < 1 || width > 65535 || height > 65535) return SPLOTCH_ERR_ARG;
    if (!(tile == 8 || tile == 16 || tile == 32)) return SPLOTCH_ERR_ARG;
    if (cap >= (1ull << 32) - 256) return SPLOTCH_ERR_ARG;
    Layout L{};
    L.n = n;
    L.width = width;
    L.height = height;
    L.tile = tile;
    L.ntx = (width + tile - 1) / tile;
    L.nty = (height + tile - 1) / tile;
    L.ntiles = (uint32_t)L.ntx * (uint32_t)L.nty;
    L.cap = cap;
    L.sort_ctas = balanced_ctas(n);
    L.ent_ctas = balanced_ctas(cap);
    L.hist_ctas = L.sort_ctas > L.ent_ctas ? L.sort_ctas : L.ent_ctas;
    uint64_t o = kHeaderBytes;
    auto take = [&](uint64_t bytes) {
        uint64_t r = o;
        o = align256(o + bytes);
        return r;
    };
    L.off_geo = take(n * 16);
    L.off_col = take(n * 16);
    L.off_key = take(n * 4);
    L.off_box = take(n * 8);
    L.off_tbox = take(n * 4);
    L.off_sbox = take(n * 8 + 256);
    L.off_pay[0] = L.off_sbox;
    L.off_pay[1] = L.off_sbox + align256(n * 4);
    for (int b = 0; b < 2; ++b) {
        L.off_sk[b] = take(n * 4);
        L.off_sv[b] = take(n * 4);
    }
    L.off_part = take((uint64_t)kMaxSortCtas * 8);
    L.off_hist = take((uint64_t)kRadix * L.hist_ctas * 4);
    L.off_htot = take((uint64_t)kRadix * 4);
    L.off_toff = take(((uint64_t)L.ntiles + 1) * 4);
    L.off_torder = take((uint64_t)L.ntiles * 4);
    L.nsx = (uint32_t)((L.ntx + kSuperSide - 1) / kSuperSide);
    L.nsy = (uint32_t)((L.nty + kSuperSide - 1) / kSuperSide);
    L.nsuper = L.nsx * L.nsy;
    L.max_units = (uint32_t)((cap + kUnit - 1) / kUnit) + L.nsuper;
    L.off_soff = take(((uint64_t)L.nsuper + 1) * 4);
    L.off_ufirst = take(((uint64_t)L.nsuper + 1) * 4);
    L.off_units = take((uint64_t)L.max_units * 16);
    L.off_ucnt = take((uint64_t)L.max_units * 64 * 4);
    for (int b = 0; b < 2; ++b) {
        L.off_ek[b] = take(cap * 4 + 64);
        L.off_ev[b] = take(cap * 4 + 64);
    }
    L.total = o;
    *out = L;
    return SPLOTCH_OK;
}

// The per-particle records come first, so their offsets depend on the
// particle count alone (not on the image or the tile-entry capacity).
static uint64_t col_offset(uint64_t n) { return align256(kHeaderBytes + n * 16); }

static int check_ws(const void *ws, size_t bytes, const Layout &L) {
    if (!ws || (reinterpret_cast<uintptr_t>(ws) & 255u)) return SPLOTCH_ERR_ARG;
    if (bytes < L.total) return SPLOTCH_ERR_WORKSPACE;
    return SPLOTCH_OK;
}

static int check_params(const splotch_render_params *pr) {
    if (!pr) return SPLOTCH_ERR_ARG;
    if (pr->mode < 0 || pr->mode > 2) return SPLOTCH_ERR_ARG;
    if (!(pr->batch == 64 || pr->batch == 128 || pr->batch == 256)) return SPLOTCH_ERR_ARG;
    if (!(pr->sigma_per_h > 0.0f) || !(pr->trunc_f > 0.0f) || pr->large_threshold_px < 0) return SPLOTCH_ERR_ARG;
    if (pr->slab != 0 && pr->slab != 1) return SPLOTCH_ERR_ARG;
    if (!(pr->t_min_cutoff >= 0.0f) || !(pr->t_min_cutoff < 1.0f)) return SPLOTCH_ERR_ARG;
    if (pr->staging != 0 && pr->staging != 1) return SPLOTCH_ERR_ARG;
    if (pr->keep_pixel_boxes != 0 && pr->keep_pixel_boxes != 1) return SPLOTCH_ERR_ARG;
    return SPLOTCH_OK;
}

static int check_camera(const splotch_camera *c) {
    if (!c || !(c->scale > 0.0) || !std::isfinite(c->scale) || c->width < 1 || c->height < 1) return SPLOTCH_ERR_ARG;
    return SPLOTCH_OK;
}

static int frame_layout(const splotch_render_params *pr, const splotch_camera *cam, uint64_t n, Layout *L) {
    int s = check_params(pr);
    if (s) return s;
    s = check_camera(cam);
    if (s) return s;
    return compute_layout(n, cam->width, cam->height, pr->tile, pr->max_tile_entries, L);
}

static int cuda_status(cudaError_t e) { return e == cudaSuccess ? SPLOTCH_OK : SPLOTCH_ERR_CUDA; }

__global__ void k_box_to_int(const ushort4 *box, const uint32_t *key, int4 *out, uint64_t n) {
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
        const ushort4 b = box[i];
        out[i] = key[i] == kInvalidKey ? make_int4(0, 0, -1, -1) : make_int4(b.x, b.y, b.z, b.w);
    }
}

__global__ void k_geo_split(const float4 *geo, float *sx, float *sy, float *r2, uint64_t n) {
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
        const float4 g = geo[i];
        if (sx) sx[i] = g.x;
        if (sy) sy[i] = g.y;
        if (r2) r2[i] = g.z;
    }
}

static int read_header(const void *ws, size_t bytes, cudaStream_t st, Header *h) {
    if (!ws || bytes < kHeaderBytes) return SPLOTCH_ERR_ARG;
    if (cudaStreamSynchronize(st) != cudaSuccess) return SPLOTCH_ERR_CUDA;
    if (cudaMemcpy(h, ws, sizeof(Header), cudaMemcpyDeviceToHost) != cudaSuccess) return SPLOTCH_ERR_CUDA;
    if (h->magic != kMagic) return SPLOTCH_ERR_STATE;
    if (h->layout.total > bytes) return SPLOTCH_ERR_WORKSPACE;
    return SPLOTCH_OK;
}

}  // namespace spl

using namespace spl;

extern "C" {

int splotch_abi_version(void) { return SPLOTCH_ABI_VERSION; }

const char *splotch_status_string(int status) {
    switch (status) {
    case SPLOTCH_OK: return "ok";
    case SPLOTCH_ERR_ARG: return "invalid argument";
    case SPLOTCH_ERR_CUDA: return "CUDA runtime error";
    case SPLOTCH_ERR_WORKSPACE: return "workspace too small or tile-entry capacity exceeded";
    case SPLOTCH_ERR_TIMEOUT: return "bounded device wait ran out";
    case SPLOTCH_ERR_OOM_ADMISSION: return "request refused: not enough memory";
    case SPLOTCH_ERR_STATE: return "workspace does not hold the required step";
    case SPLOTCH_ERR_IO: return "file could not be opened or read";
    default: return "unknown status";
    }
}

int splotch_camera_init(splotch_camera *c) {
    if (!c) return SPLOTCH_ERR_ARG;
    double f[3] = {c->target[0] - c->eye[0], c->target[1] - c->eye[1], c->target[2] - c->eye[2]};
    double fn = std::sqrt(f[0] * f[0] + f[1] * f[1] + f[2] * f[2]);
    if (!(fn > 0.0) || !std::isfinite(fn)) return SPLOTCH_ERR_ARG;
    for (double &v : f) v /= fn;
    double r[3] = {c->up[1] * f[2] - c->up[2] * f[1], c->up[2] * f[0] - c->up[0] * f[2],
                   c->up[0] * f[1] - c->up[1] * f[0]};
    double rn = std::sqrt(r[0] * r[0] + r[1] * r[1] + r[2] * r[2]);
    if (!(rn > 0.0) || !std::isfinite(rn)) return SPLOTCH_ERR_ARG;
    for (double &v : r) v /= rn;
    double u[3] = {f[1] * r[2] - f[2] * r[1], f[2] * r[0] - f[0] * r[2], f[0] * r[1] - f[1] * r[0]};
    if (!(c->fov_x_deg > 0.0 && c->fov_x_deg < 180.0) || c->width < 1 || c->height < 1) return SPLOTCH_ERR_ARG;
    const double pi = 3.14159265358979323846;
    for (int k = 0; k < 3; ++k) {
        c->fwd[k] = f[k];
        c->right[k] = r[k];
        c->upv[k] = u[k];
    }
    c->scale = (0.5 * (double)c->width) / std::tan(0.5 * c->fov_x_deg * pi / 180.0);
    c->c_right = std::fma(c->eye[2], r[2], std::fma(c->eye[1], r[1], c->eye[0] * r[0]));
    c->c_up = std::fma(c->eye[2], u[2], std::fma(c->eye[1], u[1], c->eye[0] * u[0]));
    c->c_fwd = std::fma(c->eye[2], f[2], std::fma(c->eye[1], f[1], c->eye[0] * f[0]));
    return SPLOTCH_OK;
}

int splotch_workspace_size(uint64_t n, const splotch_camera *cam, const splotch_render_params *params, size_t *bytes) {
    if (!bytes) return SPLOTCH_ERR_ARG;
    Layout L;
    int s = frame_layout(params, cam, n, &L);
    if (s) return s;
    *bytes = (size_t)L.total;
    return SPLOTCH_OK;
}

int splotch_transform(const splotch_particles *p, const splotch_camera *cam, const splotch_render_params *params,
                      void *workspace, size_t workspace_bytes, void *stream) {
    if (!p) return SPLOTCH_ERR_ARG;
    Layout L;
    int s = frame_layout(params, cam, p->n, &L);
    if (s) return s;
    if ((s = check_ws(workspace, workspace_bytes, L))) return s;
    if (p->n && (!p->x || !p->y || !p->z || !p->h)) return SPLOTCH_ERR_ARG;
    if (p->n_species < 1 || p->n_species > SPLOTCH_MAX_SPECIES) return SPLOTCH_ERR_ARG;
    if (!(cam->znear >= 0.0)) return SPLOTCH_ERR_ARG;
    TransformArgs a{};
    a.x = p->x; a.y = p->y; a.z = p->z; a.h = p->h;
    a.n = p->n;
    a.fwd0 = cam->fwd[0]; a.fwd1 = cam->fwd[1]; a.fwd2 = cam->fwd[2];
    a.c_fwd = cam->c_fwd;
    a.znear = cam->znear;
    a.r0 = (float)cam->right[0]; a.r1 = (float)cam->right[1]; a.r2 = (float)cam->right[2];
    a.cr = (float)cam->c_right;
    a.u0 = (float)cam->upv[0]; a.u1 = (float)cam->upv[1]; a.u2 = (float)cam->upv[2];
    a.cu = (float)cam->c_up;
    a.s = (float)cam->scale;
    a.half_w = 0.5f * (float)cam->width;
    a.half_h = 0.5f * (float)cam->height;
    a.w_max = (float)(cam->width - 1);
    a.h_max = (float)(cam->height - 1);
    a.sigma_per_h = params->sigma_per_h;
    a.trunc_f = params->trunc_f;
    a.slab = params->slab != 0;
    a.slab_lo = params->slab_key_lo;
    a.slab_hi = params->slab_key_hi;
    a.tshift = L.tile == 8 ? 3 : (L.tile == 16 ? 4 : 5);
    a.tbox = tile_box_packs(L) ? at<uint32_t>(workspace, L.off_tbox) : nullptr;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const bool keep_boxes = params->keep_pixel_boxes != 0 || !a.tbox;
    cudaError_t e = launch_init_header(workspace, L, p->n_species, params->mode, keep_boxes, st);
    if (e == cudaSuccess) e = launch_transform(a, workspace, L, keep_boxes, st);
    return cuda_status(e);
}

int splotch_colorize(const splotch_particles *p, const splotch_species *species, const splotch_colormap *cmap,
                     void *workspace, size_t workspace_bytes, void *stream) {
    if (!p || !species || !cmap || !workspace) return SPLOTCH_ERR_ARG;
    if (reinterpret_cast<uintptr_t>(workspace) & 255u) return SPLOTCH_ERR_ARG;
    if (p->n_species < 1 || p->n_species > SPLOTCH_MAX_SPECIES) return SPLOTCH_ERR_ARG;
    if (p->n && !p->intensity) return SPLOTCH_ERR_ARG;
    if (p->intensity_dtype < 0 || p->intensity_dtype > 2) return SPLOTCH_ERR_ARG;
    if (cmap->n_entries < 2 || cmap->n_entries > SPLOTCH_MAX_PALETTE || !cmap->rgb) return SPLOTCH_ERR_ARG;
    if (p->species_begin[0] != 0 || p->species_begin[p->n_species] != p->n) return SPLOTCH_ERR_ARG;
    for (int s = 0; s < p->n_species; ++s)
        if (p->species_begin[s + 1] < p->species_begin[s]) return SPLOTCH_ERR_ARG;
    for (int s = 0; s < p->n_species; ++s) {
        if (p->species_begin[s + 1] == p->species_begin[s]) continue;
        if (species[s].use_vector && (!p->vector[0] || !p->vector[1] || !p->vector[2])) return SPLOTCH_ERR_ARG;
        if (species[s].modulate && !p->modulator) return SPLOTCH_ERR_ARG;
    }
    if (workspace_bytes < col_offset(p->n) + p->n * 16) return SPLOTCH_ERR_WORKSPACE;
    ColorizeArgs a{};
    a.v = p->intensity;
    for (int c = 0; c < 3; ++c) a.vec[c] = p->vector[c];
    a.q = p->modulator;
    a.dtype = p->intensity_dtype;
    a.n = p->n;
    a.n_species = p->n_species;
    for (int s = 0; s <= p->n_species; ++s) a.begin[s] = p->species_begin[s];
    for (int s = p->n_species + 1; s <= SPLOTCH_MAX_SPECIES; ++s) a.begin[s] = p->n;
    for (int s = 0; s < p->n_species; ++s) a.sp[s] = species[s];
    a.palette = cmap->rgb;
    a.n_entries = cmap->n_entries;
    Layout L{};
    L.off_col = col_offset(p->n);
    return cuda_status(launch_colorize(a, workspace, L, static_cast<cudaStream_t>(stream)));
}

int splotch_sort(const splotch_render_params *params, const splotch_camera *cam, uint64_t n, void *workspace,
                 size_t workspace_bytes, void *stream) {
    Layout L;
    int s = frame_layout(params, cam, n, &L);
    if (s) return s;
    if ((s = check_ws(workspace, workspace_bytes, L))) return s;
    return cuda_status(launch_sort(workspace, L, params->mode, static_cast<cudaStream_t>(stream)));
}

int splotch_bin(const splotch_render_params *params, const splotch_camera *cam, uint64_t n, void *workspace,
                size_t workspace_bytes, void *stream) {
    Layout L;
    int s = frame_layout(params, cam, n, &L);
    if (s) return s;
    if ((s = check_ws(workspace, workspace_bytes, L))) return s;
    const int64_t px = params->large_threshold_px > 0 ? params->large_threshold_px
                                                       : (int64_t)(cam->width + cam->height) / 2;
    const int64_t side = (int64_t)params->tile * kSuperSide;   // entries are per super-tile
    const int64_t area = side * side;
    uint32_t large_tiles = (uint32_t)((px + area - 1) / area);
    if (large_tiles < 1) large_tiles = 1;
    return cuda_status(launch_bin(workspace, L, large_tiles, static_cast<cudaStream_t>(stream)));
}

int splotch_render_tiles(const splotch_render_params *params, const splotch_camera *cam, uint64_t n,
                         void *workspace, size_t workspace_bytes, float *image, void *stream) {
    Layout L;
    int s = frame_layout(params, cam, n, &L);
    if (s) return s;
    if ((s = check_ws(workspace, workspace_bytes, L))) return s;
    if (!image) return SPLOTCH_ERR_ARG;
    return cuda_status(launch_render(workspace, L, params->mode, params->batch, image, nullptr,
                                     params->t_min_cutoff, params->staging, static_cast<cudaStream_t>(stream)));
}

int splotch_render_partial(const splotch_render_params *params, const splotch_camera *cam, uint64_t n,
                           void *workspace, size_t workspace_bytes, float *color, float *trans, void *stream) {
    if (!color || !trans) return SPLOTCH_ERR_ARG;
    int s = splotch_sort(params, cam, n, workspace, workspace_bytes, stream);
    if (!s) s = splotch_bin(params, cam, n, workspace, workspace_bytes, stream);
    if (s) return s;
    Layout L;
    frame_layout(params, cam, n, &L);
    return cuda_status(launch_render(workspace, L, params->mode, params->batch, color, trans, params->t_min_cutoff,
                                     params->staging, static_cast<cudaStream_t>(stream)));
}

int splotch_compose(const float *c_front, const float *t_front, const float *c_back, const float *t_back,
                    float *c_out, float *t_out, uint64_t n_values, void *stream) {
    if (!c_front || !t_front || !c_back || !t_back || !c_out) return SPLOTCH_ERR_ARG;
    const uintptr_t bits = reinterpret_cast<uintptr_t>(c_front) | reinterpret_cast<uintptr_t>(t_front) |
                           reinterpret_cast<uintptr_t>(c_back) | reinterpret_cast<uintptr_t>(t_back) |
                           reinterpret_cast<uintptr_t>(c_out) | reinterpret_cast<uintptr_t>(t_out);
    if (bits & 15u) return SPLOTCH_ERR_ARG;
    return cuda_status(launch_compose(c_front, t_front, c_back, t_back, c_out, t_out, n_values,
                                      static_cast<cudaStream_t>(stream)));
}

int splotch_render_tiles_batch(const splotch_batch_item *items, int32_t n_items, int32_t tile, int32_t batch,
                               uint32_t *counter, void *stream) {
    if (!items || n_items < 1 || n_items > kMaxBatchItems || !counter) return SPLOTCH_ERR_ARG;
    if (!(tile == 8 || tile == 16 || tile == 32) || !(batch == 64 || batch == 128 || batch == 256))
        return SPLOTCH_ERR_ARG;
    std::vector<int> order(n_items);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return items[a].n > items[b].n; });
    static thread_local BatchArgs b;   // ~10 KB: kept off the stack
    b.counter = counter;
    b.n_items = n_items;
    uint64_t tasks = 0;
    for (int k = 0; k < n_items; ++k) {
        const splotch_batch_item &it = items[order[k]];
        if (check_camera(it.camera) || it.mode < 0 || it.mode > 2 || !it.image) return SPLOTCH_ERR_ARG;
        Layout L;
        int s = compute_layout(it.n, it.camera->width, it.camera->height, tile, it.max_tile_entries, &L);
        if (s) return s;
        if ((s = check_ws(it.workspace, it.workspace_bytes, L))) return s;
        b.item[k].args = make_render_args(it.workspace, L, it.mode, batch, it.image);
        b.item[k].task_begin = (uint32_t)tasks;
        tasks += L.ntiles;
        if (tasks >= (1ull << 32)) return SPLOTCH_ERR_ARG;
    }
    b.n_tasks = (uint32_t)tasks;
    return cuda_status(launch_render_batch(b, tile, batch, static_cast<cudaStream_t>(stream)));
}

int splotch_roi_scratch_size(uint64_t n, size_t *bytes) {
    if (!bytes || n >= (1ull << 32)) return SPLOTCH_ERR_ARG;
    *bytes = (size_t)kMaxSortCtas * 8;
    return SPLOTCH_OK;
}

static int check_roi(const splotch_particles *src, const double box[6], const void *scratch, size_t scratch_bytes,
                     const uint64_t *count) {
    if (!src || !box || !scratch || !count || src->n >= (1ull << 32)) return SPLOTCH_ERR_ARG;
    if (src->n && (!src->x || !src->y || !src->z || !src->h || !src->intensity)) return SPLOTCH_ERR_ARG;
    if (src->intensity_dtype < 0 || src->intensity_dtype > 2) return SPLOTCH_ERR_ARG;
    if (scratch_bytes < (size_t)kMaxSortCtas * 8) return SPLOTCH_ERR_WORKSPACE;
    return SPLOTCH_OK;
}

int splotch_roi_count(const splotch_particles *src, const double box[6], void *scratch, size_t scratch_bytes,
                      uint64_t *count, void *stream) {
    int s = check_roi(src, box, scratch, scratch_bytes, count);
    if (s) return s;
    return cuda_status(launch_roi(src, box, scratch, count, nullptr, nullptr, nullptr, nullptr, nullptr, 0, false,
                                  static_cast<cudaStream_t>(stream)));
}

int splotch_roi_select(const splotch_particles *src, const double box[6], void *scratch, size_t scratch_bytes,
                       float *x, float *y, float *z, float *h, void *intensity, uint64_t capacity, uint64_t *count,
                       void *stream) {
    int s = check_roi(src, box, scratch, scratch_bytes, count);
    if (s) return s;
    if (capacity && (!x || !y || !z || !h || !intensity)) return SPLOTCH_ERR_ARG;
    return cuda_status(launch_roi(src, box, scratch, count, x, y, z, h, intensity, capacity, true,
                                  static_cast<cudaStream_t>(stream)));
}

int splotch_render(const splotch_render_params *params, const splotch_camera *cam, uint64_t n, void *workspace,
                   size_t workspace_bytes, float *image, void *stream) {
    if (!image) return SPLOTCH_ERR_ARG;
    int s = splotch_sort(params, cam, n, workspace, workspace_bytes, stream);
    if (!s) s = splotch_bin(params, cam, n, workspace, workspace_bytes, stream);
    if (!s) s = splotch_render_tiles(params, cam, n, workspace, workspace_bytes, image, stream);
    return s;
}

int splotch_frame_info(const void *workspace, size_t workspace_bytes, splotch_frame_info_t *info, void *stream) {
    if (!info) return SPLOTCH_ERR_ARG;
    Header h;
    int s = read_header(workspace, workspace_bytes, static_cast<cudaStream_t>(stream), &h);
    if (s) return s;
    std::memset(info, 0, sizeof(*info));
    info->status = h.status;
    info->visible = h.visible;
    info->tile_entries = h.tile_entries;
    info->large = h.n_large;
    info->ntiles = h.layout.ntiles;
    info->check_line = h.check_line;
    for (int k = 0; k < SPLOTCH_MAX_SPECIES; ++k) {
        info->lo[k] = h.lo[k];
        info->hi[k] = h.hi[k];
    }
    return SPLOTCH_OK;
}

int splotch_get_keys(const void *workspace, size_t workspace_bytes, uint32_t *key, int32_t *box, void *stream) {
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    Header h;
    int s = read_header(workspace, workspace_bytes, st, &h);
    if (s) return s;
    const Layout &L = h.layout;
    void *ws = const_cast<void *>(workspace);
    if (key && L.n && cudaMemcpyAsync(key, at<uint32_t>(ws, L.off_key), L.n * 4, cudaMemcpyDeviceToDevice, st))
        return SPLOTCH_ERR_CUDA;
    if (box && L.n) {
        if (!h.boxes_kept) return SPLOTCH_ERR_STATE;   // the transform did not store the pixel boxes
        k_box_to_int<<<256, 256, 0, st>>>(at<ushort4>(ws, L.off_box), at<uint32_t>(ws, L.off_key),
                                          reinterpret_cast<int4 *>(box), L.n);
        count_launches(1);
        if (cudaGetLastError() != cudaSuccess) return SPLOTCH_ERR_CUDA;
    }
    return SPLOTCH_OK;
}

int splotch_get_geometry(const void *workspace, size_t workspace_bytes, float *sx, float *sy, float *r2,
                         void *stream) {
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    Header h;
    int s = read_header(workspace, workspace_bytes, st, &h);
    if (s) return s;
    if (h.layout.n) {
        k_geo_split<<<256, 256, 0, st>>>(at<float4>(const_cast<void *>(workspace), h.layout.off_geo), sx, sy, r2,
                                         h.layout.n);
        count_launches(1);
        if (cudaGetLastError() != cudaSuccess) return SPLOTCH_ERR_CUDA;
    }
    return SPLOTCH_OK;
}

int splotch_get_order(const void *workspace, size_t workspace_bytes, uint32_t *order, void *stream) {
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    Header h;
    int s = read_header(workspace, workspace_bytes, st, &h);
    if (s) return s;
    if (!order) return SPLOTCH_ERR_ARG;
    const Layout &L = h.layout;
    if (h.visible && cudaMemcpyAsync(order, at<uint32_t>(const_cast<void *>(workspace), L.off_sv[h.sorted_buf & 1]),
                                     (size_t)h.visible * 4, cudaMemcpyDeviceToDevice, st))
        return SPLOTCH_ERR_CUDA;
    return SPLOTCH_OK;
}

int splotch_get_tile_lists(const void *workspace, size_t workspace_bytes, uint32_t *offsets, uint32_t *list,
                           uint64_t capacity, void *stream) {
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    Header h;
    int s = read_header(workspace, workspace_bytes, st, &h);
    if (s) return s;
    const Layout &L = h.layout;
    if (h.status != SPLOTCH_OK) return h.status;
    if (list && capacity < h.tile_entries) return SPLOTCH_ERR_WORKSPACE;
    void *ws = const_cast<void *>(workspace);
    if (offsets && cudaMemcpyAsync(offsets, at<uint32_t>(ws, L.off_toff), ((size_t)L.ntiles + 1) * 4,
                                   cudaMemcpyDeviceToDevice, st))
        return SPLOTCH_ERR_CUDA;
    if (list && h.tile_entries &&
        cudaMemcpyAsync(list, at<uint32_t>(ws, fine_list_offset(L)), (size_t)h.tile_entries * 4,
                        cudaMemcpyDeviceToDevice, st))
        return SPLOTCH_ERR_CUDA;
    return SPLOTCH_OK;
}

int splotch_get_colors(const void *workspace, size_t workspace_bytes, float *ea, void *stream) {
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    Header h;
    int s = read_header(workspace, workspace_bytes, st, &h);
    if (s) return s;
    if (!ea) return SPLOTCH_ERR_ARG;
    if (h.layout.n && cudaMemcpyAsync(ea, at<float>(const_cast<void *>(workspace), h.layout.off_col), h.layout.n * 16,
                                      cudaMemcpyDeviceToDevice, st))
        return SPLOTCH_ERR_CUDA;
    return SPLOTCH_OK;
}

int splotch_count_fragments(const splotch_render_params *params, const splotch_camera *cam, uint64_t n,
                            void *workspace, size_t workspace_bytes, uint64_t *out, void *stream) {
    Layout L;
    int s = frame_layout(params, cam, n, &L);
    if (s) return s;
    if ((s = check_ws(workspace, workspace_bytes, L))) return s;
    if (!out) return SPLOTCH_ERR_ARG;
    return cuda_status(launch_count_fragments(workspace, L, out, static_cast<cudaStream_t>(stream)));
}

uint64_t splotch_launch_count(void) { return g_launches.load(std::memory_order_relaxed); }

}  // extern "C"
