// Internal declarations of the GB300 Splotch library: workspace layout,
// device header and the launchers of each kernel file.
#pragma once

#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

#include "splotch.h"

namespace spl {

constexpr uint32_t kInvalidKey = 0xFFFFFFFFu;
constexpr uint32_t kMagic = 0x5350'4C54u;  // "SPLT"

// Radix sort geometry: items are ranked in tiles of kSortTile.
constexpr int kSortThreads = 256;
constexpr int kSortTile = 4096;
constexpr int kRadix = 256;
constexpr int kMaxSortCtas = 2048;

// Launch with programmatic stream serialization: the kernel's CTAs may be
// scheduled while the previous kernel on the stream drains (every kernel of
// the frame path starts with pdl_enter(), which waits for that kernel's
// completion before touching memory), so the launch gap and the previous
// kernel's last wave overlap.
template <typename... KArgs, typename... Args>
cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                       Args &&...args) {
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...);
}

// Byte offsets of every workspace section.  Sections that depend only on the
// particle count come first, so colorize can find its output from n alone.
struct Layout {
    uint64_t n;
    int32_t width, height, tile, ntx, nty;
    uint32_t ntiles;
    uint64_t cap;            // tile-entry capacity
    uint32_t sort_ctas;      // CTAs of a radix pass over particles
    uint32_t ent_ctas;       // CTAs of a radix pass over tile entries
    uint32_t hist_ctas;      // max(sort_ctas, ent_ctas): rows of the histogram table
    uint32_t pad0;
    uint64_t off_geo, off_col, off_key, off_box, off_sbox;   // geo: {sx, sy, r2, -log2(e)/sigma_pix^2}; col: {Er, Eg, Eb, A}
    uint64_t off_pay[2];     // tile-box payload of the depth sort (ping-pong), inside the sbox section
    uint64_t off_tbox;       // packed tile box per particle (index order), written by the transform
    uint64_t off_sk[2], off_sv[2];
    uint64_t off_part;
    uint64_t off_hist, off_htot;
    uint64_t off_toff;                 // fine-tile offsets (ntiles + 1)
    uint64_t off_torder;               // render order of the tiles (ntiles): heaviest lists first
    uint64_t off_soff, off_ufirst;     // super-tile offsets (nsuper + 1), first unit of each super-tile (nsuper + 1)
    uint64_t off_units, off_ucnt;      // units (super-tile, begin, end), per-unit counts of the 64 fine tiles
    uint64_t off_ek[2], off_ev[2];     // super-tile entries (ping-pong); the final fine list reuses the free key buffer
    uint32_t nsx, nsy, nsuper, max_units;
    uint64_t total;
};

struct Header {
    uint32_t magic;
    int32_t status;
    uint32_t visible;          // V
    uint32_t n_large;
    uint64_t tile_entries;     // D (may exceed cap on overflow)
    uint32_t tile_entries32;   // min(D, cap): the fine entries written
    uint32_t key_min, key_max; // over visible particles
    uint32_t sorted_buf;       // ping-pong buffer holding the ordered visible list
    uint64_t super_entries;    // entries (particle, super-tile) (may exceed cap on overflow)
    uint32_t super32;          // min(super_entries, cap)
    uint32_t n_units;
    uint32_t n_species;
    uint32_t mode;
    uint32_t series_only;      // every species with particles has A <= kSeriesMaxA
    uint32_t boxes_kept;       // the transform stored every particle's pixel box
    uint32_t check_line;       // checked builds: source line of the first failed index check (0: none)
    uint32_t range_lo_enc[SPLOTCH_MAX_SPECIES];   // order-preserving encodings for atomic min/max
    uint32_t range_hi_enc[SPLOTCH_MAX_SPECIES];
    float lo[SPLOTCH_MAX_SPECIES], hi[SPLOTCH_MAX_SPECIES];
    float inv_span[SPLOTCH_MAX_SPECIES];     // 1 / (hi - lo) (0 when hi <= lo)
    uint32_t vlo_enc[SPLOTCH_MAX_SPECIES][3], vhi_enc[SPLOTCH_MAX_SPECIES][3];   // vector components
    uint32_t qlo_enc[SPLOTCH_MAX_SPECIES], qhi_enc[SPLOTCH_MAX_SPECIES];         // modulating scalar
    float vlo[SPLOTCH_MAX_SPECIES][3], vhi[SPLOTCH_MAX_SPECIES][3], qmax[SPLOTCH_MAX_SPECIES];
    float eoa_max[3];          // per channel, an upper bound of |E_c| / A over the particles (inf if some A = 0 emits)
    Layout layout;
};

constexpr uint64_t kHeaderBytes = 4096;

// Index checks of the checked build (-DSPLOTCH_DEVICE_CHECKS): a failed check
// records its source line and SPLOTCH_ERR_STATE in the header and the caller
// skips the access (no trap).  In the release build the condition is not
// evaluated and the check is always true.
#ifdef __CUDACC__
__device__ __forceinline__ bool device_check(const Header *hdr, bool ok, int line) {
    if (!ok) {
        Header *h = const_cast<Header *>(hdr);
        atomicCAS(&h->check_line, 0u, (uint32_t)line);
        atomicExch(&h->status, (int)SPLOTCH_ERR_STATE);
    }
    return ok;
}
#ifdef SPLOTCH_DEVICE_CHECKS
#define SPL_CHECK(hdr, cond) (::spl::device_check((hdr), (cond), __LINE__))
#else
#define SPL_CHECK(hdr, cond) (true)
#endif
#endif

// Absorption up to which the renderer takes a layer's source and transmission
// from a series in A g instead of an exponential.
constexpr float kSeriesMaxA = 0.125f;
static_assert(sizeof(Header) <= kHeaderBytes, "header too large");

// Transform parameters in the form the kernels use (host computes once).
struct TransformArgs {
    const float *x, *y, *z, *h;
    uint64_t n;
    double fwd0, fwd1, fwd2, c_fwd, znear;
    float r0, r1, r2, cr, u0, u1, u2, cu;
    float s, half_w, half_h, w_max, h_max;
    float sigma_per_h, trunc_f;
    int slab;                  // keep only slab_lo <= key < slab_hi
    uint32_t slab_lo, slab_hi;
    uint32_t *tbox;            // packed tile boxes (nullptr: the tile counts do not fit 8 bits)
    int tshift;                // log2(tile side)
};

struct ColorizeArgs {
    const void *v;
    const void *vec[3];        // vector components (species with use_vector)
    const void *q;             // modulating scalar (species with modulate)
    int dtype;
    uint64_t n;
    int n_species;
    uint64_t begin[SPLOTCH_MAX_SPECIES + 1];
    splotch_species sp[SPLOTCH_MAX_SPECIES];
    const float *palette;
    int n_entries;
};

// One radix pass: digit = ((key - kmin) >> shift) & mask.
struct RadixPass {
    const uint32_t *key_in;
    const uint32_t *val_in;    // nullptr: value = item index (first pass over particles)
    uint32_t *key_out, *val_out;
    const uint32_t *n_dev;     // device item count (nullptr: n_host)
    uint32_t n_host;
    uint32_t shift, mask;
    int depth_pass;            // >= 0: pass index of the depth sort (kmin from header, skip test); -1: plain
    int skip_invalid;          // drop kInvalidKey items (first pass over particles)
    uint32_t ctas;             // grid size of upsweep/downsweep
    uint32_t *hist;            // [256][ctas] (row stride hist_ctas)
    uint32_t hist_stride;
    uint32_t *htot;            // [256]
    Header *hdr;
    // Optional payload carried with each item (nullptr pay_out: none); the
    // first pass over particles reads it in index order, like the keys.
    const uint32_t *pay_in;
    uint32_t *pay_out;
};

// Emission of (super-tile, particle) entries in render order.
// A (super-tile, particle) entry key: the super-tile id in the low kSidBits
// bits (the only bits the grouping pass sorts on) and, above them, the
// particle's rectangle of fine tiles inside that super-tile (c0, c1, r0, r1,
// 3 bits each), so the fine expansion needs no gather of the particle's box.
constexpr int kSidBits = 20;
constexpr uint32_t kSidMask = (1u << kSidBits) - 1u;

struct BinArgs {
    Header *hdr;
    const uint32_t *list[2];   // ordered visible list candidates (sorted_buf selects)
    const ushort4 *box;
    ushort4 *sbox;             // tile-level box per ordered position (written by the reduce, read by the emission)
    const uint32_t *tbox;      // packed tile boxes per particle (index order), or nullptr
    uint32_t *psbox;           // packed tile box per ordered position (the sbox section), when tbox is used
    const uint32_t *pk[2];     // packed tile boxes in render order read by the emission (sorted_buf selects)
    int tshift;                // log2(tile side)
    uint64_t *part;            // per-CTA partial sums
    uint32_t ctas;
    uint32_t *ek, *ev;         // emitted entries (super-tile id, particle)
    uint64_t cap;
    int nsx;                   // super-tile columns
    uint32_t large_tiles;      // particles touching more super-tiles than this have their entries dealt over the CTA
};

// Expansion of super-tile lists into fine-tile lists (64 fine tiles per super-tile).
constexpr int kSuperSide = 8;      // fine tiles per super-tile side
constexpr int kUnit = 2048;        // super-tile entries per unit of work
struct FineArgs {
    Header *hdr;
    const uint32_t *skey, *sval;   // super-tile sorted entries
    const uint32_t *soff;          // super-tile offsets
    uint32_t *ufirst;              // first unit of each super-tile (nsuper + 1)
    uint4 *units;                  // (super-tile, begin, end, 0)
    uint32_t *ucnt;                // [unit][64]
    uint32_t *toff;                // fine-tile offsets (ntiles + 1)
    uint32_t *list;                // fine-tile lists
    uint32_t *torder;              // render order of the tiles (ntiles)
    uint64_t cap;
    uint32_t nsuper, nsx, ntx, nty, ntiles, max_units;
};

struct RenderArgs {
    const Header *hdr;
    const uint32_t *toff;      // ntiles + 1
    const uint32_t *torder;    // ntiles: tiles in render order (a permutation)
    const uint32_t *list;      // tile-sorted particle indices
    const float4 *geo;         // sx, sy, r2, -log2(e)/sigma_pix^2
    const float4 *col;         // Er, Eg, Eb, A
    float *image;
    float *trans;              // partial render: transmittance per pixel and channel (nullptr: none)
    float cutoff;              // absorptive early termination bound (0: off)
    int width, height, tile, ntx, mode, batch;
};

// Render of many frames in one persistent launch: per frame its render
// arguments and the index of its first (frame, tile) task.
constexpr int kMaxBatchItems = 128;
struct BatchItemArgs {
    RenderArgs args;
    uint32_t task_begin;
    uint32_t pad;
};
struct BatchArgs {
    unsigned int *counter;     // task counter (zeroed before the launch)
    int n_items;
    uint32_t n_tasks;
    BatchItemArgs item[kMaxBatchItems];
};

// Layout of a workspace for n particles with this camera/params.
int compute_layout(uint64_t n, int width, int height, int tile, uint64_t cap, Layout *out);

inline Header *header(void *ws) { return reinterpret_cast<Header *>(ws); }
template <class T> inline T *at(void *ws, uint64_t off) {
    return reinterpret_cast<T *>(static_cast<char *>(ws) + off);
}

// Kernel launches made by this library (a process-wide counter).
void count_launches(uint64_t k);

// Launchers (each returns cudaGetLastError()).
cudaError_t launch_init_header(void *ws, const Layout &L, int n_species, int mode, bool boxes_kept, cudaStream_t st);
cudaError_t launch_transform(const TransformArgs &a, void *ws, const Layout &L, bool keep_boxes, cudaStream_t st);
cudaError_t launch_colorize(const ColorizeArgs &a, void *ws, const Layout &L, cudaStream_t st);
// Tile boxes fit 32 bits (8 bits per edge) when both tile counts are at most 256.
inline bool tile_box_packs(const Layout &L) { return L.ntx <= 256 && L.nty <= 256; }

// L2 cache size of the current device (bytes).
uint64_t device_l2_bytes();

// Whether the depth sort carries each visible particle's tile box for the
// binning (the packed 32-bit form).  It replaces binning's one random gather (the box of each
// particle in render order) by sequential reads, at the price of a third
// array in every sort pass; that pays only when the boxes (8 B per particle)
// do not stay in L2.
// The environment variable SPLOTCH_TILE_PAYLOAD=1 (or 0) forces the choice
// where the tile counts allow it (both paths give the same lists; tests use
// it to cover both at small sizes).
int tile_payload_override();   // -1: automatic, 0 or 1: forced
inline bool tile_payload(const Layout &L) {
    if (!tile_box_packs(L)) return false;
    const int o = tile_payload_override();
    return o >= 0 ? o == 1 : L.n * 8 > device_l2_bytes();
}
cudaError_t launch_sort(void *ws, const Layout &L, int mode, cudaStream_t st);
cudaError_t launch_radix_pass(const RadixPass &p, cudaStream_t st);
cudaError_t launch_sort_finish(Header *hdr, cudaStream_t st);   // absorptive ordering of a depth sort
cudaError_t launch_bin(void *ws, const Layout &L, uint32_t large_tiles, cudaStream_t st);
int super_passes(uint32_t nsuper);             // radix passes that group entries by super-tile
uint64_t fine_list_offset(const Layout &L);    // workspace offset of the fine-tile lists
cudaError_t launch_render(void *ws, const Layout &L, int mode, int batch, float *image, float *trans, float cutoff,
                          int staging, cudaStream_t st);
cudaError_t launch_compose(const float *cf, const float *tf, const float *cb, const float *tb, float *co, float *to,
                           uint64_t n, cudaStream_t st);
cudaError_t launch_count_fragments(void *ws, const Layout &L, uint64_t *out, cudaStream_t st);
RenderArgs make_render_args(void *ws, const Layout &L, int mode, int batch, float *image, float *trans = nullptr,
                            float cutoff = 0.0f);
cudaError_t launch_render_batch(const BatchArgs &b, int tile, int batch, cudaStream_t st);
uint32_t roi_ctas(uint64_t n);
cudaError_t launch_roi(const splotch_particles *p, const double box[6], void *scratch, uint64_t *count, float *ox,
                       float *oy, float *oz, float *oh, void *ov, uint64_t capacity, bool scatter, cudaStream_t st);

}  // namespace spl
