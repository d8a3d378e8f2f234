/*
 * splotch.h -- C ABI of the GB300 Splotch per-frame rendering path.
 *
 * The method is the particle renderer of Jin et al., "High-performance
 * astrophysical visualization using Splotch" (ICCS 2010): every particle is a
 * Gaussian density cut at f sigma (Section 2, first item), colour comes from
 * a scalar through a palette (Section 2, third item), and the intensity along
 * each line of sight obeys the transfer equation dI/dx = (E_p - A_p I) rho_p
 * (Section 2, Eq. 1) for red, green and blue independently (Section 2,
 * second item).  A frame is "process" (normalisation) then "display"
 * (transform, colour, render) (Section 3.2).
 *
 * Conventions that the paper leaves open (camera model, pixel centres, the
 * single-precision geometry that decides which pixels a particle reaches,
 * normalisation, palette interpolation, ordering) are stated next to the
 * call that applies them.
 *
 * Memory and streams.  Every pointer marked "device" is CUDA device memory
 * owned by the caller; the library never allocates, frees or keeps a pointer
 * beyond the call (the workspace is caller-owned too).  Inputs are read only.
 * Every call that takes `stream` (a cudaStream_t passed as void*, NULL = the
 * legacy default stream) only enqueues work and returns; results are ready
 * when the stream reaches that point.  Calls return SPLOTCH_OK or a negative
 * status; argument errors are reported before anything is enqueued.  Errors
 * found on the device (for example a tile-entry capacity overflow) are
 * written to a status word inside the workspace and reported by
 * splotch_frame_info.  No call aborts, traps or throws.
 *
 * The kernels of a frame are launched with programmatic stream
 * serialization (programmatic dependent launch): a kernel may be scheduled
 * while the one before it on the stream drains, but waits for it to complete
 * before it touches memory, so stream order holds for the caller's own work
 * before and after these calls.
 */
#ifndef SPLOTCH_H
#define SPLOTCH_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define SPLOTCH_ABI_VERSION 4
#define SPLOTCH_MAX_SPECIES 8
#define SPLOTCH_MAX_PALETTE 256

typedef enum {
    SPLOTCH_OK = 0,
    SPLOTCH_ERR_ARG = -1,         /* invalid argument, detected on the host */
    SPLOTCH_ERR_CUDA = -2,        /* a CUDA runtime call failed */
    SPLOTCH_ERR_WORKSPACE = -3,   /* workspace too small (on the host) or tile entries over capacity (device) */
    SPLOTCH_ERR_TIMEOUT = -4,     /* a bounded device wait ran out */
    SPLOTCH_ERR_OOM_ADMISSION = -5,
    SPLOTCH_ERR_STATE = -6,       /* workspace does not hold the step this call needs */
    SPLOTCH_ERR_IO = -7           /* a file could not be opened or read (short file, I/O error) */
} splotch_status;

typedef enum { SPLOTCH_F32 = 0, SPLOTCH_F16 = 1, SPLOTCH_BF16 = 2 } splotch_dtype;

/* SPLOTCH_EMISSION: A = 0, I = sum_p E_p g_p, order-independent.
 * SPLOTCH_ABSORPTIVE: Eq. 1 with per-species scalar A, front to back over
 *   particles sorted by depth (ascending key, ties by ascending index).
 * SPLOTCH_E_EQ_A: the paper's E = A setting (Section 2): I = 1 - exp(-sum_p E_p g_p). */
typedef enum { SPLOTCH_EMISSION = 0, SPLOTCH_ABSORPTIVE = 1, SPLOTCH_E_EQ_A = 2 } splotch_mode;

/* Particle block in structure-of-arrays form, one array per property, as in
 * the block file layout of Section 3.1.  Species are contiguous index ranges
 * [species_begin[s], species_begin[s+1]).  The vector quantity and the
 * modulating scalar (Section 2, third item) are optional: NULL when no
 * species uses them. */
typedef struct {
    uint64_t n;                 /* number of particles, < 2^32 */
    const float *x, *y, *z;     /* device, n each: world position */
    const float *h;             /* device, n: smoothing length */
    const void *intensity;      /* device, n values of intensity_dtype: the scalar mapped to colour */
    int32_t intensity_dtype;    /* splotch_dtype, also the type of vector[] and modulator */
    int32_t n_species;          /* 1..SPLOTCH_MAX_SPECIES */
    uint64_t species_begin[SPLOTCH_MAX_SPECIES + 1];  /* host values; begin[0] = 0, begin[n_species] = n */
    const void *vector[3];      /* device, n values each, or NULL: components of a vector quantity
                                   (for example velocity) for species with use_vector */
    const void *modulator;      /* device, n values, or NULL: scalar q (for example density) for
                                   species with modulate */
} splotch_particles;

/* Perspective camera.  The caller fills eye, target, up, fov_x_deg (full
 * horizontal angle), width, height, znear; splotch_camera_init fills the rest. */
typedef struct {
    double eye[3], target[3], up[3];
    double fov_x_deg;
    int32_t width, height;
    double znear;
    double right[3], upv[3], fwd[3];   /* derived: right = up x fwd, upv = fwd x right */
    double scale;                      /* derived: (width/2) / tan(fov/2), px per unit at unit depth */
    double c_right, c_up, c_fwd;       /* derived: eye . right, eye . upv, eye . fwd */
} splotch_camera;

/* Palette: n_entries rgb triples (device, float, n_entries x 3), 2..256 entries. */
typedef struct {
    int32_t n_entries;
    const float *rgb;
} splotch_colormap;

/* Render settings of one species (Section 2: E and A per particle, colour
 * through a palette or fixed). */
typedef struct {
    int32_t use_log;         /* normalise log10(max(v, 1e-37)) instead of v */
    int32_t use_colormap;    /* 1: palette(t); 0: fixed_rgb */
    float lo, hi;            /* normalisation range; NaN = min/max over the species (computed on the device) */
    float brightness;        /* E = brightness * colour */
    float absorption;        /* A = absorption * (1, 1, 1); 0 = pure emission */
    float fixed_rgb[3];
    int32_t use_vector;      /* 1: E_c = brightness * t_c, t_c = clamp((v_c - lo_c)/(hi_c - lo_c), 0, 1),
                                lo_c/hi_c = min/max of component c over the species (a vector quantity
                                mapped to red, green and blue, Section 2, third item); overrides use_colormap */
    int32_t modulate;        /* 1: the particle's column density, and so E and A, scaled by
                                m = clamp(q / q_max, 0, 1), q_max = max of q over the species
                                (m = 0 if q_max <= 0): optical depth proportional to q (Section 2, third item) */
} splotch_species;

typedef struct {
    int32_t mode;                 /* splotch_mode */
    int32_t tile;                 /* screen tile side in px: 8, 16 or 32 */
    float sigma_per_h;            /* sigma = sigma_per_h * h (default 1) */
    float trunc_f;                /* footprint cut at f sigma (default 2) */
    int32_t batch;                /* particles staged per renderer batch: 64, 128 or 256 */
    int32_t large_threshold_px;   /* footprint area (px) above which a particle's tile entries are
                                     emitted cooperatively; 0 = (width + height) / 2 (Section 3.2) */
    uint64_t max_tile_entries;    /* capacity of the tile-entry arrays in the workspace, < 2^32 */
    int32_t slab;                 /* 1: the transform keeps only the depth slab slab_key_lo <= key < slab_key_hi
                                     (key = bit pattern of (float)Z, so the bounds are depths); every
                                     other particle is culled.  The normalisation range still covers
                                     every particle of a species.  0: no slab */
    uint32_t slab_key_lo, slab_key_hi;
    float t_min_cutoff;           /* absorptive early termination, 0 = off (the default; results are then
                                     bit-for-bit those of the full integral).  > 0: a warp's pixels stop
                                     taking particles once, for every channel c, T_max * M_c <=
                                     t_min_cutoff * C_max,c, with T_max the largest transmittance of its
                                     pixels, C_max,c the largest intensity they have reached and M_c the
                                     largest E_c / A of any species (the light still to come through a
                                     pixel is at most T * M_c, Eq. 1 integrated over the remaining
                                     layers).  Never stops while a species with A = 0 emits.  Changes
                                     each channel by at most t_min_cutoff times its image maximum */
    int32_t staging;              /* how the renderer stages a batch of a tile's list in shared memory:
                                     0 (default): every thread loads its entries' records through registers;
                                     1: cp.async.bulk.tensor tile::gather4 copies (TMA) land them directly,
                                     for tiles of 16 and 32 px in the plain render (8-px tiles, partial
                                     images and early termination load through registers).  The image is
                                     the same bit for bit either way */
    int32_t keep_pixel_boxes;     /* 1: the transform also stores every particle's pixel box (8 B each)
                                     for splotch_get_keys.  0 (default): it stores them only when binning
                                     reads them (more than 256 tiles in a row or column); otherwise
                                     binning reads the packed tile boxes, the pass writes 8 B less per
                                     particle, and a box request to splotch_get_keys is refused with
                                     SPLOTCH_ERR_STATE.  Nothing else depends on it */
} splotch_render_params;

/* Result summary read back by splotch_frame_info (synchronises the stream). */
typedef struct {
    int32_t status;               /* device-side status (splotch_status) */
    uint32_t visible;             /* V: particles that reach the image */
    uint64_t tile_entries;        /* D: sum over visible particles of tiles touched (after a capacity
                                     overflow: a lower bound to grow max_tile_entries to) */
    uint32_t large;               /* particles sent to the cooperative emission path */
    uint32_t ntiles;
    float lo[SPLOTCH_MAX_SPECIES], hi[SPLOTCH_MAX_SPECIES];   /* normalisation range used */
    uint32_t check_line;          /* library built with device index checks: source line of the first
                                     failed check (status then SPLOTCH_ERR_STATE); 0 otherwise */
} splotch_frame_info_t;

/* Library ABI version (SPLOTCH_ABI_VERSION). */
int splotch_abi_version(void);

/* Text for a status code; never NULL. */
const char *splotch_status_string(int status);

/*
 * Fill the derived camera fields on the host in double precision.
 * forward = normalize(target - eye), right = normalize(up x forward),
 * upv = forward x right (right-handed, +y up on screen), scale =
 * (width/2)/tan(fov_x/2).  Camera coordinates of p are X = p.right - c_right,
 * Y = p.upv - c_up, Z = p.fwd - c_fwd.  SPLOTCH_ERR_ARG when target == eye,
 * up is parallel to the view, fov is not in (0, 180), or a size is < 1.
 */
int splotch_camera_init(splotch_camera *cam);

/*
 * Bytes of workspace for up to n particles with this camera and parameters
 * (tile size and max_tile_entries matter).  The workspace must be 256-byte
 * aligned device memory.  One workspace serves one frame at a time.
 */
int splotch_workspace_size(uint64_t n, const splotch_camera *cam, const splotch_render_params *params,
                           size_t *bytes);

/*
 * Transform (Section 3.2, "transformation into screen coordinates";
 * footprint of Section 2, first item).  Per particle, in this order, each
 * operation rounded separately:
 *   Z  = fma(z, fwd2, fma(y, fwd1, x * fwd0)) - c_fwd          in double;
 *        culled when Z <= znear; depth key = bit pattern of (float)Z
 *   X  = fmaf(z, r2, fmaf(y, r1, x * r0)) - (float)c_right      in float (basis rounded to float), Y likewise
 *   inv = 1 / (float)Z;  sx = W/2 + (s * X) * inv;  sy = H/2 - (s * Y) * inv    (s = (float)scale)
 *   sigma_pix = (s * (sigma_per_h * h)) * inv;  r = trunc_f * sigma_pix;  r2 = r * r
 *   box x0 = max(0, ceil(((sx - r) - 0.5) - 1/64)), x1 = min(W - 1, floor(((sx + r) - 0.5) + 1/64)),
 *       y likewise; culled when empty (no pixel centre within reach) or not finite
 * Pixel (i, j) (centre (i + 0.5, j + 0.5), row 0 on top) receives the
 * particle iff fmaf(dy, dy, dx * dx) < r2 with dx = (i + 0.5f) - sx,
 * dy = (j + 0.5f) - sy; such a pixel always lies in the box.
 * Writes the per-particle record, key and box into the workspace.
 */
int splotch_transform(const splotch_particles *p, const splotch_camera *cam, const splotch_render_params *params,
                      void *workspace, size_t workspace_bytes, void *stream);

/*
 * Normalise and colour (Section 3.2 "normalizing of some
 * particle values"; Section 2 colour look-up table).  species[s] applies to
 * range s of p.  Per species, u = log10(max(v, 1e-37)) (use_log) or v;
 * [lo, hi] = the given range, or min/max of u over every particle of the
 * species when lo or hi is NaN; t = clamp((u - lo)/(hi - lo), 0, 1) (0 when
 * hi == lo); palette value by linear interpolation, w = t (K - 1),
 * k = min(floor(w), K - 2); E = brightness * colour (or * fixed_rgb),
 * A = absorption.  A species with use_vector takes E from the three
 * components of p->vector instead, each normalised linearly over the
 * species; one with modulate scales E and A by q / q_max of the species
 * (p->modulator).  Half-precision values are widened to float exactly.
 * Errors: SPLOTCH_ERR_ARG when a species asks for a vector or modulator
 * array that p does not provide.
 */
int splotch_colorize(const splotch_particles *p, const splotch_species *species, const splotch_colormap *cmap,
                     void *workspace, size_t workspace_bytes, void *stream);

/*
 * Depth sort, tile binning and tile render into image
 * (device, float, height x width x 3, row 0 on top).  Absorptive mode sorts
 * visible particles by ascending key, ties by ascending index (a stable LSD
 * radix sort); the other modes keep index order.  Binning lists, for every
 * tile (row-major), the particles whose box meets it, in that order
 * (bit-exact).  The render integrates Eq. 1 per pixel over its tile's list
 * with g = exp(-d^2 / sigma_pix^2): emission sum E g; absorptive front to
 * back C += T S, T *= exp(-A g), S = E (1 - exp(-A g)) / A (E g when A = 0);
 * E = A: 1 - exp(-sum E g).  Background 0.  The same params as the
 * transform call, and its particle count n, must be given.  Runs
 * splotch_sort, splotch_bin and splotch_render_tiles in order.
 */
int splotch_render(const splotch_render_params *params, const splotch_camera *cam, uint64_t n, void *workspace,
                   size_t workspace_bytes, float *image, void *stream);

/* The three parts of splotch_render, callable one by one (same arguments).
 * splotch_bin also records the order in which splotch_render_tiles starts
 * the tiles (longest lists first); it changes when a tile is rendered, never
 * the image.  splotch_render_tiles needs a workspace that splotch_bin has
 * processed for this frame. */
int splotch_sort(const splotch_render_params *params, const splotch_camera *cam, uint64_t n, void *workspace,
                 size_t workspace_bytes, void *stream);
int splotch_bin(const splotch_render_params *params, const splotch_camera *cam, uint64_t n, void *workspace,
                size_t workspace_bytes, void *stream);
int splotch_render_tiles(const splotch_render_params *params, const splotch_camera *cam, uint64_t n,
                         void *workspace, size_t workspace_bytes, float *image, void *stream);

/*
 * Partial image of a depth slab, for depth-sharded rendering (the reduction
 * of partial images of Section 3.1, generalised to E != A by Eq. 1).  Light
 * entering the rendered particles from behind leaves them as C + T I_in per
 * pixel and channel: `color` receives C (the front-to-back render with a
 * background of 0, as splotch_render_tiles writes it, except in E = A mode)
 * and `trans` receives T (device, height x width x 3 floats each):
 *   absorptive  T = prod_p exp(-A_p g_p) (the same in every channel)
 *   emission    T = 1
 *   E = A       C = 1 - exp(-tau), T = exp(-tau), tau = sum_p E_p g_p per channel
 * Slabs rendered from the same set with params.slab and consecutive key
 * ranges combine, nearest first, with splotch_compose into the image of the
 * whole set.  Runs splotch_sort, splotch_bin and the tile render.
 */
int splotch_render_partial(const splotch_render_params *params, const splotch_camera *cam, uint64_t n,
                           void *workspace, size_t workspace_bytes, float *color, float *trans, void *stream);

/*
 * Ordered composition of two partial images, `front` nearer the camera:
 *   c_out = c_front + t_front * c_back,  t_out = t_front * t_back
 * element by element over n_values floats (height x width x 3 for an
 * image), each product rounded once, then the sum (no fused multiply-add).
 * The operator is associative, not commutative: fold slabs in depth order.
 * All pointers are device floats; c_out and t_out may each be the same array
 * as an input (not a partial overlap); t_out may be NULL when only the
 * colour is wanted (the last fold).  Pointers must be
 * 16-byte aligned.  SPLOTCH_ERR_ARG for NULL or misaligned pointers.
 */
int splotch_compose(const float *c_front, const float *t_front, const float *c_back, const float *t_back,
                    float *c_out, float *t_out, uint64_t n_values, void *stream);

/* Synchronises `stream` and reads the frame summary from the workspace
 * (written by the last transform/colorize/render on it). */
int splotch_frame_info(const void *workspace, size_t workspace_bytes, splotch_frame_info_t *info, void *stream);

/*
 * Test access.  Each call synchronises `stream`, reads the workspace layout
 * recorded by splotch_transform, then enqueues device-to-device copies.
 * splotch_get_keys: key (n x uint32, 0xFFFFFFFF when culled) and box
 *   (n x 4 int32: x0, y0, x1, y1; 0, 0, -1, -1 when culled); either may be NULL.
 *   A box request after a transform that did not store the pixel boxes
 *   (splotch_render_params.keep_pixel_boxes) returns SPLOTCH_ERR_STATE.
 * splotch_get_geometry: sx, sy, r2 (n floats each; 0 when culled); any may be NULL.
 * splotch_get_order: the V visible particle indices in render order.
 * splotch_get_tile_lists: offsets (ntiles + 1 uint32) and list (capacity
 *   uint32, first D used); SPLOTCH_ERR_WORKSPACE when capacity < D (read D first).
 * splotch_get_colors: E and A (n x 4 floats: Er, Eg, Eb, A).
 */
int splotch_get_keys(const void *workspace, size_t workspace_bytes, uint32_t *key, int32_t *box, void *stream);
int splotch_get_geometry(const void *workspace, size_t workspace_bytes, float *sx, float *sy, float *r2,
                         void *stream);
int splotch_get_order(const void *workspace, size_t workspace_bytes, uint32_t *order, void *stream);
int splotch_get_tile_lists(const void *workspace, size_t workspace_bytes, uint32_t *offsets, uint32_t *list,
                           uint64_t capacity, void *stream);
int splotch_get_colors(const void *workspace, size_t workspace_bytes, float *ea, void *stream);

/*
 * One frame of a batch render: a workspace that has been through
 * splotch_transform, splotch_colorize, splotch_sort and splotch_bin for n
 * particles with this camera, mode, max_tile_entries and the batch's tile
 * size, and the frame's image (device, height x width x 3 floats).
 */
typedef struct {
    uint64_t n;
    const splotch_camera *camera;   /* host */
    int32_t mode;                   /* splotch_mode of this frame */
    int32_t reserved;
    uint64_t max_tile_entries;
    void *workspace;
    size_t workspace_bytes;
    float *image;
} splotch_batch_item;

#define SPLOTCH_MAX_BATCH 128

/*
 * Tile render of up to SPLOTCH_MAX_BATCH frames (views of one particle set,
 * or independent snapshots) in one persistent launch: as many CTAs as fit on
 * the GPU take (frame, tile) tasks from `counter` (device, one uint32 owned
 * by the caller; zeroed by this call on `stream`), larger frames first.  Each
 * frame's image equals what splotch_render_tiles gives for it with
 * register staging, no early termination and no partial image (the batch
 * items carry no such settings).  The frames' workspaces must be distinct.  Makes no allocation and no host
 * synchronisation, so a sequence of these calls can be captured in a CUDA
 * graph.  SPLOTCH_ERR_ARG for a bad item, a tile size other than 8, 16 or
 * 32, or more than SPLOTCH_MAX_BATCH items.
 */
int splotch_render_tiles_batch(const splotch_batch_item *items, int32_t n_items, int32_t tile, int32_t batch,
                               uint32_t *counter, void *stream);

/*
 * Region-of-interest cut of a resident particle set (serving): the particles
 * of `src` inside the box {x_lo, y_lo, z_lo, x_hi, y_hi, z_hi}, i.e. with
 * lo <= p < hi on every axis (compared in single precision, bounds rounded
 * to float), copied in index order.  Only x, y, z, h and the intensity are
 * copied; species ranges of `src` are not tracked (cut one range at a time).
 * scratch: device, at least splotch_roi_scratch_size bytes, caller-owned.
 * splotch_roi_count writes the number of particles inside to *count (device
 * uint64).  splotch_roi_select also writes the first min(count, capacity)
 * of them to x, y, z, h (device floats) and intensity (device, src's dtype).
 * Both are asynchronous on `stream` and allocate nothing.
 */
int splotch_roi_scratch_size(uint64_t n, size_t *bytes);
int splotch_roi_count(const splotch_particles *src, const double box[6], void *scratch, size_t scratch_bytes,
                      uint64_t *count, void *stream);
int splotch_roi_select(const splotch_particles *src, const double box[6], void *scratch, size_t scratch_bytes,
                       float *x, float *y, float *z, float *h, void *intensity, uint64_t capacity, uint64_t *count,
                       void *stream);

/*
 * Measurement helpers.
 * splotch_count_fragments: enqueues a count, over the visible particles of
 *   the last transform, of the (pixel, particle) pairs that pass the
 *   membership test of splotch_transform (the fragments F of the frame);
 *   writes one uint64 to `out` (device).  Not part of a frame.
 * splotch_launch_count: kernels this library has launched in this process.
 */
int splotch_count_fragments(const splotch_render_params *params, const splotch_camera *cam, uint64_t n,
                            void *workspace, size_t workspace_bytes, uint64_t *out, void *stream);
uint64_t splotch_launch_count(void);

/*
 * Depth sort without any device allocation, for callers that cannot call
 * cudaMalloc while they run (for example a renderer embedded in a host
 * application that owns all device memory through its own fixed pool, or a
 * real-time loop where an allocation, which can synchronise the device, is
 * not allowed after start-up).  The paper has no counterpart: it is a
 * deployment convenience of this library.
 *
 * key: device, n depth keys as splotch_transform writes them (0xFFFFFFFF for
 * a culled particle), 16-byte aligned (the keys are read four at a time).
 * order: device, room for n uint32; receives the indices of the non-culled
 * keys in ascending key order, ties by ascending index (the order
 * splotch_sort gives).  count: device, one uint32, receives how many indices
 * were written (0xFFFFFFFF, and no order, if a library built with device
 * index checks found a failed check).  The caller owns all three buffers.
 *
 * The sort's scratch is a fixed array inside the library (about 4.3 MB on
 * every GPU that loads it, held until the process exits); no call allocates
 * or frees memory.  n above SPLOTCH_NO_ALLOC_MAX_KEYS, a key pointer that is
 * not 16-byte aligned or an order/count pointer that is not 4-byte aligned
 * returns SPLOTCH_ERR_ARG without enqueuing anything.  Every call looks up
 * the array's device address on the current device; the first call on a
 * device can load the library's device code there, so make it before
 * capturing a stream.  All calls share the one array and it keeps the last
 * call's contents, so calls whose work overlaps on the GPU (different
 * streams, or different host threads on one device) race and must be
 * serialised by the caller.  Asynchronous on `stream` like the other calls.
 */
#define SPLOTCH_NO_ALLOC_MAX_KEYS (1u << 18)
int splotch_sort_keys_no_alloc(const uint32_t *key, uint32_t n, uint32_t *order, uint32_t *count, void *stream);

/*
 * Block-structured particle files (Section 3.1, MPI implementation): a file
 * holds n_blocks contiguous blocks, one per particle property, each of
 * n_particles 32-bit floats; seen as a 2-D array A of n_blocks x n_particles
 * floats (row-major), block b, particle i is at byte
 * offset + 4 (b n_particles + i).  A reader takes the same slice
 * [first, first + count) of each block it needs (the n x N/nprocs subarray
 * of a process), converting the byte order when the file's differs from the
 * host's.  Host-side I/O: these calls are the "read" stage of Section 3,
 * outside the rendering path.
 */
typedef struct {
    const char *path;          /* host, NUL-terminated */
    uint64_t offset;           /* byte offset of block 0 in the file */
    int32_t n_blocks;          /* n: properties per particle */
    int32_t big_endian;        /* 1: the file stores big-endian floats; 0: little-endian */
    uint64_t n_particles;      /* N: floats per block */
} splotch_block_file;

/* Read particles [first, first + count) of block `block` into host memory
 * (count floats, caller-owned, any alignment), in host byte order.
 * Synchronous.  Errors: SPLOTCH_ERR_ARG (block or range outside the file
 * description, NULL pointers), SPLOTCH_ERR_IO (open/read failure, file
 * shorter than the description). */
int splotch_block_read(const splotch_block_file *file, int32_t block, uint64_t first, uint64_t count, float *dst);

/* Loader: reads block slices on host threads of its own, each into two
 * pinned staging buffers (chunk_bytes each, allocated at creation), and
 * enqueues their copies to device arrays on the caller's stream, so a file's
 * read overlaps the copies and whatever else runs on the device (for example
 * the render of the previous snapshot on another stream).  Reader t takes
 * chunks t, t + T, ... of a load.  One load at a time per loader. */
typedef struct splotch_loader splotch_loader;

/* Create a loader on the current CUDA device with n_threads readers (1..64).
 * chunk_bytes: multiple of 4, at least 4096.  Errors: SPLOTCH_ERR_ARG,
 * SPLOTCH_ERR_CUDA (pinned allocation failed). */
int splotch_loader_create(size_t chunk_bytes, int32_t n_threads, splotch_loader **out);

/* Start loading: for d < n_dst, particles [first, first + count) of block
 * blocks[d] go to device array dst[d] (count floats each, device memory
 * owned by the caller, host byte order).  Returns at once; the copies are
 * ordered on `stream` (a cudaStream_t as void*).  The arrays and `file`'s
 * path must stay valid until splotch_loader_wait returns.  Errors:
 * SPLOTCH_ERR_ARG (bad description or range, a load already running). */
int splotch_loader_start(splotch_loader *loader, const splotch_block_file *file, int32_t n_dst,
                         const int32_t *blocks, uint64_t first, uint64_t count, float *const *dst, void *stream);

/* Wait for the host side of the current load (every chunk read and its copy
 * enqueued) and return its status (SPLOTCH_ERR_IO on a read failure; the
 * arrays are then incomplete).  The device copies complete in stream order.
 * Without a running load, returns the status of the last one. */
int splotch_loader_wait(splotch_loader *loader);

/* Free the staging buffers (waits for a running load first). */
int splotch_loader_destroy(splotch_loader *loader);

#ifdef __cplusplus
}
#endif
#endif /* SPLOTCH_H */
