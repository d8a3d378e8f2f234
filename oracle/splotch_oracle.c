/*
 * FP64 CPU oracle of the Splotch per-frame rendering path.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the CPU
 * baseline leg of the benchmark may load this library.  It shares no code,
 * header or table with the CUDA path.
 *
 * What it computes (Jin et al., "High-performance astrophysical visualization
 * using Splotch", Section 2 and Section 3.2):
 *   - each particle p carries a Gaussian density rho_p(r) = rho_0 exp(-r^2/sigma_p^2)
 *     cut to zero beyond f * sigma_p (Section 2, first item);
 *   - red, green and blue are transported independently (Section 2, second item);
 *   - the intensity along a ray obeys dI/dx = (E_p - A_p I) rho_p(x) (Section 2, Eq. 1);
 *   - E_p comes from a scalar through a colour look-up table, or from the three
 *     components of a vector quantity, and a particle's optical depth may be
 *     scaled by another scalar (Section 2, third item);
 *   - the "process" stage normalises particle values and the "display" stage
 *     transforms to screen coordinates, colours and renders (Section 3.2).
 *
 * The paper leaves the camera, the sigma-h relation, the normalisation, the
 * palette interpolation and the discretisation of Eq. 1 open.  The readings
 * used here (the project's conventions C1-C12) are:
 *   C1  horizontal field of view; scale s = (W/2) / tan(fov/2) pixels per unit at unit depth.
 *   C2  pixel (i, j) has its centre at (i + 1/2, j + 1/2); row 0 is the top.
 *   C3  a particle with camera depth Z <= znear is culled.
 *   C4  sigma = sigma_per_h * h.
 *   C5  each particle is a thin layer at its centre depth with a circular screen
 *       footprint: sigma_pix = s sigma / Z, r_pix = f sigma_pix; along a ray at
 *       screen distance d its column density is g = exp(-d^2 / sigma_pix^2)
 *       (the constant sigma sqrt(pi) of the line-of-sight integral is folded into E and A).
 *   C6  hard cut: the particle reaches pixel (i, j) only if d^2 < r_pix^2,
 *       tested in single precision exactly as written in oracle_geometry and
 *       pixel_weight below.
 *   C7  per species, u = log10(max(v, 1e-37)) (or v), lo/hi = min/max of u over
 *       all particles of the species, t = clamp((u - lo)/(hi - lo), 0, 1), t = 0 if hi == lo.
 *   C8  K-entry palette, linear interpolation: w = t (K - 1), k = min(floor(w), K - 2),
 *       colour = (1 - (w - k)) P[k] + (w - k) P[k + 1].
 *   C9  E = brightness * colour (or brightness * fixed rgb); A = absorption * (1, 1, 1).
 *   C10 absorptive order: ascending depth key, ties by ascending particle index;
 *       emission order: ascending index.
 *   C11 Eq. 1 integrated exactly over each layer with constant E_p, A_p:
 *       T_p = exp(-A_p g), S_p = E_p (1 - T_p) / A_p (E_p g when A_p = 0).
 *       Background intensity 0, linear output.
 *   C12 the single-precision screen geometry, bbox and depth key written in
 *       oracle_geometry (each operation rounded separately; build with
 *       -ffp-contract=off).
 */
#include <math.h>
#ifdef _OPENMP
#include <omp.h>
#endif
#include <stddef.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

enum { OR_EMISSION = 0, OR_ABSORPTIVE = 1, OR_E_EQ_A = 2 };

typedef struct {
    double eye[3], target[3], up[3];
    double fov_x_deg;
    int32_t width, height;
    double znear;
    /* filled by oracle_camera */
    double right[3], upv[3], fwd[3];
    double scale;
    double c_right, c_up, c_fwd;
} ocam;

static void cross3(const double a[3], const double b[3], double o[3])
{
    o[0] = a[1] * b[2] - a[2] * b[1];
    o[1] = a[2] * b[0] - a[0] * b[2];
    o[2] = a[0] * b[1] - a[1] * b[0];
}

static int normalize3(double v[3])
{
    double n = sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
    if (!(n > 0.0)) return -1;
    v[0] /= n; v[1] /= n; v[2] /= n;
    return 0;
}

/* C1-C2: right-handed camera basis (forward, right = up x forward, up' =
 * forward x right) and the screen scale.  The eye's projections on the basis
 * are kept so that camera coordinates are p.basis - eye.basis. */
int oracle_camera(ocam *c)
{
    const double pi = 3.14159265358979323846;
    for (int k = 0; k < 3; ++k) c->fwd[k] = c->target[k] - c->eye[k];
    if (normalize3(c->fwd)) return -1;
    cross3(c->up, c->fwd, c->right);
    if (normalize3(c->right)) return -1;
    cross3(c->fwd, c->right, c->upv);
    if (!(c->fov_x_deg > 0.0 && c->fov_x_deg < 180.0) || c->width <= 0 || c->height <= 0) return -1;
    c->scale = (0.5 * (double)c->width) / tan(0.5 * c->fov_x_deg * pi / 180.0);
    c->c_right = fma(c->eye[2], c->right[2], fma(c->eye[1], c->right[1], c->eye[0] * c->right[0]));
    c->c_up = fma(c->eye[2], c->upv[2], fma(c->eye[1], c->upv[1], c->eye[0] * c->upv[0]));
    c->c_fwd = fma(c->eye[2], c->fwd[2], fma(c->eye[1], c->fwd[1], c->eye[0] * c->fwd[0]));
    return 0;
}

/*
 * C3-C6, C12: per particle screen geometry.
 *   Z    = fma(z, f2, fma(y, f1, x * f0)) - c_fwd           (double; the depth key is bits((float)Z))
 *   X, Y = fmaf(z, b2, fmaf(y, b1, x * b0)) - c_b            (float, basis and c_b rounded to float)
 *   inv  = 1 / (float)Z
 *   sx   = W/2 + (s * X) * inv,  sy = H/2 - (s * Y) * inv
 *   sigma_pix = (s * (sigma_per_h * h)) * inv, r = f * sigma_pix, r2 = r * r
 *   bbox: ceil(((sx - r) - 1/2) - 1/64) .. floor(((sx + r) - 1/2) + 1/64),
 *         clipped to the image; culled when empty (no pixel centre can pass
 *         the cut).  Pixel i passes the C6 test only if its centre lies within
 *         r of sx up to single-precision rounding: fl(dx*dx) <= the fused sum
 *         and both squares are rounded once, so |(i + 1/2) - sx| < r (1 + 2^-22)
 *         roughly; the 1/64 px guard covers that and the rounding of the box
 *         arithmetic itself (a few ulp of values below 2^16), so every pixel
 *         that passes the C6 test lies inside the box.
 * Outputs are per input index; bbox holds x0, y0, x1, y1.
 */
void oracle_geometry(const ocam *c, size_t n, const float *x, const float *y, const float *z, const float *h,
                     float sigma_per_h, float trunc_f,
                     uint32_t *key, uint8_t *visible, float *sx, float *sy, float *sigma_pix, float *r2,
                     int32_t *bbox)
{
    const float s = (float)c->scale;
    const float wh = 0.5f * (float)c->width, hh = 0.5f * (float)c->height;
    const float r0 = (float)c->right[0], r1 = (float)c->right[1], rr2 = (float)c->right[2];
    const float u0 = (float)c->upv[0], u1 = (float)c->upv[1], u2 = (float)c->upv[2];
    const float cr = (float)c->c_right, cu = (float)c->c_up;
    const float wmax = (float)(c->width - 1), hmax = (float)(c->height - 1);
#pragma omp parallel for schedule(static)
    for (long long i = 0; i < (long long)n; ++i) {
        double Z = fma((double)z[i], c->fwd[2], fma((double)y[i], c->fwd[1], (double)x[i] * c->fwd[0])) - c->c_fwd;
        key[i] = 0xFFFFFFFFu;
        visible[i] = 0;
        sx[i] = sy[i] = sigma_pix[i] = r2[i] = 0.0f;
        bbox[4 * i + 0] = bbox[4 * i + 1] = 0;
        bbox[4 * i + 2] = bbox[4 * i + 3] = -1;
        if (!(Z > c->znear))
            continue; /* C3 */
        float Zf = (float)Z;
        float X = fmaf(z[i], rr2, fmaf(y[i], r1, x[i] * r0)) - cr;
        float Y = fmaf(z[i], u2, fmaf(y[i], u1, x[i] * u0)) - cu;
        float inv = 1.0f / Zf;
        float px = wh + (s * X) * inv;
        float py = hh - (s * Y) * inv;
        float sg = (s * (sigma_per_h * h[i])) * inv;
        float r = trunc_f * sg;
        const float G = 0.015625f; /* 1/64 px guard, see the comment above */
        float lx = ceilf(((px - r) - 0.5f) - G), hx = floorf(((px + r) - 0.5f) + G);
        float ly = ceilf(((py - r) - 0.5f) - G), hy = floorf(((py + r) - 0.5f) + G);
        float x0 = lx > 0.0f ? lx : 0.0f, x1 = hx < wmax ? hx : wmax;
        float y0 = ly > 0.0f ? ly : 0.0f, y1 = hy < hmax ? hy : hmax;
        if (!(lx <= hx) || !(ly <= hy) || !(x0 <= x1) || !(y0 <= y1))
            continue; /* off screen (or not finite) */
        uint32_t kb;
        memcpy(&kb, &Zf, sizeof kb);
        key[i] = kb;
        visible[i] = 1;
        sx[i] = px; sy[i] = py; sigma_pix[i] = sg; r2[i] = r * r;
        bbox[4 * i + 0] = (int32_t)x0; bbox[4 * i + 1] = (int32_t)y0;
        bbox[4 * i + 2] = (int32_t)x1; bbox[4 * i + 3] = (int32_t)y1;
    }
}

/* C7 (Section 3.2, "normalizing of some particle values"): lo/hi of the
 * (log10) values of one species.  v holds the values as doubles. */
void oracle_range(size_t n, const double *v, int use_log, double *lo, double *hi)
{
    double a = INFINITY, b = -INFINITY;
    for (size_t i = 0; i < n; ++i) {
        double u = use_log ? log10(v[i] > 1e-37 ? v[i] : 1e-37) : v[i];
        if (u < a) a = u;
        if (u > b) b = u;
    }
    *lo = a;
    *hi = b;
}

/* C7-C9 (Section 2, third item: colour look-up table): emission colour and
 * absorption of the particles of one species.  palette is K x 3 (K >= 2). */
void oracle_colour(size_t n, const double *v, int use_log, double lo, double hi,
                   double brightness, double absorption, int use_colormap, const double fixed_rgb[3],
                   int n_entries, const double *palette, double *E, double *A)
{
    for (size_t i = 0; i < n; ++i) {
        double rgb[3];
        if (use_colormap) {
            double u = use_log ? log10(v[i] > 1e-37 ? v[i] : 1e-37) : v[i];
            double t = hi > lo ? (u - lo) / (hi - lo) : 0.0;
            t = t < 0.0 ? 0.0 : (t > 1.0 ? 1.0 : t);
            double w = t * (double)(n_entries - 1);
            int k = (int)floor(w);
            if (k > n_entries - 2) k = n_entries - 2;
            double fr = w - (double)k;
            for (int c = 0; c < 3; ++c)
                rgb[c] = (1.0 - fr) * palette[3 * k + c] + fr * palette[3 * (k + 1) + c];
        } else {
            for (int c = 0; c < 3; ++c) rgb[c] = fixed_rgb[c];
        }
        for (int c = 0; c < 3; ++c) {
            E[3 * i + c] = brightness * rgb[c];
            A[3 * i + c] = absorption;
        }
    }
}

/* Vector colouring (Section 2, third item: a vector quantity's three
 * components give the red, green and blue of E).  Reading: each component is
 * normalised like a scalar without the logarithm (C7 per component, over the
 * particles of the species): t_c = clamp((v_c - lo_c)/(hi_c - lo_c), 0, 1),
 * t_c = 0 if hi_c == lo_c; E_c = brightness * t_c, A = absorption * (1, 1, 1).
 * vx, vy, vz hold the components as doubles. */
void oracle_colour_vector(size_t n, const double *vx, const double *vy, const double *vz, const double lo[3],
                          const double hi[3], double brightness, double absorption, double *E, double *A)
{
    const double *v[3] = {vx, vy, vz};
    for (size_t i = 0; i < n; ++i) {
        for (int c = 0; c < 3; ++c) {
            double t = hi[c] > lo[c] ? (v[c][i] - lo[c]) / (hi[c] - lo[c]) : 0.0;
            t = t < 0.0 ? 0.0 : (t > 1.0 ? 1.0 : t);
            E[3 * i + c] = brightness * t;
            A[3 * i + c] = absorption;
        }
    }
}

/* Optical-depth modulation (Section 2, third item: the optical depth of a
 * particle made proportional to another scalar q).  Reading: q scales the
 * particle's column density rho_0 (C5 sets rho_0 = 1) to m = clamp(q / q_max,
 * 0, 1), q_max the largest q of the species (m = 0 if q_max <= 0).  In Eq. 1
 * rho multiplies both terms, so E and A are both scaled by m. */
void oracle_modulate(size_t n, const double *q, double q_max, double *E, double *A)
{
    for (size_t i = 0; i < n; ++i) {
        double m = q_max > 0.0 ? q[i] / q_max : 0.0;
        m = m < 0.0 ? 0.0 : (m > 1.0 ? 1.0 : m);
        for (int c = 0; c < 3; ++c) {
            E[3 * i + c] *= m;
            A[3 * i + c] *= m;
        }
    }
}

typedef struct {
    uint32_t key;
    uint32_t idx;
} okey;

static int cmp_okey(const void *a, const void *b)
{
    const okey *p = (const okey *)a, *q = (const okey *)b;
    if (p->key != q->key) return p->key < q->key ? -1 : 1;
    return p->idx < q->idx ? -1 : (p->idx > q->idx ? 1 : 0);
}

/* C10: order of the visible particles.  Absorptive rendering needs depth
 * order because Eq. 1 does not commute when E != A (Section 2). */
size_t oracle_order(size_t n, const uint32_t *key, const uint8_t *visible, int by_depth, uint32_t *order)
{
    size_t v = 0;
    if (!by_depth) {
        for (size_t i = 0; i < n; ++i)
            if (visible[i]) order[v++] = (uint32_t)i;
        return v;
    }
    okey *tmp = (okey *)malloc(sizeof(okey) * (n ? n : 1));
    if (!tmp) return (size_t)-1;
    for (size_t i = 0; i < n; ++i)
        if (visible[i]) { tmp[v].key = key[i]; tmp[v].idx = (uint32_t)i; ++v; }
    qsort(tmp, v, sizeof(okey), cmp_okey);
    for (size_t k = 0; k < v; ++k) order[k] = tmp[k].idx;
    free(tmp);
    return v;
}

/* Screen tiles of side `tile`, numbered row-major.  Per tile, the visible
 * particles (in `order`) whose bbox meets it.  With offsets == NULL only the
 * total number of entries is returned; otherwise offsets (ntiles + 1) and
 * list are filled. */
size_t oracle_tile_lists(int width, int height, int tile, size_t v, const uint32_t *order,
                         const int32_t *bbox, uint64_t *offsets, uint32_t *list)
{
    int ntx = (width + tile - 1) / tile, nty = (height + tile - 1) / tile;
    size_t ntiles = (size_t)ntx * (size_t)nty;
    size_t total = 0;
    uint64_t *count = (uint64_t *)calloc(ntiles + 1, sizeof(uint64_t));
    if (!count) return (size_t)-1;
    for (size_t k = 0; k < v; ++k) {
        const int32_t *b = &bbox[4 * (size_t)order[k]];
        for (int ty = b[1] / tile; ty <= b[3] / tile; ++ty)
            for (int tx = b[0] / tile; tx <= b[2] / tile; ++tx) {
                count[(size_t)ty * ntx + tx] += 1;
                total += 1;
            }
    }
    if (offsets) {
        offsets[0] = 0;
        for (size_t t = 0; t < ntiles; ++t) offsets[t + 1] = offsets[t] + count[t];
        memset(count, 0, sizeof(uint64_t) * ntiles);
        for (size_t k = 0; k < v; ++k) {
            const int32_t *b = &bbox[4 * (size_t)order[k]];
            for (int ty = b[1] / tile; ty <= b[3] / tile; ++ty)
                for (int tx = b[0] / tile; tx <= b[2] / tile; ++tx) {
                    size_t t = (size_t)ty * ntx + tx;
                    list[offsets[t] + count[t]] = order[k];
                    count[t] += 1;
                }
        }
    }
    free(count);
    return total;
}

/* C6 membership in single precision, then g of C5 in double precision.
 * Returns 0 when the pixel is outside the particle's footprint. */
static double pixel_weight(int i, int j, float sx, float sy, float sigma_pix, float r2, int *inside)
{
    float dx = ((float)i + 0.5f) - sx;
    float dy = ((float)j + 0.5f) - sy;
    float d2 = fmaf(dy, dy, dx * dx);
    *inside = d2 < r2;
    if (!*inside) return 0.0;
    double ddx = ((double)i + 0.5) - (double)sx;
    double ddy = ((double)j + 0.5) - (double)sy;
    double sg = (double)sigma_pix;
    return exp(-(ddx * ddx + ddy * ddy) / (sg * sg));
}

/* Composite one pixel over the particles plist[0..m) (already in C10 order).
 * Section 2, Eq. 1 integrated layer by layer (C11):
 *   emission:   I = sum_p E_p g_p
 *   absorptive: front to back, C += T S_p then T *= T_p (back_to_front = 0), or
 *               back to front, I = I T_p + S_p (back_to_front = 1)
 *   E = A:      I = 1 - exp(-sum_p A_p g_p) with A_p = E_p per channel. */
static void composite_pixel(int i, int j, int mode, int back_to_front, size_t m, const uint32_t *plist,
                            const float *sx, const float *sy, const float *sigma_pix, const float *r2,
                            const double *E, const double *A, double out[3])
{
    double acc[3] = {0.0, 0.0, 0.0};
    if (mode == OR_EMISSION || mode == OR_E_EQ_A) {
        for (size_t k = 0; k < m; ++k) {
            uint32_t p = plist[k];
            int inside;
            double g = pixel_weight(i, j, sx[p], sy[p], sigma_pix[p], r2[p], &inside);
            if (!inside) continue;
            for (int c = 0; c < 3; ++c) acc[c] += E[3 * (size_t)p + c] * g;
        }
        for (int c = 0; c < 3; ++c) out[c] = mode == OR_E_EQ_A ? -expm1(-acc[c]) : acc[c];
        return;
    }
    double T[3] = {1.0, 1.0, 1.0};
    for (size_t kk = 0; kk < m; ++kk) {
        size_t k = back_to_front ? m - 1 - kk : kk;
        uint32_t p = plist[k];
        int inside;
        double g = pixel_weight(i, j, sx[p], sy[p], sigma_pix[p], r2[p], &inside);
        if (!inside) continue;
        for (int c = 0; c < 3; ++c) {
            double a = A[3 * (size_t)p + c], e = E[3 * (size_t)p + c];
            double Tp = exp(-a * g);
            double Sp = a > 0.0 ? e * (-expm1(-a * g)) / a : e * g;
            if (back_to_front) {
                acc[c] = acc[c] * Tp + Sp;
            } else {
                acc[c] += T[c] * Sp;
                T[c] *= Tp;
            }
        }
    }
    for (int c = 0; c < 3; ++c) out[c] = acc[c];
}

/* Whole image (H x W x 3, row-major, row 0 at the top) from the tile lists. */
void oracle_render(int width, int height, int tile, int mode, int back_to_front,
                   const uint64_t *offsets, const uint32_t *list,
                   const float *sx, const float *sy, const float *sigma_pix, const float *r2,
                   const double *E, const double *A, double *image)
{
    int ntx = (width + tile - 1) / tile;
#pragma omp parallel for schedule(dynamic, 1)
    for (int j = 0; j < height; ++j) {
        for (int i = 0; i < width; ++i) {
            size_t t = (size_t)(j / tile) * ntx + (size_t)(i / tile);
            composite_pixel(i, j, mode, back_to_front, (size_t)(offsets[t + 1] - offsets[t]), &list[offsets[t]],
                            sx, sy, sigma_pix, r2, E, A, &image[3 * ((size_t)j * width + i)]);
        }
    }
}

/* Selected pixels only (pix holds (i, j) pairs); out is npix x 3. */
void oracle_render_pixels(int width, int tile, int mode, size_t npix, const int32_t *pix,
                          const uint64_t *offsets, const uint32_t *list,
                          const float *sx, const float *sy, const float *sigma_pix, const float *r2,
                          const double *E, const double *A, double *out)
{
    int ntx = (width + tile - 1) / tile;
#pragma omp parallel for schedule(dynamic, 16)
    for (long long q = 0; q < (long long)npix; ++q) {
        int i = pix[2 * q], j = pix[2 * q + 1];
        size_t t = (size_t)(j / tile) * ntx + (size_t)(i / tile);
        composite_pixel(i, j, mode, 0, (size_t)(offsets[t + 1] - offsets[t]), &list[offsets[t]],
                        sx, sy, sigma_pix, r2, E, A, &out[3 * q]);
    }
}

/* No tiles and no bbox: every pixel against every particle of `order`. */
void oracle_render_brute(int width, int height, int mode, int back_to_front, size_t v, const uint32_t *order,
                         const float *sx, const float *sy, const float *sigma_pix, const float *r2,
                         const double *E, const double *A, double *image)
{
#pragma omp parallel for schedule(dynamic, 1)
    for (int j = 0; j < height; ++j)
        for (int i = 0; i < width; ++i)
            composite_pixel(i, j, mode, back_to_front, v, order, sx, sy, sigma_pix, r2, E, A,
                            &image[3 * ((size_t)j * width + i)]);
}

int oracle_num_threads(void)
{
    int n = 1;
#pragma omp parallel
    {
#pragma omp single
        {
#ifdef _OPENMP
            n = omp_get_num_threads();
#endif
        }
    }
    return n;
}
