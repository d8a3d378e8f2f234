/*
 * Seeded synthetic particle sets shaped like cosmological N-body snapshots.
 *
 * This module only draws inputs.  It holds none of the rendering method's
 * arithmetic (no camera, projection, colouring or compositing), so the FP64
 * oracle and the CUDA path can both consume its output without sharing any
 * code of the method.
 *
 * Every random number is a pure function of (seed, set id, particle index,
 * draw block): Philox4x32-10 (Salmon, Moraes, Dror and Shaw, "Parallel random
 * numbers: as easy as 1, 2, 3", SC'11) keyed by (seed, set id) with the counter
 * (index low word, index high word, block, 0).  A set therefore comes out the
 * same whatever the thread count or the slice [i0, i0+n) asked for.
 *
 * Build with -ffp-contract=off.  Transcendentals come from the C library, so
 * the last bit of a drawn value may differ between C libraries; every
 * comparison in this project uses inputs drawn in the same process.
 */
#include <math.h>
#include <stddef.h>
#include <stdint.h>

#define PHILOX_M0 0xD2511F53u
#define PHILOX_M1 0xCD9E8D57u
#define PHILOX_W0 0x9E3779B9u
#define PHILOX_W1 0xBB67AE85u

void synth_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        uint64_t p0 = (uint64_t)PHILOX_M0 * (uint64_t)c0;
        uint64_t p1 = (uint64_t)PHILOX_M1 * (uint64_t)c2;
        uint32_t n0 = (uint32_t)(p1 >> 32) ^ c1 ^ k0;
        uint32_t n1 = (uint32_t)p1;
        uint32_t n2 = (uint32_t)(p0 >> 32) ^ c3 ^ k1;
        uint32_t n3 = (uint32_t)p0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
        k0 += PHILOX_W0;
        k1 += PHILOX_W1;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* One Philox block for (key, index, block). */
static void draw_block(uint32_t seed, uint32_t set_id, uint64_t index, uint32_t block, uint32_t w[4])
{
    uint32_t ctr[4] = {(uint32_t)index, (uint32_t)(index >> 32), block, 0u};
    uint32_t key[2] = {seed, set_id};
    synth_philox4x32_10(ctr, key, w);
}

/* Uniform in the open interval (0, 1) from one 32-bit word. */
static double unit_open(uint32_t w) { return ((double)w + 0.5) * (1.0 / 4294967296.0); }

/* Standard normal from two words (Box-Muller, cosine branch). */
static double normal2(uint32_t a, uint32_t b)
{
    const double two_pi = 6.283185307179586476925286766559;
    return sqrt(-2.0 * log(unit_open(a))) * cos(two_pi * unit_open(b));
}

/* Fills out[k] = lo + (hi - lo) * U_k for k in [0, n): used for sphere
 * centres and scale radii.  Stream `block` keeps the draws apart. */
void synth_uniform(uint32_t seed, uint32_t set_id, uint32_t block, size_t n, double lo, double hi, double *out)
{
    for (size_t k = 0; k < n; ++k) {
        uint32_t w[4];
        draw_block(seed, set_id, (uint64_t)k, block, w);
        out[k] = lo + (hi - lo) * unit_open(w[0]);
    }
}

typedef struct {
    uint32_t seed;          /* Philox key word 0 */
    uint32_t set_id;        /* Philox key word 1 */
    int32_t n_spheres;      /* sphere j holds particles i with i % n_spheres == j */
    int32_t max_tries;      /* rejection attempts for a position inside the unit cube */
    const double *centre;   /* n_spheres x 3 */
    const double *radius;   /* n_spheres Plummer scale radii */
    double radius_factor;   /* multiplies every scale radius (2 for a wider halo) */
    double bg_fraction;     /* probability that a particle is uniform background */
    double r_cap;           /* Plummer radius cut, in scale radii */
    int32_t h_mode;         /* 0: lognormal(h_mu, h_sigma); 1: eta a (1 + r^2/a^2)^(5/6), background h_bg */
    int32_t v_mode;         /* 0: lognormal(v_mu, v_sigma); 1: v_const */
    double h_mu, h_sigma, eta, h_bg, h_min, h_max;
    double v_mu, v_sigma, v_const;
} synth_cluster_cfg;

/* Isotropic Plummer draw around centre c with scale radius a.  Returns 1 and
 * writes the position and the radius when a draw inside [0,1)^3 was found. */
static int plummer_point(const synth_cluster_cfg *c, uint64_t i, const double *centre, double a,
                         double p[3], double *rad)
{
    const double two_pi = 6.283185307179586476925286766559;
    for (int t = 0; t < c->max_tries; ++t) {
        uint32_t w[4];
        draw_block(c->seed, c->set_id, i, 2u + (uint32_t)t, w);
        double u = unit_open(w[0]);
        /* enclosed mass fraction of a Plummer sphere: m = r^3 / (r^2 + a^2)^{3/2} */
        double r = a / sqrt(pow(u, -2.0 / 3.0) - 1.0);
        if (!(r <= c->r_cap * a))
            continue;
        double ct = 2.0 * unit_open(w[1]) - 1.0;
        double st = sqrt(1.0 - ct * ct);
        double ph = two_pi * unit_open(w[2]);
        double q0 = centre[0] + r * st * cos(ph);
        double q1 = centre[1] + r * st * sin(ph);
        double q2 = centre[2] + r * ct;
        if (q0 >= 0.0 && q0 < 1.0 && q1 >= 0.0 && q1 < 1.0 && q2 >= 0.0 && q2 < 1.0) {
            p[0] = q0; p[1] = q1; p[2] = q2;
            *rad = r;
            return 1;
        }
    }
    p[0] = centre[0]; p[1] = centre[1]; p[2] = centre[2];
    *rad = 0.0;
    return 0;
}

static double clampd(double v, double lo, double hi) { return v < lo ? lo : (v > hi ? hi : v); }

/* Particles [i0, i0 + n) of a Plummer-sphere mixture with optional uniform
 * background.  Returns the number of particles whose rejection loop ran out
 * (they sit at their sphere centre). */
long synth_cluster_set(const synth_cluster_cfg *c, uint64_t i0, size_t n,
                       float *x, float *y, float *z, float *h, float *v)
{
    long fallbacks = 0;
#pragma omp parallel for schedule(static) reduction(+ : fallbacks)
    for (long long k = 0; k < (long long)n; ++k) {
        uint64_t i = i0 + (uint64_t)k;
        uint32_t w0[4], w1[4];
        draw_block(c->seed, c->set_id, i, 0u, w0);
        draw_block(c->seed, c->set_id, i, 1u, w1);
        int sphere = (int)(i % (uint64_t)c->n_spheres);
        double a = c->radius[sphere] * c->radius_factor;
        double p[3], rad = 0.0;
        int background = unit_open(w0[0]) < c->bg_fraction;
        if (background) {
            uint32_t wb[4];
            draw_block(c->seed, c->set_id, i, 2u, wb);
            p[0] = unit_open(wb[0]); p[1] = unit_open(wb[1]); p[2] = unit_open(wb[2]);
        } else if (!plummer_point(c, i, &c->centre[3 * sphere], a, p, &rad)) {
            fallbacks += 1;
        }
        double hh;
        if (c->h_mode == 0) {
            hh = exp(c->h_mu + c->h_sigma * normal2(w0[1], w0[2]));
        } else if (background) {
            hh = c->h_bg;
        } else {
            double q = rad / a;
            hh = c->eta * a * pow(1.0 + q * q, 5.0 / 6.0);
        }
        hh = clampd(hh, c->h_min, c->h_max);
        double vv = c->v_mode == 0 ? exp(c->v_mu + c->v_sigma * normal2(w1[0], w1[1])) : c->v_const;
        x[k] = (float)p[0]; y[k] = (float)p[1]; z[k] = (float)p[2];
        h[k] = (float)hh;
        v[k] = (float)vv;
    }
    return fallbacks;
}

typedef struct {
    uint32_t seed, set_id;
    int32_t n_side;          /* lattice of n_side^3 particles, spacing 1/n_side */
    int32_t n_spheres;       /* overdensities */
    int32_t max_tries;
    int32_t pad;
    const double *centre;    /* n_spheres x 3 */
    const double *radius;    /* n_spheres */
    double disp_sigma;       /* Gaussian displacement, in cells */
    double reloc_fraction;   /* probability that a particle moves into a sphere */
    double r_cap, eta, h_min, h_max;
    double v_mu, v_sigma;
} synth_lattice_cfg;

/* Particles [i0, i0 + n) of a displaced unit lattice in which a fraction of
 * the particles (chosen by their own draw) is moved into Plummer spheres.
 * Lattice particles get h = one cell; moved ones the density-based h. */
long synth_lattice_set(const synth_lattice_cfg *c, uint64_t i0, size_t n,
                       float *x, float *y, float *z, float *h, float *v)
{
    synth_cluster_cfg pc = {0};
    pc.seed = c->seed; pc.set_id = c->set_id; pc.n_spheres = c->n_spheres;
    pc.max_tries = c->max_tries; pc.r_cap = c->r_cap;
    const double cell = 1.0 / (double)c->n_side;
    long fallbacks = 0;
#pragma omp parallel for schedule(static) reduction(+ : fallbacks)
    for (long long k = 0; k < (long long)n; ++k) {
        uint64_t i = i0 + (uint64_t)k;
        uint32_t w0[4], w1[4];
        draw_block(c->seed, c->set_id, i, 0u, w0);
        draw_block(c->seed, c->set_id, i, 1u, w1);
        uint64_t ns = (uint64_t)c->n_side;
        uint64_t ix = i % ns, iy = (i / ns) % ns, iz = i / (ns * ns);
        double p[3], hh;
        if (unit_open(w1[0]) < c->reloc_fraction) {
            int sphere = (int)(unit_open(w1[1]) * (double)c->n_spheres);
            if (sphere >= c->n_spheres) sphere = c->n_spheres - 1;
            double a = c->radius[sphere], rad = 0.0;
            if (!plummer_point(&pc, i, &c->centre[3 * sphere], a, p, &rad))
                fallbacks += 1;
            double q = rad / a;
            hh = clampd(c->eta * a * pow(1.0 + q * q, 5.0 / 6.0), c->h_min, c->h_max);
        } else {
            double g0 = normal2(w0[0], w0[1]);
            double g1 = normal2(w0[2], w0[3]);
            double g2 = normal2(w1[2], w1[3]);
            p[0] = ((double)ix + 0.5 + c->disp_sigma * g0) * cell;
            p[1] = ((double)iy + 0.5 + c->disp_sigma * g1) * cell;
            p[2] = ((double)iz + 0.5 + c->disp_sigma * g2) * cell;
            hh = cell;
        }
        uint32_t wv[4];
        draw_block(c->seed, c->set_id, i, 40u, wv);
        double vv = exp(c->v_mu + c->v_sigma * normal2(wv[0], wv[1]));
        x[k] = (float)p[0]; y[k] = (float)p[1]; z[k] = (float)p[2];
        h[k] = (float)hh;
        v[k] = (float)vv;
    }
    return fallbacks;
}
