/*
 * larsim_oracle.c -- plain, slow FP64 CPU oracle of the charge-readout path of
 * "Highly-parallelized simulation of a pixelated LArTPC on a GPU"
 * (DUNE collaboration, arXiv:2212.09807, Sec. 3).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg may load this library.  It shares no code,
 * header, table or constant generator with the CUDA path; the only thing both
 * sides receive is the seeded synthetic input (segments, configuration
 * numbers, response table).
 *
 * Every step follows the paper's statement in its own order and notation:
 *   ora_recomb          Sec. 3.1, Eq. (birks) and Eq. (box)
 *   ora_quench_drift    Sec. 3.1 + Sec. 3.2, Eq. (drift), Eq. (lifetime) and
 *                       the diffusion width sigma = sqrt(2 D t_drift)
 *   ora_map_segment     Sec. 3.3.2 (pixels a segment can induce on): brute
 *                       force over every pixel of the anode
 *   ora_pixel_current   Sec. 3.3.2, the charge density rho (N points x M
 *                       perturbations) and Eq. (current), with the table of
 *                       Sec. 3.3.1 interpolated trilinearly
 *   ora_electronics     Sec. 3.4 (CSA integration, discriminator with noise,
 *                       hold, ADC, reset)
 *   ora_map_event, ora_pixel_currents_many, ora_electronics_many
 *                       the same three steps for a whole event: every
 *                       segment's map, and the current and front end of many
 *                       pixels, each pixel exactly as the single-pixel
 *                       functions compute it (the pixels are independent and
 *                       are shared among the host cores with OpenMP when the
 *                       library is built with it)
 *   ora_hit_intervals   Sec. 3.4: the ticks whose current a hit digitises
 *                       (per-hit charge truth: the per-segment sums over these
 *                       intervals are formed from ora_pixel_current of each
 *                       segment alone, in oracle/__init__.py)
 *   ora_hit_point       Sec. 6: hit -> 3-D point (pixel centre, inverse of
 *                       Eq. (drift))
 *   ora_track_dqdx      Sec. 6: dQ/dx in pieces of a known straight track
 *   ora_light_segment   Sec. 4.1: photons and photoelectrons per photosensor
 *   ora_light_photocurrent  Sec. 4.2, Eq. (photocurrent)
 *   ora_light_scintillation Sec. 4.2, the truncated scintillation convolution
 *   ora_light_fluctuate Sec. 4.2, Poisson / normal counting fluctuations
 *   ora_light_electronics   Sec. 4.3, response, noise, sampling, ADC
 *   ora_light_truth     Sec. 4.4, mean arrival time per segment and photosensor
 *   ora_philox4x32_10   counter-based generator of Salmon et al., SC'11
 *                       ("Parallel random numbers: as easy as 1, 2, 3")
 *
 * Arithmetic is FP64 throughout.  Integer decisions that the path takes from
 * floating-point values (which drift volume a segment belongs to, how many
 * points it is cut into) are taken in FP64 from the FP32 inputs with plain
 * IEEE operations in the order written here; the electronics' threshold and
 * ADC decisions are taken in FP64.  Where a decision lies within a stated band
 * of its threshold, the oracle reports it so that tests can exclude that tie
 * (the band then also covers a device's FP32 decisions).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORA_PI 3.14159265358979323846

typedef struct ora_cfg {
    /* geometry */
    int32_t n_mod_x, n_mod_y, n_tpc, tiles_x, tiles_y, px_per_tile;
    double pitch, drift_len;
    /* recombination and drift */
    int32_t recomb_model;
    double Ab, kb, alpha, beta, efield, density, w_ion;
    double vdrift, lifetime, DL, DT; /* D in cm^2/s */
    /* sampling */
    double step;
    int32_t M;
    double clip;
    /* readout */
    double tick;
    int32_t n_ticks;
    double t_w0;
    /* front end */
    double thr, s_reset, s_disc, s_unc, gain, lsb_mV;
    int32_t hold, min_int, periodic, adc_bits;
    uint64_t seed;
    /* response table */
    int32_t nb, nt, bins_per_pitch;
    /* 0: lifetime and diffusion evaluated once per segment, at its midpoint;
     * 1: at each point's own drift distance (the segment's sigma_T/L outputs
     * are then those of its farther end, which bound every point's) */
    int32_t per_point;
    /* 0: table read bilinearly in the offset and linearly in the arrival
     * tick; 1: nearest node and nearest tick (halves round up) */
    int32_t nearest;
    int32_t pad2;
} ora_cfg;

size_t ora_cfg_size(void) { return sizeof(ora_cfg); }

/* ------------------------------------------------------------------ RNG -- */

static void mulhilo32(uint32_t a, uint32_t b, uint32_t *hi, uint32_t *lo)
{
    uint64_t p = (uint64_t)a * (uint64_t)b;
    *hi = (uint32_t)(p >> 32);
    *lo = (uint32_t)p;
}

/* Philox4x32 with 10 rounds: each round multiplies words 0 and 2 by the two
 * round multipliers, exchanges the words and mixes in the key; the key is
 * bumped by the two Weyl constants between rounds. */
void ora_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int r = 0; r < 10; ++r) {
        uint32_t hi0, lo0, hi1, lo1;
        mulhilo32(0xD2511F53u, c0, &hi0, &lo0);
        mulhilo32(0xCD9E8D57u, c2, &hi1, &lo1);
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        c0 = n0; c1 = lo1; c2 = n2; c3 = lo0;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* Uniform in (0,1): (x + 1/2) 2^-32, exact in FP64. */
static double ora_u01(uint32_t x) { return ((double)x + 0.5) * (1.0 / 4294967296.0); }

/* Four standard normals from one Philox block by the Box-Muller transform:
 * (n0, n1) from (u0, u1) and (n2, n3) from (u2, u3).  Key = seed ^ event id. */
void ora_normals(uint64_t seed, uint64_t event_id, uint32_t c0, uint32_t c1,
                 uint32_t c2, uint32_t c3, double n[4])
{
    uint64_t k = seed ^ event_id;
    uint32_t key[2] = {(uint32_t)k, (uint32_t)(k >> 32)};
    uint32_t ctr[4] = {c0, c1, c2, c3};
    uint32_t x[4];
    ora_philox4x32_10(ctr, key, x);
    double r0 = sqrt(-2.0 * log(ora_u01(x[0])));
    double a0 = 2.0 * ORA_PI * ora_u01(x[1]);
    double r1 = sqrt(-2.0 * log(ora_u01(x[2])));
    double a1 = 2.0 * ORA_PI * ora_u01(x[3]);
    n[0] = r0 * cos(a0);
    n[1] = r0 * sin(a0);
    n[2] = r1 * cos(a1);
    n[3] = r1 * sin(a1);
}

/* ------------------------------------------------------- recombination -- */

/* Recombination factor at stopping power dEdx (MeV/cm), Sec. 3.1.
 * epsilon = E-field (kV/cm) x LAr density (g/cm^3).
 * Birks, Eq. (birks):  R = A_b / (1 + (k_b/epsilon) dE/dx)
 * modified Box, Eq. (box):  R = ln(alpha + (beta/epsilon) dE/dx) / ((beta/epsilon) dE/dx) */
double ora_recomb(const ora_cfg *c, double dEdx)
{
    double eps = c->efield * c->density;
    if (c->recomb_model == 1) {
        double xi = c->beta / eps * dEdx;
        return log(c->alpha + xi) / xi;
    }
    return c->Ab / (1.0 + c->kb / eps * dEdx);
}

/* ------------------------------------------------------------ geometry -- */

typedef struct {
    int ok, anode, mx, my, tpc;
    double ox, oy, za;
} ora_loc;

/* Drift volume of a point.  Modules tile x-y from the origin, each
 * npx*pitch wide; TPC 0 spans z in [0, D) with its anode at z = 0, TPC 1
 * spans [D, 2D] with its anode at z = 2D (cathode at z = D). */
static ora_loc ora_locate(const ora_cfg *c, double x, double y, double z)
{
    ora_loc L;
    memset(&L, 0, sizeof L);
    double Wx = (double)(c->tiles_x * c->px_per_tile) * c->pitch;
    double Wy = (double)(c->tiles_y * c->px_per_tile) * c->pitch;
    double xmax = (double)c->n_mod_x * Wx;
    double ymax = (double)c->n_mod_y * Wy;
    double zmax = (double)c->n_tpc * c->drift_len;
    if (!(x >= 0.0 && x < xmax && y >= 0.0 && y < ymax && z >= 0.0 && z <= zmax)) {
        L.ok = 0;
        L.anode = -1;
        return L;
    }
    int mx = (int)floor(x / Wx);
    int my = (int)floor(y / Wy);
    if (mx > c->n_mod_x - 1) mx = c->n_mod_x - 1;
    if (my > c->n_mod_y - 1) my = c->n_mod_y - 1;
    int tpc = (c->n_tpc == 2 && z >= c->drift_len) ? 1 : 0;
    L.ok = 1;
    L.mx = mx;
    L.my = my;
    L.tpc = tpc;
    L.anode = (my * c->n_mod_x + mx) * c->n_tpc + tpc;
    L.ox = (double)mx * Wx;
    L.oy = (double)my * Wy;
    L.za = tpc == 0 ? 0.0 : 2.0 * c->drift_len;
    return L;
}

/* Centre (global cm) of a pixel and its anode's z. */
static void ora_pixel_centre(const ora_cfg *c, int32_t pixel, double *xc, double *yc,
                             double *za, int32_t *anode)
{
    int32_t nx = c->tiles_x * c->px_per_tile;
    int32_t ny = c->tiles_y * c->px_per_tile;
    int32_t g = pixel / (nx * ny);
    int32_t rem = pixel % (nx * ny);
    int32_t iy = rem / nx, ix = rem % nx;
    int32_t m = g / c->n_tpc, tpc = g % c->n_tpc;
    int32_t mx = m % c->n_mod_x, my = m / c->n_mod_x;
    double Wx = (double)nx * c->pitch, Wy = (double)ny * c->pitch;
    *xc = (double)mx * Wx + ((double)ix + 0.5) * c->pitch;
    *yc = (double)my * Wy + ((double)iy + 0.5) * c->pitch;
    *za = tpc == 0 ? 0.0 : 2.0 * c->drift_len;
    *anode = g;
}

/* --------------------------------------------------- quench and drift -- */

/* Steps 1-2 for n segments (SoA FP32 input, cm / us / MeV).
 * Outputs per segment: dx (cm), dE/dx, R, Q_R and Q_a (electrons), t_drift
 * (us), sigma_T and sigma_L (cm), anode (-1 = inactive) and the number of
 * points N along the segment (10 um spacing, Sec. 3.3.2).
 * A segment is active when its midpoint lies in a drift volume and its
 * length is at least 1e-6 cm (dE/dx is undefined for a point deposit). */
void ora_quench_drift(const ora_cfg *c, int64_t n,
                      const float *x0, const float *y0, const float *z0, const float *t0,
                      const float *x1, const float *y1, const float *z1, const float *t1,
                      const float *dE,
                      double *dx_out, double *dedx_out, double *R_out, double *QR_out,
                      double *Qa, double *t_drift, double *sigma_T, double *sigma_L,
                      int32_t *anode, int32_t *n_samples)
{
    (void)t0; (void)t1;
    for (int64_t i = 0; i < n; ++i) {
        double ddx = (double)x1[i] - (double)x0[i];
        double ddy = (double)y1[i] - (double)y0[i];
        double ddz = (double)z1[i] - (double)z0[i];
        double dx = sqrt(ddx * ddx + ddy * ddy + ddz * ddz);
        double xm = 0.5 * ((double)x0[i] + (double)x1[i]);
        double ym = 0.5 * ((double)y0[i] + (double)y1[i]);
        double zm = 0.5 * ((double)z0[i] + (double)z1[i]);
        ora_loc L = ora_locate(c, xm, ym, zm);
        dx_out[i] = dx;
        if (!L.ok || dx < 1e-6) {
            dedx_out[i] = R_out[i] = QR_out[i] = 0.0;
            Qa[i] = t_drift[i] = sigma_T[i] = sigma_L[i] = 0.0;
            anode[i] = -1;
            n_samples[i] = 0;
            continue;
        }
        /* Sec. 3.1: Q_0 = E / W_ion, Q_R = R Q_0 */
        double dedx = (double)dE[i] / dx;
        double R = ora_recomb(c, dedx);
        double Q0 = (double)dE[i] / c->w_ion;
        double QR = R * Q0;
        /* Sec. 3.2, Eq. (drift): t = |z - z_anode| / v_drift, at the midpoint */
        double td = fabs(zm - L.za) / c->vdrift;
        /* Eq. (lifetime) */
        double qa = QR * exp(-td / c->lifetime);
        /* sigma = sqrt(2 D t), D converted from cm^2/s to cm^2/us */
        double tsig = td;
        if (c->per_point) {
            double t0d = fabs((double)z0[i] - L.za) / c->vdrift;
            double t1d = fabs((double)z1[i] - L.za) / c->vdrift;
            tsig = t0d > t1d ? t0d : t1d;
        }
        double sT = sqrt(2.0 * (c->DT * 1e-6) * tsig);
        double sL = sqrt(2.0 * (c->DL * 1e-6) * tsig);
        double N = ceil(dx / c->step);
        if (N < 1.0) N = 1.0;
        dedx_out[i] = dedx;
        R_out[i] = R;
        QR_out[i] = QR;
        Qa[i] = qa;
        t_drift[i] = td;
        sigma_T[i] = sT;
        sigma_L[i] = sL;
        anode[i] = L.anode;
        n_samples[i] = (int32_t)N;
    }
}

/* ------------------------------------------------------------ pixel map -- */

/* Chebyshev (L-infinity) distance between the 2-D segment (ax,ay)-(bx,by)
 * and the point (px,py): min over t in [0,1] of
 * max(|ax + t(bx-ax) - px|, |ay + t(by-ay) - py|).  The function is convex
 * and piecewise linear in t, so its minimum sits at t = 0, t = 1, a zero of
 * one of the two terms, or a point where the two terms are equal. */
double ora_cheb_distance(double ax, double ay, double bx, double by, double px, double py)
{
    double u0 = ax - px, du = bx - ax;
    double v0 = ay - py, dv = by - ay;
    double cand[8];
    int nc = 0;
    cand[nc++] = 0.0;
    cand[nc++] = 1.0;
    if (du != 0.0) cand[nc++] = -u0 / du;
    if (dv != 0.0) cand[nc++] = -v0 / dv;
    if (du - dv != 0.0) cand[nc++] = (v0 - u0) / (du - dv);
    if (du + dv != 0.0) cand[nc++] = -(u0 + v0) / (du + dv);
    double best = INFINITY;
    for (int i = 0; i < nc; ++i) {
        double t = cand[i];
        if (!(t >= 0.0 && t <= 1.0)) continue;
        double a = fabs(u0 + t * du), b = fabs(v0 + t * dv);
        double f = a > b ? a : b;
        if (f < best) best = f;
    }
    return best;
}

/* Half-width of the square around a pixel centre inside which a segment can
 * induce current on it: the table reaches (nb + 1/2) bins (its last node sits
 * at (nb - 1/2) bins and interpolation runs to the next, zero, node) and every
 * diffusion offset is clipped at clip * sigma_T. */
double ora_map_radius(const ora_cfg *c, double sigma_T)
{
    double h = c->pitch / (double)c->bins_per_pitch;
    return ((double)c->nb + 0.5) * h + c->clip * sigma_T;
}

/* Pixels of the segment's own anode that the segment can induce on
 * (Sec. 3.3.2): brute force over every pixel of that anode.  Writes up to
 * ``cap`` pixel ids in increasing order and, per id, the distance margin
 * R_map - d (>= 0).  Returns the number of mapped pixels (may exceed cap). */
int64_t ora_map_segment(const ora_cfg *c, float x0, float y0, float x1, float y1,
                        double sigma_T, int32_t anode, int32_t *ids, double *margin,
                        int64_t cap)
{
    if (anode < 0) return 0;
    int32_t nx = c->tiles_x * c->px_per_tile;
    int32_t ny = c->tiles_y * c->px_per_tile;
    double R = ora_map_radius(c, sigma_T);
    int64_t cnt = 0;
    for (int32_t iy = 0; iy < ny; ++iy) {
        for (int32_t ix = 0; ix < nx; ++ix) {
            int32_t pid = anode * nx * ny + iy * nx + ix;
            double xc, yc, za;
            int32_t g;
            ora_pixel_centre(c, pid, &xc, &yc, &za, &g);
            double d = ora_cheb_distance(x0, y0, x1, y1, xc, yc);
            if (d <= R) {
                if (cnt < cap) {
                    ids[cnt] = pid;
                    if (margin) margin[cnt] = R - d;
                }
                ++cnt;
            }
        }
    }
    return cnt;
}

/* Same map as ora_map_segment, with the brute force restricted to the pixels
 * of the segment's bounding box widened by R_map (+1 pixel): a pixel outside
 * that box is farther than R_map in Chebyshev distance from every point of the
 * segment, so the result is identical.  Ids in increasing order. */
int64_t ora_map_segment_box(const ora_cfg *c, float x0, float y0, float x1, float y1,
                            double sigma_T, int32_t anode, int32_t *ids, double *margin,
                            int64_t cap)
{
    if (anode < 0) return 0;
    int32_t nx = c->tiles_x * c->px_per_tile;
    int32_t ny = c->tiles_y * c->px_per_tile;
    double R = ora_map_radius(c, sigma_T);
    int32_t m = anode / c->n_tpc;
    double ox = (double)(m % c->n_mod_x) * (double)nx * c->pitch;
    double oy = (double)(m / c->n_mod_x) * (double)ny * c->pitch;
    double xlo = fmin((double)x0, (double)x1) - R - ox, xhi = fmax((double)x0, (double)x1) + R - ox;
    double ylo = fmin((double)y0, (double)y1) - R - oy, yhi = fmax((double)y0, (double)y1) + R - oy;
    int64_t ix0 = (int64_t)floor(xlo / c->pitch - 0.5) - 1, ix1 = (int64_t)ceil(xhi / c->pitch - 0.5) + 1;
    int64_t iy0 = (int64_t)floor(ylo / c->pitch - 0.5) - 1, iy1 = (int64_t)ceil(yhi / c->pitch - 0.5) + 1;
    if (ix0 < 0) ix0 = 0;
    if (iy0 < 0) iy0 = 0;
    if (ix1 > nx - 1) ix1 = nx - 1;
    if (iy1 > ny - 1) iy1 = ny - 1;
    int64_t cnt = 0;
    for (int64_t iy = iy0; iy <= iy1; ++iy) {
        for (int64_t ix = ix0; ix <= ix1; ++ix) {
            int32_t pid = anode * nx * ny + (int32_t)iy * nx + (int32_t)ix;
            double xc, yc, za;
            int32_t g;
            ora_pixel_centre(c, pid, &xc, &yc, &za, &g);
            double d = ora_cheb_distance(x0, y0, x1, y1, xc, yc);
            if (d <= R) {
                if (cnt < cap) {
                    ids[cnt] = pid;
                    if (margin) margin[cnt] = R - d;
                }
                ++cnt;
            }
        }
    }
    return cnt;
}

/* Margin R_map - d of one (segment, pixel) pair; negative when not mapped. */
double ora_pair_margin(const ora_cfg *c, float x0, float y0, float x1, float y1,
                       double sigma_T, int32_t anode, int32_t pixel)
{
    double xc, yc, za;
    int32_t g;
    ora_pixel_centre(c, pixel, &xc, &yc, &za, &g);
    if (g != anode || anode < 0) return -INFINITY;
    return ora_map_radius(c, sigma_T) - ora_cheb_distance(x0, y0, x1, y1, xc, yc);
}

/* ------------------------------------------------------ induced current -- */

/* Response value R[bx][by][j] with out-of-table nodes and ticks reading 0. */
static double ora_lut(const ora_cfg *c, const double *lut, int bx, int by, int64_t j)
{
    if (bx >= c->nb || by >= c->nb || j < 0 || j >= c->nt) return 0.0;
    return lut[((int64_t)bx * c->nb + by) * c->nt + j];
}

/* Current I[k], k in [0, n_ticks), induced on one pixel by the listed
 * segments (Sec. 3.3.2).  Each segment s is cut into N_s points at
 * r_mu = r_s + (mu + 1/2)/N_s (r_e - r_s) (same for the time coordinate); each
 * point gets M perturbations (sigma_T n0, sigma_T n1, sigma_L n2) with standard
 * normals from Philox counter (s, mu M + nu, 1, 0), clipped at +-clip; each
 * perturbed point carries q = Q_a / (N_s M) and arrives at
 * t_a = t_mu + |z_mu + dz - z_anode| / v_drift (Eq. (drift) per point).
 * With nearest, the table is read at the nearest node (bx, by) =
 * (floor(xi + 1/2), floor(yi + 1/2)) (none when it is node nb) and the
 * nearest tick A = floor(a + 1/2): I[k] += q R[bx][by][k - A + L - 1];
 * *n_ties (if non-null) receives the number of perturbed points with one of
 * these roundings within tie_band (bins or ticks) of its half-way point:
 * FP32 arithmetic may round those the other way.
 * With per_point, the point's own drift time t = |z_mu - z_anode| / v_drift
 * sets its charge q exp(-(t - t_drift)/tau) (Eq. (lifetime) at the point
 * instead of the midpoint) and its widths sigma = sqrt(2 D t).
 * The table is read at the folded offset (|dx|, |dy|) by bilinear
 * interpolation between bin-centred nodes (node nb reads 0; offsets below
 * half a bin read node 0) and at the fractional arrival tick by linear
 * interpolation, as in Eq. (current):
 *   I[k] += q ((1-f) Rxy[k - A + L - 1] + f Rxy[k - A + L - 2]),
 *   a = (t_a - t_window0) / tick, A = floor(a), f = a - A.
 * The pixel's current is written to I (zeroed first). */
void ora_pixel_current(const ora_cfg *c, const double *lut,
                       const float *x0, const float *y0, const float *z0, const float *t0,
                       const float *x1, const float *y1, const float *z1, const float *t1,
                       const double *Qa, const double *t_drift, const double *sigma_T,
                       const double *sigma_L, const int32_t *anode, const int32_t *n_samples,
                       uint64_t event_id, int32_t pixel, const int64_t *segs, int64_t n_segs,
                       double *I, double tie_band, int64_t *n_ties)
{
    int64_t ties = 0;
    int T = c->n_ticks;
    int L = c->nt;
    double h = c->pitch / (double)c->bins_per_pitch;
    double xc, yc, za;
    int32_t g;
    ora_pixel_centre(c, pixel, &xc, &yc, &za, &g);
    for (int k = 0; k < T; ++k) I[k] = 0.0;
    double *Rxy = (double *)malloc(sizeof(double) * (size_t)L);
    for (int64_t si = 0; si < n_segs; ++si) {
        int64_t s = segs[si];
        if (anode[s] != g) continue;
        int64_t N = n_samples[s];
        double q = Qa[s] / ((double)N * (double)c->M);
        for (int64_t mu = 0; mu < N; ++mu) {
            double u = ((double)mu + 0.5) / (double)N;
            double x = (double)x0[s] + u * ((double)x1[s] - (double)x0[s]);
            double y = (double)y0[s] + u * ((double)y1[s] - (double)y0[s]);
            double z = (double)z0[s] + u * ((double)z1[s] - (double)z0[s]);
            double t = (double)t0[s] + u * ((double)t1[s] - (double)t0[s]);
            double qp = q, sTp = sigma_T[s], sLp = sigma_L[s];
            if (c->per_point) {
                double tp = fabs(z - za) / c->vdrift;
                qp = q * exp(-(tp - t_drift[s]) / c->lifetime);
                sTp = sqrt(2.0 * (c->DT * 1e-6) * tp);
                sLp = sqrt(2.0 * (c->DL * 1e-6) * tp);
            }
            for (int nu = 0; nu < c->M; ++nu) {
                double n[4];
                ora_normals(c->seed, event_id, (uint32_t)s, (uint32_t)(mu * c->M + nu), 1u, 0u, n);
                for (int d = 0; d < 3; ++d) {
                    if (n[d] > c->clip) n[d] = c->clip;
                    if (n[d] < -c->clip) n[d] = -c->clip;
                }
                double dxp = x + sTp * n[0] - xc;
                double dyp = y + sTp * n[1] - yc;
                double zz = z + sLp * n[2];
                double ta = t + fabs(zz - za) / c->vdrift;
                double xi = fabs(dxp) / h - 0.5;
                double yi = fabs(dyp) / h - 0.5;
                if (xi < 0.0) xi = 0.0;
                if (yi < 0.0) yi = 0.0;
                if (xi >= (double)c->nb || yi >= (double)c->nb) continue;
                if (c->nearest) {
                    double a = (ta - c->t_w0) / c->tick;
                    double mx = fabs(xi - floor(xi) - 0.5), my = fabs(yi - floor(yi) - 0.5);
                    double ma = fabs(a - floor(a) - 0.5);
                    if (mx < tie_band || my < tie_band || ma < tie_band) ++ties;
                    int nx = (int)floor(xi + 0.5), ny = (int)floor(yi + 0.5);
                    if (nx >= c->nb || ny >= c->nb) continue;
                    int64_t A = (int64_t)floor(a + 0.5);
                    for (int k = 0; k < T; ++k) {
                        int64_t j = (int64_t)k - A + L - 1;
                        if (j >= 0 && j < L) I[k] += qp * ora_lut(c, lut, nx, ny, j);
                    }
                    continue;
                }
                int bx = (int)floor(xi), by = (int)floor(yi);
                double wx = xi - bx, wy = yi - by;
                for (int j = 0; j < L; ++j) {
                    Rxy[j] = (1.0 - wx) * (1.0 - wy) * ora_lut(c, lut, bx, by, j)
                           + wx * (1.0 - wy) * ora_lut(c, lut, bx + 1, by, j)
                           + (1.0 - wx) * wy * ora_lut(c, lut, bx, by + 1, j)
                           + wx * wy * ora_lut(c, lut, bx + 1, by + 1, j);
                }
                double a = (ta - c->t_w0) / c->tick;
                double Af = floor(a);
                double f = a - Af;
                int64_t A = (int64_t)Af;
                for (int k = 0; k < T; ++k) {
                    int64_t j1 = (int64_t)k - A + L - 1;
                    int64_t j2 = j1 - 1;
                    double r1 = (j1 >= 0 && j1 < L) ? Rxy[j1] : 0.0;
                    double r2 = (j2 >= 0 && j2 < L) ? Rxy[j2] : 0.0;
                    I[k] += qp * ((1.0 - f) * r1 + f * r2);
                }
            }
        }
    }
    free(Rxy);
    if (n_ties) *n_ties = ties;
}

/* ---------------------------------------------------------- electronics -- */

/* Front end of one pixel (Sec. 3.4), tick by tick:
 *   q += I[k] (charge-sensitive amplifier integrates the current);
 *   idle: v = q + s_unc n_unc(k) is compared with thr + s_disc n_disc(k)
 *     (Philox counter (pixel, k, 2, 0): n_unc = n0, n_disc = n1); on a
 *     crossing the digitisation is scheduled at
 *     t_adc = max(k + hold, last_adc + min_interval);
 *   at k == t_adc: v = q + s_unc n_unc(k), ADC = clamp(floor(v / lsb_e), 0,
 *     2^bits - 1) with lsb_e = gain x lsb_mV, the hit (pixel, t_cross, t_adc,
 *     ADC, v) is stored, and the CSA resets to a pedestal s_reset n0 of
 *     counter (pixel, k, 3, 0);
 *   optional periodic reset (period > 0, idle, k % period == 0, k > 0):
 *     q = s_reset n0 of counter (pixel, k, 4, 0) before the tick's current.
 * A digitisation still pending at the end of the window is dropped.
 * Threshold and ADC decisions are taken in FP64 (a device that decides in
 * FP32 can differ only where v lies within its FP32 rounding of the decision
 * point, i.e. inside the tie band).
 * ``tie_tick`` receives the first tick whose decision lies within ``band``
 * electrons of its threshold (or -1).  ``p_tie`` (if non-null) receives the
 * probability, under the noise model, that some decision of this trace lies
 * within the band: each idle tick's margin v - thr is normal with mean q - thr
 * (q: the CSA charge of the trace) and variance s_unc^2 + s_disc^2, so it falls
 * within the band with probability ~ 2 band phi((q - thr)/s) / s, and an ADC
 * decision's fractional code with probability 2 band / lsb_e; p_tie = 1 - prod
 * (1 - p).  Tests use it to bound how many pixels a band may exclude.
 * Returns the number of hits (may exceed cap; only cap are written). */
int64_t ora_electronics(const ora_cfg *c, uint64_t event_id, int32_t pixel, const double *I,
                        int64_t cap, int32_t *t_cross, int32_t *t_adc, int32_t *adc,
                        double *qv, double band, int32_t *tie_tick, double *p_tie)
{
    const double sd = sqrt(c->s_unc * c->s_unc + c->s_disc * c->s_disc);
    double log_none = 0.0;                     /* log P(no decision within the band) */
    int T = c->n_ticks;
    double lsb_e = c->gain * c->lsb_mV;
    int adc_max = (1 << c->adc_bits) - 1;
    double q = 0.0;
    int idle = 1;
    int64_t last_adc = -(int64_t)1 << 40;
    int64_t tc = -1, ta = -1;
    int64_t nh = 0;
    int32_t tie = -1;
    for (int k = 0; k < T; ++k) {
        double n[4];
        if (c->periodic > 0 && idle && k > 0 && k % c->periodic == 0) {
            ora_normals(c->seed, event_id, (uint32_t)pixel, (uint32_t)k, 4u, 0u, n);
            q = c->s_reset * n[0];
        }
        q += I[k];
        ora_normals(c->seed, event_id, (uint32_t)pixel, (uint32_t)k, 2u, 0u, n);
        if (idle) {
            double v = q + c->s_unc * n[0];
            double thr = c->thr + c->s_disc * n[1];
            if (tie < 0 && fabs(v - thr) < band) tie = k;
            if (p_tie && sd > 0.0) {
                double z = (q - c->thr) / sd;
                double p = 2.0 * band * exp(-0.5 * z * z) / (sd * sqrt(2.0 * ORA_PI));
                log_none += log1p(-(p < 1.0 ? p : 1.0 - 1e-16));
            }
            if (v >= thr) {
                tc = k;
                ta = k + c->hold;
                if (last_adc + c->min_int > ta) ta = last_adc + c->min_int;
                idle = 0;
            }
        }
        if (!idle && k == ta) {
            double v = q + c->s_unc * n[0];
            double code = floor(v / lsb_e);
            if (tie < 0 && fabs(v / lsb_e - floor(v / lsb_e + 0.5)) * lsb_e < band) tie = k;
            if (p_tie) {
                double p = 2.0 * band / lsb_e;
                log_none += log1p(-(p < 1.0 ? p : 1.0 - 1e-16));
            }
            if (code < 0) code = 0;
            if (code > adc_max) code = adc_max;
            if (nh < cap) {
                t_cross[nh] = (int32_t)tc;
                t_adc[nh] = (int32_t)ta;
                adc[nh] = (int32_t)code;
                qv[nh] = v;
            }
            ++nh;
            double m[4];
            ora_normals(c->seed, event_id, (uint32_t)pixel, (uint32_t)k, 3u, 0u, m);
            q = c->s_reset * m[0];
            last_adc = k;
            idle = 1;
        }
    }
    if (tie_tick) *tie_tick = tie;
    if (p_tie) *p_tie = -expm1(log_none);
    return nh;
}

/* ------------------------------------------------------- whole events -- */

/* Host threads the many-pixel functions use for a request of n_threads
 * (0 = all available); 1 when the library was built without OpenMP. */
int ora_threads(int n_threads)
{
#ifdef _OPENMP
    return n_threads > 0 ? n_threads : omp_get_max_threads();
#else
    (void)n_threads;
    return 1;
#endif
}

/* Map of every segment of an event (Sec. 3.3.2): the pairs of
 * ora_map_segment_box, segment by segment in increasing segment order, pixel
 * ids increasing within a segment.  Writes up to cap pairs (segment index,
 * pixel id, margin R_map - d) and returns the number of pairs (which may
 * exceed cap). */
int64_t ora_map_event(const ora_cfg *c, int64_t n, const float *x0, const float *y0, const float *x1,
                      const float *y1, const double *sigma_T, const int32_t *anode, int64_t cap,
                      int64_t *pair_seg, int32_t *pair_pix, double *pair_margin)
{
    int64_t bcap = 4096;
    int32_t *ids = (int32_t *)malloc(sizeof(int32_t) * (size_t)bcap);
    double *mg = (double *)malloc(sizeof(double) * (size_t)bcap);
    int64_t total = 0;
    for (int64_t s = 0; s < n; ++s) {
        if (anode[s] < 0) continue;
        int64_t m = ora_map_segment_box(c, x0[s], y0[s], x1[s], y1[s], sigma_T[s], anode[s], ids, mg, bcap);
        if (m > bcap) {
            bcap = m;
            ids = (int32_t *)realloc(ids, sizeof(int32_t) * (size_t)bcap);
            mg = (double *)realloc(mg, sizeof(double) * (size_t)bcap);
            m = ora_map_segment_box(c, x0[s], y0[s], x1[s], y1[s], sigma_T[s], anode[s], ids, mg, bcap);
        }
        for (int64_t j = 0; j < m; ++j, ++total) {
            if (total < cap) {
                pair_seg[total] = s;
                pair_pix[total] = ids[j];
                pair_margin[total] = mg[j];
            }
        }
    }
    free(ids);
    free(mg);
    return total;
}

/* ora_pixel_current of n_pix pixels: pixel pixels[i] with the segment list
 * segs[off[i] .. off[i+1]) writes row i of I [n_pix][n_ticks]. */
void ora_pixel_currents_many(const ora_cfg *c, const double *lut,
                             const float *x0, const float *y0, const float *z0, const float *t0,
                             const float *x1, const float *y1, const float *z1, const float *t1,
                             const double *Qa, const double *t_drift, const double *sigma_T,
                             const double *sigma_L, const int32_t *anode, const int32_t *n_samples,
                             uint64_t event_id, int64_t n_pix, const int32_t *pixels, const int64_t *off,
                             const int64_t *segs, double *I, int n_threads)
{
    (void)n_threads;
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 1) num_threads(ora_threads(n_threads))
#endif
    for (int64_t i = 0; i < n_pix; ++i)
        ora_pixel_current(c, lut, x0, y0, z0, t0, x1, y1, z1, t1, Qa, t_drift, sigma_T, sigma_L, anode,
                          n_samples, event_id, pixels[i], segs + off[i], off[i + 1] - off[i],
                          I + (size_t)i * (size_t)c->n_ticks, 0.0, NULL);
}

/* ora_electronics of n_pix pixels: pixel pixels[i] with the current row i of
 * I and tie band band[i] (NULL: 0) writes up to cap hits to entries
 * [i cap, (i+1) cap) of the hit arrays, its hit count to n_hits[i], its
 * first tied tick to tie_tick[i] and its tie probability to p_tie[i] (if
 * non-null). */
void ora_electronics_many(const ora_cfg *c, uint64_t event_id, int64_t n_pix, const int32_t *pixels,
                          const double *I, const double *band, int64_t cap, int32_t *t_cross, int32_t *t_adc,
                          int32_t *adc, double *qv, int64_t *n_hits, int32_t *tie_tick, double *p_tie,
                          int n_threads)
{
    (void)n_threads;
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 4) num_threads(ora_threads(n_threads))
#endif
    for (int64_t i = 0; i < n_pix; ++i) {
        const size_t o = (size_t)i * (size_t)cap;
        n_hits[i] = ora_electronics(c, event_id, pixels[i], I + (size_t)i * (size_t)c->n_ticks, cap, t_cross + o,
                                    t_adc + o, adc + o, qv + o, band ? band[i] : 0.0, tie_tick + i,
                                    p_tie ? p_tie + i : NULL);
    }
}

/* ------------------------------------------------- per-hit charge truth -- */

/* Integration interval [k0, k1] of each hit of one pixel, hits in tick order
 * (Sec. 3.4: the CSA integrates the current from its last reset until the
 * ADC samples it).  The interval ends at the hit's ADC tick.  It starts after
 * the previous hit's ADC tick (that conversion reset the CSA), or at the
 * window start for the pixel's first hit, or, when periodic resets are on, at
 * the latest reset tick r = j * period (0 < r <= the crossing tick) after it:
 * a reset at tick r clears the charge before tick r's current is added, and
 * resets only happen while the front end is idle, i.e. before the crossing. */
void ora_hit_intervals(const ora_cfg *c, int64_t n, const int32_t *t_cross, const int32_t *t_adc,
                       int32_t *k0, int32_t *k1)
{
    int64_t prev_end = -1;
    for (int64_t h = 0; h < n; ++h) {
        int64_t start = prev_end + 1;
        if (c->periodic > 0) {
            int64_t r = ((int64_t)t_cross[h] / c->periodic) * c->periodic;
            if (r > 0 && r > start) start = r;
        }
        k0[h] = (int32_t)start;
        k1[h] = t_adc[h];
        prev_end = t_adc[h];
    }
}

/* ------------------------------------------------------ hits -> 3-D points -- */

/* 3-D point of a hit (Sec. 6, the reconstruction's input): x and y at the
 * centre of the hit's pixel, z from the hit's crossing tick by the inverse of
 * Eq. (drift): the tick starts at t = t_w0 + t_cross * tick, the charge
 * drifted for t - t_event, and z = z_anode + v_d (t - t_event) for the anode
 * at z = 0 (TPC 0), z_anode - v_d (t - t_event) for the anode at z = 2D. */
void ora_hit_point(const ora_cfg *c, int32_t pixel, int32_t t_cross, double t_event, double out[3])
{
    double xc, yc, za;
    int32_t anode;
    ora_pixel_centre(c, pixel, &xc, &yc, &za, &anode);
    double t = c->t_w0 + (double)t_cross * c->tick;
    double dz = c->vdrift * (t - t_event);
    out[0] = xc;
    out[1] = yc;
    out[2] = za == 0.0 ? za + dz : za - dz;
}

/* dQ/dx along a known straight track (Sec. 6: the charge of the hits of a
 * track per unit length, in pieces of fixed length).  The track starts at o
 * with unit direction u; a point p at arc length s = (p - o) . u and distance
 * d = |p - o - s u| from the line belongs to piece floor(s / dx) when
 * 0 <= s < n_bins dx and d <= r_max.  dq[b] = sum of the charges of piece b,
 * cnt[b] = its points; margin[i] = distance (cm) of point i's decisions from
 * the nearest edge (a piece boundary or r_max), so that tests can exclude
 * points whose assignment a rounding could flip. */
void ora_track_dqdx(int64_t n, const double *x, const double *y, const double *z, const double *q,
                    const double o[3], const double u[3], double dx, int32_t n_bins, double r_max,
                    double *dq, int64_t *cnt, double *margin)
{
    for (int32_t b = 0; b < n_bins; ++b) {
        dq[b] = 0.0;
        cnt[b] = 0;
    }
    for (int64_t i = 0; i < n; ++i) {
        double px = x[i] - o[0], py = y[i] - o[1], pz = z[i] - o[2];
        double s = px * u[0] + py * u[1] + pz * u[2];
        double ex = px - s * u[0], ey = py - s * u[1], ez = pz - s * u[2];
        double d = sqrt(ex * ex + ey * ey + ez * ez);
        double fb = floor(s / dx);
        double m = fabs(d - r_max);
        double ms = fmin(fabs(s - fb * dx), fabs((fb + 1.0) * dx - s));
        if (ms < m) m = ms;
        margin[i] = m;
        if (d > r_max || s < 0.0 || fb >= (double)n_bins) continue;
        int32_t b = (int32_t)fb;
        dq[b] += q[i];
        cnt[b] += 1;
    }
}

/* ================================================================ light == */
/* Sec. 4: scintillation light on the same segments.  Tables (synthetic
 * stand-ins for the Geant4 visibility / arrival-time tables) are inputs:
 * vis [nv][n_det], tdist [nv][n_det][nt] with nv = nvx * nvy * nvz voxels of
 * one TPC in local coordinates (x, y from the module corner, z = distance
 * from the anode). */
typedef struct ora_light {
    int32_t nvx, nvy, nvz, n_det, nt, n_ticks, n_trunc, n_resp, noise_block, adc_bits;
    double vox, w_ph, tick, t_start;
    double fast_frac, tau_fast, tau_slow, poisson_max;
    double sample, pedestal;
} ora_light;

size_t ora_light_size(void) { return sizeof(ora_light); }

/* Sec. 4.1: photons of one segment, N_gamma = (1/W_ph - R/W_ion) dE, i.e.
 * dE / W_ph - Q_R (Q_R = R dE / W_ion, the quenched ionisation of Sec. 3.1),
 * and the photoelectrons of each photosensor of its TPC,
 * N_pe,i = eps_i V_i[voxel] N_gamma, with the voxel of the segment's
 * midpoint; the arrival tick shift floor((t_mid - t_start) / tick) of its
 * midpoint time.  The voxel and the tick are integer decisions taken in FP32
 * (the precision the GPU decides them in) with IEEE single operations in the
 * order written.  Returns 0 for an inactive segment (anode < 0). */
int ora_light_segment(const ora_cfg *c, const ora_light *L, const float *p /* x0 y0 z0 t0 x1 y1 z1 t1 dE */,
                      double QR, int32_t anode, const double *vis, const double *eff, double *npe,
                      int32_t *tick, int32_t *vox)
{
    for (int k = 0; k < L->n_det; ++k) npe[k] = 0.0;
    *tick = 0;
    *vox = -1;
    if (anode < 0) return 0;
    int32_t tpc = anode % c->n_tpc, m = anode / c->n_tpc;
    int32_t mx = m % c->n_mod_x, my = m / c->n_mod_x;
    float pitch = (float)c->pitch, D = (float)c->drift_len;
    float Wx = (float)(c->tiles_x * c->px_per_tile) * pitch;
    float Wy = (float)(c->tiles_y * c->px_per_tile) * pitch;
    float xm = 0.5f * (p[0] + p[4]), ym = 0.5f * (p[1] + p[5]), zm = 0.5f * (p[2] + p[6]);
    float tm = 0.5f * (p[3] + p[7]);
    float xl = xm - (float)mx * Wx, yl = ym - (float)my * Wy;
    float za = tpc == 0 ? 0.0f : 2.0f * D;
    float zl = fabsf(zm - za);
    float vx = (float)L->vox;
    int ix = (int)floorf(xl / vx), iy = (int)floorf(yl / vx), iz = (int)floorf(zl / vx);
    if (ix < 0) ix = 0;
    if (ix > L->nvx - 1) ix = L->nvx - 1;
    if (iy < 0) iy = 0;
    if (iy > L->nvy - 1) iy = L->nvy - 1;
    if (iz < 0) iz = 0;
    if (iz > L->nvz - 1) iz = L->nvz - 1;
    int v = (ix * L->nvy + iy) * L->nvz + iz;
    *vox = v;
    *tick = (int32_t)floorf((tm - (float)L->t_start) / (float)L->tick);
    double ngam = (double)p[8] / L->w_ph - QR;
    if (ngam < 0.0) ngam = 0.0;
    for (int k = 0; k < L->n_det; ++k) npe[k] = eff[k] * vis[(size_t)v * L->n_det + k] * ngam;
    return 1;
}

/* Sec. 4.2, Eq. (photocurrent) with equal table and simulation ticks: the
 * expected photoelectrons of photosensor k of anode a arriving in tick t,
 * I[t] = sum over the anode's segments j of f[vox_j][k][t - tick_j] N_pe,jk,
 * for 0 <= t - tick_j < nt; summed in segment order. */
void ora_light_photocurrent(const ora_light *L, int64_t n, const double *npe, const int32_t *tick,
                            const int32_t *vox, const int32_t *anode, const double *tdist, int32_t a, int32_t k,
                            double *I)
{
    for (int t = 0; t < L->n_ticks; ++t) I[t] = 0.0;
    for (int64_t j = 0; j < n; ++j) {
        if (anode[j] != a || vox[j] < 0) continue;
        double q = npe[j * L->n_det + k];
        const double *f = tdist + ((size_t)vox[j] * L->n_det + k) * L->nt;
        for (int u = 0; u < L->nt; ++u) {
            int64_t t = (int64_t)tick[j] + u;
            if (t >= 0 && t < L->n_ticks) I[t] += q * f[u];
        }
    }
}

/* Sec. 4.2, the truncated scintillation convolution:
 * S[t] = sum_{u=0}^{min(t, n_trunc)} I[t - u] f_scint(u tick), with
 * f_scint(t) = f_p / tau_p e^(-t / tau_p) + (1 - f_p) / tau_s e^(-t / tau_s)
 * (a rate: photoelectrons per us). */
void ora_light_scintillation(const ora_light *L, const double *I, double *S)
{
    for (int t = 0; t < L->n_ticks; ++t) {
        double s = 0.0;
        int umax = t < L->n_trunc ? t : L->n_trunc;
        for (int u = 0; u <= umax; ++u) {
            double tu = (double)u * L->tick;
            double f = L->fast_frac / L->tau_fast * exp(-tu / L->tau_fast) +
                       (1.0 - L->fast_frac) / L->tau_slow * exp(-tu / L->tau_slow);
            s += I[t - u] * f;
        }
        S[t] = s;
    }
}

/* Sec. 4.2, counting fluctuations: the observed photoelectrons of tick t of
 * photosensor `det` (global id), from the mean lambda = S[t] tick: for
 * lambda <= poisson_max, inverse transform sampling of the Poisson law with
 * the uniform u of Philox block (det, t, 5, 0) (the smallest n with
 * u <= F(n), F the Poisson CDF accumulated term by term, at most 1000 terms);
 * above, a normal N(lambda, sqrt(lambda)) from the Box-Muller pair of block
 * (det, t, 6, 0), floored at 0.  margin[t]: the distance of the decisions
 * from their thresholds (|u - F| at the last two comparisons; |lambda - max|). */
void ora_light_fluctuate(const ora_cfg *c, const ora_light *L, uint64_t event_id, int32_t det, const double *S,
                         double *nout, double *margin)
{
    uint32_t key[2] = {(uint32_t)((c->seed ^ event_id) & 0xFFFFFFFFu), (uint32_t)((c->seed ^ event_id) >> 32)};
    for (int t = 0; t < L->n_ticks; ++t) {
        double lam = S[t] * L->tick;
        double mg = fabs(lam - L->poisson_max);
        if (lam <= L->poisson_max) {
            uint32_t ctr[4] = {(uint32_t)det, (uint32_t)t, 5u, 0u}, x[4];
            ora_philox4x32_10(ctr, key, x);
            double u = ora_u01(x[0]);
            double pk = exp(-lam), F = pk;
            int k = 0;
            double m2 = fabs(u - F);
            while (u > F && k < 1000) {
                ++k;
                pk *= lam / (double)k;
                F += pk;
                double d = fabs(u - F);
                m2 = d;
                if (k >= 1) {
                    /* the previous comparison (u > F_prev) also decided */
                    double dp = fabs(u - (F - pk));
                    if (dp < m2) m2 = dp;
                }
            }
            if (m2 < mg) mg = m2;
            nout[t] = (double)k;
        } else {
            double nn[4];
            ora_normals(c->seed, event_id, (uint32_t)det, (uint32_t)t, 6u, 0u, nn);
            double v = lam + sqrt(lam) * nn[0];
            nout[t] = v > 0.0 ? v : 0.0;
        }
        margin[t] = mg;
    }
}

/* Sec. 4.3, Eq. (light response) with equal response and simulation ticks:
 * V[t] = noise(t) + G sum_{u=0}^{n_resp-1} n[t - u] resp[u], and the noise of
 * each block of noise_block ticks, b = t / N, tau = t - b N:
 * noise(t) = sum_{k=0}^{N/2} A_k cos(2 pi k tau / N + phi_k), phi_k = 2 pi u
 * with u of Philox block (det, b, 7, k).  Then the digitiser: sample m at
 * position p = m * ratio (ratio = sampling period / tick) read linearly
 * between ticks floor(p) and floor(p) + 1, code = clamp(floor(v + pedestal +
 * 1/2), 0, 2^bits - 1); margin[m] = distance of v + pedestal + 1/2 from the
 * nearest integer. */
void ora_light_electronics(const ora_cfg *c, const ora_light *L, uint64_t event_id, int32_t det, double gain,
                           const double *n, const double *resp, const double *amp, double ratio,
                           int32_t n_samples, double *V, double *vs, int32_t *code, double *margin)
{
    uint32_t key[2] = {(uint32_t)((c->seed ^ event_id) & 0xFFFFFFFFu), (uint32_t)((c->seed ^ event_id) >> 32)};
    int N = L->noise_block;
    int nblk = (L->n_ticks + N - 1) / N;
    double *phi = (double *)malloc(sizeof(double) * (size_t)(N / 2 + 1));
    for (int b = 0; b < nblk; ++b) {
        for (int k = 0; k <= N / 2; ++k) {
            uint32_t ctr[4] = {(uint32_t)det, (uint32_t)b, 7u, (uint32_t)k}, x[4];
            ora_philox4x32_10(ctr, key, x);
            phi[k] = 2.0 * ORA_PI * ora_u01(x[0]);
        }
        for (int tau = 0; tau < N; ++tau) {
            int t = b * N + tau;
            if (t >= L->n_ticks) break;
            double s = 0.0;
            for (int k = 0; k <= N / 2; ++k) s += amp[k] * cos(2.0 * ORA_PI * (double)k * (double)tau / (double)N + phi[k]);
            double r = 0.0;
            for (int u = 0; u < L->n_resp && u <= t; ++u) r += n[t - u] * resp[u];
            V[t] = s + gain * r;
        }
    }
    free(phi);
    double top = (double)((1 << L->adc_bits) - 1);
    for (int m = 0; m < n_samples; ++m) {
        double p = (double)m * ratio;
        double fl = floor(p);
        int i = (int)fl;
        double fr = p - fl;
        double v = i + 1 < L->n_ticks ? (1.0 - fr) * V[i] + fr * V[i + 1] : V[i];
        vs[m] = v;
        double w = v + L->pedestal + 0.5;
        double cd = floor(w);
        margin[m] = fmin(w - cd, cd + 1.0 - w);
        if (cd < 0.0) cd = 0.0;
        if (cd > top) cd = top;
        code[m] = (int32_t)cd;
    }
}

/* Sec. 4.4 (the default light truth): with the photoelectrons of each
 * segment and photosensor (ora_light_segment), their mean arrival time on the
 * simulation's tick grid, before the scintillation delay:
 * t = t_start + (tick_j + sum_u (u + 1/2) f[vox_j][k][u]) tick.  Inactive
 * segments (vox < 0) get 0. */
void ora_light_truth(const ora_light *L, int64_t n, const int32_t *tick, const int32_t *vox, const double *tdist,
                     double *t_arr)
{
    for (int64_t j = 0; j < n; ++j) {
        for (int k = 0; k < L->n_det; ++k) {
            if (vox[j] < 0) {
                t_arr[j * L->n_det + k] = 0.0;
                continue;
            }
            const double *f = tdist + ((size_t)vox[j] * L->n_det + k) * L->nt;
            double m = 0.0;
            for (int u = 0; u < L->nt; ++u) m += ((double)u + 0.5) * f[u];
            t_arr[j * L->n_det + k] = L->t_start + ((double)tick[j] + m) * L->tick;
        }
    }
}
