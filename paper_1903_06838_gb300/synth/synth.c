/*
 * synth.c — seeded synthetic pixel-detector frames with ground truth.
 *
 * Input generator only: it models what a detector records (pedestal,
 * per-unit common-mode offset, Gaussian electronic noise, photons whose
 * charge cloud spreads over a 3x3 neighbourhood) and holds none of the
 * correction chain's arithmetic.  Both the CPU oracle and the CUDA path
 * consume its output.
 *
 * Random numbers come from SplitMix64 (Steele, Lea and Flood, "Fast
 * splittable pseudorandom number generators", OOPSLA 2014): a 64-bit
 * counter advanced by the golden-ratio increment and finalised by the
 * published two-multiply mix.  Every (frame, module, purpose) triple has
 * its own stream, keyed by hashing those indices with the seed, so a
 * frame's content does not depend on which other frames are generated.
 * Normal deviates use the Box-Muller transform; Poisson counts use
 * inversion of the CDF with one uniform.
 *
 * Charge cloud: a photon landing at continuous position (x, y) with cloud
 * width sigma deposits, in the pixel at column offset i and row offset j
 * (i, j in {-1, 0, 1}) from its landing pixel, the fraction
 * fx(i) * fy(j), where fx(i) is the Gaussian mass over that column's
 * extent (from erf), renormalised over the three columns so the 3x3
 * fractions sum to one.  Deposits are in ADU: energy * gain of the
 * receiving pixel.  Pixels outside the module receive nothing (the charge
 * is lost), matching a sensor edge.
 *
 * Build: gcc -O2 -fPIC -shared -ffp-contract=off synth.c -lm
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
    uint32_t n_modules, rows, cols, unit_rows, unit_cols, reserved;
    double ped_mean, ped_sigma;   /* pedestal per pixel, ADU               */
    double gain_mean, gain_sigma; /* relative gain per pixel               */
    double adu_per_kev;           /* nominal gain, ADU per keV             */
    double noise_sigma;           /* electronic noise per pixel, ADU       */
    double cm_sigma;              /* common-mode offset per unit, ADU      */
    double occ_lo, occ_hi;        /* mean photons per pixel per frame;
                                     log-uniform per frame when hi > lo    */
    double photon_kev;            /* photon energy                         */
    double cloud_lo, cloud_hi;    /* cloud sigma in pixels; uniform per
                                     photon when hi > lo                   */
    double multi_frac;            /* probability that a landing site gets
                                     1-3 extra photons at the same spot    */
    uint64_t seed;
} ps_config;

typedef struct {
    uint32_t frame, module;
    float x, y;     /* landing position: column / row coordinate in module */
    float kev;      /* energy deposited inside the module                  */
    float sigma;    /* cloud width used                                    */
} ps_photon;

enum { TAG_PED = 1, TAG_GAIN = 2, TAG_CM = 3, TAG_NOISE = 4, TAG_PHOT = 5,
       TAG_OCC = 6 };

typedef struct { uint64_t s; int have; double spare; } rng_t;

static uint64_t mix64(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

static uint64_t next64(rng_t* r) {
    r->s += 0x9E3779B97F4A7C15ull;
    return mix64(r->s);
}

static rng_t stream(uint64_t seed, uint64_t tag, uint64_t a, uint64_t b) {
    rng_t r;
    uint64_t k = mix64(seed ^ 0x5851F42D4C957F2Dull);
    k = mix64(k ^ (tag * 0xD1B54A32D192ED03ull));
    k = mix64(k ^ (a * 0x8CB92BA72F3D8DD7ull));
    k = mix64(k ^ (b * 0xABC98388FB8FAC03ull));
    r.s = k;
    r.have = 0;
    r.spare = 0.0;
    return r;
}

/* uniform in the open interval (0, 1) */
static double unif(rng_t* r) {
    return ((double)(next64(r) >> 11) + 0.5) * (1.0 / 9007199254740992.0);
}

static double gauss(rng_t* r) {
    if (r->have) { r->have = 0; return r->spare; }
    double u1 = unif(r), u2 = unif(r);
    double rad = sqrt(-2.0 * log(u1));
    double th = 6.283185307179586 * u2;
    r->spare = rad * sin(th);
    r->have = 1;
    return rad * cos(th);
}

static int poisson(rng_t* r, double lam) {
    double u = unif(r);
    double p = exp(-lam), c = p;
    int k = 0;
    while (u > c && k < 64) {
        k++;
        p *= lam / k;
        c += p;
    }
    return k;
}

/* Gaussian mass of [a, b) for a cloud centred at x with width s */
static double gmass(double a, double b, double x, double s) {
    const double k = 0.7071067811865476 / s;
    return 0.5 * (erf((b - x) * k) - erf((a - x) * k));
}

int ps_check(const ps_config* c) {
    if (!c || !c->n_modules || !c->rows || !c->cols || !c->unit_rows ||
        !c->unit_cols)
        return 1;
    if (c->rows % c->unit_rows || c->cols % c->unit_cols) return 1;
    return 0;
}

/* Pedestal (ADU) and gain (ADU/keV) maps, float32 [n_modules][rows][cols]. */
int ps_maps(const ps_config* c, float* ped, float* gain) {
    if (ps_check(c)) return 1;
    const size_t mpx = (size_t)c->rows * c->cols;
    for (uint32_t m = 0; m < c->n_modules; m++) {
        rng_t rp = stream(c->seed, TAG_PED, m, 0);
        rng_t rg = stream(c->seed, TAG_GAIN, m, 0);
        for (size_t p = 0; p < mpx; p++) {
            ped[m * mpx + p] = (float)(c->ped_mean + c->ped_sigma * gauss(&rp));
            gain[m * mpx + p] = (float)((c->gain_mean + c->gain_sigma *
                                                        gauss(&rg)) *
                                        c->adu_per_kev);
        }
    }
    return 0;
}

/* Occupancy of absolute frame index f. */
double ps_frame_occupancy(const ps_config* c, uint32_t f) {
    if (!(c->occ_hi > c->occ_lo)) return c->occ_lo;
    rng_t r = stream(c->seed, TAG_OCC, f, 0);
    double lo = log(c->occ_lo), hi = log(c->occ_hi);
    return exp(lo + unif(&r) * (hi - lo));
}

/* Generate frames [f0, f0 + n) into raw (uint16 [n][modules][rows][cols]).
 * If cm_out is not NULL it receives the injected common-mode offsets
 * (double [n][units]).  Photons are written to truth (up to cap records);
 * the return value is the total number of photons (may exceed cap), or -1
 * on invalid input.  scratch: double [rows*cols] work buffer or NULL. */
long long ps_frames(const ps_config* c, const float* ped, const float* gain,
                    uint32_t f0, uint32_t n, uint16_t* raw, double* cm_out,
                    ps_photon* truth, long long cap) {
    if (ps_check(c)) return -1;
    const uint32_t R = c->rows, C = c->cols;
    const size_t mpx = (size_t)R * C;
    const uint32_t ucols = C / c->unit_cols, urows = R / c->unit_rows;
    const uint32_t upm = ucols * urows;
    double* acc = (double*)malloc(mpx * sizeof(double));
    double* off = (double*)malloc((size_t)upm * sizeof(double));
    if (!acc || !off) { free(acc); free(off); return -1; }
    long long nph = 0;
    for (uint32_t fi = 0; fi < n; fi++) {
        const uint32_t f = f0 + fi;
        const double occ = ps_frame_occupancy(c, f);
        for (uint32_t m = 0; m < c->n_modules; m++) {
            const float* pm = ped + m * mpx;
            const float* gm = gain + m * mpx;
            rng_t rc = stream(c->seed, TAG_CM, f, m);
            for (uint32_t u = 0; u < upm; u++) off[u] = c->cm_sigma * gauss(&rc);
            if (cm_out)
                for (uint32_t u = 0; u < upm; u++)
                    cm_out[((size_t)fi * c->n_modules + m) * upm + u] = off[u];
            rng_t rn = stream(c->seed, TAG_NOISE, f, m);
            for (uint32_t r = 0; r < R; r++) {
                const uint32_t ur = r / c->unit_rows;
                for (uint32_t q = 0; q < C; q++) {
                    const size_t p = (size_t)r * C + q;
                    acc[p] = (double)pm[p] + off[ur * ucols + q / c->unit_cols] +
                             c->noise_sigma * gauss(&rn);
                }
            }
            if (occ > 0.0) {
                rng_t rph = stream(c->seed, TAG_PHOT, f, m);
                for (uint32_t r = 0; r < R; r++) {
                    for (uint32_t q = 0; q < C; q++) {
                        int k = poisson(&rph, occ);
                        if (k && c->multi_frac > 0.0 && unif(&rph) < c->multi_frac)
                            k += 1 + (int)(unif(&rph) * 3.0);
                        double x = 0, y = 0, s = 0;
                        for (int i = 0; i < k; i++) {
                            /* extra photons of a multi-photon site share its
                               landing point and cloud */
                            if (i == 0 || !(c->multi_frac > 0.0)) {
                                x = q + unif(&rph);
                                y = r + unif(&rph);
                                s = c->cloud_lo;
                                if (c->cloud_hi > c->cloud_lo)
                                    s = c->cloud_lo +
                                        unif(&rph) * (c->cloud_hi - c->cloud_lo);
                            }
                            double fx[3], fy[3], sx = 0, sy = 0;
                            for (int d = -1; d <= 1; d++) {
                                /* signed pixel edges: q + d wraps in
                                   unsigned arithmetic at column / row 0 */
                                const double qe = (double)q + d, re = (double)r + d;
                                fx[d + 1] = gmass(qe, qe + 1.0, x, s);
                                fy[d + 1] = gmass(re, re + 1.0, y, s);
                                sx += fx[d + 1];
                                sy += fy[d + 1];
                            }
                            double kev_in = 0.0;
                            for (int dy = -1; dy <= 1; dy++) {
                                const long rr = (long)r + dy;
                                if (rr < 0 || rr >= (long)R) continue;
                                for (int dx = -1; dx <= 1; dx++) {
                                    const long cc = (long)q + dx;
                                    if (cc < 0 || cc >= (long)C) continue;
                                    const double fr = fx[dx + 1] / sx *
                                                      (fy[dy + 1] / sy);
                                    const size_t pp = (size_t)rr * C + cc;
                                    acc[pp] += c->photon_kev * fr * gm[pp];
                                    kev_in += c->photon_kev * fr;
                                }
                            }
                            if (truth && nph < cap) {
                                ps_photon* t = &truth[nph];
                                t->frame = f;
                                t->module = m;
                                t->x = (float)x;
                                t->y = (float)y;
                                t->kev = (float)kev_in;
                                t->sigma = (float)s;
                            }
                            nph++;
                        }
                    }
                }
            }
            uint16_t* out = raw + ((size_t)fi * c->n_modules + m) * mpx;
            for (size_t p = 0; p < mpx; p++) {
                double v = nearbyint(acc[p]);
                if (v < 0.0) v = 0.0;
                if (v > 65535.0) v = 65535.0;
                out[p] = (uint16_t)v;
            }
        }
    }
    free(acc);
    free(off);
    return nph;
}
