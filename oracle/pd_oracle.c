/*
 * pd_oracle.c — CPU oracle of the pixel-detector correction chain.
 *
 * TEST INFRASTRUCTURE.  This file defines what the chain computes; it is a
 * plain, slow, single-threaded restatement of the method, step by step, in
 * the paper's order.  Only the tests, the smoke check and the benchmark's
 * CPU-baseline leg may load it.  It shares no code, header or constant with
 * the CUDA library: its structs below mirror the public layout field by
 * field but are declared here.
 *
 * Paper: G. Blaj, C.-E. Chang, C. J. Kenney, "Ultrafast Processing of Pixel
 * Detector Data with Machine Learning Frameworks", AIP Conf. Proc. 2054,
 * 060077 (2019).  Section names below refer to it.
 *
 * Arithmetic: IEEE binary32, round to nearest, one rounding per written
 * operation (build with -ffp-contract=off, never -ffast-math).  For each
 * frame, each module in order:
 *
 *  1. Dark: d = (float)raw - pedestal                 (Fig. b, "Frames0")
 *  2. Common mode, per unit u (section "Common Mode", Fig. c): the set of
 *     pixels of u whose d < cm_cut ("pixels without signal" are segmented
 *     by a threshold).  With n pixels in the set and n >= n_min, cm_u is
 *     the element of rank floor((n-1)/2) of the set sorted ascending (the
 *     lower median; the paper's figure averages the set, the median is the
 *     robust estimator this library uses); otherwise cm_u = 0, which plays
 *     the role of the figure's sqrt(HW) guard against estimating from too
 *     few pixels.  n_min defaults to ceil(sqrt(unit pixels)).
 *     Ascending order is IEEE order refined so -0 sorts below +0.
 *     The paper's own estimator (Fig. c) is available too, as
 *     cm_mode = MEAN: per group of G pixels, N0 = number of values v with
 *     v < cm_cut (and v > -inf), S = their sum, and
 *     cm = S / max(N0, sqrt(G)); the sqrt(G) term keeps a group with few
 *     background pixels from correcting by a noisy estimate.  The sum is
 *     defined exactly, independent of order: with M the largest |v| of the
 *     set and E = max(floor(log2 M), -60), every v is rounded to the grid
 *     2^(E-38) (rint, ties to even), the integers are added exactly, and the
 *     total is rounded once to binary32.  Values down to M * 2^-15 lie on
 *     that grid, so for detector data the sum is the exactly rounded sum.
 *     cm_mode = MEAN_STACKED stacks three such stages, as the paper's
 *     benchmark model does (section "Performance"; the text of section
 *     "Common Mode" names row, column and block groups): stage 1 over each
 *     unit gives cm_u; stage 2 over each row of the module, on d - cm_u,
 *     gives cm_r; stage 3 over each column of the module, on
 *     (d - cm_u) - cm_r, gives cm_c.  G is the group's pixel count.
 *  3. c = d - cm_u  (stacked: c = ((d - cm_u) - cm_r) - cm_c)
 *  4. Gain: e = c * inv_gain with inv_gain = 1.0f / gain computed once
 *     (Fig. b divides by the gain map; the reciprocal is taken once per
 *     pixel); gain <= 0 or non-finite masks the pixel (inv_gain = 0).
 *  5. Noise zeroing (Fig. e "Signal? / Signal"): s = e > zero_thr ? e : 0.
 *  6. Seed (charge goes to the pixel with the highest signal, section
 *     "Photon Charge Summing"): p is a seed iff s_p > seed_thr and, for each
 *     of its 8 neighbours q inside the module, s_p > s_q when q comes before
 *     p in the module's raster order and s_p >= s_q when q comes after it.
 *     Neighbours outside the module do not exist (zero padding; since
 *     s_p > 0 they never block a seed).
 *  7. Charge sum: E = sum of s over the 3x3 around the seed (out-of-module
 *     terms are 0), accumulated row-major from 0.0f (Fig. e "Frames3").
 *     Photon count (same section, high-flux paragraph): n = rint(E /
 *     photon_kev), ties to even, clipped to [0, 255].  A hit is emitted iff
 *     n >= 1.
 *  8. Centroid (section "Photon Subpixel Resolution", Fig. f): with column
 *     offsets ox and row offsets oy in {-1, 0, 1},
 *     Mx = sum s_q * ox_q, My = sum s_q * oy_q in the same row-major order,
 *     dx = Mx / E, dy = My / E, in pixel pitches from the seed centre.
 *  9. Summaries (section "Summarization"): count_map[seed] += n for every
 *     hit; hist_pix[bin(e)] += 1 for every pixel; hist_hit[bin(E)] += 1 for
 *     every seed.  The paper does not define its bins; here bin b covers
 *     [lo + b*width, lo + (b+1)*width) in the sense bin(v) = floor(t) with
 *     t = fmaf(v, inv_w, -lo_s), inv_w = 1.0f / width and lo_s = lo * inv_w
 *     (each rounded to nearest once; fmaf rounds once), clipped to
 *     [0, bins-1].
 *
 * Matched filters (oracle_process_matched; section "Photon Charge
 * Summing", Figs. d and e; section "Photon Subpixel Resolution", Fig. f).
 * Steps 6.-8. are replaced by the paper's filter model, with a filter bank
 * supplied by the caller (the paper prints its values only as a picture).
 * Each of the bank's F features has four 4 x 5 filters F0, F1, F1dx, F1dy
 * and a threshold F1Nmin.  A filter is applied at pixel (r, c) as TF's
 * conv2d with "SAME" padding does for a 4 x 5 kernel: tap (i, j) meets the
 * pixel (r + i - 1, c + j - 2), zero outside the module; the taps are
 * accumulated row-major from 0.0f, each term a product.  With T = (s > 0)
 * (the "Signal?" mask; s > 0 iff e > zero_thr since zero_thr >= 0):
 *     Size_f     = sum T * F1_f        Droplet_f = sum s * F1_f
 *     Overflow_f = sum T * F0_f        Mx_f = sum s * F1dx_f,  My_f likewise
 *     Valid_f    = (Overflow_f == 0) and (Size_f >= F1Nmin_f)
 * and, over the valid features in order,
 *     E  = sum Droplet_f                        (Frames3)
 *     dx = sum Mx_f / Droplet_f,  dy = sum My_f / Droplet_f
 * where a feature whose Droplet_f is 0 adds nothing to dx, dy.  A pixel
 * with a valid feature and E != 0 counts as a seed (hist_hit[bin(E)]); its
 * count is n = rint(E / photon_kev) as in 7., a hit iff n >= 1, with npix
 * the number of signal pixels under the nonzero taps of the first valid
 * feature's F1.  The model is pinned (correlation against a library routine,
 * the alignment, hand-worked cloud shapes); the paper's own filter values are
 * not in its text, so parity with the paper's bank is unpinned.
 *
 * Auto-ranging multi-gain (oracle_process_ext with n_gains > 0; the
 * caption of Fig. b notes that several darks and gains per pixel are
 * accommodated the same way and does not show how).  Each raw word carries
 * its gain stage in its top bits: stage = raw >> gain_shift, value =
 * raw & (2^gain_shift - 1), and the pedestal and gain maps hold one map per
 * stage.  Step 1 becomes d = (float)value - pedestal[stage]; only stage-0
 * pixels enter the common-mode set (step 2 adds stage == 0 to d < cut);
 * step 3-4 become e = (d - cm_u) * inv_gain[0] for stage 0 and
 * e = d * inv_gain[stage] for the other stages (a pixel switched to a lower
 * gain carries a signal far above the common mode's scale); a stage
 * >= n_gains marks the pixel bad: e = 0.  Only the median and no common
 * mode are defined with several gains.
 *
 * The paper's order (cm_after_gain = 1; Fig. a lists gain before common
 * mode, and Fig. c takes the gain-corrected Frames1): step 4 comes first,
 * e0 = d * inv_gain, the common-mode set is {e0 < cm_cut_kev} over the
 * unit's unmasked pixels (inv_gain != 0), the estimators (median, mean,
 * stacked stages) work on e0 in keV exactly as on d, and e = e0 - cm_u
 * (stacked: ((e0 - cm_u) - cm_r) - cm_c); a masked pixel reads e = 0.  Not
 * defined with several gains.
 *
 * Inputs must be finite (pedestal finite; non-finite gains are masked).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
    uint32_t n_modules, rows, cols, unit_rows, unit_cols, cm_mode, cm_after_gain;
} og_geometry;

typedef struct {
    float cm_cut_adu, zero_thr_kev, seed_thr_kev, photon_kev;
    uint32_t cm_min_count;
    float hist_lo_kev, hist_bin_kev;
    uint32_t hist_bins;
    float cm_cut_kev;
} og_thresholds;

typedef struct {
    uint32_t frame, pixel;
    float energy_kev, dx, dy;
    uint8_t count, npix;
    uint16_t flags;
} og_hit;

enum { OG_CM_MEDIAN = 0, OG_CM_NONE = 1, OG_CM_MEAN = 2, OG_CM_MEAN_STACKED = 3 };
enum { OG_EDGE = 1, OG_SATURATED = 2 };

#define OG_MAX_FEATURES 8
typedef struct {
    uint32_t n_features;
    float f0[OG_MAX_FEATURES][4][5];
    float f1[OG_MAX_FEATURES][4][5];
    float f1_dx[OG_MAX_FEATURES][4][5];
    float f1_dy[OG_MAX_FEATURES][4][5];
    float f1_nmin[OG_MAX_FEATURES];
} og_filters;

static int filters_ok(const og_filters* fb) {
    if (fb->n_features < 1 || fb->n_features > OG_MAX_FEATURES) return 0;
    for (uint32_t f = 0; f < fb->n_features; f++) {
        if (isnan(fb->f1_nmin[f])) return 0;
        for (int i = 0; i < 4; i++)
            for (int j = 0; j < 5; j++)
                if (!isfinite(fb->f0[f][i][j]) || !isfinite(fb->f1[f][i][j]) ||
                    !isfinite(fb->f1_dx[f][i][j]) || !isfinite(fb->f1_dy[f][i][j]))
                    return 0;
    }
    return 1;
}

/* The 32-bit pattern of a float mapped so that unsigned comparison of the
 * keys is the ascending IEEE order with -0 below +0. */
static uint32_t order_key(float v) {
    uint32_t b;
    memcpy(&b, &v, 4);
    return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}

static int cmp_float(const void* a, const void* b) {
    uint32_t ka = order_key(*(const float*)a), kb = order_key(*(const float*)b);
    return (ka > kb) - (ka < kb);
}

/* smallest k with k*k >= n */
static uint32_t ceil_sqrt(uint32_t n) {
    uint32_t k = 0;
    while ((uint64_t)k * k < n) k++;
    return k;
}

uint32_t oracle_default_min_count(uint32_t unit_pixels) {
    return ceil_sqrt(unit_pixels);
}

static uint32_t bin_of(float v, float lo_s, float inv_w, uint32_t bins) {
    const float t = fmaf(v, inv_w, -lo_s);
    if (!(t >= 0.0f)) return 0;
    if (t >= (float)bins) return bins - 1;
    return (uint32_t)t; /* truncation == floor for t >= 0 */
}

/* Lower median of the values of `set` (n of them), sorted in place. */
float oracle_lower_median(float* set, uint32_t n) {
    qsort(set, n, sizeof(float), cmp_float);
    return set[(n - 1) / 2];
}

/* A value enters the paper's mean iff it is below the cut and not -inf. */
static int mean_selects(float v, float cut) { return v < cut && v > -INFINITY; }

/* The paper's common-mode estimator (Fig. c) over the n values of one
 * group, with the exactly defined sum of step 2 above.  Values that must
 * not enter the set (masked pixels in the paper's order) are passed as NaN,
 * which no comparison selects. */
float oracle_paper_mean(const float* v, uint32_t n, float cut) {
    uint32_t n0 = 0;
    float mx = 0.0f;
    for (uint32_t i = 0; i < n; i++) {
        if (!mean_selects(v[i], cut)) continue;
        n0++;
        if (fabsf(v[i]) > mx) mx = fabsf(v[i]);
    }
    float sum = 0.0f;
    if (n0 > 0 && mx > 0.0f) {
        int ex;
        frexpf(mx, &ex); /* mx = f * 2^ex, f in [0.5, 1) */
        int e = ex - 1;
        if (e < -60) e = -60;
        const int k = 38 - e;
        long long total = 0;
        for (uint32_t i = 0; i < n; i++)
            if (mean_selects(v[i], cut)) total += llrintf(ldexpf(v[i], k));
        sum = ldexpf((float)total, -k);
    }
    const float guard = sqrtf((float)n);
    const float den = (float)n0 > guard ? (float)n0 : guard;
    return sum / den;
}

/* Common-mode values per frame: units, then (stacked) module rows and
 * module columns. */
uint32_t oracle_cm_values_per_frame(const og_geometry* g) {
    const uint32_t units = g->n_modules * (g->rows / g->unit_rows) * (g->cols / g->unit_cols);
    if (g->cm_mode != OG_CM_MEAN_STACKED) return units;
    return units + g->n_modules * (g->rows + g->cols);
}

int oracle_check(const og_geometry* g, const og_thresholds* t) {
    if (!g || !t) return 1;
    if (!g->n_modules || !g->rows || !g->cols || !g->unit_rows ||
        !g->unit_cols)
        return 1;
    if (g->rows % g->unit_rows || g->cols % g->unit_cols) return 1;
    if (g->cm_mode > OG_CM_MEAN_STACKED || g->cm_after_gain > 1) return 1;
    if (g->cm_after_gain && isnan(t->cm_cut_kev)) return 1;
    /* the exact sum of the mean stays within 64 bits below 2^24 values */
    if (g->cm_mode >= OG_CM_MEAN &&
        ((uint64_t)g->unit_rows * g->unit_cols >= (1u << 24) || g->rows >= (1u << 24) ||
         g->cols >= (1u << 24)))
        return 1;
    if (!(t->zero_thr_kev >= 0.0f) || !(t->seed_thr_kev >= t->zero_thr_kev))
        return 1;
    if (!(t->photon_kev > 0.0f) || !(t->hist_bin_kev > 0.0f)) return 1;
    if (!isfinite(t->seed_thr_kev) || !isfinite(t->photon_kev) ||
        !isfinite(t->hist_lo_kev) || !isfinite(t->hist_bin_kev) ||
        isnan(t->cm_cut_adu))
        return 1;
    if (t->hist_bins < 1 || t->hist_bins > 4096) return 1;
    return 0;
}

/*
 * oracle_process — run the chain on n_frames raw frames.
 *   ped, gain:  float [n_modules][rows][cols] (ADU, ADU/keV)
 *   raw:        uint16 [n_frames][n_modules][rows][cols]
 *   hits:       up to cap records, written in (frame, module, row, col)
 *               order; *n_hits receives the true number of hits
 *   count_map:  u32 [pixels]   (accumulated, not cleared)
 *   hist_pix, hist_hit: u64 [hist_bins] (accumulated, not cleared)
 *   corrected:  float [n_frames][pixels] e values, or NULL
 *   cm_out:     float [n_frames][oracle_cm_values_per_frame] common mode
 *               (units, then for MEAN_STACKED n_modules x rows row terms
 *               and n_modules x cols column terms), or NULL
 *   n_seeds:    receives the number of seeds (hits plus seeds with n = 0),
 *               or NULL
 * Returns 0, or 1 on invalid input.
 */
static int process_impl(const og_geometry* g, const og_thresholds* t,
                        const og_filters* fb, uint32_t n_gains, uint32_t gain_shift,
                        const float* ped, const float* gain,
                        const uint16_t* raw, uint32_t n_frames, uint32_t frame_base,
                        og_hit* hits, uint32_t cap, uint32_t* n_hits, uint32_t* count_map,
                        uint64_t* hist_pix, uint64_t* hist_hit, float* corrected,
                        float* cm_out, uint64_t* n_seeds);

int oracle_process(const og_geometry* g, const og_thresholds* t,
                   const float* ped, const float* gain, const uint16_t* raw,
                   uint32_t n_frames, uint32_t frame_base, og_hit* hits,
                   uint32_t cap, uint32_t* n_hits, uint32_t* count_map,
                   uint64_t* hist_pix, uint64_t* hist_hit, float* corrected,
                   float* cm_out, uint64_t* n_seeds) {
    return process_impl(g, t, NULL, 0, 0, ped, gain, raw, n_frames, frame_base, hits, cap,
                        n_hits, count_map, hist_pix, hist_hit, corrected, cm_out, n_seeds);
}

/* The chain with the matched-filter charge summing of the bank fb. */
int oracle_process_matched(const og_geometry* g, const og_thresholds* t,
                           const og_filters* fb, const float* ped, const float* gain,
                           const uint16_t* raw, uint32_t n_frames, uint32_t frame_base,
                           og_hit* hits, uint32_t cap, uint32_t* n_hits,
                           uint32_t* count_map, uint64_t* hist_pix, uint64_t* hist_hit,
                           float* corrected, float* cm_out, uint64_t* n_seeds) {
    if (!fb || !filters_ok(fb)) return 1;
    return process_impl(g, t, fb, 0, 0, ped, gain, raw, n_frames, frame_base, hits, cap,
                        n_hits, count_map, hist_pix, hist_hit, corrected, cm_out, n_seeds);
}

/* The chain with an optional filter bank (NULL: 3x3 local maximum) and
 * n_gains gain stages (0: plain single-gain data; 1..4: auto-ranging words
 * with the stage in bits gain_shift.., pedestal and gain [n_gains][pixels]). */
int oracle_process_ext(const og_geometry* g, const og_thresholds* t, const og_filters* fb,
                       uint32_t n_gains, uint32_t gain_shift, const float* ped,
                       const float* gain, const uint16_t* raw, uint32_t n_frames,
                       uint32_t frame_base, og_hit* hits, uint32_t cap, uint32_t* n_hits,
                       uint32_t* count_map, uint64_t* hist_pix, uint64_t* hist_hit,
                       float* corrected, float* cm_out, uint64_t* n_seeds) {
    if (fb && !filters_ok(fb)) return 1;
    if (n_gains > 4 || (n_gains && (gain_shift < 1 || gain_shift > 15))) return 1;
    if (n_gains && g->cm_mode != OG_CM_MEDIAN && g->cm_mode != OG_CM_NONE) return 1;
    if (n_gains && g->cm_after_gain) return 1;
    return process_impl(g, t, fb, n_gains, gain_shift, ped, gain, raw, n_frames, frame_base,
                        hits, cap, n_hits, count_map, hist_pix, hist_hit, corrected, cm_out,
                        n_seeds);
}

/* The matched-filter model at pixel (r, c) of a module's zeroed signal s
 * (R x C).  Returns 1 when a feature is valid; fills E, dx, dy, npix. */
static int matched_at(const og_filters* fb, const float* s, uint32_t R, uint32_t C,
                      uint32_t r, uint32_t c, float* E_out, float* dx_out, float* dy_out,
                      uint32_t* npix_out) {
    float E = 0.0f, dx = 0.0f, dy = 0.0f;
    uint32_t npix = 0;
    int any = 0;
    for (uint32_t f = 0; f < fb->n_features; f++) {
        float size = 0.0f, over = 0.0f, drop = 0.0f, mx = 0.0f, my = 0.0f;
        uint32_t under = 0;
        for (int i = 0; i < 4; i++) {
            for (int j = 0; j < 5; j++) {
                const long rr = (long)r + i - 1, cc = (long)c + j - 2;
                float sv = 0.0f;
                if (rr >= 0 && rr < (long)R && cc >= 0 && cc < (long)C)
                    sv = s[(size_t)rr * C + cc];
                const float tv = sv > 0.0f ? 1.0f : 0.0f;
                size = size + tv * fb->f1[f][i][j];
                over = over + tv * fb->f0[f][i][j];
                drop = drop + sv * fb->f1[f][i][j];
                mx = mx + sv * fb->f1_dx[f][i][j];
                my = my + sv * fb->f1_dy[f][i][j];
                if (sv > 0.0f && fb->f1[f][i][j] != 0.0f) under++;
            }
        }
        if (!(over == 0.0f && size >= fb->f1_nmin[f])) continue;
        if (!any) npix = under;
        any = 1;
        E = E + drop;
        if (drop != 0.0f) {
            dx = dx + mx / drop;
            dy = dy + my / drop;
        }
    }
    *E_out = E;
    *dx_out = dx;
    *dy_out = dy;
    *npix_out = npix;
    return any;
}

static int process_impl(const og_geometry* g, const og_thresholds* t,
                        const og_filters* fb, uint32_t n_gains, uint32_t gain_shift,
                        const float* ped, const float* gain,
                        const uint16_t* raw, uint32_t n_frames, uint32_t frame_base,
                        og_hit* hits, uint32_t cap, uint32_t* n_hits, uint32_t* count_map,
                        uint64_t* hist_pix, uint64_t* hist_hit, float* corrected,
                        float* cm_out, uint64_t* n_seeds) {
    if (oracle_check(g, t)) return 1;
    /* one pedestal and gain map per stage; plain data is one stage of raw words */
    const uint32_t stages = n_gains ? n_gains : 1;
    const uint32_t vmask = n_gains ? (1u << gain_shift) - 1u : 0xFFFFu;
    const uint32_t sshift = n_gains ? gain_shift : 16;
    const int ag = g->cm_after_gain != 0;
    const float cut = ag ? t->cm_cut_kev : t->cm_cut_adu;
    const uint32_t R = g->rows, C = g->cols;
    const size_t mpx = (size_t)R * C;
    const size_t fpx = mpx * g->n_modules;
    const uint32_t urows = R / g->unit_rows, ucols = C / g->unit_cols;
    const uint32_t upm = urows * ucols;
    const uint32_t unit_px = g->unit_rows * g->unit_cols;
    const uint32_t n_min =
        t->cm_min_count ? t->cm_min_count : ceil_sqrt(unit_px);
    const float inv_w = 1.0f / t->hist_bin_kev;
    const float lo_s = t->hist_lo_kev * inv_w;

    float* inv_gain = (float*)malloc(stages * fpx * sizeof(float));
    uint8_t* stage = (uint8_t*)malloc(mpx);
    float* d = (float*)malloc(mpx * sizeof(float));
    float* e = (float*)malloc(mpx * sizeof(float));
    float* s = (float*)malloc(mpx * sizeof(float));
    const int stacked = g->cm_mode == OG_CM_MEAN_STACKED;
    const uint32_t cpf = oracle_cm_values_per_frame(g);
    const uint32_t upf = g->n_modules * upm;
    size_t set_n = unit_px;
    if (R > set_n) set_n = R;
    if (C > set_n) set_n = C;
    float* set = (float*)malloc(set_n * sizeof(float));
    float* cmu = (float*)malloc((size_t)upm * sizeof(float));
    float* cmr = (float*)calloc(R, sizeof(float));
    float* cmc = (float*)calloc(C, sizeof(float));
    if (!inv_gain || !stage || !d || !e || !s || !set || !cmu || !cmr || !cmc) {
        free(inv_gain); free(stage); free(d); free(e); free(s); free(set); free(cmu);
        free(cmr); free(cmc);
        return 1;
    }
    for (size_t p = 0; p < stages * fpx; p++) {
        if (!isfinite(ped[p])) {
            free(inv_gain); free(stage); free(d); free(e); free(s); free(set); free(cmu);
            free(cmr); free(cmc);
            return 1;
        }
        const float gp = gain[p];
        inv_gain[p] = (gp > 0.0f && isfinite(gp)) ? 1.0f / gp : 0.0f;
    }

    uint32_t nh = 0;
    uint64_t ns = 0;
    for (uint32_t f = 0; f < n_frames; f++) {
        for (uint32_t m = 0; m < g->n_modules; m++) {
            const size_t base = m * mpx;
            const uint16_t* rw = raw + (size_t)f * fpx + base;
            /* 1. dark (per gain stage); in the paper's order 4. gain first:
             * d then holds e0 = d * inv_gain, NaN for masked pixels so that
             * no common-mode set takes them */
            for (size_t p = 0; p < mpx; p++) {
                const uint32_t st = (uint32_t)rw[p] >> sshift;
                const uint32_t v = (uint32_t)rw[p] & vmask;
                stage[p] = (uint8_t)(st < stages ? st : 255);
                d[p] = st < stages ? (float)v - ped[(size_t)st * fpx + base + p] : 0.0f;
                if (ag) d[p] = inv_gain[base + p] != 0.0f ? d[p] * inv_gain[base + p] : NAN;
            }
            /* 2. common mode per unit */
            for (uint32_t ur = 0; ur < urows; ur++) {
                for (uint32_t uc = 0; uc < ucols; uc++) {
                    float cm = 0.0f;
                    if (g->cm_mode == OG_CM_MEDIAN) {
                        uint32_t n = 0;
                        for (uint32_t r = 0; r < g->unit_rows; r++) {
                            for (uint32_t c = 0; c < g->unit_cols; c++) {
                                const size_t p =
                                    (size_t)(ur * g->unit_rows + r) * C +
                                    uc * g->unit_cols + c;
                                if (stage[p] == 0 && d[p] < cut) set[n++] = d[p];
                            }
                        }
                        if (n >= n_min && n > 0) cm = oracle_lower_median(set, n);
                    } else if (g->cm_mode != OG_CM_NONE) {
                        uint32_t n = 0;
                        for (uint32_t r = 0; r < g->unit_rows; r++)
                            for (uint32_t c = 0; c < g->unit_cols; c++)
                                set[n++] = d[(size_t)(ur * g->unit_rows + r) * C +
                                             uc * g->unit_cols + c];
                        cm = oracle_paper_mean(set, n, cut);
                    }
                    cmu[ur * ucols + uc] = cm;
                    if (cm_out)
                        cm_out[(size_t)f * cpf + m * upm + ur * ucols + uc] = cm;
                }
            }
            if (stacked) {
                /* stage 2: each module row, on d - cm_u */
                for (uint32_t r = 0; r < R; r++) {
                    for (uint32_t c = 0; c < C; c++)
                        set[c] = d[(size_t)r * C + c] -
                                 cmu[(r / g->unit_rows) * ucols + c / g->unit_cols];
                    cmr[r] = oracle_paper_mean(set, C, cut);
                    if (cm_out) cm_out[(size_t)f * cpf + upf + (size_t)m * R + r] = cmr[r];
                }
                /* stage 3: each module column, on (d - cm_u) - cm_r */
                for (uint32_t c = 0; c < C; c++) {
                    for (uint32_t r = 0; r < R; r++)
                        set[r] = (d[(size_t)r * C + c] -
                                  cmu[(r / g->unit_rows) * ucols + c / g->unit_cols]) -
                                 cmr[r];
                    cmc[c] = oracle_paper_mean(set, R, cut);
                    if (cm_out)
                        cm_out[(size_t)f * cpf + upf + (size_t)g->n_modules * R +
                               (size_t)m * C + c] = cmc[c];
                }
            }
            /* 3.-5. subtract common mode, gain, zero noise; pixel histogram */
            for (uint32_t r = 0; r < R; r++) {
                for (uint32_t c = 0; c < C; c++) {
                    const size_t p = (size_t)r * C + c;
                    const float cm =
                        cmu[(r / g->unit_rows) * ucols + c / g->unit_cols];
                    float ev = 0.0f;
                    if (ag) {
                        if (inv_gain[base + p] != 0.0f) {
                            ev = d[p] - cm;
                            if (stacked) ev = (ev - cmr[r]) - cmc[c];
                        }
                    } else if (stage[p] == 0) {
                        float cc = d[p] - cm;
                        if (stacked) cc = (cc - cmr[r]) - cmc[c];
                        ev = cc * inv_gain[base + p];
                    } else if (stage[p] != 255) {
                        ev = d[p] * inv_gain[(size_t)stage[p] * fpx + base + p];
                    }
                    e[p] = ev;
                    s[p] = ev > t->zero_thr_kev ? ev : 0.0f;
                    hist_pix[bin_of(ev, lo_s, inv_w, t->hist_bins)]++;
                    if (corrected) corrected[(size_t)f * fpx + base + p] = ev;
                }
            }
            /* 6.-9. seeds, charge sum, count, centroid, summaries */
            for (uint32_t r = 0; fb && r < R; r++) {
                for (uint32_t c = 0; c < C; c++) {
                    float E, dxm, dym;
                    uint32_t npix;
                    if (!matched_at(fb, s, R, C, r, c, &E, &dxm, &dym, &npix)) continue;
                    if (E == 0.0f) continue;
                    ns++;
                    hist_hit[bin_of(E, lo_s, inv_w, t->hist_bins)]++;
                    const float qr = nearbyintf(E / t->photon_kev);
                    uint32_t n;
                    uint16_t flags = 0;
                    if (!(qr >= 0.0f)) n = 0;
                    else if (qr > 255.0f) { n = 255; flags |= OG_SATURATED; }
                    else n = (uint32_t)qr;
                    if (n < 1) continue;
                    if (r == 0 || c == 0 || r == R - 1 || c == C - 1) flags |= OG_EDGE;
                    const uint32_t pix = (uint32_t)(base + (size_t)r * C + c);
                    count_map[pix] += n;
                    if (nh < cap) {
                        og_hit* h = &hits[nh];
                        h->frame = frame_base + f;
                        h->pixel = pix;
                        h->energy_kev = E;
                        h->dx = dxm;
                        h->dy = dym;
                        h->count = (uint8_t)n;
                        h->npix = (uint8_t)(npix > 255 ? 255 : npix);
                        h->flags = flags;
                    }
                    nh++;
                }
            }
            for (uint32_t r = 0; !fb && r < R; r++) {
                for (uint32_t c = 0; c < C; c++) {
                    const size_t p = (size_t)r * C + c;
                    const float sp = s[p];
                    if (!(sp > t->seed_thr_kev)) continue;
                    int seed = 1;
                    for (int dy = -1; dy <= 1 && seed; dy++) {
                        for (int dx = -1; dx <= 1; dx++) {
                            if (!dy && !dx) continue;
                            const long rr = (long)r + dy, cc = (long)c + dx;
                            if (rr < 0 || rr >= (long)R || cc < 0 || cc >= (long)C)
                                continue;
                            const float sq = s[(size_t)rr * C + cc];
                            const int before = dy < 0 || (dy == 0 && dx < 0);
                            if (before ? !(sp > sq) : !(sp >= sq)) {
                                seed = 0;
                                break;
                            }
                        }
                    }
                    if (!seed) continue;
                    float E = 0.0f, Mx = 0.0f, My = 0.0f;
                    uint32_t npix = 0;
                    for (int dy = -1; dy <= 1; dy++) {
                        for (int dx = -1; dx <= 1; dx++) {
                            const long rr = (long)r + dy, cc = (long)c + dx;
                            float sq = 0.0f;
                            if (rr >= 0 && rr < (long)R && cc >= 0 && cc < (long)C)
                                sq = s[(size_t)rr * C + cc];
                            E = E + sq;
                            Mx = Mx + sq * (float)dx;
                            My = My + sq * (float)dy;
                            if (sq > 0.0f) npix++;
                        }
                    }
                    ns++;
                    hist_hit[bin_of(E, lo_s, inv_w, t->hist_bins)]++;
                    const float q = E / t->photon_kev;
                    const float qr = nearbyintf(q);
                    uint32_t n;
                    uint16_t flags = 0;
                    if (!(qr >= 0.0f)) n = 0;
                    else if (qr > 255.0f) { n = 255; flags |= OG_SATURATED; }
                    else n = (uint32_t)qr;
                    if (n < 1) continue;
                    if (r == 0 || c == 0 || r == R - 1 || c == C - 1)
                        flags |= OG_EDGE;
                    const uint32_t pix = (uint32_t)(base + p);
                    count_map[pix] += n;
                    if (nh < cap) {
                        og_hit* h = &hits[nh];
                        h->frame = frame_base + f;
                        h->pixel = pix;
                        h->energy_kev = E;
                        h->dx = Mx / E;
                        h->dy = My / E;
                        h->count = (uint8_t)n;
                        h->npix = (uint8_t)npix;
                        h->flags = flags;
                    }
                    nh++;
                }
            }
        }
    }
    *n_hits = nh;
    if (n_seeds) *n_seeds = ns;
    free(inv_gain); free(stage); free(d); free(e); free(s); free(set); free(cmu);
    free(cmr); free(cmc);
    return 0;
}
