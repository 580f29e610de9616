/*
 * spd_oracle.c -- plain, slow, FP64 CPU oracle for the single-pulse search of
 * Adamek & Armour, "A Real-time Single Pulse Detection Algorithm for GPUs"
 * (arXiv:1611.09704).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, loads or
 * calls this file.  Only the test suite, the smoke check and the CPU-baseline
 * leg of the benchmark may use it.  It shares no code, header, table or
 * helper with the CUDA path.
 *
 * Every function is the plain definition of what the paper computes, or the
 * paper's algorithm taken step by step in the paper's order:
 *   - mean / standard deviation: the two-pass definition (population sd,
 *     sigma = sqrt(S/j) as in Sec. 2.1), plus Chan's streaming update (Eq. 1)
 *     and pairwise merge (Eq. 2) as separate functions that the tests pin
 *     against the two-pass definition;
 *   - sigma after an N-sample boxcar: Eq. 4 (sqrt(N) sigma) and the linear
 *     approximation of Eq. 5 (two readings, see oracle_sigma_table);
 *   - per-sample highest SNR over boxcar widths with the winning width:
 *     Algorithm 1 of Sec. 2.3, boxcar grown one sample at a time, strict ">";
 *   - candidate selection: keep x_i >= f_T (Sec. 2.4), unordered list
 *     returned here in (dm, sample) order;
 *   - the detector's input, the de-dispersed DM x time plane (Sec. 1): the
 *     definition of incoherent de-dispersion, a sum over frequency channels
 *     each shifted by its delay for the DM trial.
 *
 * Readings of silent or garbled points (each is pinned by a test):
 *   - Eq. 1's S update is read with the square, (j x_j - T_j)^2/(j(j-1)),
 *     T_j taken after adding x_j (Chan et al. 1983); S_1 = 0.
 *   - Algorithm 1's window is forward: B_w(i) = x[i] + ... + x[i+w-1]; the
 *     SNR of a width-w boxcar is (B_w - w mu)/sigma_w; widths with
 *     i + w > n_samp are not evaluated (row end); width 1 is always the
 *     starting value.
 *
 * Input samples are FP32, or FP16 / BF16 bit patterns with an optional FP32
 * per-row scale and offset; the value searched is the FP32 number
 * fmaf(scale, q, offset) (q exactly converted), promoted to double.
 *
 * Build: gcc -O2 -std=c11 -fopenmp -ffp-contract=off -shared -fPIC.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ---------------------------------------------------------------- values */

/* IEEE binary16 -> binary32, exact (every half is a float). */
static float half_bits_to_float(uint16_t h)
{
    uint32_t sign = (uint32_t)(h >> 15) & 1u;
    uint32_t expo = (uint32_t)(h >> 10) & 0x1fu;
    uint32_t mant = (uint32_t)h & 0x3ffu;
    float mag;
    if (expo == 0u) {
        mag = ldexpf((float)mant, -24);               /* zero or subnormal */
    } else if (expo == 31u) {
        mag = mant ? NAN : INFINITY;
    } else {
        mag = ldexpf((float)(mant | 0x400u), (int)expo - 25);
    }
    return sign ? -mag : mag;
}

/* bfloat16 -> binary32, exact: the bf16 bits are the top half of a float. */
static float bf16_bits_to_float(uint16_t b)
{
    uint32_t u = (uint32_t)b << 16;
    float f;
    memcpy(&f, &u, sizeof f);
    return f;
}

/* The value of element t of row r as the search sees it. */
static double sample_value(const void *data, int dtype, int64_t stride,
                           const float *scale, const float *offset,
                           int64_t r, int64_t t)
{
    int64_t idx = r * stride + t;
    float q;
    if (dtype == 0)
        q = ((const float *)data)[idx];
    else if (dtype == 1)
        q = half_bits_to_float(((const uint16_t *)data)[idx]);
    else
        q = bf16_bits_to_float(((const uint16_t *)data)[idx]);
    if (scale) {
        float off = offset ? offset[r] : 0.0f;
        q = fmaf(scale[r], q, off);
    }
    return (double)q;
}

/* Public helper: the dequantised row r as doubles (length n_samp). */
void oracle_dequant_row(const void *data, int dtype, int64_t stride,
                        const float *scale, const float *offset,
                        int64_t r, int64_t n_samp, double *out)
{
    for (int64_t t = 0; t < n_samp; ++t)
        out[t] = sample_value(data, dtype, stride, scale, offset, r, t);
}

/* -------------------------------------------------- Sec. 2.1: mean and sd */

/* Definition: two-pass mean and population standard deviation. */
void oracle_twopass(const double *x, int64_t n, double *mean, double *sd)
{
    double s = 0.0;
    for (int64_t i = 0; i < n; ++i) s += x[i];
    double mu = s / (double)n;
    double q = 0.0;
    for (int64_t i = 0; i < n; ++i) q += (x[i] - mu) * (x[i] - mu);
    *mean = mu;
    *sd = sqrt(q / (double)n);
}

/* Eq. 1: Chan's serial update over x[0..n).  T_j = T_{j-1} + x_j and
 * S_j = S_{j-1} + (j x_j - T_j)^2 / (j (j-1)); S_1 = 0. */
void oracle_chan_stream(const double *x, int64_t n, double *T, double *S)
{
    double t = 0.0, s = 0.0;
    for (int64_t j = 1; j <= n; ++j) {
        double xj = x[j - 1];
        t = t + xj;
        if (j > 1) {
            double d = (double)j * xj - t;
            s = s + d * d / ((double)j * (double)(j - 1));
        }
    }
    *T = t;
    *S = s;
}

/* Eq. 2: merge the (T, S) of m samples with the (T, S) of the next n
 * samples:  S = S_a + S_b + m/(n(m+n)) * (n/m T_a - T_b)^2,  T = T_a + T_b.
 * Either side may be empty. */
void oracle_chan_merge(double m, double Ta, double Sa,
                       double n, double Tb, double Sb,
                       double *T, double *S)
{
    if (m == 0.0) { *T = Tb; *S = Sb; return; }
    if (n == 0.0) { *T = Ta; *S = Sa; return; }
    double d = (n / m) * Ta - Tb;
    *S = Sa + Sb + m / (n * (m + n)) * d * d;
    *T = Ta + Tb;
}

/* Two-pass MSD of the plane.  scope 0: one (mean, sd) over every sample of
 * every row (the dataset of Sec. 2.1); scope 1: one per row.  Row sums are
 * formed per row and added in row order, so the result is deterministic
 * under OpenMP. */
int oracle_plane_msd(const void *data, int dtype, int64_t n_dm, int64_t n_samp,
                     int64_t stride, const float *scale, const float *offset,
                     int scope, double *mean_out, double *sd_out)
{
    if (n_dm <= 0 || n_samp <= 0) return -1;
    double *rsum = (double *)malloc(sizeof(double) * (size_t)n_dm);
    double *rsq = (double *)malloc(sizeof(double) * (size_t)n_dm);
    if (!rsum || !rsq) { free(rsum); free(rsq); return -2; }

    #pragma omp parallel for schedule(dynamic, 1)
    for (int64_t r = 0; r < n_dm; ++r) {
        double s = 0.0;
        for (int64_t t = 0; t < n_samp; ++t)
            s += sample_value(data, dtype, stride, scale, offset, r, t);
        rsum[r] = s;
    }
    double gmean = 0.0;
    if (scope == 0) {
        double s = 0.0;
        for (int64_t r = 0; r < n_dm; ++r) s += rsum[r];
        gmean = s / ((double)n_dm * (double)n_samp);
    }
    #pragma omp parallel for schedule(dynamic, 1)
    for (int64_t r = 0; r < n_dm; ++r) {
        double mu = scope == 0 ? gmean : rsum[r] / (double)n_samp;
        double q = 0.0;
        for (int64_t t = 0; t < n_samp; ++t) {
            double d = sample_value(data, dtype, stride, scale, offset, r, t) - mu;
            q += d * d;
        }
        rsq[r] = q;
    }
    if (scope == 0) {
        double q = 0.0;
        for (int64_t r = 0; r < n_dm; ++r) q += rsq[r];
        mean_out[0] = gmean;
        sd_out[0] = sqrt(q / ((double)n_dm * (double)n_samp));
    } else {
        for (int64_t r = 0; r < n_dm; ++r) {
            mean_out[r] = rsum[r] / (double)n_samp;
            sd_out[r] = sqrt(rsq[r] / (double)n_samp);
        }
    }
    free(rsum);
    free(rsq);
    return 0;
}

/* The block-partial scheme of Sec. 2.1 written out serially: each row is cut
 * into consecutive blocks of `block` samples (the last may be short); Eq. 1
 * gives each block's (T, S); Eq. 2 adds the blocks left to right, rows in
 * order.  Used by the tests to pin Eq. 1/2 against the two-pass definition. */
int oracle_plane_msd_chan(const void *data, int dtype, int64_t n_dm, int64_t n_samp,
                          int64_t stride, const float *scale, const float *offset,
                          int64_t block, int scope, double *mean_out, double *sd_out)
{
    if (n_dm <= 0 || n_samp <= 0 || block <= 0) return -1;
    double *buf = (double *)malloc(sizeof(double) * (size_t)block);
    if (!buf) return -2;
    double gn = 0.0, gT = 0.0, gS = 0.0;
    for (int64_t r = 0; r < n_dm; ++r) {
        double rn = 0.0, rT = 0.0, rS = 0.0;
        for (int64_t t0 = 0; t0 < n_samp; t0 += block) {
            int64_t len = n_samp - t0 < block ? n_samp - t0 : block;
            for (int64_t k = 0; k < len; ++k)
                buf[k] = sample_value(data, dtype, stride, scale, offset, r, t0 + k);
            double bT, bS;
            oracle_chan_stream(buf, len, &bT, &bS);
            double T, S;
            oracle_chan_merge(rn, rT, rS, (double)len, bT, bS, &T, &S);
            rn += (double)len; rT = T; rS = S;
        }
        if (scope == 0) {
            double T, S;
            oracle_chan_merge(gn, gT, gS, rn, rT, rS, &T, &S);
            gn += rn; gT = T; gS = S;
        } else {
            mean_out[r] = rT / rn;
            sd_out[r] = sqrt(rS / rn);
        }
    }
    if (scope == 0) {
        mean_out[0] = gT / gn;
        sd_out[0] = sqrt(gS / gn);
    }
    free(buf);
    return 0;
}

/* ------------------------------------- Sec. 2.2: sigma after N-sample boxcar */

/* sigma_Nmax of Eq. 5: the measured (population) standard deviation of the
 * series B_Nmax(i) = x[i] + ... + x[i+Nmax-1] over full windows
 * i = 0 .. n_samp - Nmax of each row, pooled over the scope (two-pass).
 * Rows shorter than Nmax contribute nothing. */
int oracle_plane_sd_nmax(const void *data, int dtype, int64_t n_dm, int64_t n_samp,
                         int64_t stride, const float *scale, const float *offset,
                         int nmax, int scope, double *sd_out)
{
    if (n_dm <= 0 || n_samp <= 0 || nmax <= 0) return -1;
    int64_t nwin = n_samp - nmax + 1;
    if (nwin <= 0) return -3;
    double *rsum = (double *)malloc(sizeof(double) * (size_t)n_dm);
    double *rsq = (double *)malloc(sizeof(double) * (size_t)n_dm);
    if (!rsum || !rsq) { free(rsum); free(rsq); return -2; }

    #pragma omp parallel for schedule(dynamic, 1)
    for (int64_t r = 0; r < n_dm; ++r) {
        double s = 0.0;
        for (int64_t i = 0; i < nwin; ++i) {
            double b = 0.0;
            for (int k = 0; k < nmax; ++k)
                b += sample_value(data, dtype, stride, scale, offset, r, i + k);
            s += b;
        }
        rsum[r] = s;
    }
    double gmean = 0.0;
    if (scope == 0) {
        double s = 0.0;
        for (int64_t r = 0; r < n_dm; ++r) s += rsum[r];
        gmean = s / ((double)n_dm * (double)nwin);
    }
    #pragma omp parallel for schedule(dynamic, 1)
    for (int64_t r = 0; r < n_dm; ++r) {
        double mu = scope == 0 ? gmean : rsum[r] / (double)nwin;
        double q = 0.0;
        for (int64_t i = 0; i < nwin; ++i) {
            double b = 0.0;
            for (int k = 0; k < nmax; ++k)
                b += sample_value(data, dtype, stride, scale, offset, r, i + k);
            q += (b - mu) * (b - mu);
        }
        rsq[r] = q;
    }
    if (scope == 0) {
        double q = 0.0;
        for (int64_t r = 0; r < n_dm; ++r) q += rsq[r];
        sd_out[0] = sqrt(q / ((double)n_dm * (double)nwin));
    } else {
        for (int64_t r = 0; r < n_dm; ++r) sd_out[r] = sqrt(rsq[r] / (double)nwin);
    }
    free(rsum);
    free(rsq);
    return 0;
}

/* sigma_N for each listed width N.
 *   mode 0, Eq. 4:            sigma_N = sqrt(N) sigma
 *   mode 1, Eq. 5 as printed: sigma_N = sqrt(N) sigma + (N-1) sigma_Nmax/(Nmax-1)
 *   mode 2, Eq. 5 read as a linear excess over Eq. 4, exact at N = 1 and at
 *           N = Nmax: sigma_N = sqrt(N) sigma
 *                               + (N-1) (sigma_Nmax - sqrt(Nmax) sigma)/(Nmax-1)
 * Modes 1 and 2 need nmax >= 2. */
int oracle_sigma_table(int mode, double sd, double sd_nmax, int nmax,
                       const int32_t *widths, int n_widths, double *sigma_out)
{
    if (mode != 0 && nmax < 2) return -1;
    for (int k = 0; k < n_widths; ++k) {
        double N = (double)widths[k];
        double base = sqrt(N) * sd;
        if (mode == 0)
            sigma_out[k] = base;
        else if (mode == 1)
            sigma_out[k] = base + (N - 1.0) * sd_nmax / (double)(nmax - 1);
        else
            sigma_out[k] = base + (N - 1.0) * (sd_nmax - sqrt((double)nmax) * sd)
                                      / (double)(nmax - 1);
    }
    return 0;
}

/* ------------------------------------------- Sec. 2.3: boxcars, Algorithm 1 */

/* Plain boxcar sums B_w(i) = x[i] + ... + x[i+w-1] for i = 0..n_samp-w of each
 * row; NaN where the window runs past the row end.  out: [n_dm][n_samp]. */
int oracle_boxcar_sums(const void *data, int dtype, int64_t n_dm, int64_t n_samp,
                       int64_t stride, const float *scale, const float *offset,
                       int w, double *out)
{
    if (w <= 0) return -1;
    #pragma omp parallel for schedule(dynamic, 1)
    for (int64_t r = 0; r < n_dm; ++r) {
        for (int64_t i = 0; i < n_samp; ++i) {
            double b = NAN;
            if (i + w <= n_samp) {
                b = 0.0;
                for (int k = 0; k < w; ++k)
                    b += sample_value(data, dtype, stride, scale, offset, r, i + k);
            }
            out[r * n_samp + i] = b;
        }
    }
    return 0;
}

/* Algorithm 1 for rows [row0, row1).  For every start sample i:
 *   best = (x[i] - mu)/sigma, W = 1            (SNR of the unprocessed sample)
 *   B = 0;  grow B one sample at a time; at each listed width w (ascending,
 *   w <= n_samp - i): SNR = (B - w mu)/sigma_w; if SNR > best: best, W = SNR, w.
 * mean[e], sd[e]: the MSD of scope entry e (e = 0 for the global scope, e = row
 * for the per-row scope); sigma_tab[e * n_widths + k]: sigma_w of width k for
 * entry e.  Outputs are [row1 - row0][n_samp]. */
int oracle_boxcar_snr(const void *data, int dtype, int64_t n_dm, int64_t n_samp,
                      int64_t stride, const float *scale, const float *offset,
                      int scope, const double *mean, const double *sd,
                      const double *sigma_tab, const int32_t *widths, int n_widths,
                      int64_t row0, int64_t row1, double *best_out, int32_t *width_out,
                      int start_w1)
{
    if (row0 < 0 || row1 > n_dm || row0 > row1 || n_widths < 0) return -1;
    for (int k = 1; k < n_widths; ++k)
        if (widths[k] <= widths[k - 1]) return -1;
    if (n_widths > 0 && widths[0] < 1) return -1;
    int wmax = n_widths > 0 ? widths[n_widths - 1] : 1;

    #pragma omp parallel
    {
        double *x = (double *)malloc(sizeof(double) * (size_t)(n_samp > 0 ? n_samp : 1));
        #pragma omp for schedule(dynamic, 1)
        for (int64_t r = row0; r < row1; ++r) {
            int64_t e = scope == 0 ? 0 : r;
            double mu = mean[e], sg = sd[e];
            const double *sig = sigma_tab + e * (int64_t)n_widths;
            for (int64_t t = 0; t < n_samp; ++t)
                x[t] = sample_value(data, dtype, stride, scale, offset, r, t);
            for (int64_t i = 0; i < n_samp; ++i) {
                /* Algorithm 1 starts from width 1; start_w1 = 0 evaluates the
                   listed widths only (best -inf, width 0 when none fits) */
                double best = start_w1 ? (x[i] - mu) / sg : -INFINITY;
                int32_t W = start_w1 ? 1 : 0;
                double B = 0.0;
                int64_t grown = 0;
                for (int k = 0; k < n_widths; ++k) {
                    int64_t w = widths[k];
                    if (i + w > n_samp) break;
                    while (grown < w) { B += x[i + grown]; ++grown; }
                    double snr = (B - (double)w * mu) / sig[k];
                    if (snr > best) { best = snr; W = (int32_t)w; }
                }
                (void)wmax;
                best_out[(r - row0) * n_samp + i] = best;
                width_out[(r - row0) * n_samp + i] = W;
            }
        }
        free(x);
    }
    return 0;
}

/* --------------------------------------------- Sec. 2.4: candidate selection */

/* Keep every (dm, sample) with best >= thr.  Returns the number kept; writes
 * the first min(count, cap) of them in (dm, sample) order.  dm is row0 + row
 * index of the given planes. */
int64_t oracle_threshold(const double *best, const int32_t *width, int64_t n_rows,
                         int64_t n_samp, int64_t row0, double thr,
                         int32_t *dm_out, int32_t *sample_out, double *snr_out,
                         int32_t *width_out, int64_t cap)
{
    int64_t c = 0;
    for (int64_t r = 0; r < n_rows; ++r) {
        for (int64_t i = 0; i < n_samp; ++i) {
            double v = best[r * n_samp + i];
            if (v >= thr) {
                if (c < cap) {
                    dm_out[c] = (int32_t)(row0 + r);
                    sample_out[c] = (int32_t)i;
                    snr_out[c] = v;
                    width_out[c] = width[r * n_samp + i];
                }
                ++c;
            }
        }
    }
    return c;
}

int oracle_num_threads(void)
{
#ifdef _OPENMP
    extern int omp_get_max_threads(void);
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* SNR of one (row, start, width) pair, Sec. 2.3: (B_w(i) - w mu) / sigma_w with
 * B_w(i) summed directly in FP64.  NaN when the window passes the row end.
 * Used to check that a reported width is one of the (near-)tied maxima. */
double oracle_snr_at(const void *data, int dtype, int64_t n_samp, int64_t stride,
                     const float *scale, const float *offset, int64_t r, int64_t i,
                     int w, double mean, double sigma_w)
{
    if (i < 0 || w < 1 || i + w > n_samp) return NAN;
    double b = 0.0;
    for (int k = 0; k < w; ++k)
        b += sample_value(data, dtype, stride, scale, offset, r, i + k);
    return (b - (double)w * mean) / sigma_w;
}

/* Incoherent de-dispersion, the step that produces the DM x time plane the
 * detector searches (Sec. 1), written as its definition: for DM trial d and
 * output sample t, the sum over channels c of the channel's value at
 * t + delays[d * n_chan + c], in FP64 in channel order.  The filterbank is a
 * "plane" of n_chan channel rows.  Returns -1 (and writes nothing) if a delay
 * lies outside 0 .. n_samp - n_out. */
int oracle_dedisperse(const void *data, int dtype, int64_t n_chan, int64_t n_samp,
                      int64_t stride, const float *scale, const float *offset,
                      const int32_t *delays, int64_t n_dm, int64_t n_out, double *out)
{
    if (n_out < 0 || n_out > n_samp) return -1;
    for (int64_t k = 0; k < n_dm * n_chan; ++k)
        if (delays[k] < 0 || (int64_t)delays[k] > n_samp - n_out) return -1;
#pragma omp parallel for schedule(static)
    for (int64_t d = 0; d < n_dm; ++d) {
        for (int64_t t = 0; t < n_out; ++t) {
            double s = 0.0;
            for (int64_t c = 0; c < n_chan; ++c)
                s += sample_value(data, dtype, stride, scale, offset, c,
                                  t + (int64_t)delays[d * n_chan + c]);
            out[d * n_out + t] = s;
        }
    }
    return 0;
}
