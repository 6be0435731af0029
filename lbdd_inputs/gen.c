/*
 * Seeded synthetic LBDD instances.
 *
 * This module only manufactures inputs: demand/center coordinates, the
 * demand-service cost matrix CM, capacities and per-unit overload penalties.
 * It holds none of the solver's arithmetic, and both the CPU oracle and the
 * CUDA path consume exactly the same bytes from it.
 *
 * The instances follow the shape of the paper's experimental set-up (Section
 * 5, "Datasets"): unit demand, service centers placed at random, a total
 * capacity theta*n < n split randomly across centers, and one constant
 * penalty per center drawn from a range.  The road network of the paper is
 * not available, so Euclidean distances (optionally stretched by a random
 * per-pair road factor) stand in for shortest-path distances; Section 3.4
 * names Euclidean distance as a valid CM construction.
 *
 * Determinism across machines (x86-64 here, aarch64 on the GPU host):
 *  - random numbers come from a counter-based splitmix64 stream keyed on
 *    (seed, stream, index), so the result does not depend on thread count;
 *  - floating point uses only +, -, *, /, sqrt and floor, which IEEE 754
 *    rounds identically everywhere; the file must be compiled with
 *    -ffp-contract=off so that no multiply-add is fused;
 *  - logarithm and exponential (needed for Gaussian draws, Zipf weights and
 *    log-uniform sizes) are computed by the fixed-operation-order series
 *    below instead of libm, whose last-bit results differ between platforms.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>

#define GEN_OK 0
#define GEN_ERR_ARG (-1)
#define GEN_ERR_RANGE (-2)
#define GEN_ERR_OOM (-3)

/* ---------------------------------------------------------------- RNG --- */

static const uint64_t GOLDEN_GAMMA = 0x9E3779B97F4A7C15ull;

/* splitmix64 output function (S. Vigna, public domain reference). */
static inline uint64_t splitmix64_out(uint64_t state) {
    uint64_t z = state + GOLDEN_GAMMA;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

/* Element `idx` of stream `stream` under `seed`. */
uint64_t lbdd_gen_u64(uint64_t seed, uint32_t stream, uint64_t idx) {
    uint64_t base = splitmix64_out(seed ^ ((uint64_t)stream * 0xD1B54A32D192ED03ull));
    return splitmix64_out(base + idx * GOLDEN_GAMMA);
}

/* Uniform double in [0, 1) with 53 random bits. */
double lbdd_gen_u01(uint64_t seed, uint32_t stream, uint64_t idx) {
    return (double)(lbdd_gen_u64(seed, stream, idx) >> 11) * (1.0 / 9007199254740992.0);
}

enum {
    ST_DEMAND_XY = 1,
    ST_CENTER_XY = 2,
    ST_ROAD = 3,
    ST_CAP_W = 4,
    ST_PEN = 5,
    ST_GMM_PARAM = 6,
    ST_GMM_PICK = 7,
    ST_GMM_NORMAL = 8,
    ST_PERM = 9,
    ST_SIZES = 10,
};

/* ------------------------------------------- deterministic log / exp --- */

static const double LN2 = 0.6931471805599453;

/* Natural log for x > 0: exact frexp split, then 2*atanh((m-1)/(m+1)) by a
 * fixed Horner series.  Accurate to a few ulps; identical on every IEEE
 * machine because the operation sequence is fixed. */
double lbdd_gen_log(double x) {
    int e;
    double m = frexp(x, &e); /* x = m * 2^e, m in [0.5, 1) */
    if (m < 0.70710678118654752) { m = m * 2.0; e = e - 1; }
    double t = (m - 1.0) / (m + 1.0);
    double t2 = t * t;
    double s = 1.0 / 25.0;
    s = s * t2 + 1.0 / 23.0;
    s = s * t2 + 1.0 / 21.0;
    s = s * t2 + 1.0 / 19.0;
    s = s * t2 + 1.0 / 17.0;
    s = s * t2 + 1.0 / 15.0;
    s = s * t2 + 1.0 / 13.0;
    s = s * t2 + 1.0 / 11.0;
    s = s * t2 + 1.0 / 9.0;
    s = s * t2 + 1.0 / 7.0;
    s = s * t2 + 1.0 / 5.0;
    s = s * t2 + 1.0 / 3.0;
    s = s * t2 + 1.0;
    return 2.0 * t * s + (double)e * LN2;
}

/* Exponential: x = m*ln2 + r with |r| <= ln2/2, Taylor series for e^r,
 * exact ldexp for 2^m. */
double lbdd_gen_exp(double x) {
    double mf = floor(x / LN2 + 0.5);
    double r = x - mf * LN2;
    double term = 1.0, sum = 1.0;
    for (int i = 1; i <= 22; ++i) {
        term = term * r / (double)i;
        sum = sum + term;
    }
    return ldexp(sum, (int)mf);
}

/* ------------------------------------------------------------ points --- */

/* `count` points uniform in the unit square, xy interleaved. */
int lbdd_gen_points_uniform(uint64_t seed, uint32_t stream, int64_t count, double *xy) {
    if (count < 0 || (count > 0 && !xy)) return GEN_ERR_ARG;
    for (int64_t i = 0; i < count; ++i) {
        xy[2 * i] = lbdd_gen_u01(seed, stream, 2 * (uint64_t)i);
        xy[2 * i + 1] = lbdd_gen_u01(seed, stream, 2 * (uint64_t)i + 1);
    }
    return GEN_OK;
}

/* `count` demand points from an `ncomp`-component isotropic Gaussian
 * mixture: means uniform in the unit square, sigma uniform in
 * [sig_lo, sig_hi], component weights uniform in (0, 1] and normalised.
 * Normal deviates use Marsaglia's polar method. */
int lbdd_gen_points_gmm(uint64_t seed, int64_t count, int ncomp, double sig_lo,
                        double sig_hi, double *xy) {
    if (count < 0 || ncomp < 1 || (count > 0 && !xy)) return GEN_ERR_ARG;
    double *mx = (double *)malloc(sizeof(double) * 4 * (size_t)ncomp);
    if (!mx) return GEN_ERR_OOM;
    double *my = mx + ncomp, *sg = my + ncomp, *cw = sg + ncomp;
    double wsum = 0.0;
    for (int c = 0; c < ncomp; ++c) {
        mx[c] = lbdd_gen_u01(seed, ST_GMM_PARAM, 4 * (uint64_t)c);
        my[c] = lbdd_gen_u01(seed, ST_GMM_PARAM, 4 * (uint64_t)c + 1);
        sg[c] = sig_lo + (sig_hi - sig_lo) * lbdd_gen_u01(seed, ST_GMM_PARAM, 4 * (uint64_t)c + 2);
        double w = 1.0 - lbdd_gen_u01(seed, ST_GMM_PARAM, 4 * (uint64_t)c + 3);
        wsum = wsum + w;
        cw[c] = wsum;
    }
    for (int c = 0; c < ncomp; ++c) cw[c] = cw[c] / wsum;
    int rc = GEN_OK;
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < count; ++i) {
        double u = lbdd_gen_u01(seed, ST_GMM_PICK, (uint64_t)i);
        int c = ncomp - 1;
        for (int q = 0; q < ncomp; ++q) {
            if (u < cw[q]) { c = q; break; }
        }
        double z1 = 0.0, z2 = 0.0;
        int found = 0;
        for (uint64_t a = 0; a < 64 && !found; ++a) {
            uint64_t base = ((uint64_t)i * 64 + a) * 2;
            double u1 = 2.0 * lbdd_gen_u01(seed, ST_GMM_NORMAL, base) - 1.0;
            double u2 = 2.0 * lbdd_gen_u01(seed, ST_GMM_NORMAL, base + 1) - 1.0;
            double s = u1 * u1 + u2 * u2;
            if (s > 0.0 && s < 1.0) {
                double f = sqrt(-2.0 * lbdd_gen_log(s) / s);
                z1 = u1 * f;
                z2 = u2 * f;
                found = 1;
            }
        }
        xy[2 * i] = mx[c] + sg[c] * z1;
        xy[2 * i + 1] = my[c] + sg[c] * z2;
    }
    free(mx);
    return rc;
}

/* ------------------------------------------------------- cost matrix --- */

/* One CM entry: max(1, floor(scale * dist * rf + 0.5)), rf = 1 when road_lo
 * == road_hi == 1, else uniform in [road_lo, road_hi] per (d, s) pair. */
static inline double cm_value(const double *dxy, const double *sxy, int64_t d, int64_t s,
                              int64_t k, double scale, double road_lo, double road_hi,
                              uint64_t seed) {
    double dx = dxy[2 * d] - sxy[2 * s];
    double dy = dxy[2 * d + 1] - sxy[2 * s + 1];
    double sq = dx * dx;
    double sq2 = dy * dy;
    double dist = sqrt(sq + sq2);
    double v = scale * dist;
    if (road_hi != 1.0 || road_lo != 1.0) {
        double rf = road_lo + (road_hi - road_lo) * lbdd_gen_u01(seed, ST_ROAD, (uint64_t)(d * k + s));
        v = v * rf;
    }
    double c = floor(v + 0.5);
    if (c < 1.0) c = 1.0;
    return c;
}

/* Fill CM (n x k, demand-major).  elem_bytes = 4 (int32) or 2 (int16).
 * Returns GEN_ERR_RANGE if a value does not fit the element type. */
int lbdd_gen_cm(int64_t n, int64_t k, const double *dxy, const double *sxy, double scale,
                double road_lo, double road_hi, uint64_t seed, int elem_bytes, void *out) {
    if (n < 1 || k < 1 || !dxy || !sxy || !out) return GEN_ERR_ARG;
    if (elem_bytes != 4 && elem_bytes != 2) return GEN_ERR_ARG;
    const double lim = elem_bytes == 4 ? 2147483647.0 : 32767.0;
    int bad = 0;
#pragma omp parallel for schedule(static) reduction(| : bad)
    for (int64_t d = 0; d < n; ++d) {
        for (int64_t s = 0; s < k; ++s) {
            double c = cm_value(dxy, sxy, d, s, k, scale, road_lo, road_hi, seed);
            if (c > lim) { bad = 1; c = lim; }
            if (elem_bytes == 4) ((int32_t *)out)[d * k + s] = (int32_t)c;
            else ((int16_t *)out)[d * k + s] = (int16_t)c;
        }
    }
    return bad ? GEN_ERR_RANGE : GEN_OK;
}

/* Entries (d, s) listed in idx pairs, for spot checks of very large CMs. */
int lbdd_gen_cm_sample(int64_t m, const int64_t *pairs, int64_t k, const double *dxy,
                       const double *sxy, double scale, double road_lo, double road_hi,
                       uint64_t seed, int64_t *out) {
    if (m < 0 || !pairs || !dxy || !sxy || !out) return GEN_ERR_ARG;
    for (int64_t i = 0; i < m; ++i)
        out[i] = (int64_t)cm_value(dxy, sxy, pairs[2 * i], pairs[2 * i + 1], k, scale, road_lo,
                                   road_hi, seed);
    return GEN_OK;
}

/* ------------------------------------------------- capacities, penalties */

typedef struct { double frac; int64_t idx; } frac_item;

static int frac_cmp(const void *a, const void *b) {
    const frac_item *x = (const frac_item *)a, *y = (const frac_item *)b;
    if (x->frac > y->frac) return -1;
    if (x->frac < y->frac) return 1;
    return (x->idx > y->idx) - (x->idx < y->idx);
}

/* Split `total` units over k centers in proportion to w: every center gets 1,
 * the remaining total-k go by floor of the proportional share plus largest
 * remainder (ties to the lower index). */
static int split_total(int64_t k, const double *w, int64_t total, int32_t *cap) {
    if (total < k) return GEN_ERR_ARG;
    double wsum = 0.0;
    for (int64_t s = 0; s < k; ++s) wsum = wsum + w[s];
    int64_t rest = total - k, given = 0;
    frac_item *it = (frac_item *)malloc(sizeof(frac_item) * (size_t)k);
    if (!it) return GEN_ERR_OOM;
    for (int64_t s = 0; s < k; ++s) {
        double q = w[s] / wsum * (double)rest;
        double f = floor(q);
        cap[s] = 1 + (int32_t)f;
        given += (int64_t)f;
        it[s].frac = q - f;
        it[s].idx = s;
    }
    qsort(it, (size_t)k, sizeof(frac_item), frac_cmp);
    int64_t left = rest - given;
    for (int64_t i = 0; i < left && i < k; ++i) cap[it[i].idx] += 1;
    free(it);
    return GEN_OK;
}

/* Capacities with uniform (0, 1] random weights, summing to `total`. */
int lbdd_gen_caps_uniform(uint64_t seed, int64_t k, int64_t total, int32_t *cap) {
    if (k < 1 || !cap) return GEN_ERR_ARG;
    double *w = (double *)malloc(sizeof(double) * (size_t)k);
    if (!w) return GEN_ERR_OOM;
    for (int64_t s = 0; s < k; ++s) w[s] = 1.0 - lbdd_gen_u01(seed, ST_CAP_W, (uint64_t)s);
    int rc = split_total(k, w, total, cap);
    free(w);
    return rc;
}

/* Zipf capacities: a seeded random permutation ranks the centers 1..k and
 * the center of rank r gets weight r^(-expo); the weights are split to sum to
 * `total`. */
int lbdd_gen_caps_zipf(uint64_t seed, int64_t k, int64_t total, double expo, int32_t *cap) {
    if (k < 1 || !cap) return GEN_ERR_ARG;
    int64_t *perm = (int64_t *)malloc(sizeof(int64_t) * (size_t)k);
    double *w = (double *)malloc(sizeof(double) * (size_t)k);
    if (!perm || !w) { free(perm); free(w); return GEN_ERR_OOM; }
    for (int64_t i = 0; i < k; ++i) perm[i] = i;
    for (int64_t i = k - 1; i >= 1; --i) {
        int64_t j = (int64_t)(lbdd_gen_u64(seed, ST_PERM, (uint64_t)i) % (uint64_t)(i + 1));
        int64_t t = perm[i]; perm[i] = perm[j]; perm[j] = t;
    }
    for (int64_t r = 0; r < k; ++r)
        w[perm[r]] = lbdd_gen_exp(-expo * lbdd_gen_log((double)(r + 1)));
    int rc = split_total(k, w, total, cap);
    free(perm); free(w);
    return rc;
}

/* One constant per-unit overload penalty per center, uniform in [lo, hi]. */
int lbdd_gen_pens(uint64_t seed, int64_t k, int32_t lo, int32_t hi, int32_t *pen) {
    if (k < 1 || !pen || lo > hi) return GEN_ERR_ARG;
    uint64_t span = (uint64_t)((int64_t)hi - (int64_t)lo + 1);
    for (int64_t s = 0; s < k; ++s)
        pen[s] = lo + (int32_t)(lbdd_gen_u64(seed, ST_PEN, (uint64_t)s) % span);
    return GEN_OK;
}

/* Log-uniform instance size in [10^lo_exp, 10^hi_exp), floored. */
int64_t lbdd_gen_logu_size(uint64_t seed, uint64_t which, double lo_exp, double hi_exp) {
    const double LN10 = 2.302585092994046;
    double u = lbdd_gen_u01(seed, ST_SIZES, which);
    double e = lo_exp + (hi_exp - lo_exp) * u;
    return (int64_t)floor(lbdd_gen_exp(e * LN10));
}
