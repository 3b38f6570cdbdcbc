/*
 * cf_oracle.c -- plain, slow FP64 CPU oracle of the exact circulant-embedding
 * survey-field sampler (Carron, Wolk & Szapudi 2014).
 *
 * TEST INFRASTRUCTURE ONLY: loaded by the tests, the smoke check and the CPU
 * baseline leg of the benchmark; never by the product library.
 *
 * Written for a reader to check against the paper by eye: every step follows
 * the paper's order and notation, transforms are a naive DFT or a textbook
 * recursive radix-2 FFT, loops are plain, nothing is blocked, fused or
 * reordered.  Compile with -ffp-contract=off: the noise specification is a
 * fixed sequence of correctly rounded IEEE operations (explicit fma where
 * wanted), so that an independent implementation can reproduce it bit for bit.
 *
 * Readings of the paper where it is silent (all listed in the design notes):
 *  - DFT sign convention: forward e^{-2 pi i k.m/M}, inverse e^{+...}.
 *  - Embedding lag of index m on an axis of size M = 2N: m if m < N else m - M
 *    (the grid of eq. (grid) runs -N..N-1, so index N carries lag -N).
 *  - Eigenvalues within tau = 1e-12 lambda_max of zero are set to zero; below
 *    -tau the embedding fails unless clamping is requested.
 *  - One complex draw gives two fields (Re, Im) with the target covariance.
 *  - The noise is Philox4x32-10 + Box-Muller with the bit layout below.
 *  - Poisson counts by inverse CDF with a strict "<" comparison.
 *  - Power spectrum bins are half-open intervals of |n| in fundamental units.
 */
#include "cf_oracle.h"

#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

static const double OR_PI = 3.14159265358979323846;

/* ======================================================================
 * Philox4x32-10, as published by Salmon, Moraes, Dror & Shaw, "Parallel
 * random numbers: as easy as 1, 2, 3" (SC'11).  Ten rounds; each round
 * multiplies counter words 0 and 2 by the round multipliers, swaps and
 * xors in the key; the key is bumped by the Weyl constants between rounds.
 * ==================================================================== */
void or_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    const uint32_t MULT0 = 0xD2511F53u, MULT1 = 0xCD9E8D57u;
    const uint32_t WEYL0 = 0x9E3779B9u, WEYL1 = 0xBB67AE85u;
    uint32_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k0 += WEYL0;
            k1 += WEYL1;
        }
        uint64_t prod0 = (uint64_t)MULT0 * (uint64_t)x0;
        uint64_t prod1 = (uint64_t)MULT1 * (uint64_t)x2;
        uint32_t hi0 = (uint32_t)(prod0 >> 32), lo0 = (uint32_t)prod0;
        uint32_t hi1 = (uint32_t)(prod1 >> 32), lo1 = (uint32_t)prod1;
        uint32_t y0 = hi1 ^ x1 ^ k0;
        uint32_t y1 = lo1;
        uint32_t y2 = hi0 ^ x3 ^ k1;
        uint32_t y3 = lo0;
        x0 = y0; x1 = y1; x2 = y2; x3 = y3;
    }
    out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

/* ======================================================================
 * Natural logarithm on (0,1], own implementation.
 * Method: reduce u = 2^e m with m in (sqrt(1/2), sqrt(2)], then
 * ln m = 2 atanh(s), s = (m-1)/(m+1), summed as the Gregory series
 * 2 (s + s^3/3 + s^5/5 + ...), and ln u = e ln2 + ln m with ln 2 split in
 * a leading and a trailing part (Cody & Waite style).  Coefficients are the
 * correctly rounded reciprocals 1/(2j+1).
 * ==================================================================== */
static const double OR_SQRT2 = 1.41421356237309504880;
static const double OR_LN2 = 0.69314718055994530942;        /* nearest binary64 to ln 2 */
static const double OR_LN2_LO = 2.3190468138462996e-17;     /* ln 2 - OR_LN2 */

double or_log_unit(double u)
{
    uint64_t bits;
    memcpy(&bits, &u, sizeof bits);
    int e = (int)((bits >> 52) & 0x7ff) - 1023;
    uint64_t mbits = (bits & 0x000fffffffffffffULL) | 0x3ff0000000000000ULL;
    double m;
    memcpy(&m, &mbits, sizeof m);
    if (m > OR_SQRT2) {
        m = m * 0.5;
        e += 1;
    }
    double s = (m - 1.0) / (m + 1.0);
    double z = s * s;
    /* terms j = 1..9 of sum z^j / (2j+1) */
    double p = 1.0 / 19.0;
    for (int j = 8; j >= 1; --j) p = fma(p, z, 1.0 / (double)(2 * j + 1));
    double t = fma(s * z, p, s);
    double lnm = 2.0 * t;
    double de = (double)e;
    return fma(de, OR_LN2, fma(de, OR_LN2_LO, lnm));
}

static const float OR_SQRT2F = 1.41421356f;
static const float OR_LN2F = 0.693147182f;          /* nearest binary32 to ln 2 */
static const float OR_LN2F_LO = -1.9046542e-09f;    /* ln 2 - OR_LN2F */

float or_logf_unit(float u)
{
    uint32_t bits;
    memcpy(&bits, &u, sizeof bits);
    int e = (int)((bits >> 23) & 0xff) - 127;
    uint32_t mbits = (bits & 0x007fffffu) | 0x3f800000u;
    float m;
    memcpy(&m, &mbits, sizeof m);
    if (m > OR_SQRT2F) {
        m = m * 0.5f;
        e += 1;
    }
    float s = (m - 1.0f) / (m + 1.0f);
    float z = s * s;
    /* terms j = 1..4 of sum z^j / (2j+1) */
    float p = 1.0f / 9.0f;
    p = fmaf(p, z, 1.0f / 7.0f);
    p = fmaf(p, z, 1.0f / 5.0f);
    p = fmaf(p, z, 1.0f / 3.0f);
    float t = fmaf(s * z, p, s);
    float lnm = 2.0f * t;
    float fe = (float)e;
    return fmaf(fe, OR_LN2F, fmaf(fe, OR_LN2F_LO, lnm));
}

/* ======================================================================
 * cos(2 pi u), sin(2 pi u) for a dyadic u in (0,1], own implementation.
 * Method: t = 4u and q = nearest integer to t are exact, f = t - q in
 * [-1/2, 1/2] is exact, x = (pi/2) f; Taylor series of sin x and cos x with
 * the correctly rounded coefficients 1/n!, then rotation by q quarter turns.
 * ==================================================================== */
static const double OR_PIO2 = 1.57079632679489661923;

static double or_fact(int n)
{
    double r = 1.0;
    for (int i = 2; i <= n; ++i) r *= (double)i; /* exact up to 22! */
    return r;
}

void or_cossin_2pi(double u, double* c, double* s)
{
    double t = 4.0 * u;
    double q = rint(t);
    double f = t - q;
    double x = OR_PIO2 * f;
    double z = x * x;
    /* sin x = x + x z (S1 + z (S2 + ... S8)),  Sj = (-1)^j / (2j+1)! */
    double ps = 1.0 / or_fact(17);
    for (int j = 7; j >= 1; --j) {
        double sj = ((j & 1) ? -1.0 : 1.0) / or_fact(2 * j + 1);
        ps = fma(ps, z, sj);
    }
    double sn = fma(x * z, ps, x);
    /* cos x = 1 + z (C1 + z (C2 + ... C8)),  Cj = (-1)^j / (2j)! */
    double pc = 1.0 / or_fact(16);
    for (int j = 7; j >= 1; --j) {
        double cj = ((j & 1) ? -1.0 : 1.0) / or_fact(2 * j);
        pc = fma(pc, z, cj);
    }
    double cs = fma(z, pc, 1.0);
    int quadrant = ((int)q) & 3;
    switch (quadrant) {
    case 0: *c = cs; *s = sn; break;
    case 1: *c = -sn; *s = cs; break;
    case 2: *c = -cs; *s = -sn; break;
    default: *c = sn; *s = -cs; break;
    }
}

static const float OR_PIO2F = 1.57079637f;

void or_cossin_2pif(float u, float* c, float* s)
{
    float t = 4.0f * u;
    float q = rintf(t);
    float f = t - q;
    float x = OR_PIO2F * f;
    float z = x * x;
    /* sin: S1..S4 = -1/3!, 1/5!, -1/7!, 1/9! */
    float ps = 1.0f / 362880.0f;
    ps = fmaf(ps, z, -1.0f / 5040.0f);
    ps = fmaf(ps, z, 1.0f / 120.0f);
    ps = fmaf(ps, z, -1.0f / 6.0f);
    float sn = fmaf(x * z, ps, x);
    /* cos: C1..C5 = -1/2!, 1/4!, -1/6!, 1/8!, -1/10! */
    float pc = -1.0f / 3628800.0f;
    pc = fmaf(pc, z, 1.0f / 40320.0f);
    pc = fmaf(pc, z, -1.0f / 720.0f);
    pc = fmaf(pc, z, 1.0f / 24.0f);
    pc = fmaf(pc, z, -1.0f / 2.0f);
    float cs = fmaf(z, pc, 1.0f);
    int quadrant = ((int)q) & 3;
    switch (quadrant) {
    case 0: *c = cs; *s = sn; break;
    case 1: *c = -sn; *s = cs; break;
    case 2: *c = -cs; *s = -sn; break;
    default: *c = sn; *s = -cs; break;
    }
}

/* ======================================================================
 * Noise specification: the paper's modes are independent zero-mean
 * Gaussians (section 2, eq. (Papos2)); the generator is not specified.
 *
 * binary64: embedded cell k, realization r: Philox4x32-10 with key
 *   (seed_lo, seed_hi) and counter (k_lo, k_hi, r, 0); uniforms
 *   u1 = (((x0>>5) 2^26 + (x1>>6)) + 1) 2^-53, u2 likewise from (x2, x3);
 *   Box-Muller: rad = sqrt(-2 ln u1), eps = rad (cos 2 pi u2, sin 2 pi u2).
 * binary32: cells are paired along the last axis (column c with c + M/2);
 *   pair index p = row (M/2) + (c mod M/2); counter (p_lo, p_hi, r, 0);
 *   the lower column uses (x0, x1), the upper (x2, x3);
 *   u = ((x>>8) + 1) 2^-24; Box-Muller in binary32.
 * ==================================================================== */
static void or_noise_f64_cell(uint64_t seed, uint64_t r, uint64_t k, double* e1, double* e2)
{
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t ctr[4] = {(uint32_t)k, (uint32_t)(k >> 32), (uint32_t)r, 0u};
    uint32_t x[4];
    or_philox4x32_10(ctr, key, x);
    uint64_t i1 = ((uint64_t)(x[0] >> 5) << 26) | (uint64_t)(x[1] >> 6);
    uint64_t i2 = ((uint64_t)(x[2] >> 5) << 26) | (uint64_t)(x[3] >> 6);
    double u1 = ((double)i1 + 1.0) * 0x1p-53;
    double u2 = ((double)i2 + 1.0) * 0x1p-53;
    double rad = sqrt(-2.0 * or_log_unit(u1));
    double c, s;
    or_cossin_2pi(u2, &c, &s);
    *e1 = rad * c;
    *e2 = rad * s;
}

static void or_noise_f32_cell(uint64_t seed, uint64_t r, uint64_t k, int64_t m_last,
                              float* e1, float* e2)
{
    uint64_t half = (uint64_t)m_last / 2;
    uint64_t row = k / (uint64_t)m_last;
    uint64_t col = k % (uint64_t)m_last;
    uint64_t p = row * half + (col % half);
    int upper = col >= half;
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t ctr[4] = {(uint32_t)p, (uint32_t)(p >> 32), (uint32_t)r, 0u};
    uint32_t x[4];
    or_philox4x32_10(ctr, key, x);
    uint32_t a = upper ? x[2] : x[0];
    uint32_t b = upper ? x[3] : x[1];
    float u1 = (float)((a >> 8) + 1u) * 0x1p-24f;
    float u2 = (float)((b >> 8) + 1u) * 0x1p-24f;
    float rad = sqrtf(-2.0f * or_logf_unit(u1));
    float c, s;
    or_cossin_2pif(u2, &c, &s);
    *e1 = rad * c;
    *e2 = rad * s;
}

void or_draw_noise(uint64_t seed, uint64_t r0, int32_t R, int64_t ncells, int64_t m_last,
                   int32_t dtype, double* out)
{
    for (int32_t rr = 0; rr < R; ++rr) {
        uint64_t r = r0 + (uint64_t)rr;
        double* o = out + (size_t)rr * (size_t)ncells * 2;
        for (int64_t k = 0; k < ncells; ++k) {
            if (dtype == 0) {
                or_noise_f64_cell(seed, r, (uint64_t)k, &o[2 * k], &o[2 * k + 1]);
            } else {
                float a, b;
                or_noise_f32_cell(seed, r, (uint64_t)k, m_last, &a, &b);
                o[2 * k] = (double)a;
                o[2 * k + 1] = (double)b;
            }
        }
    }
}

/* ======================================================================
 * Transforms.  Unnormalised: X_k = sum_j x_j exp(sign 2 pi i j k / n).
 * ==================================================================== */
static void or_twiddle(int64_t num, int64_t n, int sign, double* wr, double* wi)
{
    /* exp(sign 2 pi i num/n), with num reduced mod n first */
    num %= n;
    double ang = 2.0 * OR_PI * (double)num / (double)n;
    *wr = cos(ang);
    *wi = (double)sign * sin(ang);
}

void or_dft_naive(const double* in, double* out, int64_t n, int sign)
{
    for (int64_t k = 0; k < n; ++k) {
        double sr = 0.0, si = 0.0;
        for (int64_t j = 0; j < n; ++j) {
            double wr, wi;
            or_twiddle((j * k) % n, n, sign, &wr, &wi);
            double xr = in[2 * j], xi = in[2 * j + 1];
            sr += xr * wr - xi * wi;
            si += xr * wi + xi * wr;
        }
        out[2 * k] = sr;
        out[2 * k + 1] = si;
    }
}

/* Textbook recursive radix-2 decimation in time; tmp has room for n values. */
static void or_fft_rec(double* a, int64_t n, double* tmp, int sign)
{
    if (n == 1) return;
    int64_t h = n / 2;
    for (int64_t j = 0; j < h; ++j) {
        tmp[2 * j] = a[4 * j];
        tmp[2 * j + 1] = a[4 * j + 1];
        tmp[2 * (h + j)] = a[4 * j + 2];
        tmp[2 * (h + j) + 1] = a[4 * j + 3];
    }
    or_fft_rec(tmp, h, a, sign);
    or_fft_rec(tmp + 2 * h, h, a + 2 * h, sign);
    for (int64_t k = 0; k < h; ++k) {
        double wr, wi;
        or_twiddle(k, n, sign, &wr, &wi);
        double er = tmp[2 * k], ei = tmp[2 * k + 1];
        double orr = tmp[2 * (h + k)], oi = tmp[2 * (h + k) + 1];
        double tr = wr * orr - wi * oi;
        double ti = wr * oi + wi * orr;
        a[2 * k] = er + tr;
        a[2 * k + 1] = ei + ti;
        a[2 * (k + h)] = er - tr;
        a[2 * (k + h) + 1] = ei - ti;
    }
}

void or_fft_recursive(double* a, int64_t n, int sign)
{
    double* tmp = (double*)malloc(sizeof(double) * 2 * (size_t)n);
    or_fft_rec(a, n, tmp, sign);
    free(tmp);
}

static int or_is_pow2(int64_t n) { return n > 0 && (n & (n - 1)) == 0; }

void or_fft_nd(double* a, int32_t ndim, const int64_t* dims, int sign)
{
    int64_t total = 1;
    for (int d = 0; d < ndim; ++d) total *= dims[d];
    for (int axis = 0; axis < ndim; ++axis) {
        int64_t n = dims[axis];
        int64_t inner = 1;
        for (int d = axis + 1; d < ndim; ++d) inner *= dims[d];
        int64_t outer = total / (n * inner);
        double* line = (double*)malloc(sizeof(double) * 2 * (size_t)n);
        double* res = (double*)malloc(sizeof(double) * 2 * (size_t)n);
        for (int64_t o = 0; o < outer; ++o) {
            for (int64_t i = 0; i < inner; ++i) {
                for (int64_t j = 0; j < n; ++j) {
                    size_t idx = (size_t)((o * n + j) * inner + i);
                    line[2 * j] = a[2 * idx];
                    line[2 * j + 1] = a[2 * idx + 1];
                }
                if (or_is_pow2(n) && n > 16) {
                    or_fft_recursive(line, n, sign);
                    memcpy(res, line, sizeof(double) * 2 * (size_t)n);
                } else {
                    or_dft_naive(line, res, n, sign);
                }
                for (int64_t j = 0; j < n; ++j) {
                    size_t idx = (size_t)((o * n + j) * inner + i);
                    a[2 * idx] = res[2 * j];
                    a[2 * idx + 1] = res[2 * j + 1];
                }
            }
        }
        free(line);
        free(res);
    }
}

/* ======================================================================
 * Section 2, eq. (grid) and eq. (Specd): the survey grid of n_i points per
 * axis is enlarged to M_i = 2 n_i points at lags -n_i..n_i-1; the first row
 * of the circulant covariance is xi at those lags, and the "ad-hoc" spectrum
 * is its DFT.  The cell volume factor (L/N)^2 of eq. (Specd) is absorbed into
 * the normalisation of the inverse transform, so lambda = DFT(c) exactly.
 * ==================================================================== */
static double or_xi(int32_t kind, double amp, double scale, double beta, double r2)
{
    switch (kind) {
    case OR_XI_GAUSSIAN: return amp * exp(-r2 / (2.0 * scale * scale));
    case OR_XI_GEN_CAUCHY: return amp * pow(1.0 + r2 / (scale * scale), -beta);
    case OR_XI_EXPONENTIAL: return amp * exp(-sqrt(r2) / scale);
    default: return 0.0;
    }
}

void or_embed_row(int32_t ndim, const int64_t* M, const double* cell, int32_t kind,
                  double amp, double scale, double beta, const double* table, double* c)
{
    int64_t total = 1;
    for (int d = 0; d < ndim; ++d) total *= M[d];
    for (int64_t idx = 0; idx < total; ++idx) {
        if (kind == OR_XI_TABLE) {
            c[idx] = table[idx];
            continue;
        }
        int64_t rem = idx;
        double r2 = 0.0;
        for (int d = ndim - 1; d >= 0; --d) {
            int64_t m = rem % M[d];
            rem /= M[d];
            int64_t lag = (2 * m < M[d]) ? m : m - M[d];
            double x = (double)lag * cell[d];
            r2 += x * x;
        }
        c[idx] = or_xi(kind, amp, scale, beta, r2);
    }
}

void or_eigenvalues(int32_t ndim, const int64_t* M, const double* c, double* lambda)
{
    int64_t total = 1;
    for (int d = 0; d < ndim; ++d) total *= M[d];
    double* z = (double*)calloc((size_t)total * 2, sizeof(double));
    for (int64_t i = 0; i < total; ++i) z[2 * i] = c[i];
    or_fft_nd(z, ndim, M, -1);
    for (int64_t i = 0; i < total; ++i) lambda[i] = z[2 * i];
    free(z);
}

/* Section 2, eq. (condition) and the remark after eq. (Papos2): the method
 * needs every eigenvalue non-negative. */
void or_psd(int32_t ndim, const int64_t* n, const int64_t* M, const double* c, const double* lambda,
            int32_t clamp, double* lambda_plus, double* sqrt_lambda, or_embed_report* rep)
{
    int64_t total = 1;
    for (int d = 0; d < ndim; ++d) total *= M[d];
    memset(rep, 0, sizeof *rep);
    double lmin = lambda[0], lmax = lambda[0];
    for (int64_t i = 1; i < total; ++i) {
        if (lambda[i] < lmin) lmin = lambda[i];
        if (lambda[i] > lmax) lmax = lambda[i];
    }
    rep->lambda_min = lmin;
    rep->lambda_max = lmax;
    double tau = 1e-12 * lmax;
    rep->tau = tau;
    if (!(lmax > 0.0)) {
        rep->status = 2;
        rep->n_negative = total;
        for (int64_t i = 0; i < total; ++i) {
            lambda_plus[i] = 0.0;
            sqrt_lambda[i] = 0.0;
        }
        return;
    }
    for (int64_t i = 0; i < total; ++i) {
        double l = lambda[i];
        double lp;
        if (l > tau) {
            lp = l;
        } else if (l >= -tau) {
            lp = 0.0;
            rep->n_zeroed += 1;
        } else {
            lp = 0.0;
            rep->n_negative += 1;
            rep->neg_mass += -l;
        }
        lambda_plus[i] = lp;
        sqrt_lambda[i] = sqrt(lp);
    }
    if (rep->n_negative > 0 && !clamp) {
        rep->status = 2;
        return;
    }
    rep->clamped = rep->n_negative > 0;
    if (rep->clamped) {
        /* realised covariance = inverse DFT of lambda+ / M^d, compared with
         * the embedded row on survey lags (|lag| < n on every axis: index
         * m < n or m > M - n). */
        double* z = (double*)calloc((size_t)total * 2, sizeof(double));
        for (int64_t i = 0; i < total; ++i) z[2 * i] = lambda_plus[i];
        or_fft_nd(z, ndim, M, +1);
        double err = 0.0;
        for (int64_t idx = 0; idx < total; ++idx) {
            int64_t rem = idx;
            int survey = 1;
            for (int d = ndim - 1; d >= 0; --d) {
                int64_t m = rem % M[d];
                rem /= M[d];
                if (m >= n[d] && m <= M[d] - n[d]) survey = 0;
            }
            if (!survey) continue;
            double e = fabs(z[2 * idx] / (double)total - c[idx]);
            if (e > err) err = e;
        }
        rep->cov_error = err;
        free(z);
    }
}

/* ======================================================================
 * Section 2, eqs. (Papos2) and the closing paragraph: independent Gaussian
 * modes with variance lambda, inverse DFT, restriction to the survey box.
 * W_m = M^{-d/2} sum_k sqrt(lambda_k) eps_k exp(+2 pi i k.m/M), m_i < n_i;
 * Re W and Im W are two independent fields with covariance xi.
 * ==================================================================== */
void or_sample_given_noise(int32_t ndim, const int64_t* n, const int64_t* M, const double* s,
                           const double* eps, double* w)
{
    int64_t total = 1;
    for (int d = 0; d < ndim; ++d) total *= M[d];
    double* x = (double*)malloc(sizeof(double) * 2 * (size_t)total);
    for (int64_t k = 0; k < total; ++k) {
        x[2 * k] = s[k] * eps[2 * k];
        x[2 * k + 1] = s[k] * eps[2 * k + 1];
    }
    or_fft_nd(x, ndim, M, +1);
    double norm = 1.0 / sqrt((double)total);
    /* crop: survey indices m_i in [0, n_i) */
    int64_t ncell = 1;
    for (int d = 0; d < ndim; ++d) ncell *= n[d];
    for (int64_t i = 0; i < ncell; ++i) {
        int64_t rem = i, idx = 0, mul = 1;
        for (int d = ndim - 1; d >= 0; --d) {
            int64_t m = rem % n[d];
            rem /= n[d];
            idx += m * mul;
            mul *= M[d];
        }
        w[2 * i] = x[2 * idx] * norm;
        w[2 * i + 1] = x[2 * idx + 1] * norm;
    }
    free(x);
}

void or_sample(int32_t ndim, const int64_t* n, const int64_t* M, const double* s, uint64_t seed,
               uint64_t r0, int32_t R, int32_t dtype, double* fields)
{
    int64_t total = 1, ncell = 1;
    for (int d = 0; d < ndim; ++d) {
        total *= M[d];
        ncell *= n[d];
    }
    double* eps = (double*)malloc(sizeof(double) * 2 * (size_t)total);
    double* w = (double*)malloc(sizeof(double) * 2 * (size_t)ncell);
    for (int32_t rr = 0; rr < R; ++rr) {
        or_draw_noise(seed, r0 + (uint64_t)rr, 1, total, M[ndim - 1], dtype, eps);
        or_sample_given_noise(ndim, n, M, s, eps, w);
        double* re = fields + (size_t)rr * 2 * (size_t)ncell;
        double* im = re + ncell;
        for (int64_t i = 0; i < ncell; ++i) {
            re[i] = w[2 * i];
            im[i] = w[2 * i + 1];
        }
    }
    free(eps);
    free(w);
}

/* ======================================================================
 * Section 3.1: rho = 1 + delta is lognormal, A = ln rho Gaussian with mean
 * -sigma_A^2/2 (the centring used in section 3.4's counts-in-cells integral),
 * and counts are Poisson with intensity nbar f_i rho_i, eq. (sampling).
 * ==================================================================== */
double or_poisson_uniform(uint64_t seed, uint64_t cell, uint64_t field)
{
    uint64_t pair = field >> 1;
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t ctr[4] = {(uint32_t)cell, (uint32_t)(cell >> 32), (uint32_t)pair, 1u};
    uint32_t x[4];
    or_philox4x32_10(ctr, key, x);
    uint32_t a = (field & 1) ? x[2] : x[0];
    uint32_t b = (field & 1) ? x[3] : x[1];
    uint64_t i = ((uint64_t)(a >> 5) << 26) | (uint64_t)(b >> 6);
    return (double)i * 0x1p-53; /* [0, 1) */
}

/* Inverse CDF: n = min{ j >= 0 : U < F(j; mu) } with p_0 = e^{-mu},
 * p_{j+1} = p_j (mu/(j+1)), F summed left to right.  The sum stops growing
 * once the tail is below binary64 resolution; then the current j is taken.
 * margin: relative change of mu that would flip the decision,
 * using dF(j;mu)/dmu = -p(j;mu). */
static int32_t or_icdf_small(double U, double mu, double* margin)
{
    int32_t j = 0;
    double p = exp(-mu);
    double F = p;
    double Fprev = 0.0, pprev = 0.0;
    while (!(U < F)) {
        j += 1;
        pprev = p;
        Fprev = F;
        p = p * (mu / (double)j);
        double Fn = F + p;
        if (Fn == F && (double)j > mu) {
            F = Fn;
            break;
        }
        F = Fn;
    }
    if (margin) {
        double up = (p > 0.0) ? (F - U) / p : INFINITY;
        double down = INFINITY;
        if (j > 0 && pprev > 0.0) down = (U - Fprev) / pprev;
        double m = up < down ? up : down;
        *margin = m / mu;
    }
    return j;
}

/* For mu > 700, e^{-mu} underflows: start at the mode m = floor(mu) with
 * p_m = exp(-mu + m ln mu - lnGamma(m+1)), sum F(m) downwards, then walk. */
static int32_t or_icdf_large(double U, double mu, double* margin)
{
    int32_t m = (int32_t)floor(mu);
    double pm = exp(-mu + (double)m * log(mu) - lgamma((double)m + 1.0));
    double S = pm, q = pm;
    for (int32_t j = m; j >= 1; --j) {
        q = q * ((double)j / mu);
        double Sn = S + q;
        if (Sn == S) break;
        S = Sn;
    }
    int32_t j = m;
    double F = S, p = pm;
    if (U < F) {
        /* walk down while U < F(j-1) = F(j) - p(j) */
        while (j > 0 && U < F - p) {
            F = F - p;
            p = p * ((double)j / mu);
            j -= 1;
        }
    } else {
        while (!(U < F)) {
            j += 1;
            p = p * (mu / (double)j);
            double Fn = F + p;
            if (Fn == F) {
                F = Fn;
                break;
            }
            F = Fn;
        }
    }
    if (margin) {
        double up = (p > 0.0) ? (F - U) / p : INFINITY;
        double pprev = p * ((double)j / mu);
        double down = (j > 0 && pprev > 0.0) ? (U - (F - p)) / pprev : INFINITY;
        double mm = up < down ? up : down;
        *margin = mm / mu;
    }
    return j;
}

int32_t or_poisson_icdf(double U, double mu, double* margin)
{
    if (!(mu > 0.0)) {
        if (margin) *margin = INFINITY;
        return 0;
    }
    if (!(mu < 1e9)) {
        /* an intensity this large (or infinite, from an overflowing exp) has
         * no count that an int32 map can hold reliably: saturate */
        if (margin) *margin = INFINITY;
        return INT32_MAX;
    }
    if (mu > 700.0) return or_icdf_large(U, mu, margin);
    return or_icdf_small(U, mu, margin);
}

void or_lognormal_poisson(const double* G, int64_t cells, int64_t nfields, double sigma2,
                          double nbar, const double* f_or_null, uint64_t seed,
                          uint64_t field0, double* delta_out, int32_t* counts_out,
                          double* margin_out)
{
    for (int64_t j = 0; j < nfields; ++j) {
        uint64_t field = field0 + (uint64_t)j;
        for (int64_t i = 0; i < cells; ++i) {
            size_t at = (size_t)(j * cells + i);
            double rho = exp(G[at] - 0.5 * sigma2);
            double f = f_or_null ? f_or_null[i] : 1.0;
            double mu = nbar * f * rho;
            if (delta_out) delta_out[at] = rho - 1.0;
            double U = or_poisson_uniform(seed, (uint64_t)i, field);
            double margin = INFINITY;
            counts_out[at] = or_poisson_icdf(U, mu, &margin);
            if (margin_out) margin_out[at] = margin;
        }
    }
}

/* ======================================================================
 * Section 3.2, eq. (Def spec): P(l) = (1/V)(1/N_l) sum_{l' in bin} |phi~(l')|^2
 * over all Fourier modes of the map (both +k and -k), V = prod(n_i) cell^d,
 * phi~ = cell^d DFT(phi).  Bins are half-open [e_b, e_{b+1}) in |k| in units
 * of the fundamental frequency of the longest side (on a cube the mode index
 * length |n|, n_i in (-n/2, n/2]); the DC mode is excluded.
 * ==================================================================== */
void or_bin_edges(int32_t kind, int32_t nbins, double kmin, double kmax,
                  const double* edges_in, double* edges_out)
{
    for (int32_t b = 0; b <= nbins; ++b) {
        if (kind == OR_BINS_LINEAR)
            edges_out[b] = kmin + (double)b * ((kmax - kmin) / (double)nbins);
        else if (kind == OR_BINS_LOG)
            edges_out[b] = kmin * exp((double)b * (log(kmax / kmin) / (double)nbins));
        else
            edges_out[b] = edges_in[b];
    }
}

void or_power_spectrum(const double* fields, int32_t ndim, const int64_t* n, const double* cell,
                       int64_t nfields, int32_t nbins, const double* edges, double* pk,
                       int64_t* nmodes)
{
    /* Section 3.2, eq. (Def spec): mode m of the survey box has wavevector
     * k_d = 2 pi s_d / L_d with s_d the signed index and L_d = n_d cell_d the
     * side.  |k| is measured in units of the fundamental 2 pi / L_ref of the
     * longest side L_ref: q = sqrt(sum_d (s_d r_d)^2), r_d = L_ref / L_d, each
     * operation rounded in binary64 in this order (for a cube r_d = 1 and q is
     * the integer index length sqrt(sum s_d^2)). */
    int64_t total = 1;
    for (int d = 0; d < ndim; ++d) total *= n[d];
    double vol_cell = 1.0, lref = 0.0, r[3] = {1.0, 1.0, 1.0};
    for (int d = 0; d < ndim; ++d) {
        vol_cell *= cell[d];
        if ((double)n[d] * cell[d] > lref) lref = (double)n[d] * cell[d];
    }
    for (int d = 0; d < ndim; ++d) r[d] = lref / ((double)n[d] * cell[d]);
    double* z = (double*)malloc(sizeof(double) * 2 * (size_t)total);
    double* sums = (double*)malloc(sizeof(double) * (size_t)nbins);
    for (int32_t b = 0; b < nbins; ++b) nmodes[b] = 0;
    for (int64_t f = 0; f < nfields; ++f) {
        for (int64_t i = 0; i < total; ++i) {
            z[2 * i] = fields[f * total + i];
            z[2 * i + 1] = 0.0;
        }
        or_fft_nd(z, ndim, n, -1);
        for (int32_t b = 0; b < nbins; ++b) sums[b] = 0.0;
        for (int64_t idx = 0; idx < total; ++idx) {
            int64_t rem = idx, sv[3] = {0, 0, 0};
            for (int d = ndim - 1; d >= 0; --d) {
                int64_t i = rem % n[d];
                rem /= n[d];
                sv[d] = (2 * i <= n[d]) ? i : i - n[d];
            }
            double q2 = 0.0;
            for (int d = 0; d < ndim; ++d) {
                const double t = (double)sv[d] * r[d];
                q2 = q2 + t * t;
            }
            if (q2 == 0.0) continue;
            double kn = sqrt(q2);
            if (!(kn >= edges[0] && kn < edges[nbins])) continue;
            int32_t b = 0;
            while (!(kn < edges[b + 1])) ++b;
            sums[b] += z[2 * idx] * z[2 * idx] + z[2 * idx + 1] * z[2 * idx + 1];
            if (f == 0) nmodes[b] += 1;
        }
        for (int32_t b = 0; b < nbins; ++b) {
            pk[f * nbins + b] =
                nmodes[b] > 0 ? vol_cell * sums[b] / ((double)total * (double)nmodes[b]) : 0.0;
        }
    }
    free(z);
    free(sums);
}

/* Section 3.2, eq. (Estim) and the map before it:
 * delta_g = (N/f - Nhat)/Nhat where f != 0, 0 elsewhere; Nhat = N_tot / sum f. */
void or_counts_to_delta(const int32_t* counts, const double* f_or_null, int64_t cells,
                        int64_t nfields, double* delta_g)
{
    double fsum = 0.0;
    for (int64_t i = 0; i < cells; ++i) fsum += f_or_null ? f_or_null[i] : 1.0;
    for (int64_t j = 0; j < nfields; ++j) {
        const int32_t* N = counts + j * cells;
        double* out = delta_g + j * cells;
        double ntot = 0.0;
        for (int64_t i = 0; i < cells; ++i) ntot += (double)N[i];
        double nhat = (fsum > 0.0) ? ntot / fsum : 0.0;
        for (int64_t i = 0; i < cells; ++i) {
            double f = f_or_null ? f_or_null[i] : 1.0;
            if (f != 0.0 && nhat > 0.0)
                out[i] = ((double)N[i] / f - nhat) / nhat;
            else
                out[i] = 0.0;
        }
    }
}

/* Section 3.2: prediction and covariance from many simulations -- mean and
 * unbiased (1/(F-1)) covariance of the binned spectra over F fields. */
void or_mean_cov(const double* pk, int64_t nfields, int32_t nbins, double* mean, double* cov)
{
    for (int32_t b = 0; b < nbins; ++b) {
        double s = 0.0;
        for (int64_t f = 0; f < nfields; ++f) s += pk[f * nbins + b];
        mean[b] = nfields > 0 ? s / (double)nfields : 0.0;
    }
    for (int32_t a = 0; a < nbins; ++a) {
        for (int32_t b = 0; b < nbins; ++b) {
            double s = 0.0;
            for (int64_t f = 0; f < nfields; ++f)
                s += (pk[f * nbins + a] - mean[a]) * (pk[f * nbins + b] - mean[b]);
            cov[a * nbins + b] = nfields > 1 ? s / (double)(nfields - 1) : 0.0;
        }
    }
}
