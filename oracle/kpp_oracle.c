/*
 * kpp_oracle.c -- plain, serial, FP64 CPU oracle for k-means++ D^2 seeding.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the correctness reference that the
 * CUDA library is checked against.  Only the test suite, the smoke check in
 * __graft_entry__.py and the CPU-baseline leg of bench.py may load or run it.
 * It shares no code, header, table or helper with the CUDA path, and the CUDA
 * path never calls it.
 *
 * What it computes (Heydarpour Shahrezaei & Tavoli, "Parallelization of
 * Kmeans++ using CUDA", arXiv:1908.02136):
 *   - Algorithm 1 (Serial K-means++): the first seed is a uniformly random
 *     point; every point's nearest distance starts at infinity; for each new
 *     seed the distance of every point to that seed is taken, the nearest
 *     squared distance d_sn is kept, and the next seed is drawn with
 *     probability P(n_l) = d_sn / sum_w d_sn_w (Algorithm 1, the probability
 *     line; the upper summation limit is read as N).
 *   - Section II: the index of every chosen centre is kept in an array and the
 *     centre coordinates are looked up from the point array by that index.
 *   - Section II (Thrust reduction): the sum of all D^2 is taken in double.
 *
 * Readings where the paper is silent (the CUDA library implements the same):
 *   R1  The random draw is u_m = Philox4x64-10(key = {seed, stream},
 *       counter = {m, 0, 0, 0}), word 0 mapped to [0,1) as (w0 >> 11) * 2^-53.
 *       Philox4x64-10 follows Salmon, Moraes, Dror and Shaw, "Parallel Random
 *       Numbers: As Easy as 1, 2, 3", SC'11 (round function, multipliers and
 *       Weyl key increments as published there).
 *   R2  First seed: i_0 = min(floor(u_0 * N), N - 1).
 *   R3  Draw of seed m (m >= 1) by inverse CDF in index order: with
 *       P_i = sum_{k <= i} D^2_k (sequential FP64), T = P_{N-1}, t = u_m * T,
 *       i_m is the smallest i with P_i > t (strict, so zero-weight points are
 *       never drawn).  If rounding leaves no P_i > t, i_m is the largest i
 *       with D^2_i > 0.
 *   R4  Degenerate data: if T == 0 at a draw (fewer distinct points than K),
 *       seeding stops; the remaining indices are -1 and the status is
 *       KPP_ORACLE_DEGENERATE.
 *   R5  Distances are squared Euclidean, summed over j = 0..d-1 in order, in
 *       FP64, in the difference form sum_j (x_ij - c_j)^2.  Stored BF16 and
 *       FP8-e4m3 coordinates are decoded exactly (value = s_i * q_ij for FP8,
 *       formed in double).
 *   R6  There are K distance passes and K-1 draws; the D^2 returned is the one
 *       after the pass for the last centre, and phi = sum_i D^2_i (FP64,
 *       sequential).
 *
 * Quantisers (precision forms; not in the paper):
 *   BF16  round-to-nearest-even of the FP32 value (IEEE 754 rounding applied
 *         to the 8-bit-exponent, 7-bit-fraction format).
 *   FP8   OCP 8-bit floating point, E4M3 ("fn": no infinities, max 448):
 *         per row s_i = max_j |x_ij| / 448 (FP32 division; s_i = 1 for an
 *         all-zero row), q_ij = RNE-with-saturation of the FP32 quotient
 *         x_ij / s_i.
 *
 * Lloyd iteration (the clustering stage after seeding; Section II says it is
 * implemented as the standard K-means algorithm, i.e. Lloyd's):
 *   L1  Assignment: label_i = argmin_k sum_j (x_ij - c_kj)^2 in FP64, the
 *       difference form summed over j in order; the smallest k wins a tie.
 *   L2  Update: c'_k = (sum of the points labelled k, FP64, index order) /
 *       count_k; a centre that no point chose keeps its position (the paper
 *       is silent on empty clusters).
 *   L3  phi = sum_i of the assigned squared distances (FP64, index order),
 *       the cost of the assignment, before the update.
 *
 * k-means|| (the oversampling initialisation of Bahmani et al., the
 * technique the paper cites as an alternative to k-means++):
 *   P1  c_0 = the first seed of R2; D^2 = squared distance to it, phi = sum.
 *   P2  For rounds r = 0 .. R-1: point i joins the candidates iff
 *       u_{r,i} < ell * D^2_i / phi, with u_{r,i} = Philox4x64-10(key = {seed,
 *       stream}, counter = {i, r + 1, 0, 0}), word 0 mapped as in R1 (a point
 *       already chosen has D^2 = 0 and is never chosen again).  The round's
 *       new candidates are appended in increasing point index; D^2 then takes
 *       the minimum over them and phi is recomputed (FP64).
 *   P3  Weight of candidate c = the number of points whose nearest candidate
 *       is c (the earliest candidate in list order on a tie).
 *   P4  Recluster: weighted k-means++ over the candidates in list order --
 *       the first centre by inverse CDF on the weights, then by inverse CDF
 *       on w_c * D^2_c (D^2 to the centres chosen so far), rules of R3, with
 *       draws v_m = Philox4x64-10(key = {seed, stream}, counter = {m, 0, 1,
 *       0}) word 0 mapped as in R1.  Fewer than K candidates with weight, or
 *       a zero total, is a degenerate stop (R4).
 *
 * Build: gcc -O2 -ffp-contract=off -shared -fPIC (no fused multiply-add, so
 * the arithmetic is the one written here on every host).
 */
#define _POSIX_C_SOURCE 200809L /* pthread barriers under -std=c11 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define KPP_ORACLE_OK 0
#define KPP_ORACLE_INVALID 1
#define KPP_ORACLE_DEGENERATE 5

#define KPP_ORACLE_F32 0
#define KPP_ORACLE_BF16 1
#define KPP_ORACLE_FP8_E4M3 2

/* ------------------------------------------------------------------------ */
/* Philox4x64-10 (Salmon et al., SC'11).                                      */
/* ------------------------------------------------------------------------ */

static void mul_hi_lo_64(uint64_t a, uint64_t b, uint64_t *hi, uint64_t *lo)
{
    /* Schoolbook 64x64 -> 128 with 32-bit halves. */
    uint64_t a_lo = a & 0xffffffffu, a_hi = a >> 32;
    uint64_t b_lo = b & 0xffffffffu, b_hi = b >> 32;
    uint64_t p0 = a_lo * b_lo;
    uint64_t p1 = a_lo * b_hi;
    uint64_t p2 = a_hi * b_lo;
    uint64_t p3 = a_hi * b_hi;
    uint64_t mid = (p0 >> 32) + (p1 & 0xffffffffu) + (p2 & 0xffffffffu);
    *lo = (p0 & 0xffffffffu) | (mid << 32);
    *hi = p3 + (p1 >> 32) + (p2 >> 32) + (mid >> 32);
}

void kpp_oracle_philox4x64_10(const uint64_t ctr_in[4], const uint64_t key_in[2],
                              uint64_t out[4])
{
    /* Round multipliers and key (Weyl) increments of Philox4x64. */
    const uint64_t M0 = 0xD2E7470EE14C6C93ull;
    const uint64_t M1 = 0xCA5A826395121157ull;
    const uint64_t W0 = 0x9E3779B97F4A7C15ull; /* golden ratio */
    const uint64_t W1 = 0xBB67AE8584CAA73Bull; /* sqrt(3) - 1 */
    uint64_t x[4] = {ctr_in[0], ctr_in[1], ctr_in[2], ctr_in[3]};
    uint64_t k0 = key_in[0], k1 = key_in[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k0 += W0;
            k1 += W1;
        }
        uint64_t hi0, lo0, hi1, lo1;
        mul_hi_lo_64(M0, x[0], &hi0, &lo0);
        mul_hi_lo_64(M1, x[2], &hi1, &lo1);
        uint64_t y0 = hi1 ^ x[1] ^ k0;
        uint64_t y1 = lo1;
        uint64_t y2 = hi0 ^ x[3] ^ k1;
        uint64_t y3 = lo0;
        x[0] = y0;
        x[1] = y1;
        x[2] = y2;
        x[3] = y3;
    }
    memcpy(out, x, sizeof(x));
}

/* Reading R1: u_m in [0, 1) with 53 random bits. */
double kpp_oracle_uniform(uint64_t seed, uint64_t stream, uint64_t m)
{
    uint64_t ctr[4] = {m, 0, 0, 0};
    uint64_t key[2] = {seed, stream};
    uint64_t out[4];
    kpp_oracle_philox4x64_10(ctr, key, out);
    return (double)(out[0] >> 11) * 0x1.0p-53;
}

/* ------------------------------------------------------------------------ */
/* Stored formats.                                                            */
/* ------------------------------------------------------------------------ */

double kpp_oracle_decode_bf16(uint16_t h)
{
    uint32_t bits = (uint32_t)h << 16; /* BF16 is the top half of FP32 */
    float f;
    memcpy(&f, &bits, sizeof(f));
    return (double)f;
}

double kpp_oracle_decode_e4m3(uint8_t q)
{
    int sign = (q >> 7) & 1;
    int e = (q >> 3) & 0xf;
    int man = q & 0x7;
    double v;
    if (e == 0xf && man == 0x7)
        return NAN;
    if (e == 0)
        v = ldexp((double)man, -9); /* subnormal: man * 2^(1-7) / 8 */
    else
        v = ldexp(1.0 + (double)man / 8.0, e - 7);
    return sign ? -v : v;
}

uint16_t kpp_oracle_encode_bf16(float f)
{
    uint32_t bits;
    memcpy(&bits, &f, sizeof(bits));
    if ((bits & 0x7fffffffu) > 0x7f800000u) /* NaN: keep it a quiet NaN */
        return (uint16_t)((bits >> 16) | 0x0040u);
    /* Round to nearest, ties to even, on the 16 dropped bits. */
    uint32_t lsb = (bits >> 16) & 1u;
    uint32_t rounded = bits + 0x7fffu + lsb;
    return (uint16_t)(rounded >> 16);
}

uint8_t kpp_oracle_encode_e4m3_sat(float f)
{
    if (isnan(f))
        return 0x7f;
    uint8_t sign = signbit(f) ? 0x80 : 0x00;
    double a = fabs((double)f);
    if (a >= 448.0)
        return sign | 0x7e; /* saturate to the largest finite value */
    if (a < 0x1.0p-6) {
        /* Subnormal range: quantum 2^-9; a code of 8 is the smallest normal. */
        double c = rint(a * 512.0); /* default rounding mode: ties to even */
        return sign | (uint8_t)c;
    }
    int ex;
    frexp(a, &ex);      /* a = f * 2^ex, f in [0.5, 1) */
    int e = ex - 1;     /* a in [2^e, 2^(e+1)) with e in [-6, 8] */
    double scaled = rint(ldexp(a, 3 - e)); /* in [8, 16] */
    if (scaled >= 16.0) {
        scaled = 8.0;
        e += 1;
    }
    int biased = e + 7;
    uint8_t code = (uint8_t)((biased << 3) | ((int)scaled - 8));
    if (code > 0x7e)
        code = 0x7e;
    return sign | code;
}

void kpp_oracle_quantize_bf16(const float *x, int64_t n, uint16_t *out)
{
    for (int64_t i = 0; i < n; ++i)
        out[i] = kpp_oracle_encode_bf16(x[i]);
}

void kpp_oracle_quantize_fp8(const float *x, int64_t N, int32_t d, uint8_t *q,
                             float *scales)
{
    for (int64_t i = 0; i < N; ++i) {
        const float *row = x + i * (int64_t)d;
        float mx = 0.0f;
        for (int32_t j = 0; j < d; ++j) {
            float a = fabsf(row[j]);
            if (a > mx)
                mx = a;
        }
        float s = (mx > 0.0f) ? mx / 448.0f : 1.0f;
        scales[i] = s;
        for (int32_t j = 0; j < d; ++j) {
            volatile float v = row[j] / s; /* the FP32 quotient is what is rounded */
            q[i * (int64_t)d + j] = kpp_oracle_encode_e4m3_sat(v);
        }
    }
}

/* Decoded value of coordinate j of point i, in double (reading R5). */
static double coord(const void *pts, const float *scales, int dtype, int64_t i,
                    int32_t d, int32_t j)
{
    int64_t k = i * (int64_t)d + j;
    switch (dtype) {
    case KPP_ORACLE_F32:
        return (double)((const float *)pts)[k];
    case KPP_ORACLE_BF16:
        return kpp_oracle_decode_bf16(((const uint16_t *)pts)[k]);
    default:
        return (double)scales[i] * kpp_oracle_decode_e4m3(((const uint8_t *)pts)[k]);
    }
}

/* ------------------------------------------------------------------------ */
/* The draw (reading R3).                                                     */
/* ------------------------------------------------------------------------ */

/* Inverse-CDF draw over D2[0..N) at uniform u; returns -1 if sum is zero. */
int64_t kpp_oracle_pick(const double *D2, int64_t N, double u, double *t_out,
                        double *T_out)
{
    double T = 0.0;
    for (int64_t i = 0; i < N; ++i)
        T += D2[i];
    double t = u * T;
    if (t_out)
        *t_out = t;
    if (T_out)
        *T_out = T;
    if (T == 0.0)
        return -1;
    double P = 0.0;
    for (int64_t i = 0; i < N; ++i) {
        P += D2[i];
        if (P > t)
            return i;
    }
    for (int64_t i = N - 1; i >= 0; --i)
        if (D2[i] > 0.0)
            return i;
    return -1;
}

/* Per-draw record, used to compare a replayed trajectory with the oracle's own
 * choices.  For draw m: own = the index the oracle draws from its own D^2;
 * t, T as in R3; P_before / P_at = the sequential prefix sums just before and
 * at the replayed index (the one actually taken). */
typedef struct {
    int64_t own;
    double t;
    double T;
    double P_before;
    double P_at;
} kpp_oracle_draw;

/*
 * Algorithm 1, with readings R1-R6.
 *   points     N x d row-major stored values (dtype F32, BF16 or FP8-E4M3)
 *   scales     FP8 per-row scales [N] (NULL otherwise)
 *   forced     optional index prefix of length n_forced that replaces the
 *              oracle's own draws (replay / teacher forcing); NULL if none
 *   idx_out    [K] chosen indices (-1 after a degenerate stop)
 *   d2_out     [N] nearest squared distance after the last pass (FP64)
 *   phi_out    [1] sum of d2_out (FP64), or NULL
 *   draws_out  [K] per-draw records (entry 0: own = first uniform pick), or NULL
 *   d2_hist    [K x N] D^2 after each pass, or NULL (tiny cases only)
 * Returns KPP_ORACLE_OK, KPP_ORACLE_INVALID or KPP_ORACLE_DEGENERATE.
 */
int kpp_oracle_seed(const void *points, const float *scales, int dtype, int64_t N,
                    int32_t d, int32_t K, uint64_t seed, uint64_t stream,
                    const int64_t *forced, int32_t n_forced, int64_t *idx_out,
                    double *d2_out, double *phi_out, kpp_oracle_draw *draws_out,
                    double *d2_hist)
{
    if (!points || !idx_out || !d2_out || N < 1 || d < 1 || K < 1 || K > N ||
        n_forced < 0 || n_forced > K || (n_forced > 0 && !forced) ||
        dtype < 0 || dtype > 2 || (dtype == KPP_ORACLE_FP8_E4M3 && !scales))
        return KPP_ORACLE_INVALID;
    for (int32_t m = 0; m < n_forced; ++m)
        if (forced[m] < 0 || forced[m] >= N)
            return KPP_ORACLE_INVALID;

    /* Decode every stored coordinate to double once (reading R5). */
    double *X = (double *)malloc(sizeof(double) * (size_t)N * (size_t)d);
    if (!X)
        return KPP_ORACLE_INVALID;
    for (int64_t i = 0; i < N; ++i)
        for (int32_t j = 0; j < d; ++j)
            X[i * (int64_t)d + j] = coord(points, scales, dtype, i, d, j);

    for (int32_t m = 0; m < K; ++m)
        idx_out[m] = -1;

    /* First seed, uniformly at random (Algorithm 1; reading R2). */
    double u0 = kpp_oracle_uniform(seed, stream, 0);
    int64_t first = (int64_t)floor(u0 * (double)N);
    if (first > N - 1)
        first = N - 1;
    if (draws_out) {
        memset(draws_out, 0, sizeof(kpp_oracle_draw) * (size_t)K);
        draws_out[0].own = first;
    }
    idx_out[0] = (n_forced > 0) ? forced[0] : first;

    /* O(l) = infinity for every point (Algorithm 1). */
    for (int64_t i = 0; i < N; ++i)
        d2_out[i] = INFINITY;

    int status = KPP_ORACLE_OK;
    for (int32_t m = 0; m < K; ++m) {
        /* Centre coordinates looked up by index (Section II). */
        const double *c = X + idx_out[m] * (int64_t)d;
        /* Distance to the newest seed and nearest squared distance. */
        for (int64_t i = 0; i < N; ++i) {
            double delta = 0.0;
            for (int32_t j = 0; j < d; ++j) {
                double diff = X[i * (int64_t)d + j] - c[j];
                delta += diff * diff;
            }
            if (delta < d2_out[i])
                d2_out[i] = delta;
        }
        if (d2_hist)
            memcpy(d2_hist + (size_t)m * (size_t)N, d2_out, sizeof(double) * (size_t)N);
        if (m == K - 1)
            break;

        /* Draw of seed m+1 with probability D^2 / sum D^2 (reading R3). */
        double u = kpp_oracle_uniform(seed, stream, (uint64_t)(m + 1));
        double t, T;
        int64_t own = kpp_oracle_pick(d2_out, N, u, &t, &T);
        if (T == 0.0) { /* reading R4 */
            status = KPP_ORACLE_DEGENERATE;
            break;
        }
        int64_t taken = (m + 1 < n_forced) ? forced[m + 1] : own;
        idx_out[m + 1] = taken;
        if (draws_out) {
            double P = 0.0;
            for (int64_t i = 0; i < taken; ++i)
                P += d2_out[i];
            draws_out[m + 1].own = own;
            draws_out[m + 1].t = t;
            draws_out[m + 1].T = T;
            draws_out[m + 1].P_before = P;
            draws_out[m + 1].P_at = P + d2_out[taken];
        }
    }
    if (phi_out) {
        double phi = 0.0;
        for (int64_t i = 0; i < N; ++i)
            phi += d2_out[i];
        *phi_out = phi;
    }
    free(X);
    return status;
}

/* ------------------------------------------------------------------------ */
/* One Lloyd iteration (readings L1-L3).                                      */
/* ------------------------------------------------------------------------ */

/*
 * points [N x d] stored values (decoded as in R5), centres [K x d] FP64.
 * Outputs: labels [N], d2 [N] (squared distance to the assigned centre),
 * centres_out [K x d], counts [K], phi.  Any output may be NULL except
 * labels.  Returns KPP_ORACLE_OK or KPP_ORACLE_INVALID.
 */
int kpp_oracle_lloyd_step(const void *points, const float *scales, int dtype, int64_t N,
                          int32_t d, const double *centres, int32_t K, int32_t *labels,
                          double *d2, double *centres_out, int64_t *counts, double *phi)
{
    if (!points || !centres || !labels || N < 1 || d < 1 || K < 1)
        return KPP_ORACLE_INVALID;
    if (dtype == KPP_ORACLE_FP8_E4M3 && !scales)
        return KPP_ORACLE_INVALID;
    double *x = (double *)malloc(sizeof(double) * (size_t)d);
    double *sum = (double *)calloc((size_t)K * (size_t)d, sizeof(double));
    int64_t *cnt = (int64_t *)calloc((size_t)K, sizeof(int64_t));
    if (!x || !sum || !cnt) {
        free(x);
        free(sum);
        free(cnt);
        return KPP_ORACLE_INVALID;
    }
    double total = 0.0;
    for (int64_t i = 0; i < N; ++i) {
        for (int32_t j = 0; j < d; ++j)
            x[j] = coord(points, scales, dtype, i, d, j);
        int32_t best = 0;
        double best_d = INFINITY;
        for (int32_t k = 0; k < K; ++k) {
            const double *c = centres + (int64_t)k * d;
            double s = 0.0;
            for (int32_t j = 0; j < d; ++j) {
                double t = x[j] - c[j];
                s += t * t;
            }
            if (s < best_d) { /* strict: the smallest k wins a tie (L1) */
                best_d = s;
                best = k;
            }
        }
        labels[i] = best;
        if (d2)
            d2[i] = best_d;
        total += best_d;
        cnt[best] += 1;
        double *acc = sum + (int64_t)best * d;
        for (int32_t j = 0; j < d; ++j)
            acc[j] += x[j];
    }
    if (centres_out) {
        for (int32_t k = 0; k < K; ++k)
            for (int32_t j = 0; j < d; ++j)
                centres_out[(int64_t)k * d + j] =
                    cnt[k] > 0 ? sum[(int64_t)k * d + j] / (double)cnt[k]
                               : centres[(int64_t)k * d + j]; /* L2: empty keeps */
    }
    if (counts)
        memcpy(counts, cnt, sizeof(int64_t) * (size_t)K);
    if (phi)
        *phi = total;
    free(x);
    free(sum);
    free(cnt);
    return KPP_ORACLE_OK;
}

/* ------------------------------------------------------------------------ */
/* k-means|| (readings P1-P4).                                                */
/* ------------------------------------------------------------------------ */

/* A uniform in [0, 1) from word 0 of Philox at an explicit counter. */
double kpp_oracle_uniform_ctr(uint64_t seed, uint64_t stream, uint64_t c0, uint64_t c1,
                              uint64_t c2, uint64_t c3)
{
    const uint64_t ctr[4] = {c0, c1, c2, c3};
    const uint64_t key[2] = {seed, stream};
    uint64_t out[4];
    kpp_oracle_philox4x64_10(ctr, key, out);
    return (double)(out[0] >> 11) * (1.0 / 9007199254740992.0);
}

/* FP64 squared distance between point i and point j (decoded, R5). */
static double sqdist(const void *pts, const float *scales, int dtype, int32_t d, int64_t i,
                     int64_t j)
{
    double s = 0.0;
    for (int32_t k = 0; k < d; ++k) {
        double t = coord(pts, scales, dtype, i, d, k) - coord(pts, scales, dtype, j, d, k);
        s += t * t;
    }
    return s;
}

/* D2[i] = min(D2[i], min over the listed centres of the distance to them);
 * with init != 0 D2 starts at +infinity.  Returns the sum (index order). */
double kpp_oracle_min_update(const void *points, const float *scales, int dtype, int64_t N,
                             int32_t d, const int64_t *centres, int64_t n, double *D2, int init)
{
    double phi = 0.0;
    for (int64_t i = 0; i < N; ++i) {
        double best = init ? INFINITY : D2[i];
        for (int64_t c = 0; c < n; ++c) {
            double v = sqdist(points, scales, dtype, d, i, centres[c]);
            if (v < best)
                best = v;
        }
        D2[i] = best;
        phi += best;
    }
    return phi;
}

/* Round r's Bernoulli decisions (P2): flags[i] = 1 iff u_{r,i} < ell D2[i] / phi;
 * p_out[i] (may be NULL) = ell D2[i] / phi, u_out[i] (may be NULL) = u_{r,i}.
 * Returns the number selected. */
int64_t kpp_oracle_kmpar_select(const double *D2, int64_t N, double phi, double ell,
                                uint64_t seed, uint64_t stream, int32_t r, uint8_t *flags,
                                double *p_out, double *u_out)
{
    int64_t n = 0;
    for (int64_t i = 0; i < N; ++i) {
        double p = phi > 0.0 ? ell * D2[i] / phi : 0.0;
        double u = kpp_oracle_uniform_ctr(seed, stream, (uint64_t)i, (uint64_t)r + 1, 0, 0);
        flags[i] = u < p ? 1 : 0;
        n += flags[i];
        if (p_out)
            p_out[i] = p;
        if (u_out)
            u_out[i] = u;
    }
    return n;
}

/* Weights (P3): w[c] = number of points whose nearest candidate is cand[c]. */
void kpp_oracle_kmpar_weights(const void *points, const float *scales, int dtype, int64_t N,
                              int32_t d, const int64_t *cand, int64_t nc, int64_t *w)
{
    for (int64_t c = 0; c < nc; ++c)
        w[c] = 0;
    for (int64_t i = 0; i < N; ++i) {
        int64_t best = 0;
        double best_d = INFINITY;
        for (int64_t c = 0; c < nc; ++c) {
            double v = sqdist(points, scales, dtype, d, i, cand[c]);
            if (v < best_d) {
                best_d = v;
                best = c;
            }
        }
        w[best] += 1;
    }
}

/* Recluster (P4): weighted k-means++ over the candidates; out[m] = position in
 * cand of centre m (-1 after a degenerate stop).  forced (may be NULL) replays
 * the first n_forced positions; own_out[m] (may be NULL) = the oracle's own
 * draw at step m. */
int kpp_oracle_weighted_seed(const void *points, const float *scales, int dtype, int32_t d,
                             const int64_t *cand, int64_t nc, const int64_t *w, int32_t K,
                             uint64_t seed, uint64_t stream, const int64_t *forced,
                             int32_t n_forced, int64_t *out, int64_t *own_out)
{
    if (K < 1 || nc < 1)
        return KPP_ORACLE_INVALID;
    double *D2 = (double *)malloc(sizeof(double) * (size_t)nc);
    double *val = (double *)malloc(sizeof(double) * (size_t)nc);
    if (!D2 || !val) {
        free(D2);
        free(val);
        return KPP_ORACLE_INVALID;
    }
    int status = KPP_ORACLE_OK;
    for (int32_t m = 0; m < K; ++m)
        out[m] = -1;
    for (int64_t c = 0; c < nc; ++c) {
        D2[c] = INFINITY;
        val[c] = (double)w[c];
    }
    for (int32_t m = 0; m < K; ++m) {
        double v = kpp_oracle_uniform_ctr(seed, stream, (uint64_t)m, 0, 1, 0);
        double t, T;
        int64_t own = kpp_oracle_pick(val, nc, v, &t, &T);
        if (own_out)
            own_out[m] = own;
        if (T == 0.0) {
            status = KPP_ORACLE_DEGENERATE;
            break;
        }
        int64_t taken = m < n_forced ? forced[m] : own;
        if (taken < 0 || taken >= nc) {
            status = KPP_ORACLE_INVALID;
            break;
        }
        out[m] = taken;
        for (int64_t c = 0; c < nc; ++c) {
            double dd = sqdist(points, scales, dtype, d, cand[c], cand[taken]);
            if (dd < D2[c])
                D2[c] = dd;
            val[c] = (double)w[c] * D2[c];
        }
    }
    free(D2);
    free(val);
    return status;
}

/*
 * The whole of k-means|| (P1-P4).  cand_out has room for cand_cap indices;
 * n_cand_out gets the number of candidates (the run stops with
 * KPP_ORACLE_INVALID if they do not fit).  idx_out [K]: the chosen points.
 */
int kpp_oracle_kmeans_par(const void *points, const float *scales, int dtype, int64_t N,
                          int32_t d, int32_t K, double ell, int32_t rounds, uint64_t seed,
                          uint64_t stream, int64_t *idx_out, int64_t *cand_out, int64_t cand_cap,
                          int64_t *n_cand_out, int64_t *w_out)
{
    if (!points || N < 1 || d < 1 || K < 1 || K > N || rounds < 0 || !(ell > 0.0) ||
        !idx_out || !cand_out || cand_cap < 1)
        return KPP_ORACLE_INVALID;
    double *D2 = (double *)malloc(sizeof(double) * (size_t)N);
    uint8_t *flags = (uint8_t *)malloc((size_t)N);
    if (!D2 || !flags) {
        free(D2);
        free(flags);
        return KPP_ORACLE_INVALID;
    }
    int status = KPP_ORACLE_OK;
    double u0 = kpp_oracle_uniform(seed, stream, 0);
    int64_t c0 = (int64_t)floor(u0 * (double)N);
    if (c0 > N - 1)
        c0 = N - 1;
    int64_t nc = 0;
    cand_out[nc++] = c0;
    double phi = kpp_oracle_min_update(points, scales, dtype, N, d, &c0, 1, D2, 1);
    for (int32_t r = 0; r < rounds && status == KPP_ORACLE_OK; ++r) {
        kpp_oracle_kmpar_select(D2, N, phi, ell, seed, stream, r, flags, NULL, NULL);
        int64_t first = nc;
        for (int64_t i = 0; i < N; ++i) {
            if (!flags[i])
                continue;
            if (nc >= cand_cap) {
                status = KPP_ORACLE_INVALID;
                break;
            }
            cand_out[nc++] = i;
        }
        if (status != KPP_ORACLE_OK)
            break;
        phi = kpp_oracle_min_update(points, scales, dtype, N, d, cand_out + first, nc - first,
                                    D2, 0);
    }
    int64_t *w = (int64_t *)malloc(sizeof(int64_t) * (size_t)(nc > 0 ? nc : 1));
    int64_t *pos = (int64_t *)malloc(sizeof(int64_t) * (size_t)K);
    if (status == KPP_ORACLE_OK && w && pos) {
        kpp_oracle_kmpar_weights(points, scales, dtype, N, d, cand_out, nc, w);
        status = kpp_oracle_weighted_seed(points, scales, dtype, d, cand_out, nc, w, K, seed,
                                          stream, NULL, 0, pos, NULL);
        for (int32_t m = 0; m < K; ++m)
            idx_out[m] = pos[m] >= 0 ? cand_out[pos[m]] : -1;
        if (w_out)
            memcpy(w_out, w, sizeof(int64_t) * (size_t)nc);
    } else if (status == KPP_ORACLE_OK) {
        status = KPP_ORACLE_INVALID;
    }
    if (n_cand_out)
        *n_cand_out = nc;
    free(w);
    free(pos);
    free(D2);
    free(flags);
    return status;
}

/* ------------------------------------------------------------------------ */
/* Multi-threaded seeding (Algorithm 1, readings R1-R6), for the CPU baseline */
/* ------------------------------------------------------------------------ */

/*
 * The same seeding as kpp_oracle_seed, run by n_threads POSIX threads so that
 * a timing of the oracle uses every host core.  The points are split into
 * n_threads contiguous chunks [t*N/n, (t+1)*N/n).  In every pass each thread
 * takes the FP64 difference-form distance of each point of its chunk to the
 * newest seed (R5, the same operations as the serial oracle, so D^2 is
 * bit-identical to it), keeps the minimum, and sums its chunk's D^2
 * sequentially in FP64.  The draw (R3) then adds the chunk sums in chunk
 * order to form T and t = u_m * T, walks them in order to the first chunk
 * whose running total exceeds t, and rescans that chunk sequentially from
 * the total before it for the first point whose prefix exceeds t -- the
 * prefix P_i of R3 with the sequential sum regrouped at chunk boundaries
 * (identical on integer data, where every sum is exact).  If rounding leaves
 * the rescan short of t, the chunk's last point with D^2 > 0 is taken; if no
 * chunk total exceeds t, the last point with D^2 > 0 overall.  Coordinates are
 * decoded on the fly (no N x d FP64 copy of the points).
 *   idx_out [K], d2_out [N], phi_out [1] or NULL; n_threads >= 1.
 * Returns KPP_ORACLE_OK, KPP_ORACLE_INVALID or KPP_ORACLE_DEGENERATE (R4).
 */
typedef struct {
    const void *points;
    const float *scales;
    int dtype;
    int64_t N;
    int32_t d;
    int32_t n_threads; /* threads actually running (chunks) */
    double *d2;
    double *centre;    /* [d] decoded coordinates of the newest seed */
    double *chunk_sum; /* [n_threads] */
    int first_pass;
    int stop;
    int ready; /* barriers initialised for n_threads: workers may start */
    pthread_mutex_t mu;
    pthread_cond_t cv;
    pthread_barrier_t start, done;
} mt_shared;

typedef struct {
    mt_shared *sh;
    int32_t tid;
} mt_arg;

static int64_t mt_chunk_begin(const mt_shared *sh, int32_t t)
{
    return sh->N * (int64_t)t / sh->n_threads;
}

static void mt_pass(mt_shared *sh, int32_t t)
{
    const int64_t b = mt_chunk_begin(sh, t), e = mt_chunk_begin(sh, t + 1);
    double s = 0.0;
    for (int64_t i = b; i < e; ++i) {
        double delta = 0.0;
        for (int32_t j = 0; j < sh->d; ++j) {
            double diff = coord(sh->points, sh->scales, sh->dtype, i, sh->d, j) - sh->centre[j];
            delta += diff * diff;
        }
        if (sh->first_pass || delta < sh->d2[i])
            sh->d2[i] = delta;
        s += sh->d2[i];
    }
    sh->chunk_sum[t] = s;
}

static void *mt_worker(void *p)
{
    mt_arg *a = (mt_arg *)p;
    mt_shared *sh = a->sh;
    pthread_mutex_lock(&sh->mu);
    while (!sh->ready)
        pthread_cond_wait(&sh->cv, &sh->mu);
    pthread_mutex_unlock(&sh->mu);
    for (;;) {
        pthread_barrier_wait(&sh->start);
        if (sh->stop)
            break;
        mt_pass(sh, a->tid);
        pthread_barrier_wait(&sh->done);
    }
    return NULL;
}

int kpp_oracle_seed_mt(const void *points, const float *scales, int dtype, int64_t N,
                       int32_t d, int32_t K, uint64_t seed, uint64_t stream, int64_t *idx_out,
                       double *d2_out, double *phi_out, int32_t n_threads)
{
    if (!points || !idx_out || !d2_out || N < 1 || d < 1 || K < 1 || K > N || n_threads < 1 ||
        dtype < 0 || dtype > 2 || (dtype == KPP_ORACLE_FP8_E4M3 && !scales))
        return KPP_ORACLE_INVALID;
    if ((int64_t)n_threads > N)
        n_threads = (int32_t)N;
    mt_shared sh;
    memset(&sh, 0, sizeof(sh));
    sh.points = points;
    sh.scales = scales;
    sh.dtype = dtype;
    sh.N = N;
    sh.d = d;
    sh.d2 = d2_out;
    sh.centre = (double *)malloc(sizeof(double) * (size_t)d);
    sh.chunk_sum = (double *)malloc(sizeof(double) * (size_t)n_threads);
    pthread_t *th = (pthread_t *)malloc(sizeof(pthread_t) * (size_t)n_threads);
    mt_arg *args = (mt_arg *)malloc(sizeof(mt_arg) * (size_t)n_threads);
    if (!sh.centre || !sh.chunk_sum || !th || !args) {
        free(sh.centre);
        free(sh.chunk_sum);
        free(th);
        free(args);
        return KPP_ORACLE_INVALID;
    }
    pthread_mutex_init(&sh.mu, NULL);
    pthread_cond_init(&sh.cv, NULL);
    /* workers wait until the barriers exist; if a thread cannot be created,
       the chunks are split over the threads that were */
    int32_t started = 1;
    for (int32_t t = 1; t < n_threads; ++t) {
        args[t].sh = &sh;
        args[t].tid = t;
        if (pthread_create(&th[t], NULL, mt_worker, &args[t]) != 0)
            break;
        ++started;
    }
    sh.n_threads = started;
    pthread_barrier_init(&sh.start, NULL, (unsigned)started);
    pthread_barrier_init(&sh.done, NULL, (unsigned)started);
    pthread_mutex_lock(&sh.mu);
    sh.ready = 1;
    pthread_cond_broadcast(&sh.cv);
    pthread_mutex_unlock(&sh.mu);

    int status = KPP_ORACLE_OK;
    for (int32_t m = 0; m < K; ++m)
        idx_out[m] = -1;
    double u0 = kpp_oracle_uniform(seed, stream, 0); /* R2 */
    int64_t first = (int64_t)floor(u0 * (double)N);
    idx_out[0] = first > N - 1 ? N - 1 : first;
    for (int32_t m = 0; m < K; ++m) {
        for (int32_t j = 0; j < d; ++j)
            sh.centre[j] = coord(points, scales, dtype, idx_out[m], d, j);
        sh.first_pass = (m == 0);
        pthread_barrier_wait(&sh.start);
        mt_pass(&sh, 0);
        pthread_barrier_wait(&sh.done);
        if (m == K - 1)
            break;
        double T = 0.0;
        for (int32_t t = 0; t < sh.n_threads; ++t)
            T += sh.chunk_sum[t];
        if (T == 0.0) { /* R4 */
            status = KPP_ORACLE_DEGENERATE;
            break;
        }
        const double tt = kpp_oracle_uniform(seed, stream, (uint64_t)(m + 1)) * T;
        int64_t pick = -1;
        double run = 0.0;
        for (int32_t c = 0; c < sh.n_threads; ++c) {
            if (run + sh.chunk_sum[c] > tt) {
                const int64_t b = mt_chunk_begin(&sh, c), e = mt_chunk_begin(&sh, c + 1);
                double P = run;
                int64_t lastpos = -1;
                for (int64_t i = b; i < e && pick < 0; ++i) {
                    if (d2_out[i] > 0.0)
                        lastpos = i;
                    P += d2_out[i];
                    if (P > tt)
                        pick = i;
                }
                if (pick < 0)
                    pick = lastpos;
                break;
            }
            run += sh.chunk_sum[c];
        }
        for (int64_t i = N - 1; pick < 0 && i >= 0; --i)
            if (d2_out[i] > 0.0)
                pick = i;
        idx_out[m + 1] = pick;
    }
    sh.stop = 1;
    pthread_barrier_wait(&sh.start);
    for (int32_t t = 1; t < started; ++t)
        pthread_join(th[t], NULL);
    if (status == KPP_ORACLE_OK && phi_out) {
        double phi = 0.0;
        for (int32_t t = 0; t < sh.n_threads; ++t)
            phi += sh.chunk_sum[t];
        *phi_out = phi;
    }
    pthread_barrier_destroy(&sh.start);
    pthread_barrier_destroy(&sh.done);
    pthread_cond_destroy(&sh.cv);
    pthread_mutex_destroy(&sh.mu);
    free(sh.centre);
    free(sh.chunk_sum);
    free(th);
    free(args);
    return status;
}
