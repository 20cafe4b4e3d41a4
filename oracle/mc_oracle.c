/*
 * FP64 CPU oracle for the Monte Carlo estimator of the trial-success
 * probability (Sec. 2.2, Eq. 5-7), written for clarity, not speed.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow reference that the CUDA
 * path is checked against; it shares no code, header or constant table with
 * the CUDA library, and the CUDA library never calls it.
 *
 * What is computed, per design (Sec. 2.1, Eq. 2-4 and Sec. 2.2, Eq. 6-7):
 *   X = mu + L z,  z ~ N(0, I_d),  Sigma = L L^T  (Eq. 1 / Eq. 3)
 *   success  <=>  X_i > b_i for some i   <=>  y_i > t_i for some i,
 *   with y = L z and t = b - mu.  The estimate of P(success) is hits / N;
 *   Eq. 6-7 count the complement (all X_i <= Z_{1-alpha_i}).
 *
 * Random numbers (a reading: the paper names no generator):
 *   - Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers:
 *     as easy as 1, 2, 3", SC'11), written here from that definition.
 *   - Normal number m = n*d + i (draw n, coordinate i) of a design stream
 *     comes from Philox call c = m / 4, output word m % 4, with counter
 *     (c_lo, c_hi, key_lo, key_hi) and Philox key (seed_lo, seed_hi).
 *   - Word x -> uniform u = (2*floor(x / 2^9) + 1) * 2^-24, in (0, 1).
 *   - Box-Muller on words (0,1) and (2,3): with r = sqrt(-2 ln u0),
 *     z0 = r cos(2 pi u1), z1 = r sin(2 pi u1).
 *
 * Besides the plain hit count the oracle reports, per design, how many draws
 * are "ambiguous": draws whose smallest distance min_i |y_i - t_i| is below a
 * caller-given eps.  Any implementation that evaluates y with an error below
 * eps can disagree with this FP64 count only on those draws.
 *
 * Gradient accumulators (the derivative of P(success) with respect to the
 * mean, used for the adjoint; Appendix A.3 proves the objective smooth):
 *   A_i = sum_n 1[success_n] z_{n,i}      (likelihood ratio numerator)
 *   B_i = sum_n z_{n,i}                   (its zero-mean control variate)
 *   G_i = sum_n prod_k s_k * (1 - s_i) / h,  s_k = 1/(1+exp(-(t_k - y_k)/h))
 *         (the derivative in mu_i of the sigmoid-smoothed indicator
 *          1 - prod_k s_k).
 */
#include <math.h>
#include <stdint.h>
#include <stddef.h>
#include <string.h>

#define PHILOX_M0 0xD2511F53u
#define PHILOX_M1 0xCD9E8D57u
#define PHILOX_W0 0x9E3779B9u
#define PHILOX_W1 0xBB67AE85u

static const double TWO_PI = 6.283185307179586476925286766559;

/* Philox4x32 with 10 rounds: ctr[4], key[2] -> out[4]. */
void oracle_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        uint64_t prod0 = (uint64_t)PHILOX_M0 * (uint64_t)x0;
        uint64_t prod1 = (uint64_t)PHILOX_M1 * (uint64_t)x2;
        uint32_t hi0 = (uint32_t)(prod0 >> 32), lo0 = (uint32_t)prod0;
        uint32_t hi1 = (uint32_t)(prod1 >> 32), lo1 = (uint32_t)prod1;
        uint32_t n0 = hi1 ^ x1 ^ k0;
        uint32_t n1 = lo1;
        uint32_t n2 = hi0 ^ x3 ^ k1;
        uint32_t n3 = lo0;
        x0 = n0; x1 = n1; x2 = n2; x3 = n3;
        k0 += PHILOX_W0;
        k1 += PHILOX_W1;
    }
    out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

/* Word -> uniform in (0,1): the odd multiples of 2^-24. */
double oracle_uniform(uint32_t x)
{
    return (2.0 * (double)(x >> 9) + 1.0) * ldexp(1.0, -24);
}

/* The four standard normals of Philox call `call` of stream (seed, key). */
static void normals_of_call(uint64_t seed, uint64_t key, uint64_t call, double z[4])
{
    uint32_t ctr[4] = {(uint32_t)call, (uint32_t)(call >> 32), (uint32_t)key, (uint32_t)(key >> 32)};
    uint32_t k[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t w[4];
    oracle_philox4x32_10(ctr, k, w);
    for (int pair = 0; pair < 2; ++pair) {
        double u0 = oracle_uniform(w[2 * pair]);
        double u1 = oracle_uniform(w[2 * pair + 1]);
        double r = sqrt(-2.0 * log(u0));
        z[2 * pair] = r * cos(TWO_PI * u1);
        z[2 * pair + 1] = r * sin(TWO_PI * u1);
    }
}

/* Normals with stream indices m_begin .. m_begin+count-1 (for unit checks). */
void oracle_normals(uint64_t seed, uint64_t key, uint64_t m_begin, uint64_t count, double* out)
{
    for (uint64_t k = 0; k < count; ++k) {
        uint64_t m = m_begin + k;
        double z[4];
        normals_of_call(seed, key, m >> 2, z);
        out[k] = z[m & 3];
    }
}

/* Raw Philox words of calls c_begin .. c_begin+count-1 (4 words each). */
void oracle_philox_stream(uint64_t seed, uint64_t key, uint64_t c_begin, uint64_t count, uint32_t* out)
{
    uint32_t k[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    for (uint64_t c = 0; c < count; ++c) {
        uint64_t call = c_begin + c;
        uint32_t ctr[4] = {(uint32_t)call, (uint32_t)(call >> 32), (uint32_t)key, (uint32_t)(key >> 32)};
        oracle_philox4x32_10(ctr, k, out + 4 * c);
    }
}

/* Textbook Cholesky Sigma = L L^T (row-major d x d; L lower, zeros above).
 * Returns 0 on success, 1 + i if the i-th pivot is not positive. */
int oracle_cholesky(int d, const double* Sigma, double* L)
{
    memset(L, 0, sizeof(double) * (size_t)d * (size_t)d);
    for (int i = 0; i < d; ++i) {
        for (int j = 0; j <= i; ++j) {
            double s = Sigma[i * d + j];
            for (int k = 0; k < j; ++k) s -= L[i * d + k] * L[j * d + k];
            if (i == j) {
                if (!(s > 0.0)) return 1 + i;
                L[i * d + i] = sqrt(s);
            } else {
                L[i * d + j] = s / L[j * d + j];
            }
        }
    }
    return 0;
}

static double logistic(double u) { return 1.0 / (1.0 + exp(-u)); }

/*
 * Monte Carlo for one design over draws draw_begin .. draw_begin+n_draws-1.
 *   L: d x d row-major lower Cholesky factor.  t: d thresholds (b - mu);
 *   t_i = +inf drops coordinate i.  eps: ambiguity radius.  h: sigmoid
 *   bandwidth (<= 0 skips G).  A, B, G: d outputs each, or NULL to skip.
 */
void oracle_mc_design(int d, const double* L, const double* t,
                      uint64_t seed, uint64_t key, uint64_t draw_begin, uint64_t n_draws,
                      double eps, double h,
                      uint64_t* hits, uint64_t* ambiguous,
                      double* A, double* B, double* G)
{
    double z[20], y[20];
    uint64_t nh = 0, na = 0;
    if (A) for (int i = 0; i < d; ++i) { A[i] = 0.0; B[i] = 0.0; }
    if (G) for (int i = 0; i < d; ++i) G[i] = 0.0;
    double zc[4];
    uint64_t cached_call = UINT64_MAX;
    for (uint64_t k = 0; k < n_draws; ++k) {
        uint64_t n = draw_begin + k;
        for (int i = 0; i < d; ++i) {
            uint64_t m = n * (uint64_t)d + (uint64_t)i;
            if ((m >> 2) != cached_call) { cached_call = m >> 2; normals_of_call(seed, key, cached_call, zc); }
            z[i] = zc[m & 3];
        }
        int hit = 0;
        double margin = INFINITY;
        for (int i = 0; i < d; ++i) {
            double acc = 0.0;
            for (int j = 0; j <= i; ++j) acc += L[i * d + j] * z[j];
            y[i] = acc;
            if (y[i] > t[i]) hit = 1;
            double gap = fabs(y[i] - t[i]);
            if (gap < margin) margin = gap;
        }
        nh += (uint64_t)hit;
        if (margin < eps) na += 1;
        if (A) for (int i = 0; i < d; ++i) { A[i] += hit ? z[i] : 0.0; B[i] += z[i]; }
        if (G && h > 0.0) {
            double s[20], prod = 1.0;
            for (int i = 0; i < d; ++i) {
                s[i] = isinf(t[i]) ? 1.0 : logistic((t[i] - y[i]) / h);
                prod *= s[i];
            }
            for (int i = 0; i < d; ++i) G[i] += prod * (1.0 - s[i]) / h;
        }
    }
    *hits = nh;
    *ambiguous = na;
}

/* Batch over designs (OpenMP when compiled with -fopenmp).
 *   d: per design; L: per design d*d block at L_off[j]; t: at t_off[j];
 *   grad arrays (optional) at t_off[j].  Returns nothing; all outputs are
 *   written per design. */
void oracle_mc_batch(int64_t n_design, const int32_t* d, const double* L, const int64_t* L_off,
                     const double* t, const int64_t* t_off,
                     uint64_t seed, const uint64_t* key, const uint64_t* draw_begin,
                     const uint64_t* n_draws, double eps, double h,
                     uint64_t* hits, uint64_t* ambiguous, double* A, double* B, double* G)
{
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t j = 0; j < n_design; ++j) {
        oracle_mc_design(d[j], L + L_off[j], t + t_off[j], seed, key[j],
                         draw_begin ? draw_begin[j] : 0, n_draws[j], eps, h,
                         hits + j, ambiguous + j,
                         A ? A + t_off[j] : NULL, A ? B + t_off[j] : NULL,
                         G ? G + t_off[j] : NULL);
    }
}

/* Threads of the batch loop for the calls that follow (timing on one core
 * or on all of them); n < 1 is ignored. */
void oracle_set_num_threads(int n)
{
#ifdef _OPENMP
    extern void omp_set_num_threads(int);
    if (n >= 1) omp_set_num_threads(n);
#else
    (void)n;
#endif
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
