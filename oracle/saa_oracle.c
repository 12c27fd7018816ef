/*
 * saa_oracle.c -- plain, slow, FP64 CPU oracle for the Monte Carlo
 * sample-average (SAA) estimate of the mean-variance objective and its
 * gradient (arXiv 2404.11631, Sec. 3.1, Eqs. 3-5, Algorithm 1).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg may load this library.  It shares no code,
 * header, table or constant with the CUDA library: every constant below is
 * written here from its mathematical definition, and the tests pin the
 * oracle against closed forms, brute force and independent library routines.
 *
 * Contents
 *   1. Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers:
 *      as easy as 1, 2, 3", SC'11), the counter-based generator that draws
 *      the i.i.d. samples R_i of Sec. 3.1.
 *   2. The scenario generator: uniforms, Box-Muller normals built on this
 *      file's own LOG / SIN2PI / COS2PI / EXP, and the law transforms.
 *   3. The SAA estimator of Eq. 4 with the sample mean of Eq. 5, written out
 *      directly: R_bar first, then the sum of squared projections of the
 *      centred samples, and the gradient of Eq. 4 in w.  Also the same sums
 *      split by scenario range (partial sums that add across ranges) and the
 *      estimate finalized from their totals.
 *   4. Frank-Wolfe, Algorithm 1 (resample every M iterations, LMO over
 *      W = {w >= 0, 1'w <= 1}, step 2/(kM+m+2)).
 *   5. The relative squared error of Table 2's notes.
 *   6. The lower Cholesky factor C of Sigma (C C' = Sigma), which turns the
 *      covariance of Sec. 3.1's normal law into the sample map R = mu + C z.
 *   7. The newsvendor's Monte Carlo gradient (Sec. 3.2, the approximated
 *      gradient): per product j, k_j - v_j + (h_j + v_j) times the fraction
 *      of S normal demand samples d_j = mu_j + sigma_j z that are <= x_j.
 *   8. The binary-classification task of Sec. 3.3: the synthetic data set of
 *      Sec. 4.1's setup (binary features, labels from a random linear rule
 *      with 10 % label noise), the objective F(omega) (negative mean
 *      log-likelihood of the logistic model), its sample-average gradient
 *      and the sub-sampled Hessian applied to a vector.
 *
 * Floating-point discipline: compiled with -ffp-contract=off; every fused
 * multiply-add in the generator is an explicit fmaf()/fma() call, so each
 * operation rounds exactly once in IEEE round-to-nearest-even.
 *
 * Sums over scenarios use Neumaier compensation over a fixed partition of the
 * scenario range into chunks that are merged in chunk order, so results do
 * not depend on the number of OpenMP threads.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_OK 0
#define OR_EINVAL 1
#define OR_ENOMEM 2

/* Law codes (scenario distributions). */
#define OR_LAW_GAUSS 0     /* R = mu + C z, z ~ N(0, I): R ~ N(mu, Sigma), Sec. 3.1 */
#define OR_LAW_LOGN_STD 1  /* z replaced by standardised lognormal (sigma=1) innovations */
#define OR_LAW_STUDENT_T 2 /* R = mu + s C z, s = sqrt(nu / chi2_nu): multivariate t */
#define OR_LAW_MIX 3       /* scenarios i < N/2 Gaussian, i >= N/2 standardised lognormal */

typedef struct {
    int32_t d;        /* decision / asset dimension */
    int64_t N;        /* number of samples R_i */
    int32_t law;      /* OR_LAW_* */
    int32_t nu;       /* degrees of freedom (even) for the t law */
    double lambda;    /* weight of the variance term (1/2 in Eq. 3) */
    uint64_t seed;    /* Philox key */
    uint32_t instance;/* instance id (low 24 bits of counter word 3) */
    uint32_t epoch;   /* resample index (counter word 2) */
    const double* mu;   /* [d] mean of R */
    const double* chol; /* [d*d] row-major lower-triangular C with C C' = Sigma, or NULL */
    const double* sd;   /* [d] with chol NULL: Sigma = diag(sd^2), the independent assets of Sec. 4.1 */
} oracle_problem;

/* ------------------------------------------------------------------------- */
/* 1. Philox4x32-10                                                          */
/* ------------------------------------------------------------------------- */
/* Round multipliers and Weyl key increments of Philox4x32 (SC'11, Table 2). */
#define PHILOX_M0 0xD2511F53u
#define PHILOX_M1 0xCD9E8D57u
#define PHILOX_W0 0x9E3779B9u /* golden ratio */
#define PHILOX_W1 0xBB67AE85u /* sqrt(3) - 1 */

static void philox10(const uint32_t in[4], uint32_t k0, uint32_t k1, uint32_t out[4])
{
    uint32_t x0 = in[0], x1 = in[1], x2 = in[2], x3 = in[3];
    for (int r = 0; r < 10; ++r) {
        if (r > 0) {
            k0 += PHILOX_W0;
            k1 += PHILOX_W1;
        }
        uint64_t p0 = (uint64_t)PHILOX_M0 * (uint64_t)x0;
        uint64_t p1 = (uint64_t)PHILOX_M1 * (uint64_t)x2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t y0 = hi1 ^ x1 ^ k0;
        uint32_t y1 = lo1;
        uint32_t y2 = hi0 ^ x3 ^ k1;
        uint32_t y3 = lo0;
        x0 = y0; x1 = y1; x2 = y2; x3 = y3;
    }
    out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

void oracle_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    philox10(ctr, key[0], key[1], out);
}

void oracle_philox_batch(int64_t n, const uint32_t* ctr, const uint32_t* key, uint32_t* out)
{
    for (int64_t i = 0; i < n; ++i) philox10(ctr + 4 * i, key[2 * i], key[2 * i + 1], out + 4 * i);
}

/* ------------------------------------------------------------------------- */
/* 2. Own elementary functions                                               */
/* ------------------------------------------------------------------------- */
/* Constants, each the correctly rounded value of the stated real number.
 * Decimal literals carry 40 significant digits; the compiler rounds them
 * once to the target format.  Dyadic constants are written exactly in hex. */

/* sqrt(2) */
static const float SQRT2_F = 1.414213562373095048801688724209698078570f;
static const double SQRT2_D = 1.414213562373095048801688724209698078570;
/* Cody-Waite split of ln 2: the high part is ln 2 rounded to 16 (float) or
 * 32 (double) significant bits, so e * LN2_HI is exact for every exponent e
 * that occurs; the low part is the rounded remainder ln 2 - LN2_HI. */
static const float LN2_HI_F = 0x1.62e4p-1f;
static const float LN2_LO_F = 0x1.7f7d1cp-20f;
static const double LN2_HI_D = 0x1.62e42ffp-1;
static const double LN2_LO_D = -0x1.718432a1b0e26p-35;
/* 1 / ln 2 */
static const float LOG2E_F = 1.442695040888963407359924681001892137427f;
static const double LOG2E_D = 1.442695040888963407359924681001892137427;
/* e^(1/2) = mean of exp(Z), Z ~ N(0,1) */
static const float E_HALF_F = 1.648721270700128146848650787814163571654f;
static const double E_HALF_D = 1.648721270700128146848650787814163571654;
/* 1 / sqrt(e^2 - e) = 1 / standard deviation of exp(Z) */
static const float INV_SD_LN_F = 0.4627064573764711388582888487271463418743f;
static const double INV_SD_LN_D = 0.4627064573764711388582888487271463418743;

/* log(m) = 2 atanh(s), s = (m-1)/(m+1):  2 atanh(s) = s * sum_k 2/(2k+1) s^(2k).
 * Coefficients 2/(2k+1), k = 0..4 (float) and k = 0..10 (double). */
#define NLOG_F 5
#define NLOG_D 11
static const float LOGP_F[NLOG_F] = {
    2.0f,
    0.6666666666666666666666666666666666666667f,
    0.4000000000000000000000000000000000000000f,
    0.2857142857142857142857142857142857142857f,
    0.2222222222222222222222222222222222222222f,
};
static const double LOGP_D[NLOG_D] = {
    2.0,
    0.6666666666666666666666666666666666666667,
    0.4000000000000000000000000000000000000000,
    0.2857142857142857142857142857142857142857,
    0.2222222222222222222222222222222222222222,
    0.1818181818181818181818181818181818181818,
    0.1538461538461538461538461538461538461538,
    0.1333333333333333333333333333333333333333,
    0.1176470588235294117647058823529411764706,
    0.1052631578947368421052631578947368421053,
    0.09523809523809523809523809523809523809524,
};

/* Taylor series of sin(2 pi r) / r and cos(2 pi r) in t = r^2:
 *   sin: (-1)^k (2 pi)^(2k+1) / (2k+1)!,   cos: (-1)^k (2 pi)^(2k) / (2k)!
 * 5 / 6 terms in float, 9 / 10 terms in double (|2 pi r| <= pi/4). */
#define NSIN_F 5
#define NCOS_F 6
#define NSIN_D 9
#define NCOS_D 10
static const float SINP_F[NSIN_F] = {
    6.283185307179586476925286766559005768394f,
    -41.34170224039976023396842008946852693630f,
    81.60524927607505420339768267824949506141f,
    -76.70585975306138584163064109389312588997f,
    42.05869394489765314498681114813355254161f,
};
static const float COSP_F[NCOS_F] = {
    1.0f,
    -19.73920880217871723766898199975230227063f,
    64.93939402266829149096022179247007416649f,
    -85.45681720669372773601950610243732434375f,
    60.24464137187666036272111431051914791554f,
    -26.42625678337439745290065331496842204896f,
};
static const double SINP_D[NSIN_D] = {
    6.283185307179586476925286766559005768394,
    -41.34170224039976023396842008946852693630,
    81.60524927607505420339768267824949506141,
    -76.70585975306138584163064109389312588997,
    42.05869394489765314498681114813355254161,
    -15.09464257682299039182661623253152051448,
    3.819952584848282127733792067340466125441,
    -0.7181223017785005122317402786068623805399,
    0.1042291622081398411727104489876041109703,
};
static const double COSP_D[NCOS_D] = {
    1.0,
    -19.73920880217871723766898199975230227063,
    64.93939402266829149096022179247007416649,
    -85.45681720669372773601950610243732434375,
    60.24464137187666036272111431051914791554,
    -26.42625678337439745290065331496842204896,
    7.903536371318468804212103428857682494130,
    -1.714390711088672065421586077323089143567,
    0.2820059684557912150702701749840722854475,
    -0.03638284114254567077175122330646765486151,
};

/* exp(r) Taylor series 1/j!, degree 7 (float) and 13 (double), |r| <= ln2/2. */
#define NEXP_F 8
#define NEXP_D 14
static const float EXPP_F[NEXP_F] = {
    1.0f, 1.0f, 0.5f,
    0.1666666666666666666666666666666666666667f,
    0.04166666666666666666666666666666666666667f,
    0.008333333333333333333333333333333333333333f,
    0.001388888888888888888888888888888888888889f,
    0.0001984126984126984126984126984126984126984f,
};
static const double EXPP_D[NEXP_D] = {
    1.0, 1.0, 0.5,
    0.1666666666666666666666666666666666666667,
    0.04166666666666666666666666666666666666667,
    0.008333333333333333333333333333333333333333,
    0.001388888888888888888888888888888888888889,
    0.0001984126984126984126984126984126984126984,
    0.00002480158730158730158730158730158730158730,
    0.000002755731922398589065255731922398589065256,
    0.0000002755731922398589065255731922398589065256,
    0.00000002505210838544171877505210838544171877505,
    0.000000002087675698786809897921009032120143231254,
    0.0000000001605904383682161459939237717015494793273,
};

/* Natural log of a positive normal float u < 2^128.
 * u = 2^e m with m in [1,2); if m > sqrt(2) use m/2, e+1 so m in
 * [sqrt(2)/2, sqrt(2)]; log u = e ln2 + 2 atanh((m-1)/(m+1)). */
static float own_logf(float u)
{
    uint32_t b;
    memcpy(&b, &u, 4);
    int e = (int)((b >> 23) & 0xffu) - 127;
    uint32_t mb = (b & 0x7fffffu) | 0x3f800000u;
    float m;
    memcpy(&m, &mb, 4);
    if (m > SQRT2_F) {
        m = m * 0.5f;
        e = e + 1;
    }
    float f = m - 1.0f; /* exact (Sterbenz) */
    float g = m + 1.0f;
    float s = f / g;
    float t = s * s;
    float p = LOGP_F[NLOG_F - 1];
    for (int k = NLOG_F - 2; k >= 0; --k) p = fmaf(p, t, LOGP_F[k]);
    float ls = s * p;
    float ef = (float)e;
    float hi = ef * LN2_HI_F; /* exact */
    float lo = fmaf(ef, LN2_LO_F, ls);
    return hi + lo;
}

static double own_log(double u)
{
    uint64_t b;
    memcpy(&b, &u, 8);
    int e = (int)((b >> 52) & 0x7ffu) - 1023;
    uint64_t mb = (b & 0xfffffffffffffull) | 0x3ff0000000000000ull;
    double m;
    memcpy(&m, &mb, 8);
    if (m > SQRT2_D) {
        m = m * 0.5;
        e = e + 1;
    }
    double f = m - 1.0;
    double g = m + 1.0;
    double s = f / g;
    double t = s * s;
    double p = LOGP_D[NLOG_D - 1];
    for (int k = NLOG_D - 2; k >= 0; --k) p = fma(p, t, LOGP_D[k]);
    double ls = s * p;
    double ef = (double)e;
    double hi = ef * LN2_HI_D;
    double lo = fma(ef, LN2_LO_D, ls);
    return hi + lo;
}

/* sin(2 pi u), cos(2 pi u) for u = n 2^-24, n an odd integer in [1, 2^24).
 * The quadrant q = round(4u) and the remainder r = u - q/4 (|r| <= 1/8) are
 * exact integer operations; the result is rotated by q quarter turns. */
static void own_sincos2pif(uint32_t n, float* s_out, float* c_out)
{
    uint32_t q = (n + (1u << 21)) >> 22;
    int32_t ri = (int32_t)n - (int32_t)(q << 22);
    float r = (float)ri * 0x1p-24f; /* exact */
    float t = r * r;
    float ps = SINP_F[NSIN_F - 1];
    for (int k = NSIN_F - 2; k >= 0; --k) ps = fmaf(ps, t, SINP_F[k]);
    float sn = r * ps;
    float pc = COSP_F[NCOS_F - 1];
    for (int k = NCOS_F - 2; k >= 0; --k) pc = fmaf(pc, t, COSP_F[k]);
    float cs = pc;
    switch (q & 3u) {
    case 0: *s_out = sn; *c_out = cs; break;
    case 1: *s_out = cs; *c_out = -sn; break;
    case 2: *s_out = -sn; *c_out = -cs; break;
    default: *s_out = -cs; *c_out = sn; break;
    }
}

/* Same for u = n 2^-53, n odd in [1, 2^53). */
static void own_sincos2pi(uint64_t n, double* s_out, double* c_out)
{
    uint64_t q = (n + (1ull << 50)) >> 51;
    int64_t ri = (int64_t)n - (int64_t)(q << 51);
    double r = (double)ri * 0x1p-53;
    double t = r * r;
    double ps = SINP_D[NSIN_D - 1];
    for (int k = NSIN_D - 2; k >= 0; --k) ps = fma(ps, t, SINP_D[k]);
    double sn = r * ps;
    double pc = COSP_D[NCOS_D - 1];
    for (int k = NCOS_D - 2; k >= 0; --k) pc = fma(pc, t, COSP_D[k]);
    double cs = pc;
    switch (q & 3u) {
    case 0: *s_out = sn; *c_out = cs; break;
    case 1: *s_out = cs; *c_out = -sn; break;
    case 2: *s_out = -sn; *c_out = -cs; break;
    default: *s_out = -cs; *c_out = sn; break;
    }
}

/* exp(x) for |x| < 80: x = k ln2 + r with k = rint(x / ln2) (Cody-Waite
 * reduction with the split ln 2), exp(r) by its Taylor polynomial, and the
 * factor 2^k placed in the exponent field. */
static float own_expf(float x)
{
    float kf = rintf(x * LOG2E_F);
    float r = fmaf(-kf, LN2_HI_F, x);
    r = fmaf(-kf, LN2_LO_F, r);
    float p = EXPP_F[NEXP_F - 1];
    for (int j = NEXP_F - 2; j >= 0; --j) p = fmaf(p, r, EXPP_F[j]);
    int k = (int)kf;
    uint32_t sb = (uint32_t)(k + 127) << 23;
    float sc;
    memcpy(&sc, &sb, 4);
    return p * sc;
}

static double own_exp(double x)
{
    double kf = rint(x * LOG2E_D);
    double r = fma(-kf, LN2_HI_D, x);
    r = fma(-kf, LN2_LO_D, r);
    double p = EXPP_D[NEXP_D - 1];
    for (int j = NEXP_D - 2; j >= 0; --j) p = fma(p, r, EXPP_D[j]);
    int64_t k = (int64_t)kf;
    uint64_t sb = (uint64_t)(k + 1023) << 52;
    double sc;
    memcpy(&sc, &sb, 8);
    return p * sc;
}

/* Test hooks for the elementary functions. */
void oracle_log_f32(int64_t n, const float* u, float* out)
{
    for (int64_t i = 0; i < n; ++i) out[i] = own_logf(u[i]);
}
void oracle_log_f64(int64_t n, const double* u, double* out)
{
    for (int64_t i = 0; i < n; ++i) out[i] = own_log(u[i]);
}
void oracle_exp_f32(int64_t n, const float* x, float* out)
{
    for (int64_t i = 0; i < n; ++i) out[i] = own_expf(x[i]);
}
void oracle_exp_f64(int64_t n, const double* x, double* out)
{
    for (int64_t i = 0; i < n; ++i) out[i] = own_exp(x[i]);
}
void oracle_sincos2pi_f32(int64_t n, const uint32_t* num, float* s, float* c)
{
    for (int64_t i = 0; i < n; ++i) own_sincos2pif(num[i], s + i, c + i);
}
void oracle_sincos2pi_f64(int64_t n, const uint64_t* num, double* s, double* c)
{
    for (int64_t i = 0; i < n; ++i) own_sincos2pi(num[i], s + i, c + i);
}

/* Export of the constant tables, so that a test can compare each entry with
 * the correctly rounded value of its definition.  which: 0 = float scalars
 * {SQRT2, LN2_HI, LN2_LO, LOG2E, E_HALF, INV_SD_LN}, 1 = double scalars (same
 * order), 2 = LOGP_F, 3 = LOGP_D, 4 = SINP_F, 5 = SINP_D, 6 = COSP_F,
 * 7 = COSP_D, 8 = EXPP_F, 9 = EXPP_D.  Returns the entry count. */
int oracle_constants(int which, double* out, int cap)
{
    const float fs[6] = {SQRT2_F, LN2_HI_F, LN2_LO_F, LOG2E_F, E_HALF_F, INV_SD_LN_F};
    const double ds[6] = {SQRT2_D, LN2_HI_D, LN2_LO_D, LOG2E_D, E_HALF_D, INV_SD_LN_D};
    const float* f = NULL;
    const double* dd = NULL;
    int n = 0;
    switch (which) {
    case 0: f = fs; n = 6; break;
    case 1: dd = ds; n = 6; break;
    case 2: f = LOGP_F; n = NLOG_F; break;
    case 3: dd = LOGP_D; n = NLOG_D; break;
    case 4: f = SINP_F; n = NSIN_F; break;
    case 5: dd = SINP_D; n = NSIN_D; break;
    case 6: f = COSP_F; n = NCOS_F; break;
    case 7: dd = COSP_D; n = NCOS_D; break;
    case 8: f = EXPP_F; n = NEXP_F; break;
    case 9: dd = EXPP_D; n = NEXP_D; break;
    default: return -1;
    }
    for (int k = 0; k < n && k < cap; ++k) out[k] = f ? (double)f[k] : dd[k];
    return n;
}

/* ------------------------------------------------------------------------- */
/* 2b. Scenario generator                                                    */
/* ------------------------------------------------------------------------- */
/* Counter layout: c0 = dimension block, c1 = scenario index i, c2 = epoch
 * (resample index), c3 = (tag << 24) | instance.  Tag 0 draws the normals,
 * tag 1 the chi-square uniforms of the t law.  Key = (seed lo, seed hi). */
#define TAG_NORMAL 0u
#define TAG_CHI2 1u

static void draw(const oracle_problem* p, uint32_t block, uint32_t i, uint32_t epoch, uint32_t tag,
                 uint32_t out[4])
{
    uint32_t c[4];
    c[0] = block;
    c[1] = i;
    c[2] = epoch;
    c[3] = (tag << 24) | (p->instance & 0xffffffu);
    philox10(c, (uint32_t)(p->seed & 0xffffffffu), (uint32_t)(p->seed >> 32), out);
}

/* Odd numerators of the uniforms: u = n 2^-24 and u = n 2^-53, both in (0,1). */
static uint32_t u24_num(uint32_t x) { return 2u * (x >> 9) + 1u; }
static float u24(uint32_t x) { return (float)u24_num(x) * 0x1p-24f; }
static uint64_t u53_num(uint32_t a, uint32_t b)
{
    uint64_t v = ((uint64_t)a << 32) | (uint64_t)b;
    return 2ull * (v >> 12) + 1ull;
}
static double u53(uint32_t a, uint32_t b) { return (double)u53_num(a, b) * 0x1p-53; }

/* Box-Muller: r = sqrt(-2 log u1), (z0, z1) = (r cos 2 pi u2, r sin 2 pi u2). */
static void box_muller_f(float u1, uint32_t n2, float* z0, float* z1)
{
    float L = own_logf(u1);
    float r = sqrtf(-2.0f * L);
    float sn, cs;
    own_sincos2pif(n2, &sn, &cs);
    *z0 = r * cs;
    *z1 = r * sn;
}
static void box_muller_d(double u1, uint64_t n2, double* z0, double* z1)
{
    double L = own_log(u1);
    double r = sqrt(-2.0 * L);
    double sn, cs;
    own_sincos2pi(n2, &sn, &cs);
    *z0 = r * cs;
    *z1 = r * sn;
}

static int law_is_lognormal(const oracle_problem* p, int64_t i)
{
    if (p->law == OR_LAW_LOGN_STD) return 1;
    if (p->law == OR_LAW_MIX) return i >= p->N / 2;
    return 0;
}

/* Scenario i in float mode: d innovations zhat and the scale s. */
static void gen_f32(const oracle_problem* p, int64_t i, uint32_t epoch, float* zhat, float* s_out)
{
    const int d = p->d;
    for (int b = 0; 4 * b < d; ++b) {
        uint32_t x[4];
        draw(p, (uint32_t)b, (uint32_t)i, epoch, TAG_NORMAL, x);
        float z[4];
        box_muller_f(u24(x[0]), u24_num(x[1]), &z[0], &z[1]);
        box_muller_f(u24(x[2]), u24_num(x[3]), &z[2], &z[3]);
        for (int q = 0; q < 4 && 4 * b + q < d; ++q) zhat[4 * b + q] = z[q];
    }
    if (law_is_lognormal(p, i)) {
        for (int j = 0; j < d; ++j) zhat[j] = (own_expf(zhat[j]) - E_HALF_F) * INV_SD_LN_F;
    }
    float s = 1.0f;
    if (p->law == OR_LAW_STUDENT_T) {
        float acc = 0.0f;
        uint32_t x[4];
        for (int r = 0; r < p->nu / 2; ++r) {
            if (r % 4 == 0) draw(p, (uint32_t)(r / 4), (uint32_t)i, epoch, TAG_CHI2, x);
            acc = acc + own_logf(u24(x[r % 4]));
        }
        float W = -2.0f * acc;
        s = sqrtf((float)p->nu / W);
    }
    *s_out = s;
}

/* Scenario i in double mode. */
static void gen_f64(const oracle_problem* p, int64_t i, uint32_t epoch, double* zhat, double* s_out)
{
    const int d = p->d;
    for (int b = 0; 2 * b < d; ++b) {
        uint32_t x[4];
        draw(p, (uint32_t)b, (uint32_t)i, epoch, TAG_NORMAL, x);
        double z[2];
        box_muller_d(u53(x[0], x[1]), u53_num(x[2], x[3]), &z[0], &z[1]);
        for (int q = 0; q < 2 && 2 * b + q < d; ++q) zhat[2 * b + q] = z[q];
    }
    if (law_is_lognormal(p, i)) {
        for (int j = 0; j < d; ++j) zhat[j] = (own_exp(zhat[j]) - E_HALF_D) * INV_SD_LN_D;
    }
    double s = 1.0;
    if (p->law == OR_LAW_STUDENT_T) {
        double acc = 0.0;
        uint32_t x[4];
        for (int r = 0; r < p->nu / 2; ++r) {
            if (r % 2 == 0) draw(p, (uint32_t)(r / 2), (uint32_t)i, epoch, TAG_CHI2, x);
            int w = 2 * (r % 2);
            acc = acc + own_log(u53(x[w], x[w + 1]));
        }
        double W = -2.0 * acc;
        s = sqrt((double)p->nu / W);
    }
    *s_out = s;
}

static int check_problem(const oracle_problem* p)
{
    if (!p || p->d < 1 || p->N < 2 || p->N > 0xffffffffll) return OR_EINVAL;
    if (p->law < 0 || p->law > OR_LAW_MIX) return OR_EINVAL;
    if (p->law == OR_LAW_STUDENT_T && (p->nu < 2 || (p->nu & 1))) return OR_EINVAL;
    if (!p->mu || (!p->chol && !p->sd)) return OR_EINVAL;
    return OR_OK;
}

/* Innovations and scales of scenarios i0..i0+n-1 (promoted to double), and
 * optionally the scenarios themselves at scenario precision:
 *   xi_ij = fma(s_i, acc_j, mu_j),  acc_j = fma chain over l = 0..j of
 *   C_jl zhat_il in increasing l, with C and mu first rounded to that precision.
 * prec: 32 = float scenarios, 64 = double scenarios. */
int oracle_generate(const oracle_problem* p, int prec, uint32_t epoch, int64_t i0, int64_t n,
                    double* zhat, double* s, double* xi)
{
    if (check_problem(p) != OR_OK || (prec != 32 && prec != 64) || i0 < 0 || n < 0 || i0 + n > p->N)
        return OR_EINVAL;
    if (xi && !p->chol) return OR_EINVAL;   /* the sample map of this output needs the dense C */
    const int d = p->d;
    int err = OR_OK;
#pragma omp parallel
    {
        float* zf = (float*)malloc(sizeof(float) * (size_t)d);
        double* zd = (double*)malloc(sizeof(double) * (size_t)d);
        float* Cf = NULL;
        float* muf = NULL;
        if (xi && prec == 32) {
            Cf = (float*)malloc(sizeof(float) * (size_t)d * (size_t)d);
            muf = (float*)malloc(sizeof(float) * (size_t)d);
            if (Cf && muf) {
                for (int64_t k = 0; k < (int64_t)d * d; ++k) Cf[k] = (float)p->chol[k];
                for (int j = 0; j < d; ++j) muf[j] = (float)p->mu[j];
            }
        }
        if (!zf || !zd || (xi && prec == 32 && (!Cf || !muf))) {
#pragma omp atomic write
            err = OR_ENOMEM;
        } else {
#pragma omp for schedule(static)
            for (int64_t r = 0; r < n; ++r) {
                int64_t i = i0 + r;
                if (prec == 32) {
                    float sf;
                    gen_f32(p, i, epoch, zf, &sf);
                    for (int j = 0; j < d; ++j) zhat[r * d + j] = (double)zf[j];
                    if (s) s[r] = (double)sf;
                    if (xi) {
                        for (int j = 0; j < d; ++j) {
                            float acc = 0.0f;
                            for (int l = 0; l <= j; ++l) acc = fmaf(Cf[(int64_t)j * d + l], zf[l], acc);
                            xi[r * d + j] = (double)fmaf(sf, acc, muf[j]);
                        }
                    }
                } else {
                    double sd;
                    gen_f64(p, i, epoch, zd, &sd);
                    for (int j = 0; j < d; ++j) zhat[r * d + j] = zd[j];
                    if (s) s[r] = sd;
                    if (xi) {
                        for (int j = 0; j < d; ++j) {
                            double acc = 0.0;
                            for (int l = 0; l <= j; ++l) acc = fma(p->chol[(int64_t)j * d + l], zd[l], acc);
                            xi[r * d + j] = fma(sd, acc, p->mu[j]);
                        }
                    }
                }
            }
        }
        free(zf);
        free(zd);
        free(Cf);
        free(muf);
    }
    return err;
}

/* ------------------------------------------------------------------------- */
/* 3. SAA estimator, Eq. 4 with Eq. 5                                        */
/* ------------------------------------------------------------------------- */
/* Neumaier-compensated running sum. */
typedef struct {
    double s, c;
} nsum;
static void nadd(nsum* a, double x)
{
    double t = a->s + x;
    if (fabs(a->s) >= fabs(x))
        a->c += (a->s - t) + x;
    else
        a->c += (x - t) + a->s;
    a->s = t;
}
static double nval(const nsum* a) { return a->s + a->c; }

/* Where the samples R_i come from: an explicit N x d matrix, or the
 * generator (R_i = mu + s_i C zhat_i formed in double from the innovations
 * promoted to double). */
typedef struct {
    const oracle_problem* p; /* generator source when R == NULL */
    int prec;
    uint32_t epoch;
    const double* R;         /* explicit source, row-major N x d */
    const double* Ct;        /* transpose of C (column-major C) */
    int64_t N;
    int d;
} sample_src;

typedef struct {
    float* zf;
    double* zd;
} sample_buf;

/* Writes sample R_i into out[d]. */
static void get_sample(const sample_src* S, sample_buf* B, int64_t i, double* out)
{
    const int d = S->d;
    if (S->R) {
        memcpy(out, S->R + i * d, sizeof(double) * (size_t)d);
        return;
    }
    double s;
    if (S->prec == 32) {
        float sf;
        gen_f32(S->p, i, S->epoch, B->zf, &sf);
        for (int j = 0; j < d; ++j) B->zd[j] = (double)B->zf[j];
        s = (double)sf;
    } else {
        gen_f64(S->p, i, S->epoch, B->zd, &s);
    }
    if (!S->Ct) {
        /* C = diag(sd): out_j = mu_j + s_i * (sd_j zhat_j), the same roundings as
         * the sum below for a diagonal C (whose other terms add exact zeros). */
        for (int j = 0; j < d; ++j) out[j] = S->p->mu[j] + s * (S->p->sd[j] * B->zd[j]);
        return;
    }
    /* R_i = mu + s_i C zhat_i: out_j = mu_j + s_i * sum_{l<=j} C_jl zhat_l,
     * each sum taken in increasing l (loops interchanged over j only). */
    for (int j = 0; j < d; ++j) out[j] = 0.0;
    for (int l = 0; l < d; ++l) {
        const double zl = B->zd[l];
        const double* col = S->Ct + (int64_t)l * d;
        for (int j = l; j < d; ++j) out[j] = out[j] + col[j] * zl;
    }
    for (int j = 0; j < d; ++j) out[j] = S->p->mu[j] + s * out[j];
}

#define MAX_CHUNKS 64

/* f_k   = lambda * (1/(N-1)) sum_i (w_k'(R_i - R_bar))^2 - w_k' R_bar      (Eq. 4)
 * pbar_k = w_k' R_bar,  R_bar = (1/N) sum_i R_i                          (Eq. 5)
 * var_k = (1/(N-1)) sum_i (w_k'(R_i - R_bar))^2
 * grad_k = lambda * (2/(N-1)) sum_i (R_i - R_bar)(R_i - R_bar)' w_k - R_bar
 * (the derivative of Eq. 4 in w).  Two passes: R_bar first, then the
 * centred sums.  lambda = 1 is Eq. 4 as printed; lambda = 1/2 matches the
 * objective of Eq. 3. */
static int saa_core(const sample_src* S, int K, const double* W, double lambda, double* f, double* pbar,
                    double* var, double* grad)
{
    const int64_t N = S->N;
    const int d = S->d;
    const int nch = (int)(N < MAX_CHUNKS ? N : MAX_CHUNKS);
    nsum* rsum = (nsum*)calloc((size_t)nch * d, sizeof(nsum));
    nsum* vsum = (nsum*)calloc((size_t)nch * K, sizeof(nsum));
    nsum* gsum = grad ? (nsum*)calloc((size_t)nch * K * d, sizeof(nsum)) : NULL;
    double* Rbar = (double*)malloc(sizeof(double) * (size_t)d);
    if (!rsum || !vsum || (grad && !gsum) || !Rbar) {
        free(rsum); free(vsum); free(gsum); free(Rbar);
        return OR_ENOMEM;
    }
    int err = OR_OK;

    /* Pass 1: R_bar (Eq. 5). */
#pragma omp parallel
    {
        sample_buf B = {(float*)malloc(sizeof(float) * (size_t)d), (double*)malloc(sizeof(double) * (size_t)d)};
        double* Ri = (double*)malloc(sizeof(double) * (size_t)d);
        if (!B.zf || !B.zd || !Ri) {
#pragma omp atomic write
            err = OR_ENOMEM;
        } else {
#pragma omp for schedule(dynamic, 1)
            for (int c = 0; c < nch; ++c) {
                int64_t a = N * c / nch, e = N * (c + 1) / nch;
                nsum* acc = rsum + (int64_t)c * d;
                for (int64_t i = a; i < e; ++i) {
                    get_sample(S, &B, i, Ri);
                    for (int j = 0; j < d; ++j) nadd(&acc[j], Ri[j]);
                }
            }
        }
        free(B.zf); free(B.zd); free(Ri);
    }
    if (err != OR_OK) goto done;
    for (int j = 0; j < d; ++j) {
        nsum t = {0.0, 0.0};
        for (int c = 0; c < nch; ++c) {
            nadd(&t, rsum[(int64_t)c * d + j].s);
            nadd(&t, rsum[(int64_t)c * d + j].c);
        }
        Rbar[j] = nval(&t) / (double)N;
    }

    /* Pass 2: centred squared projections and the centred cross sums. */
#pragma omp parallel
    {
        sample_buf B = {(float*)malloc(sizeof(float) * (size_t)d), (double*)malloc(sizeof(double) * (size_t)d)};
        double* D = (double*)malloc(sizeof(double) * (size_t)d);
        if (!B.zf || !B.zd || !D) {
#pragma omp atomic write
            err = OR_ENOMEM;
        } else {
#pragma omp for schedule(dynamic, 1)
            for (int c = 0; c < nch; ++c) {
                int64_t a = N * c / nch, e = N * (c + 1) / nch;
                nsum* va = vsum + (int64_t)c * K;
                nsum* ga = gsum ? gsum + (int64_t)c * K * d : NULL;
                for (int64_t i = a; i < e; ++i) {
                    get_sample(S, &B, i, D);
                    for (int j = 0; j < d; ++j) D[j] = D[j] - Rbar[j]; /* R_i - R_bar */
                    for (int k = 0; k < K; ++k) {
                        const double* wk = W + (int64_t)k * d;
                        double proj = 0.0; /* w_k'(R_i - R_bar) */
                        for (int j = 0; j < d; ++j) proj = proj + wk[j] * D[j];
                        nadd(&va[k], proj * proj);
                        if (ga) {
                            nsum* g = ga + (int64_t)k * d;
                            for (int j = 0; j < d; ++j) nadd(&g[j], D[j] * proj);
                        }
                    }
                }
            }
        }
        free(B.zf); free(B.zd); free(D);
    }
    if (err != OR_OK) goto done;

    for (int k = 0; k < K; ++k) {
        const double* wk = W + (int64_t)k * d;
        nsum t = {0.0, 0.0};
        for (int c = 0; c < nch; ++c) {
            nadd(&t, vsum[(int64_t)c * K + k].s);
            nadd(&t, vsum[(int64_t)c * K + k].c);
        }
        double V = nval(&t) / (double)(N - 1);
        double pb = 0.0;
        for (int j = 0; j < d; ++j) pb = pb + wk[j] * Rbar[j];
        if (var) var[k] = V;
        if (pbar) pbar[k] = pb;
        if (f) f[k] = lambda * V - pb;
        if (grad) {
            for (int j = 0; j < d; ++j) {
                nsum g = {0.0, 0.0};
                for (int c = 0; c < nch; ++c) {
                    nadd(&g, gsum[((int64_t)c * K + k) * d + j].s);
                    nadd(&g, gsum[((int64_t)c * K + k) * d + j].c);
                }
                grad[(int64_t)k * d + j] = lambda * (2.0 / (double)(N - 1)) * nval(&g) - Rbar[j];
            }
        }
    }
done:
    free(rsum); free(vsum); free(gsum); free(Rbar);
    return err;
}

/* Eq. 4 on an explicit sample matrix R (N x d, row-major). */
int oracle_saa_explicit(int64_t N, int d, const double* R, int K, const double* W, double lambda, double* f,
                        double* pbar, double* var, double* grad)
{
    if (N < 2 || d < 1 || K < 1 || !R || !W) return OR_EINVAL;
    sample_src S;
    memset(&S, 0, sizeof(S));
    S.R = R;
    S.N = N;
    S.d = d;
    return saa_core(&S, K, W, lambda, f, pbar, var, grad);
}

static double* transpose_chol(const oracle_problem* p)
{
    const int d = p->d;
    double* Ct = (double*)malloc(sizeof(double) * (size_t)d * (size_t)d);
    if (!Ct) return NULL;
    for (int j = 0; j < d; ++j)
        for (int l = 0; l < d; ++l) Ct[(int64_t)l * d + j] = (l <= j) ? p->chol[(int64_t)j * d + l] : 0.0;
    return Ct;
}

/* Eq. 4 on the N generated samples of resample index `epoch`. */
int oracle_saa(const oracle_problem* p, int prec, uint32_t epoch, int K, const double* W, double* f, double* pbar,
               double* var, double* grad)
{
    if (check_problem(p) != OR_OK || (prec != 32 && prec != 64) || K < 1 || !W) return OR_EINVAL;
    double* Ct = NULL;   /* diagonal C (chol NULL): the samples use sd directly */
    if (p->chol) {
        Ct = transpose_chol(p);
        if (!Ct) return OR_ENOMEM;
    }
    sample_src S;
    memset(&S, 0, sizeof(S));
    S.p = p;
    S.prec = prec;
    S.epoch = epoch;
    S.Ct = Ct;
    S.N = p->N;
    S.d = p->d;
    int rc = saa_core(&S, K, W, p->lambda, f, pbar, var, grad);
    free(Ct);
    return rc;
}

/* Partial sums of Eq. 4 / Eq. 5 over the scenario range [i0, i0 + n): the
 * sums over i of Sec. 3.1 split by scenario, so that disjoint ranges (one
 * per device) add up to the whole sample.  With D_i = R_i - mu (the samples
 * centred at the law's mean) and p_ik = w_k'D_i, part holds, in order,
 *   P1 [K]    sum_i p_ik
 *   P2 [K]    sum_i p_ik^2
 *   P3 [d]    sum_i D_i
 *   P4 [K*d]  sum_i D_i p_ik   (row k, only when want_grad)
 * R_i is formed exactly as oracle_saa forms it; each sum is Neumaier-
 * compensated over a fixed partition of the range. */
int oracle_partials(const oracle_problem* p, int prec, uint32_t epoch, int64_t i0, int64_t n, int K, const double* W,
                    int want_grad, double* part)
{
    if (check_problem(p) != OR_OK || (prec != 32 && prec != 64) || K < 1 || !W || !part) return OR_EINVAL;
    if (i0 < 0 || n < 1 || i0 + n > p->N) return OR_EINVAL;
    const int d = p->d;
    double* Ct = NULL;
    if (p->chol) {
        Ct = transpose_chol(p);
        if (!Ct) return OR_ENOMEM;
    }
    sample_src S;
    memset(&S, 0, sizeof(S));
    S.p = p;
    S.prec = prec;
    S.epoch = epoch;
    S.Ct = Ct;
    S.N = p->N;
    S.d = d;
    const int nch = (int)(n < MAX_CHUNKS ? n : MAX_CHUNKS);
    const int64_t width = 2 * (int64_t)K + d + (want_grad ? (int64_t)K * d : 0);
    nsum* acc = (nsum*)calloc((size_t)nch * (size_t)width, sizeof(nsum));
    if (!acc) {
        free(Ct);
        return OR_ENOMEM;
    }
    int err = OR_OK;
#pragma omp parallel
    {
        sample_buf B = {(float*)malloc(sizeof(float) * (size_t)d), (double*)malloc(sizeof(double) * (size_t)d)};
        double* D = (double*)malloc(sizeof(double) * (size_t)d);
        if (!B.zf || !B.zd || !D) {
#pragma omp atomic write
            err = OR_ENOMEM;
        } else {
#pragma omp for schedule(dynamic, 1)
            for (int c = 0; c < nch; ++c) {
                const int64_t a = i0 + n * c / nch, e = i0 + n * (c + 1) / nch;
                nsum* ac = acc + (int64_t)c * width;
                for (int64_t i = a; i < e; ++i) {
                    get_sample(&S, &B, i, D);
                    for (int j = 0; j < d; ++j) D[j] = D[j] - p->mu[j]; /* R_i - mu */
                    for (int j = 0; j < d; ++j) nadd(&ac[2 * K + j], D[j]);
                    for (int k = 0; k < K; ++k) {
                        const double* wk = W + (int64_t)k * d;
                        double pk = 0.0;
                        for (int j = 0; j < d; ++j) pk = pk + wk[j] * D[j];
                        nadd(&ac[k], pk);
                        nadd(&ac[K + k], pk * pk);
                        if (want_grad) {
                            nsum* g = ac + 2 * K + d + (int64_t)k * d;
                            for (int j = 0; j < d; ++j) nadd(&g[j], D[j] * pk);
                        }
                    }
                }
            }
        }
        free(B.zf); free(B.zd); free(D);
    }
    if (err == OR_OK) {
        for (int64_t e = 0; e < width; ++e) {
            nsum t = {0.0, 0.0};
            for (int c = 0; c < nch; ++c) {
                nadd(&t, acc[(int64_t)c * width + e].s);
                nadd(&t, acc[(int64_t)c * width + e].c);
            }
            part[e] = nval(&t);
        }
    }
    free(acc);
    free(Ct);
    return err;
}

/* Eq. 4, Eq. 5 and the gradient of Eq. 4 from the partial sums of the whole
 * sample (the element-wise total of oracle_partials over ranges covering
 * [0, N)): with R_bar = mu + P3/N,
 *   pbar_k = w_k'mu + P1_k/N
 *   V_k    = (P2_k - P1_k^2/N) / (N-1)
 *   f_k    = lambda V_k - pbar_k
 *   grad_k = lambda (2/(N-1)) (P4_k - P1_k P3/N) - R_bar
 * because sum_i (R_i - R_bar)(R_i - R_bar)'w_k = P4_k - P3 P1_k/N. */
int oracle_finalize_partials(int64_t N, int d, int K, const double* W, const double* mu, double lambda,
                             const double* part, double* f, double* pbar, double* var, double* grad)
{
    if (N < 2 || d < 1 || K < 1 || !W || !mu || !part) return OR_EINVAL;
    const double* P1 = part;
    const double* P2 = part + K;
    const double* P3 = part + 2 * K;
    const double* P4 = part + 2 * K + d;
    const double Nd = (double)N;
    for (int k = 0; k < K; ++k) {
        const double* wk = W + (int64_t)k * d;
        double c = 0.0;
        for (int j = 0; j < d; ++j) c = c + wk[j] * mu[j];
        const double pb = c + P1[k] / Nd;
        const double V = (P2[k] - P1[k] * P1[k] / Nd) / (Nd - 1.0);
        if (f) f[k] = lambda * V - pb;
        if (pbar) pbar[k] = pb;
        if (var) var[k] = V;
        if (grad)
            for (int j = 0; j < d; ++j)
                grad[(int64_t)k * d + j] = lambda * (2.0 / (Nd - 1.0)) * (P4[(int64_t)k * d + j] - P1[k] * P3[j] / Nd) -
                                           (mu[j] + P3[j] / Nd);
    }
    return OR_OK;
}

/* ------------------------------------------------------------------------- */
/* 4. Frank-Wolfe, Algorithm 1                                               */
/* ------------------------------------------------------------------------- */
/* One iteration after the gradient g = grad f_hat(w_t):
 *   LMO over W = {w >= 0, 1'w <= 1}: its vertices are 0 and the unit
 *   vectors e_j, so s = e_j* with j* the first index of min_j g_j when
 *   g_j* < 0, else s = 0;
 *   gamma = 2 / (t + 2) with t = kM + m the global iteration count;
 *   w_{t+1} = w_t + gamma (s - w_t);  FW gap = g'(w_t - s) >= 0.
 * Returns j* (or -1 for the zero vertex). */
int oracle_fw_step(int d, const double* g, const double* w, int64_t t, double* w_next, double* gap)
{
    int js = 0;
    for (int j = 1; j < d; ++j)
        if (g[j] < g[js]) js = j;
    if (!(g[js] < 0.0)) js = -1;
    double gamma = 2.0 / ((double)t + 2.0);
    double gw = 0.0;
    for (int j = 0; j < d; ++j) gw = gw + g[j] * w[j];
    if (gap) *gap = gw - (js >= 0 ? g[js] : 0.0);
    for (int j = 0; j < d; ++j) {
        double sj = (j == js) ? 1.0 : 0.0;
        w_next[j] = w[j] + gamma * (sj - w[j]);
    }
    return js;
}

/* Algorithm 1 from iteration t0 for T iterations, resampling every M
 * iterations: iteration t uses the samples of resample index
 * p->epoch + t / M.  f_trace[t - t0] = f_hat(w_t) on those samples,
 * gap_trace[t - t0] = the FW gap at w_t.  w_trace (optional, T x d)
 * receives w_t before each step. */
int oracle_fw(const oracle_problem* p, int prec, const double* w0, int T, int M, int64_t t0, double* w_out,
              double* f_trace, double* gap_trace, double* w_trace)
{
    if (check_problem(p) != OR_OK || (prec != 32 && prec != 64) || T < 0 || M < 1 || t0 < 0 || !w0 || !w_out)
        return OR_EINVAL;
    const int d = p->d;
    double* w = (double*)malloc(sizeof(double) * (size_t)d);
    double* wn = (double*)malloc(sizeof(double) * (size_t)d);
    double* g = (double*)malloc(sizeof(double) * (size_t)d);
    if (!w || !wn || !g) {
        free(w); free(wn); free(g);
        return OR_ENOMEM;
    }
    memcpy(w, w0, sizeof(double) * (size_t)d);
    int rc = OR_OK;
    for (int it = 0; it < T; ++it) {
        int64_t t = t0 + it;
        uint32_t epoch = p->epoch + (uint32_t)(t / M);
        double fv;
        rc = oracle_saa(p, prec, epoch, 1, w, &fv, NULL, NULL, g);
        if (rc != OR_OK) break;
        if (w_trace) memcpy(w_trace + (int64_t)it * d, w, sizeof(double) * (size_t)d);
        if (f_trace) f_trace[it] = fv;
        double gap;
        oracle_fw_step(d, g, w, t, wn, &gap);
        if (gap_trace) gap_trace[it] = gap;
        memcpy(w, wn, sizeof(double) * (size_t)d);
    }
    if (rc == OR_OK) memcpy(w_out, w, sizeof(double) * (size_t)d);
    free(w); free(wn); free(g);
    return rc;
}

/* ------------------------------------------------------------------------- */
/* 5. RSE (Table 2 notes): ((y_t - y*) / y_t)^2 * 100 %                      */
/* ------------------------------------------------------------------------- */
/* ---------------------------------------------------------------------- */
/* 6. Cholesky factor: the textbook row-by-row (Cholesky-Banachiewicz)    */
/*    recurrence, C_jj = sqrt(S_jj - sum_{l<j} C_jl^2) and, for i > j,    */
/*    C_ij = (S_ij - sum_{l<j} C_il C_jl) / C_jj, each sum in index order.  */
/*    S is row-major [d][d]; only its lower triangle is read.  C is       */
/*    row-major lower-triangular with zeros above the diagonal.  Returns  */
/*    OR_EINVAL when a pivot is not positive (S not positive definite).   */
/* ---------------------------------------------------------------------- */
int oracle_cholesky(int d, const double* S, double* C)
{
    if (d < 1 || !S || !C) return OR_EINVAL;
    memset(C, 0, sizeof(double) * (size_t)d * (size_t)d);
    for (int i = 0; i < d; ++i) {
        for (int j = 0; j <= i; ++j) {
            double acc = S[(size_t)i * d + j];
            for (int l = 0; l < j; ++l) acc -= C[(size_t)i * d + l] * C[(size_t)j * d + l];
            if (i == j) {
                if (!(acc > 0.0)) return OR_EINVAL;
                C[(size_t)i * d + i] = sqrt(acc);
            } else {
                C[(size_t)i * d + j] = acc / C[(size_t)j * d + j];
            }
        }
    }
    return OR_OK;
}

/* ---------------------------------------------------------------------- */
/* 7. Newsvendor Monte Carlo gradient                                      */
/* ---------------------------------------------------------------------- */
/* Demand samples: product j's s-th demand is d_js = mu_j + sigma_j z_js,
 * with z_js the generator's FP32 normals on counter (s / 4, j, epoch,
 * (3 << 24) | instance), element s mod 4 of the four normals of that call.
 * The indicator d_js <= x_j is decided on the standardised demand in FP32:
 * z_js <= tau, tau = (float)((x_j - mu_j) / sigma_j) with the subtraction
 * and the division in FP64 (sigma_j > 0).  The estimate is then
 * (k_j - v_j) + (h_j + v_j) * (count / S) in FP64, in that order. */
#define TAG_DEMAND 3u

typedef struct {
    int64_t n;          /* products */
    int64_t S;          /* demand samples per product */
    uint64_t seed;
    uint32_t instance;
    uint32_t epoch;
    const double* mu;    /* [n] demand means */
    const double* sigma; /* [n] demand standard deviations, > 0 */
    const double* k;     /* [n] unit ordering cost */
    const double* h;     /* [n] unit holding cost */
    const double* v;     /* [n] unit shortage cost */
} oracle_newsvendor;

static void demand_block(const oracle_newsvendor* p, int64_t j, int64_t b, float z[4])
{
    uint32_t c[4], x[4];
    c[0] = (uint32_t)b;
    c[1] = (uint32_t)j;
    c[2] = p->epoch;
    c[3] = (TAG_DEMAND << 24) | (p->instance & 0xffffffu);
    philox10(c, (uint32_t)(p->seed & 0xffffffffu), (uint32_t)(p->seed >> 32), x);
    box_muller_f(u24(x[0]), u24_num(x[1]), &z[0], &z[1]);
    box_muller_f(u24(x[2]), u24_num(x[3]), &z[2], &z[3]);
}

static int check_newsvendor(const oracle_newsvendor* p)
{
    if (!p || p->n < 1 || p->n > 0xffffffffll || p->S < 1 || p->S > 0x3fffffffll || !p->mu || !p->sigma) return OR_EINVAL;
    for (int64_t j = 0; j < p->n; ++j)
        if (!(p->sigma[j] > 0.0)) return OR_EINVAL;
    return OR_OK;
}

/* The standardised demands z_j0 .. z_j(S-1) of product j. */
int oracle_newsvendor_demands(const oracle_newsvendor* p, int64_t j, float* z)
{
    if (check_newsvendor(p) != OR_OK || j < 0 || j >= p->n || !z) return OR_EINVAL;
    for (int64_t b = 0; 4 * b < p->S; ++b) {
        float w[4];
        demand_block(p, j, b, w);
        for (int q = 0; q < 4 && 4 * b + q < p->S; ++q) z[4 * b + q] = w[q];
    }
    return OR_OK;
}

/* Gradient estimates at the K decisions X[K][n] for the products j0 <= j < j1:
 * grad[K][j1 - j0] and counts[K][j1 - j0] (optional, the number of samples
 * with z <= tau). */
int oracle_newsvendor_grad_range(const oracle_newsvendor* p, int K, const double* X, int64_t j0, int64_t j1,
                                 double* grad, int64_t* counts)
{
    if (check_newsvendor(p) != OR_OK || K < 1 || K > 64 || !X || !grad || !p->k || !p->h || !p->v) return OR_EINVAL;
    if (j0 < 0 || j1 > p->n || j0 >= j1) return OR_EINVAL;
    const int64_t n = p->n, m = j1 - j0;
#pragma omp parallel for schedule(static)
    for (int64_t j = j0; j < j1; ++j) {
        float tau[64];
        int64_t cnt[64];
        for (int kk = 0; kk < K; ++kk) {
            tau[kk] = (float)((X[(size_t)kk * n + j] - p->mu[j]) / p->sigma[j]);
            cnt[kk] = 0;
        }
        for (int64_t b = 0; 4 * b < p->S; ++b) {
            float z[4];
            demand_block(p, j, b, z);
            for (int q = 0; q < 4 && 4 * b + q < p->S; ++q)
                for (int kk = 0; kk < K; ++kk)
                    if (z[q] <= tau[kk]) cnt[kk] += 1;
        }
        for (int kk = 0; kk < K; ++kk) {
            const double frac = (double)cnt[kk] / (double)p->S;
            grad[(size_t)kk * m + (j - j0)] = (p->k[j] - p->v[j]) + (p->h[j] + p->v[j]) * frac;
            if (counts) counts[(size_t)kk * m + (j - j0)] = cnt[kk];
        }
    }
    return OR_OK;
}

/* All products: grad[K][n], counts[K][n] (optional). */
int oracle_newsvendor_grad(const oracle_newsvendor* p, int K, const double* X, double* grad, int64_t* counts)
{
    if (!p) return OR_EINVAL;
    return oracle_newsvendor_grad_range(p, K, X, 0, p->n, grad, counts);
}

/* ------------------------------------------------------------------------- */
/* 8. Binary classification (Sec. 3.3)                                        */
/* ------------------------------------------------------------------------- */
/* Data set {(x_i, z_i)}, i < N, x_i in {0,1}^n.  Feature j = 128 b + 32 q + t
 * of point i is bit t of word q of Philox4x32-10(counter (b, i, 0,
 * (4 << 24) | instance), key seed): Bernoulli(1/2) features.  The label is
 * a random linear rule with label noise: z_i = [2 x_i'w* > 1'w*] (strict,
 * integer arithmetic) flipped when word 0 of Philox(counter (0, i, 0,
 * (5 << 24) | instance)) is below `flip` (flip = 0.1 * 2^32 gives the 10 %
 * of Sec. 4.1). */
typedef struct {
    int32_t n;            /* features */
    int64_t N;            /* data points */
    uint64_t seed;
    uint32_t instance;
    uint32_t flip;
    const int32_t* wstar; /* [n] integer weights of the labelling rule */
} oracle_logistic;

static int check_logistic(const oracle_logistic* p)
{
    if (!p || p->n < 1 || p->N < 1 || p->N > 0xffffffffll || !p->wstar) return OR_EINVAL;
    return OR_OK;
}

static void logi_features(const oracle_logistic* p, int64_t i, uint8_t* x)
{
    const uint32_t k0 = (uint32_t)(p->seed & 0xffffffffu), k1 = (uint32_t)(p->seed >> 32);
    for (int32_t b = 0; 128 * b < p->n; ++b) {
        const uint32_t c[4] = {(uint32_t)b, (uint32_t)i, 0u, (4u << 24) | (p->instance & 0xffffffu)};
        uint32_t w[4];
        philox10(c, k0, k1, w);
        for (int q = 0; q < 4; ++q)
            for (int t = 0; t < 32; ++t) {
                const int32_t j = 128 * b + 32 * q + t;
                if (j < p->n) x[j] = (uint8_t)((w[q] >> t) & 1u);
            }
    }
}

static uint8_t logi_label(const oracle_logistic* p, int64_t i, const uint8_t* x)
{
    int64_t dot = 0, tot = 0;
    for (int32_t j = 0; j < p->n; ++j) {
        tot += p->wstar[j];
        if (x[j]) dot += p->wstar[j];
    }
    uint8_t z = (uint8_t)(2 * dot > tot);
    const uint32_t c[4] = {0u, (uint32_t)i, 0u, (5u << 24) | (p->instance & 0xffffffu)};
    uint32_t w[4];
    philox10(c, (uint32_t)(p->seed & 0xffffffffu), (uint32_t)(p->seed >> 32), w);
    if (w[0] < p->flip) z ^= 1u;
    return z;
}

/* Features x[rows][n] and labels z[rows] of points i0 .. i0 + rows - 1 (either
 * output may be NULL). */
int oracle_logistic_data(const oracle_logistic* p, int64_t i0, int64_t rows, uint8_t* x, uint8_t* z)
{
    if (check_logistic(p) != OR_OK || i0 < 0 || rows < 0 || i0 + rows > p->N) return OR_EINVAL;
    uint8_t* row = (uint8_t*)malloc((size_t)p->n);
    if (!row) return OR_ENOMEM;
    for (int64_t r = 0; r < rows; ++r) {
        logi_features(p, i0 + r, row);
        if (x) memcpy(x + (size_t)r * p->n, row, (size_t)p->n);
        if (z) z[r] = logi_label(p, i0 + r, row);
    }
    free(row);
    return OR_OK;
}

/* The objective and its derivatives over the sample S (indices idx[0..b-1],
 * repeats allowed; idx == NULL means every point 0 .. N-1, b = N), for K
 * parameter vectors W[K][n] (omega_k) and optional directions V[K][n]:
 *   F[k]    = -(1/b) sum_S [ z log c + (1 - z) log(1 - c) ],  c = 1/(1 + e^(-x'omega))
 *           =  (1/b) sum_S [ log(1 + e^t) - z t ],  t = x'omega          (Sec. 3.3)
 *   grad[k] =  (1/b) sum_S (c - z) x                 (derivative of F, the
 *                                                     mini-batch gradient's mean)
 *   hvp[k]  =  (1/b) sum_S c (1 - c) (x'v_k) x       (sub-sampled Hessian times v_k)
 * Each output may be NULL (hvp needs V).  Sums run over a fixed partition of
 * S into chunks merged in chunk order with Neumaier compensation. */
int oracle_logistic_eval(const oracle_logistic* p, const int64_t* idx, int64_t b, int K, const double* W,
                         const double* V, double* F, double* grad, double* hvp)
{
    if (check_logistic(p) != OR_OK || K < 1 || !W || (hvp && !V)) return OR_EINVAL;
    if (!idx) b = p->N;
    if (b < 1) return OR_EINVAL;
    if (idx)
        for (int64_t s = 0; s < b; ++s)
            if (idx[s] < 0 || idx[s] >= p->N) return OR_EINVAL;
    const int n = p->n;
    enum { NCH = 64 };
    const size_t per = (size_t)K * (size_t)n;
    nsum* pf = (nsum*)calloc((size_t)NCH * K, sizeof(nsum));
    nsum* pg = (nsum*)calloc((size_t)NCH * per, sizeof(nsum));
    nsum* ph = hvp ? (nsum*)calloc((size_t)NCH * per, sizeof(nsum)) : NULL;
    if (!pf || !pg || (hvp && !ph)) {
        free(pf); free(pg); free(ph);
        return OR_ENOMEM;
    }
    int bad = 0;
#pragma omp parallel for schedule(static)
    for (int ch = 0; ch < NCH; ++ch) {
        const int64_t s0 = b * ch / NCH, s1 = b * (ch + 1) / NCH;
        uint8_t* x = (uint8_t*)malloc((size_t)n);
        if (!x) {
            bad = 1;
            continue;
        }
        for (int64_t s = s0; s < s1; ++s) {
            const int64_t i = idx ? idx[s] : s;
            logi_features(p, i, x);
            const double z = (double)logi_label(p, i, x);
            for (int k = 0; k < K; ++k) {
                const double* w = W + (size_t)k * n;
                double t = 0.0;
                for (int j = 0; j < n; ++j)
                    if (x[j]) t += w[j];
                const double c = 1.0 / (1.0 + exp(-t));
                /* log(1 + e^t) without overflow */
                const double sp = t > 0.0 ? t + log1p(exp(-t)) : log1p(exp(t));
                nadd(&pf[(size_t)ch * K + k], sp - z * t);
                const double r = c - z;
                double hr = 0.0;
                if (hvp) {
                    const double* v = V + (size_t)k * n;
                    double u = 0.0;
                    for (int j = 0; j < n; ++j)
                        if (x[j]) u += v[j];
                    hr = c * (1.0 - c) * u;
                }
                for (int j = 0; j < n; ++j)
                    if (x[j]) {
                        nadd(&pg[(size_t)ch * per + (size_t)k * n + j], r);
                        if (hvp) nadd(&ph[(size_t)ch * per + (size_t)k * n + j], hr);
                    }
            }
        }
        free(x);
    }
    if (!bad) {
        for (int k = 0; k < K; ++k) {
            nsum a = {0.0, 0.0};
            for (int ch = 0; ch < NCH; ++ch) nadd(&a, nval(&pf[(size_t)ch * K + k]));
            if (F) F[k] = nval(&a) / (double)b;
        }
        for (size_t e = 0; e < per; ++e) {
            nsum a = {0.0, 0.0}, h = {0.0, 0.0};
            for (int ch = 0; ch < NCH; ++ch) {
                nadd(&a, nval(&pg[(size_t)ch * per + e]));
                if (hvp) nadd(&h, nval(&ph[(size_t)ch * per + e]));
            }
            if (grad) grad[e] = nval(&a) / (double)b;
            if (hvp) hvp[e] = nval(&h) / (double)b;
        }
    }
    free(pf); free(pg); free(ph);
    return bad ? OR_ENOMEM : OR_OK;
}

double oracle_rse(double y_t, double y_star)
{
    double r = (y_t - y_star) / y_t;
    return r * r * 100.0;
}

int oracle_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
