/*
 * fl_oracle.c -- plain CPU oracle for the fast Fourier-Laplace transform.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the
 * CPU-baseline leg of the benchmark may load this library.  It shares no code,
 * header, table or helper with the CUDA library, and the CUDA library never
 * calls it.
 *
 * Every routine is the plain definition written out, term by term, in IEEE
 * double precision (long double for the brute-force variant), with compensated
 * (Neumaier) summation so that the result is accurate to a few units of
 * roundoff times sum_k |term_k|:
 *
 *   oracle_flt_direct      f_j = sum_{k=0}^{N-1} c_k z_j^k,  z_j = exp(2 pi i w_j)
 *                          Kunis & Melzer, Section 4, eq. (4.1) with xi_k = k
 *                          (the index is shifted to start at k = 0) and the polar
 *                          split (4.2): z = exp(-y) exp(2 pi i x), y = 2 pi Im w.
 *   oracle_flt_adjoint     g_k = sum_j conj(z_j)^k r_j, the adjoint C^* of the
 *                          same matrix (Section 4, remark after Algorithm 2);
 *                          oracle_flt_adjoint_at: the same at selected k.
 *   oracle_laplace_direct  f_j = sum_k c_k exp(-s_j t_k), eq. (3.2) (real data).
 *   oracle_kernel_direct   f_j = sum_k c_k kappa(s_j, t_k) for the kernels of the
 *                          generalised Algorithm 1 (Section 3, after Algorithm 1):
 *                          kind 1 exp(-s t), kind 2 the Bessel kernel of the
 *                          example there, K_{1/2}(s t) = sqrt(pi / (2 s t)) exp(-s t).
 *   oracle_xi_direct       f_j = sum_k c_k exp(2 pi i xi_k w_j) for real exponents
 *                          xi_k (the generalised polynomials of eq. (4.1) with
 *                          xi_k in [1, N]): z_j^xi_k = exp(-y xi_k) exp(2 pi i xi_k x).
 *   oracle_xi_transposed   g_k = sum_j h_j exp(2 pi i xi_k w_j): the transposed
 *                          evaluation at real exponents (Section 4, remark
 *                          after Algorithm 2: the sum over nodes at given xi).
 *   oracle_flt_brute_ld    oracle_flt_direct in long double, for tiny N.
 *
 * Phase reduction: the phase k*x is split exactly into p + e with an FMA
 * (error-free product), the integer part of p is removed exactly, so the
 * angle 2*pi*frac(k*x) carries one rounding only.  This keeps the oracle
 * accurate for k up to 2^24 and beyond, where forming z^k by repeated
 * multiplication would lose ~k ulps.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <unistd.h>

#define ORACLE_TWO_PI 6.283185307179586476925286766559

/* Neumaier compensated accumulator. */
typedef struct { double s, comp; } acc_t;

static inline void acc_add(acc_t *a, double v)
{
    double t = a->s + v;
    if (fabs(a->s) >= fabs(v))
        a->comp += (a->s - t) + v;
    else
        a->comp += (v - t) + a->s;
    a->s = t;
}

static inline double acc_get(const acc_t *a) { return a->s + a->comp; }

/* frac(k*x) in [-1/2, 1/2), with one rounding: k*x = p + e exactly (FMA). */
static inline double phase_frac(double k, double x)
{
    double p = k * x;
    double e = fma(k, x, -p);
    double ip = floor(p);
    double f = p - ip;          /* exact: a multiple of ulp(p) below 1 */
    f += e;                     /* the one rounding */
    if (f >= 0.5) f -= 1.0;     /* exact */
    if (f < -0.5) f += 1.0;     /* exact */
    return f;
}

/* ------------------------------------------------------------------------ */
/* Thread pool over an index range.                                          */

typedef void (*range_fn)(void *ctx, int64_t lo, int64_t hi);

typedef struct {
    range_fn fn;
    void *ctx;
    int64_t lo, hi;
} range_job;

static void *range_thread(void *arg)
{
    range_job *j = (range_job *)arg;
    j->fn(j->ctx, j->lo, j->hi);
    return NULL;
}

int oracle_default_threads(void)
{
    long n = sysconf(_SC_NPROCESSORS_ONLN);
    return n > 0 ? (int)n : 1;
}

static void run_parallel(range_fn fn, void *ctx, int64_t n, int nthreads)
{
    if (nthreads <= 0) nthreads = oracle_default_threads();
    if (nthreads > 256) nthreads = 256;
    if (n < nthreads) nthreads = (int)(n > 0 ? n : 1);
    if (nthreads <= 1) {
        fn(ctx, 0, n);
        return;
    }
    pthread_t tid[256];
    int joined[256];
    range_job jobs[256];
    for (int t = 0; t < nthreads; ++t) {
        jobs[t].fn = fn;
        jobs[t].ctx = ctx;
        jobs[t].lo = n * t / nthreads;
        jobs[t].hi = n * (t + 1) / nthreads;
        joined[t] = pthread_create(&tid[t], NULL, range_thread, &jobs[t]) == 0;
        if (!joined[t]) range_thread(&jobs[t]); /* run inline if no thread */
    }
    for (int t = 0; t < nthreads; ++t)
        if (joined[t]) pthread_join(tid[t], NULL);
}

/* ------------------------------------------------------------------------ */
/* Forward transform f_j = sum_k c_k exp(2 pi i k w_j).                      */

typedef struct {
    int64_t N;
    const double *c;   /* 2N: re, im interleaved */
    const double *w;   /* 2M: Re w, Im w interleaved */
    double *f;         /* 2M out */
} flt_ctx;

static void flt_range(void *vctx, int64_t lo, int64_t hi)
{
    const flt_ctx *cx = (const flt_ctx *)vctx;
    for (int64_t j = lo; j < hi; ++j) {
        const double x = cx->w[2 * j];
        const double y = ORACLE_TWO_PI * cx->w[2 * j + 1];
        acc_t re = {0.0, 0.0}, im = {0.0, 0.0};
        for (int64_t k = 0; k < cx->N; ++k) {
            const double dk = (double)k;
            const double mag = exp(-y * dk);
            if (mag == 0.0) break;     /* every later term underflows too */
            const double ang = ORACLE_TWO_PI * phase_frac(dk, x);
            const double zr = mag * cos(ang), zi = mag * sin(ang);
            const double cr = cx->c[2 * k], ci = cx->c[2 * k + 1];
            /* (cr + i ci)(zr + i zi); each product rounded once */
            acc_add(&re, cr * zr);
            acc_add(&re, -(ci * zi));
            acc_add(&im, cr * zi);
            acc_add(&im, ci * zr);
        }
        cx->f[2 * j] = acc_get(&re);
        cx->f[2 * j + 1] = acc_get(&im);
    }
}

/* Returns 0 on success, -1 on invalid arguments. */
int oracle_flt_direct(int64_t N, const double *c, int64_t M, const double *w,
                      double *f, int nthreads)
{
    if (N < 0 || M < 0 || (N > 0 && !c) || (M > 0 && (!w || !f))) return -1;
    for (int64_t j = 0; j < M; ++j)
        if (!(w[2 * j + 1] >= 0.0) || !isfinite(w[2 * j])) return -1;
    flt_ctx cx = {N, c, w, f};
    run_parallel(flt_range, &cx, M, nthreads);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Real exponents: f_j = sum_k c_k exp(2 pi i xi_k w_j).  The phase xi_k x is  */
/* split exactly with an FMA as for integer k.                               */

typedef struct {
    int64_t N;
    const double *c, *xi, *w;
    double *f;
} xi_ctx;

static void xi_range(void *vctx, int64_t lo, int64_t hi)
{
    const xi_ctx *cx = (const xi_ctx *)vctx;
    for (int64_t j = lo; j < hi; ++j) {
        const double x = cx->w[2 * j];
        const double y = ORACLE_TWO_PI * cx->w[2 * j + 1];
        acc_t re = {0.0, 0.0}, im = {0.0, 0.0};
        for (int64_t k = 0; k < cx->N; ++k) {
            const double xk = cx->xi[k];
            const double mag = exp(-y * xk);
            const double ang = ORACLE_TWO_PI * phase_frac(xk, x);
            const double zr = mag * cos(ang), zi = mag * sin(ang);
            const double cr = cx->c[2 * k], ci = cx->c[2 * k + 1];
            acc_add(&re, cr * zr);
            acc_add(&re, -(ci * zi));
            acc_add(&im, cr * zi);
            acc_add(&im, ci * zr);
        }
        cx->f[2 * j] = acc_get(&re);
        cx->f[2 * j + 1] = acc_get(&im);
    }
}

int oracle_xi_direct(int64_t N, const double *c, const double *xi, int64_t M,
                     const double *w, double *f, int nthreads)
{
    if (N < 0 || M < 0 || (N > 0 && (!c || !xi)) || (M > 0 && (!w || !f))) return -1;
    for (int64_t k = 0; k < N; ++k) if (!(xi[k] >= 0.0) || !isfinite(xi[k])) return -1;
    for (int64_t j = 0; j < M; ++j)
        if (!(w[2 * j + 1] >= 0.0) || !isfinite(w[2 * j])) return -1;
    xi_ctx cx = {N, c, xi, w, f};
    run_parallel(xi_range, &cx, M, nthreads);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Transposed evaluation at real exponents: g_k = sum_j h_j exp(2 pi i xi_k w_j), */
/* the same terms as xi_range summed over nodes instead of exponents.        */

typedef struct {
    int64_t M;
    const double *h, *xi, *w;
    double *g;
} xit_ctx;

static void xit_range(void *vctx, int64_t lo, int64_t hi)
{
    const xit_ctx *cx = (const xit_ctx *)vctx;
    for (int64_t k = lo; k < hi; ++k) {
        const double xk = cx->xi[k];
        acc_t re = {0.0, 0.0}, im = {0.0, 0.0};
        for (int64_t j = 0; j < cx->M; ++j) {
            const double x = cx->w[2 * j];
            const double y = ORACLE_TWO_PI * cx->w[2 * j + 1];
            const double mag = exp(-y * xk);
            const double ang = ORACLE_TWO_PI * phase_frac(xk, x);
            const double zr = mag * cos(ang), zi = mag * sin(ang);
            const double hr = cx->h[2 * j], hi_ = cx->h[2 * j + 1];
            acc_add(&re, hr * zr);
            acc_add(&re, -(hi_ * zi));
            acc_add(&im, hr * zi);
            acc_add(&im, hi_ * zr);
        }
        cx->g[2 * k] = acc_get(&re);
        cx->g[2 * k + 1] = acc_get(&im);
    }
}

int oracle_xi_transposed(int64_t N, const double *xi, int64_t M, const double *w,
                         const double *h, double *g, int nthreads)
{
    if (N < 0 || M < 0 || (N > 0 && (!xi || !g)) || (M > 0 && (!w || !h))) return -1;
    for (int64_t k = 0; k < N; ++k) if (!(xi[k] >= 0.0) || !isfinite(xi[k])) return -1;
    for (int64_t j = 0; j < M; ++j)
        if (!(w[2 * j + 1] >= 0.0) || !isfinite(w[2 * j])) return -1;
    xit_ctx cx = {M, h, xi, w, g};
    run_parallel(xit_range, &cx, N, nthreads);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Adjoint g_k = sum_j conj(z_j)^k r_j.                                      */

typedef struct {
    int64_t M;
    const double *r;   /* 2M */
    const double *w;   /* 2M */
    double *g;         /* 2 x (number of outputs) */
    const int64_t *ks; /* NULL: output i is k = i; else k = ks[i] */
} adj_ctx;

static void adj_range(void *vctx, int64_t lo, int64_t hi)
{
    const adj_ctx *cx = (const adj_ctx *)vctx;
    for (int64_t i = lo; i < hi; ++i) {
        const int64_t k = cx->ks ? cx->ks[i] : i;
        const double dk = (double)k;
        acc_t re = {0.0, 0.0}, im = {0.0, 0.0};
        for (int64_t j = 0; j < cx->M; ++j) {
            const double x = cx->w[2 * j];
            const double y = ORACLE_TWO_PI * cx->w[2 * j + 1];
            const double mag = exp(-y * dk);
            if (mag == 0.0) continue;
            const double ang = ORACLE_TWO_PI * phase_frac(dk, x);
            const double zr = mag * cos(ang), zi = -mag * sin(ang); /* conj */
            const double rr = cx->r[2 * j], ri = cx->r[2 * j + 1];
            acc_add(&re, rr * zr);
            acc_add(&re, -(ri * zi));
            acc_add(&im, rr * zi);
            acc_add(&im, ri * zr);
        }
        cx->g[2 * i] = acc_get(&re);
        cx->g[2 * i + 1] = acc_get(&im);
    }
}

int oracle_flt_adjoint(int64_t N, const double *r, int64_t M, const double *w,
                       double *g, int nthreads)
{
    if (N < 0 || M < 0 || (M > 0 && (!r || !w)) || (N > 0 && !g)) return -1;
    for (int64_t j = 0; j < M; ++j)
        if (!(w[2 * j + 1] >= 0.0) || !isfinite(w[2 * j])) return -1;
    adj_ctx cx = {M, r, w, g, NULL};
    run_parallel(adj_range, &cx, N, nthreads);
    return 0;
}

/* The adjoint at selected frequencies: g_i = sum_j conj(z_j)^{ks[i]} r_j. */
int oracle_flt_adjoint_at(int64_t nk, const int64_t *ks, const double *r, int64_t M,
                          const double *w, double *g, int nthreads)
{
    if (nk < 0 || M < 0 || (M > 0 && (!r || !w)) || (nk > 0 && (!g || !ks))) return -1;
    for (int64_t i = 0; i < nk; ++i) if (ks[i] < 0) return -1;
    for (int64_t j = 0; j < M; ++j)
        if (!(w[2 * j + 1] >= 0.0) || !isfinite(w[2 * j])) return -1;
    adj_ctx cx = {M, r, w, g, ks};
    run_parallel(adj_range, &cx, nk, nthreads);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Real discrete Laplace transform f_j = sum_k c_k exp(-s_j t_k).            */

typedef struct {
    int64_t N;
    const double *c, *t, *s;
    double *f;
} lap_ctx;

static void lap_range(void *vctx, int64_t lo, int64_t hi)
{
    const lap_ctx *cx = (const lap_ctx *)vctx;
    for (int64_t j = lo; j < hi; ++j) {
        acc_t a = {0.0, 0.0};
        const double sj = cx->s[j];
        for (int64_t k = 0; k < cx->N; ++k)
            acc_add(&a, cx->c[k] * exp(-sj * cx->t[k]));
        cx->f[j] = acc_get(&a);
    }
}

int oracle_laplace_direct(int64_t N, const double *c, const double *t,
                          int64_t M, const double *s, double *f, int nthreads)
{
    if (N < 0 || M < 0 || (N > 0 && (!c || !t)) || (M > 0 && (!s || !f)))
        return -1;
    for (int64_t k = 0; k < N; ++k) if (!(t[k] >= 0.0)) return -1;
    for (int64_t j = 0; j < M; ++j) if (!(s[j] >= 0.0)) return -1;
    lap_ctx cx = {N, c, t, s, f};
    run_parallel(lap_range, &cx, M, nthreads);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Asymptotically smooth kernels of the generalised Algorithm 1.             */

static double kernel_value(int kind, double y, double xi)
{
    const double x = y * xi;
    if (kind == 2) return sqrt(1.5707963267948966192313216916398 / x) * exp(-x);
    return exp(-x);
}

typedef struct {
    int kind;
    int64_t N;
    const double *c, *t, *s;
    double *f;
} ker_ctx;

static void ker_range(void *vctx, int64_t lo, int64_t hi)
{
    const ker_ctx *cx = (const ker_ctx *)vctx;
    for (int64_t j = lo; j < hi; ++j) {
        acc_t a = {0.0, 0.0};
        const double sj = cx->s[j];
        for (int64_t k = 0; k < cx->N; ++k)
            acc_add(&a, cx->c[k] * kernel_value(cx->kind, sj, cx->t[k]));
        cx->f[j] = acc_get(&a);
    }
}

int oracle_kernel_direct(int kind, int64_t N, const double *c, const double *t,
                         int64_t M, const double *s, double *f, int nthreads)
{
    if ((kind != 1 && kind != 2) || N < 0 || M < 0 || (N > 0 && (!c || !t)) ||
        (M > 0 && (!s || !f)))
        return -1;
    /* nodes finite; s, t >= 0 (kind 1) or > 0 (kind 2, singular at s t = 0) */
    for (int64_t k = 0; k < N; ++k)
        if (!isfinite(t[k]) || t[k] < 0.0 || (kind == 2 && t[k] == 0.0)) return -1;
    for (int64_t j = 0; j < M; ++j)
        if (!isfinite(s[j]) || s[j] < 0.0 || (kind == 2 && s[j] == 0.0)) return -1;
    ker_ctx cx = {kind, N, c, t, s, f};
    run_parallel(ker_range, &cx, M, nthreads);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Brute force in long double (tiny N): same definition, wider arithmetic.   */

int oracle_flt_brute_ld(int64_t N, const double *c, int64_t M, const double *w,
                        double *f)
{
    if (N < 0 || M < 0 || N > (1 << 16)) return -1;
    const long double two_pi = 6.283185307179586476925286766559005768L;
    for (int64_t j = 0; j < M; ++j) {
        const long double y = two_pi * (long double)w[2 * j + 1];
        long double re = 0.0L, im = 0.0L;
        for (int64_t k = 0; k < N; ++k) {
            /* k*x = p + e exactly (FMA); the fractional part is formed in
               long double, so it carries ~2^-64 relative error at most. */
            const double dk = (double)k;
            const double pd = dk * w[2 * j];
            const double ed = fma(dk, w[2 * j], -pd);
            long double p = (long double)(pd - floor(pd)) + (long double)ed;
            const long double ang = two_pi * p;
            const long double mag = expl(-y * (long double)k);
            const long double zr = mag * cosl(ang), zi = mag * sinl(ang);
            re += (long double)c[2 * k] * zr - (long double)c[2 * k + 1] * zi;
            im += (long double)c[2 * k] * zi + (long double)c[2 * k + 1] * zr;
        }
        f[2 * j] = (double)re;
        f[2 * j + 1] = (double)im;
    }
    return 0;
}
