/*
 * CPU oracle for the Chebyshev--Jacobi transform (TEST INFRASTRUCTURE ONLY).
 *
 * This file is the plain, slow, obviously-correct reference that the CUDA
 * library is checked against.  Only tests, the smoke check and the benchmark's
 * CPU-baseline leg and reference arm may load it; the product path never does.  It shares no
 * code, header, table or constant generator with the CUDA library.
 *
 * What it computes (the paper's definitions, written out directly):
 *   forward  c_cheb = T_N^{-1} P_N c_jac                          (Eq. "CJT", Sec. 1)
 *     y_j = sum_n c_n P_n(x_j) at x_j = cos(pi j/N) by the three-term
 *     recurrence (Sec. 1.2, DLMF 18.9.2), then the inverse of the scaled
 *     DCT-I, c_k = (2/N) kappa_k sum''_j y_j cos(pi j k/N), by a direct O(N^2) sum.
 *   inverse  c_jac = P_N^{-1} T_N c_cheb                          (Eq. "iCJT", Sec. 1)
 *     via the integral definition of the Jacobi coefficients (Eq. "cjintdefn",
 *     Sec. 3) evaluated exactly by the (2N+1)-point Clenshaw--Curtis rule with
 *     the Jacobi weight (Sec. 3.1, Eq. "CCweights"); the weights come from the
 *     modified Chebyshev moments by their three-term recurrence (Sec. 3.1; mu_1
 *     taken as (beta-alpha)/(alpha+beta+2) mu_0, the sign that matches the
 *     weight (1-x)^alpha (1+x)^beta); the normalisation constants A_n of
 *     Eq. "Anab" by the ratio Gamma(z+1) = z Gamma(z).
 *
 * Precision: every recurrence state, table and accumulator is a double-double
 * (Dekker/Knuth error-free transformations: two_sum, two_prod via fma), so the
 * reference is accurate to ~1e-30 relative before the final rounding to
 * double.  The Lobatto points are computed in double-double from an exact
 * integer argument reduction of pi*j/N and Taylor series; no libm cosine is used.
 * The file must be compiled with -ffp-contract=off (no implicit fma contraction
 * inside the error-free transformations).
 *
 * Second, plain-double paths (orc_forward_f64, orc_inverse_f64) exist only as the
 * timed "naive O(N^2) CPU" baseline; parity uses the double-double routines.
 *
 * All entry points return 0 on success and a negative value on bad arguments.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ------------------------------------------------------------------ */
/* double-double arithmetic                                            */
/* ------------------------------------------------------------------ */
typedef struct { double hi, lo; } dd;

static inline dd mk(double h, double l) { dd r; r.hi = h; r.lo = l; return r; }
static inline dd dd_d(double a) { return mk(a, 0.0); }

static inline void two_sum(double a, double b, double *s, double *e) {
    double ss = a + b;
    double bb = ss - a;
    *e = (a - (ss - bb)) + (b - bb);
    *s = ss;
}
static inline void quick_two_sum(double a, double b, double *s, double *e) {
    double ss = a + b;
    *e = b - (ss - a);
    *s = ss;
}
static inline void two_prod(double a, double b, double *p, double *e) {
    double pp = a * b;
    *e = fma(a, b, -pp);
    *p = pp;
}
static inline dd dd_add(dd x, dd y) {
    double s, e, t, f;
    two_sum(x.hi, y.hi, &s, &e);
    two_sum(x.lo, y.lo, &t, &f);
    e += t;
    quick_two_sum(s, e, &s, &e);
    e += f;
    quick_two_sum(s, e, &s, &e);
    return mk(s, e);
}
static inline dd dd_neg(dd x) { return mk(-x.hi, -x.lo); }
static inline dd dd_sub(dd x, dd y) { return dd_add(x, dd_neg(y)); }
static inline dd dd_mul(dd x, dd y) {
    double p, e;
    two_prod(x.hi, y.hi, &p, &e);
    e += x.hi * y.lo + x.lo * y.hi;
    quick_two_sum(p, e, &p, &e);
    return mk(p, e);
}
static inline dd dd_mul_d(dd x, double y) {
    double p, e;
    two_prod(x.hi, y, &p, &e);
    e += x.lo * y;
    quick_two_sum(p, e, &p, &e);
    return mk(p, e);
}
static inline dd dd_div(dd x, dd y) {
    double q1 = x.hi / y.hi;
    dd r = dd_sub(x, dd_mul_d(y, q1));
    double q2 = r.hi / y.hi;
    r = dd_sub(r, dd_mul_d(y, q2));
    double q3 = r.hi / y.hi;
    double s, e;
    quick_two_sum(q1, q2, &s, &e);
    return dd_add(mk(s, e), dd_d(q3));
}
static inline dd dd_div_d(dd x, double y) { return dd_div(x, dd_d(y)); }

/* pi as an unevaluated sum of two doubles */
static const double PI_HI = 0x1.921fb54442d18p+1;
static const double PI_LO = 0x1.1a62633145c07p-53;

/* sin or cos of a (|a| <= pi/4) by Taylor series in double-double */
static dd dd_sin_taylor(dd a) {
    dd a2 = dd_mul(a, a);
    dd term = a, sum = a;
    for (int k = 1; k < 40; ++k) {
        term = dd_div_d(dd_mul(term, dd_neg(a2)), (double)((2 * k) * (2 * k + 1)));
        sum = dd_add(sum, term);
        if (fabs(term.hi) < 1e-40) break;
    }
    return sum;
}
static dd dd_cos_taylor(dd a) {
    dd a2 = dd_mul(a, a);
    dd term = dd_d(1.0), sum = dd_d(1.0);
    for (int k = 1; k < 40; ++k) {
        term = dd_div_d(dd_mul(term, dd_neg(a2)), (double)((2 * k - 1) * (2 * k)));
        sum = dd_add(sum, term);
        if (fabs(term.hi) < 1e-40) break;
    }
    return sum;
}

/* cos(pi p / q) in double-double for integers p, q > 0, exact argument reduction */
static dd dd_cospi_frac(int64_t p, int64_t q) {
    int64_t m = p % (2 * q);
    if (m < 0) m += 2 * q;
    if (m > q) m = 2 * q - m;            /* cos(2pi - t) = cos t, m in [0, q] */
    int neg = 0;
    if (2 * m > q) { m = q - m; neg = 1; } /* cos(pi - t) = -cos t, m in [0, q/2] */
    dd r;
    if (4 * m > q) {
        /* cos(pi m/q) = sin(pi (q - 2m) / (2q)), argument in [0, pi/4) */
        dd frac = dd_div(dd_d((double)(q - 2 * m)), dd_d((double)(2 * q)));
        r = dd_sin_taylor(dd_mul(mk(PI_HI, PI_LO), frac));
    } else {
        dd frac = dd_div(dd_d((double)m), dd_d((double)q));
        r = dd_cos_taylor(dd_mul(mk(PI_HI, PI_LO), frac));
    }
    return neg ? dd_neg(r) : r;
}

/* ------------------------------------------------------------------ */
/* Jacobi three-term recurrence coefficients (DLMF 18.9.2, Sec. 1.2)    */
/*   P_{n+1} = (A_n x + B_n) P_n - C_n P_{n-1}                         */
/* n = 0 is taken from P_1 = (alpha-beta)/2 + (alpha+beta+2)/2 x, which */
/* avoids the 0/0 of the general formula when alpha+beta = 0 or -1.     */
/* ------------------------------------------------------------------ */
static void rec_coeffs_dd(int64_t n, double a, double b, dd *A, dd *B, dd *C) {
    dd ab = dd_add(dd_d(a), dd_d(b));
    if (n == 0) {
        *A = dd_mul_d(dd_add(ab, dd_d(2.0)), 0.5);
        *B = dd_mul_d(dd_sub(dd_d(a), dd_d(b)), 0.5);
        *C = dd_d(0.0);
        return;
    }
    double nn = (double)n;
    dd t1 = dd_add(ab, dd_d(2.0 * nn + 1.0));    /* 2n+a+b+1 */
    dd t2 = dd_add(ab, dd_d(2.0 * nn + 2.0));    /* 2n+a+b+2 */
    dd t0 = dd_add(ab, dd_d(2.0 * nn));          /* 2n+a+b   */
    dd s1 = dd_add(ab, dd_d(nn + 1.0));          /* n+a+b+1  */
    dd n1 = dd_d(nn + 1.0);
    /* A_n = t1 t2 / (2 (n+1) s1) */
    *A = dd_div(dd_mul(t1, t2), dd_mul_d(dd_mul(n1, s1), 2.0));
    /* B_n = (a^2-b^2) t1 / (2 (n+1) s1 t0),  a^2-b^2 = (a-b)(a+b) */
    dd a2b2 = dd_mul(dd_sub(dd_d(a), dd_d(b)), ab);
    *B = dd_div(dd_mul(a2b2, t1), dd_mul(dd_mul_d(dd_mul(n1, s1), 2.0), t0));
    /* C_n = (n+a)(n+b) t2 / ((n+1) s1 t0) */
    dd na = dd_add(dd_d(nn), dd_d(a)), nb = dd_add(dd_d(nn), dd_d(b));
    *C = dd_div(dd_mul(dd_mul(na, nb), t2), dd_mul(dd_mul(n1, s1), t0));
}

typedef struct { dd *A, *B, *C; int64_t n; } rec_table;

static int rec_table_make(rec_table *t, int64_t nmax, double a, double b) {
    t->n = nmax + 1;
    t->A = (dd *)malloc(sizeof(dd) * (size_t)(nmax + 1));
    t->B = (dd *)malloc(sizeof(dd) * (size_t)(nmax + 1));
    t->C = (dd *)malloc(sizeof(dd) * (size_t)(nmax + 1));
    if (!t->A || !t->B || !t->C) return -1;
    for (int64_t n = 0; n <= nmax; ++n) rec_coeffs_dd(n, a, b, &t->A[n], &t->B[n], &t->C[n]);
    return 0;
}
static void rec_table_free(rec_table *t) { free(t->A); free(t->B); free(t->C); }

/* sum_{n=0}^{N} c_n P_n(x) by forward recurrence, accumulating in dd */
static dd jacobi_series_at(const rec_table *t, int64_t N, const double *c, dd x) {
    dd pm = dd_d(0.0), p = dd_d(1.0);
    dd acc = dd_d(c[0]);
    for (int64_t n = 0; n < N; ++n) {
        dd pn = dd_sub(dd_mul(dd_add(dd_mul(t->A[n], x), t->B[n]), p), dd_mul(t->C[n], pm));
        pm = p;
        p = pn;
        acc = dd_add(acc, dd_mul_d(p, c[n + 1]));
    }
    return acc;
}

static int nthreads_default(int req) {
#ifdef _OPENMP
    return req > 0 ? req : omp_get_max_threads();
#else
    (void)req;
    return 1;
#endif
}

/* ------------------------------------------------------------------ */
/* public: small helpers (exposed for the pin tests)                   */
/* ------------------------------------------------------------------ */
void orc_cospi_frac(int64_t p, int64_t q, double *hi, double *lo) {
    dd r = dd_cospi_frac(p, q);
    *hi = r.hi;
    *lo = r.lo;
}

void orc_rec_coeffs(int64_t n, double a, double b, double *A, double *B, double *C) {
    dd x, y, z;
    rec_coeffs_dd(n, a, b, &x, &y, &z);
    *A = x.hi; *B = y.hi; *C = z.hi;
}

/* P_n(x_j) for n = 0..nmax at one grid point x_j = cos(pi j / grid_N) */
int orc_jacobi_values(int64_t nmax, double a, double b, int64_t j, int64_t grid_N, double *out) {
    if (nmax < 0 || grid_N < 1) return -1;
    rec_table t;
    if (rec_table_make(&t, nmax, a, b)) return -2;
    dd x = dd_cospi_frac(j, grid_N);
    dd pm = dd_d(0.0), p = dd_d(1.0);
    out[0] = 1.0;
    for (int64_t n = 0; n < nmax; ++n) {
        dd pn = dd_sub(dd_mul(dd_add(dd_mul(t.A[n], x), t.B[n]), p), dd_mul(t.C[n], pm));
        pm = p; p = pn;
        out[n + 1] = p.hi + p.lo;
    }
    rec_table_free(&t);
    return 0;
}

/* y_j = sum_{n=0}^{N} c_n P_n(x_j), x_j = cos(pi j / grid_N), for a list of j */
int orc_jacobi_series(int64_t N, double a, double b, const double *c, int64_t npts,
                      const int64_t *j, int64_t grid_N, double *y_hi, double *y_lo, int nthreads) {
    if (N < 0 || npts < 0 || grid_N < 1) return -1;
    rec_table t;
    if (rec_table_make(&t, N, a, b)) return -2;
    int nt = nthreads_default(nthreads);
#pragma omp parallel for schedule(dynamic, 1) num_threads(nt)
    for (int64_t q = 0; q < npts; ++q) {
        dd x = dd_cospi_frac(j[q], grid_N);
        dd y = jacobi_series_at(&t, N, c, x);
        y_hi[q] = y.hi;
        if (y_lo) y_lo[q] = y.lo;
    }
    rec_table_free(&t);
    return 0;
}

/* y_j = sum_{k=0}^{K} c_k T_k(x_j) by Clenshaw's recurrence for Chebyshev series */
int orc_cheb_series(int64_t K, const double *c, int64_t npts, const int64_t *j, int64_t grid_N,
                    double *y_hi, double *y_lo, int nthreads) {
    if (K < 0 || npts < 0 || grid_N < 1) return -1;
    int nt = nthreads_default(nthreads);
#pragma omp parallel for schedule(dynamic, 1) num_threads(nt)
    for (int64_t q = 0; q < npts; ++q) {
        dd x = dd_cospi_frac(j[q], grid_N);
        dd x2 = dd_mul_d(x, 2.0);
        dd b1 = dd_d(0.0), b2 = dd_d(0.0);
        for (int64_t k = K; k >= 1; --k) {
            dd b0 = dd_add(dd_sub(dd_mul(x2, b1), b2), dd_d(c[k]));
            b2 = b1; b1 = b0;
        }
        dd y = dd_add(dd_sub(dd_mul(x, b1), b2), dd_d(c[0]));
        y_hi[q] = y.hi;
        if (y_lo) y_lo[q] = y.lo;
    }
    return 0;
}

/* ------------------------------------------------------------------ */
/* forward transform (Eq. "CJT")                                       */
/* ------------------------------------------------------------------ */
/* Inverse of the scaled DCT-I: c_k = (2/N) kappa_k sum''_j y_j cos(pi jk/N),
 * kappa_0 = kappa_N = 1/2, sum'' halves the j = 0 and j = N terms.  N >= 1. */
static void inverse_dct1_dd(int64_t N, const dd *y, double *c, int nt) {
    dd *tab = (dd *)malloc(sizeof(dd) * (size_t)(2 * N));
    for (int64_t m = 0; m < 2 * N; ++m) tab[m] = dd_cospi_frac(m, N);
#pragma omp parallel for schedule(dynamic, 16) num_threads(nt)
    for (int64_t k = 0; k <= N; ++k) {
        dd s = dd_mul_d(y[0], 0.5);
        int64_t m = 0;
        for (int64_t jj = 1; jj < N; ++jj) {
            m += k;
            if (m >= 2 * N) m -= 2 * N;
            s = dd_add(s, dd_mul(y[jj], tab[m]));
        }
        dd last = dd_mul_d(y[N], 0.5);
        s = (k & 1) ? dd_sub(s, last) : dd_add(s, last);
        s = dd_mul_d(s, 2.0);
        s = dd_div_d(s, (double)N);
        if (k == 0 || k == N) s = dd_mul_d(s, 0.5);
        c[k] = s.hi + s.lo;
    }
    free(tab);
}

int orc_forward(int64_t N, double a, double b, const double *c_jac, double *c_cheb, int nthreads) {
    if (N < 0) return -1;
    if (N == 0) { c_cheb[0] = c_jac[0]; return 0; }
    rec_table t;
    if (rec_table_make(&t, N, a, b)) return -2;
    int nt = nthreads_default(nthreads);
    dd *y = (dd *)malloc(sizeof(dd) * (size_t)(N + 1));
#pragma omp parallel for schedule(dynamic, 4) num_threads(nt)
    for (int64_t jj = 0; jj <= N; ++jj) {
        dd x = dd_cospi_frac(jj, N);
        y[jj] = jacobi_series_at(&t, N, c_jac, x);
    }
    inverse_dct1_dd(N, y, c_cheb, nt);
    free(y);
    rec_table_free(&t);
    return 0;
}

/* Grid values y_j = sum_n c_n P_n(x_j) for all j = 0..N (double-double,
 * returned as hi + lo pairs).  Used by tests that compare in value space. */
int orc_forward_values(int64_t N, double a, double b, const double *c_jac, double *y_hi, double *y_lo,
                       int nthreads) {
    if (N < 0) return -1;
    int64_t *j = (int64_t *)malloc(sizeof(int64_t) * (size_t)(N + 1));
    for (int64_t q = 0; q <= N; ++q) j[q] = q;
    int r = orc_jacobi_series(N, a, b, c_jac, N + 1, j, N > 0 ? N : 1, y_hi, y_lo, nthreads);
    free(j);
    return r;
}

/* Plain-double forward (same definition, plain double arithmetic and libm
 * cosines): the naive O(N^2) CPU reference that is timed as a baseline. */
int orc_forward_f64(int64_t N, double a, double b, const double *c_jac, double *c_cheb, int nthreads) {
    if (N < 0) return -1;
    if (N == 0) { c_cheb[0] = c_jac[0]; return 0; }
    int nt = nthreads_default(nthreads);
    double *A = (double *)malloc(sizeof(double) * (size_t)(N + 1));
    double *B = (double *)malloc(sizeof(double) * (size_t)(N + 1));
    double *C = (double *)malloc(sizeof(double) * (size_t)(N + 1));
    double *y = (double *)malloc(sizeof(double) * (size_t)(N + 1));
    double *tab = (double *)malloc(sizeof(double) * (size_t)(2 * N));
    for (int64_t n = 0; n <= N; ++n) {
        dd x, yy, z;
        rec_coeffs_dd(n, a, b, &x, &yy, &z);
        A[n] = x.hi; B[n] = yy.hi; C[n] = z.hi;
    }
    for (int64_t m = 0; m < 2 * N; ++m) tab[m] = cos(M_PI * (double)m / (double)N);
#pragma omp parallel for schedule(dynamic, 4) num_threads(nt)
    for (int64_t jj = 0; jj <= N; ++jj) {
        double x = tab[jj];
        double pm = 0.0, p = 1.0, acc = c_jac[0];
        for (int64_t n = 0; n < N; ++n) {
            double pn = (A[n] * x + B[n]) * p - C[n] * pm;
            pm = p; p = pn;
            acc += c_jac[n + 1] * p;
        }
        y[jj] = acc;
    }
#pragma omp parallel for schedule(dynamic, 16) num_threads(nt)
    for (int64_t k = 0; k <= N; ++k) {
        double s = 0.5 * y[0];
        int64_t m = 0;
        for (int64_t jj = 1; jj < N; ++jj) {
            m += k;
            if (m >= 2 * N) m -= 2 * N;
            s += y[jj] * tab[m];
        }
        s += (k & 1) ? -0.5 * y[N] : 0.5 * y[N];
        s *= 2.0 / (double)N;
        if (k == 0 || k == N) s *= 0.5;
        c_cheb[k] = s;
    }
    free(A); free(B); free(C); free(y); free(tab);
    return 0;
}

/* ------------------------------------------------------------------ */
/* inverse transform (Eq. "iCJT" via Eq. "cjintdefn" and CC quadrature) */
/* ------------------------------------------------------------------ */
/* mu_0 = 2^{a+b+1} B(a+1, b+1) (Sec. 3.1).  It is computed in double: every
 * moment and every A_n is proportional to it, so its rounding cancels from
 * the Jacobi coefficients. */
static double mu0_double(double a, double b) {
    return exp2(a + b + 1.0) * tgamma(a + 1.0) * tgamma(b + 1.0) / tgamma(a + b + 2.0);
}

/* modified Chebyshev moments mu_k = int T_k w, k = 0..K (Sec. 3.1):
 *   mu_1 = (b - a)/(a + b + 2) mu_0
 *   (a+b+k+2) mu_{k+1} = -2(a-b) mu_k - (a+b-k+2) mu_{k-1}                   */
static void moments_dd(int64_t K, double a, double b, dd *mu) {
    dd ab = dd_add(dd_d(a), dd_d(b));
    mu[0] = dd_d(mu0_double(a, b));
    if (K >= 1) mu[1] = dd_div(dd_mul(dd_sub(dd_d(b), dd_d(a)), mu[0]), dd_add(ab, dd_d(2.0)));
    dd amb2 = dd_mul_d(dd_sub(dd_d(a), dd_d(b)), 2.0);
    for (int64_t k = 1; k < K; ++k) {
        dd lhs = dd_add(ab, dd_d((double)k + 2.0));           /* a+b+k+2 */
        dd c2 = dd_add(ab, dd_d(2.0 - (double)k));            /* a+b-k+2 */
        dd num = dd_neg(dd_add(dd_mul(amb2, mu[k]), dd_mul(c2, mu[k - 1])));
        mu[k + 1] = dd_div(num, lhs);
    }
}

int orc_moments(int64_t K, double a, double b, double *mu_out) {
    if (K < 0) return -1;
    dd *mu = (dd *)malloc(sizeof(dd) * (size_t)(K + 1));
    moments_dd(K, a, b, mu);
    for (int64_t k = 0; k <= K; ++k) mu_out[k] = mu[k].hi + mu[k].lo;
    free(mu);
    return 0;
}

/* Clenshaw--Curtis weights for the Jacobi weight on the Ng+1 Lobatto points
 * (Eq. "CCweights"):  w_i = (eps_i/Ng) [mu_0 + (-1)^i mu_Ng + 2 sum_{k=1}^{Ng-1} mu_k cos(pi k i/Ng)] */
static void cc_weights_dd(int64_t Ng, double a, double b, dd *w, int nt) {
    dd *mu = (dd *)malloc(sizeof(dd) * (size_t)(Ng + 1));
    moments_dd(Ng, a, b, mu);
    dd *tab = (dd *)malloc(sizeof(dd) * (size_t)(2 * Ng));
    for (int64_t m = 0; m < 2 * Ng; ++m) tab[m] = dd_cospi_frac(m, Ng);
#pragma omp parallel for schedule(dynamic, 16) num_threads(nt)
    for (int64_t i = 0; i <= Ng; ++i) {
        dd s = dd_d(0.0);
        int64_t m = 0;
        for (int64_t k = 1; k < Ng; ++k) {
            m += i;
            if (m >= 2 * Ng) m -= 2 * Ng;
            s = dd_add(s, dd_mul(mu[k], tab[m]));
        }
        s = dd_mul_d(s, 2.0);
        s = dd_add(s, mu[0]);
        s = (i & 1) ? dd_sub(s, mu[Ng]) : dd_add(s, mu[Ng]);
        s = dd_div_d(s, (double)Ng);
        if (i == 0 || i == Ng) s = dd_mul_d(s, 0.5);
        w[i] = s;
    }
    free(tab);
    free(mu);
}

int orc_cc_weights(int64_t Ng, double a, double b, double *w_out, int nthreads) {
    if (Ng < 1) return -1;
    dd *w = (dd *)malloc(sizeof(dd) * (size_t)(Ng + 1));
    cc_weights_dd(Ng, a, b, w, nthreads_default(nthreads));
    for (int64_t i = 0; i <= Ng; ++i) w_out[i] = w[i].hi + w[i].lo;
    free(w);
    return 0;
}

/* A_n = int P_n^2 w (Eq. "Anab"), by A_0 = mu_0, A_1 = mu_0 (a+1)(b+1)/(a+b+3) and
 * A_n / A_{n-1} = (n+a)(n+b)(2n+a+b-1) / ((2n+a+b+1)(n+a+b) n) for n >= 2. */
static void norm_consts_dd(int64_t N, double a, double b, dd *A) {
    dd ab = dd_add(dd_d(a), dd_d(b));
    A[0] = dd_d(mu0_double(a, b));
    if (N >= 1)
        A[1] = dd_div(dd_mul(dd_mul(A[0], dd_add(dd_d(a), dd_d(1.0))), dd_add(dd_d(b), dd_d(1.0))),
                      dd_add(ab, dd_d(3.0)));
    for (int64_t n = 2; n <= N; ++n) {
        double nn = (double)n;
        dd num = dd_mul(dd_mul(dd_add(dd_d(nn), dd_d(a)), dd_add(dd_d(nn), dd_d(b))),
                        dd_add(ab, dd_d(2.0 * nn - 1.0)));
        dd den = dd_mul_d(dd_mul(dd_add(ab, dd_d(2.0 * nn + 1.0)), dd_add(ab, dd_d(nn))), nn);
        A[n] = dd_div(dd_mul(A[n - 1], num), den);
    }
}

int orc_norm_consts(int64_t N, double a, double b, double *A_out) {
    if (N < 0) return -1;
    dd *A = (dd *)malloc(sizeof(dd) * (size_t)(N + 1));
    norm_consts_dd(N, a, b, A);
    for (int64_t n = 0; n <= N; ++n) A_out[n] = A[n].hi + A[n].lo;
    free(A);
    return 0;
}

/* c_jac_n = (1/A_n) sum_{i=0}^{2N} w_i p_N(x_i) P_n(x_i) on the 2N grid (Sec. 3.2). */
int orc_inverse(int64_t N, double a, double b, const double *c_cheb, double *c_jac, int nthreads) {
    if (N < 0) return -1;
    if (N == 0) { c_jac[0] = c_cheb[0]; return 0; }
    int nt = nthreads_default(nthreads);
    int64_t Ng = 2 * N;
    /* p_N at the 2N grid: v_i = sum_k c_k cos(pi i k / Ng) */
    dd *tab = (dd *)malloc(sizeof(dd) * (size_t)(2 * Ng));
    for (int64_t m = 0; m < 2 * Ng; ++m) tab[m] = dd_cospi_frac(m, Ng);
    dd *g = (dd *)malloc(sizeof(dd) * (size_t)(Ng + 1));
    dd *w = (dd *)malloc(sizeof(dd) * (size_t)(Ng + 1));
    cc_weights_dd(Ng, a, b, w, nt);
#pragma omp parallel for schedule(dynamic, 16) num_threads(nt)
    for (int64_t i = 0; i <= Ng; ++i) {
        dd s = dd_d(c_cheb[0]);
        int64_t m = 0;
        for (int64_t k = 1; k <= N; ++k) {
            m += i;
            if (m >= 2 * Ng) m -= 2 * Ng;
            s = dd_add(s, dd_mul_d(tab[m], c_cheb[k]));
        }
        g[i] = dd_mul(w[i], s);
    }
    free(tab);
    rec_table t;
    if (rec_table_make(&t, N, a, b)) return -2;
    /* per-thread partial inner products, reduced in a fixed order */
    dd *part = (dd *)calloc((size_t)nt * (size_t)(N + 1), sizeof(dd));
#pragma omp parallel num_threads(nt)
    {
        int tid = 0;
#ifdef _OPENMP
        tid = omp_get_thread_num();
#endif
        dd *acc = part + (size_t)tid * (size_t)(N + 1);
#pragma omp for schedule(static)
        for (int64_t i = 0; i <= Ng; ++i) {
            dd x = dd_cospi_frac(i, Ng);
            dd pm = dd_d(0.0), p = g[i];
            acc[0] = dd_add(acc[0], p);
            for (int64_t n = 0; n < N; ++n) {
                dd pn = dd_sub(dd_mul(dd_add(dd_mul(t.A[n], x), t.B[n]), p), dd_mul(t.C[n], pm));
                pm = p; p = pn;
                acc[n + 1] = dd_add(acc[n + 1], p);
            }
        }
    }
    dd *An = (dd *)malloc(sizeof(dd) * (size_t)(N + 1));
    norm_consts_dd(N, a, b, An);
    for (int64_t n = 0; n <= N; ++n) {
        dd s = dd_d(0.0);
        for (int q = 0; q < nt; ++q) s = dd_add(s, part[(size_t)q * (size_t)(N + 1) + (size_t)n]);
        dd r = dd_div(s, An[n]);
        c_jac[n] = r.hi + r.lo;
    }
    free(An); free(part); free(g); free(w);
    rec_table_free(&t);
    return 0;
}

/* Plain-double inverse (the definition of orc_inverse in plain double arithmetic and
 * libm cosines): moments by the recurrence of Sec. 3.1, Clenshaw--Curtis weights by
 * the direct cosine sum, g_i = w_i p_N(x_i) on the 2N grid, the inner products
 * sum_i g_i P_n(x_i) by the three-term recurrence and 1/A_n (Eq. "Anab").  The naive
 * O(N^2) CPU reference timed beside the forward one. */
int orc_inverse_f64(int64_t N, double a, double b, const double *c_cheb, double *c_jac, int nthreads) {
    if (N < 0) return -1;
    if (N == 0) { c_jac[0] = c_cheb[0]; return 0; }
    int nt = nthreads_default(nthreads);
    const int64_t Ng = 2 * N;
    const double ab = a + b;
    double *mu = (double *)malloc(sizeof(double) * (size_t)(Ng + 1));
    double *tab = (double *)malloc(sizeof(double) * (size_t)(2 * Ng));
    double *g = (double *)malloc(sizeof(double) * (size_t)(Ng + 1));
    double *A = (double *)malloc(sizeof(double) * (size_t)(N + 1));
    double *B = (double *)malloc(sizeof(double) * (size_t)(N + 1));
    double *C = (double *)malloc(sizeof(double) * (size_t)(N + 1));
    double *An = (double *)malloc(sizeof(double) * (size_t)(N + 1));
    double *part = (double *)calloc((size_t)nt * (size_t)(N + 1), sizeof(double));
    mu[0] = mu0_double(a, b);
    mu[1] = (b - a) / (ab + 2.0) * mu[0];
    for (int64_t k = 1; k < Ng; ++k)
        mu[k + 1] = -(2.0 * (a - b) * mu[k] + (ab + 2.0 - (double)k) * mu[k - 1]) / (ab + (double)k + 2.0);
    for (int64_t m = 0; m < 2 * Ng; ++m) tab[m] = cos(M_PI * (double)m / (double)Ng);
#pragma omp parallel for schedule(dynamic, 16) num_threads(nt)
    for (int64_t i = 0; i <= Ng; ++i) {
        /* weight w_i (Eq. "CCweights") and p_N(x_i) = sum_k c_k T_k(x_i); k = N <= Ng - 1 */
        double s = 0.0, v = c_cheb[0];
        int64_t m = 0;
        for (int64_t k = 1; k < Ng; ++k) {
            m += i;
            if (m >= 2 * Ng) m -= 2 * Ng;
            s += mu[k] * tab[m];
            if (k <= N) v += c_cheb[k] * tab[m];
        }
        double w = (2.0 * s + mu[0] + ((i & 1) ? -mu[Ng] : mu[Ng])) / (double)Ng;
        if (i == 0 || i == Ng) w *= 0.5;
        g[i] = w * v;
    }
    for (int64_t n = 0; n <= N; ++n) {
        dd x, yy, z;
        rec_coeffs_dd(n, a, b, &x, &yy, &z);
        A[n] = x.hi; B[n] = yy.hi; C[n] = z.hi;
    }
    An[0] = mu[0];
    if (N >= 1) An[1] = mu[0] * (a + 1.0) * (b + 1.0) / (ab + 3.0);
    for (int64_t n = 2; n <= N; ++n) {
        const double nn = (double)n;
        An[n] = An[n - 1] * (nn + a) * (nn + b) * (ab + 2.0 * nn - 1.0) / ((ab + 2.0 * nn + 1.0) * (ab + nn) * nn);
    }
#pragma omp parallel num_threads(nt)
    {
        int tid = 0;
#ifdef _OPENMP
        tid = omp_get_thread_num();
#endif
        double *acc = part + (size_t)tid * (size_t)(N + 1);
#pragma omp for schedule(static)
        for (int64_t i = 0; i <= Ng; ++i) {
            const double x = tab[i];
            double pm = 0.0, p = g[i];
            acc[0] += p;
            for (int64_t n = 0; n < N; ++n) {
                double pn = (A[n] * x + B[n]) * p - C[n] * pm;
                pm = p; p = pn;
                acc[n + 1] += p;
            }
        }
    }
    for (int64_t n = 0; n <= N; ++n) {
        double s = 0.0;
        for (int q = 0; q < nt; ++q) s += part[(size_t)q * (size_t)(N + 1) + (size_t)n];
        c_jac[n] = s / An[n];
    }
    free(mu); free(tab); free(g); free(A); free(B); free(C); free(An); free(part);
    return 0;
}
