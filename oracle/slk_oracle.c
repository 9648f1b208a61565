/*
 * FP64 CPU oracle for the sliced kernel summation (test infrastructure).
 *
 * This file is TEST INFRASTRUCTURE.  Only the test-suite, the smoke check and
 * the CPU-baseline leg of the benchmark load it.  It shares no code, header,
 * constant or table with the CUDA library; it is plain, slow and written to
 * be read against the paper.
 *
 * What it computes (all in double precision):
 *   - F(r), the d-dimensional radial basis functions (Section 2.1, Table 1).
 *   - f(x), the 1-D counterparts of Table 1, evaluated from the power series
 *     of Theorem 2.3 (coefficients b_n = sqrt(pi) Gamma((n+d)/2) /
 *     (Gamma(d/2) Gamma((n+1)/2)) a_n), together with f'(x).
 *   - c_d = sqrt(pi) Gamma((d+1)/2) / Gamma(d/2)  (Section 3.2).
 *   - O-direct:  s_m = sum_n w_n F(|x_n - y_m|)   (problem statement, Sec. 3).
 *   - O-sliced:  per slice p and target m, the exact 1-D sum
 *                sum_n w_n f(|z_y[m,p] - z_x[n,p]|)  (Algorithm 1 with exact
 *                1-D sums instead of a fast method), and the matching
 *                gradient sums  sum_n w_n f'(|d|) sign(d),  d = z_y - z_x,
 *                with sign(0) = 0.
 *
 * Sums use Neumaier compensation.  Threads (OpenMP) only split independent
 * outputs; every output is summed in a fixed order.
 */
#include <float.h>
#include <math.h>
#include <stdint.h>
#include <string.h>

#define ORC_GAUSSIAN 0
#define ORC_LAPLACIAN 1
#define ORC_NEGDIST 2
#define ORC_MATERN32 3


/* F(r): Gaussian exp(-r^2/(2 sigma^2)), Laplacian exp(-alpha r), negative
 * distance -r, Matern nu = 3/2 (1 + a r) exp(-a r) with a = sqrt(3) / beta
 * (Table 1, first column, and the Appendix's formula for nu = p + 1/2 at p = 1;
 * param = sigma, alpha or beta). */
double orc_F(int kernel, double param, double r) {
    switch (kernel) {
    case ORC_GAUSSIAN: return exp(-r * r / (2.0 * param * param));
    case ORC_LAPLACIAN: return exp(-param * r);
    case ORC_NEGDIST: return -r;
    case ORC_MATERN32: {
        double a = sqrt(3.0) / param;
        return (1.0 + a * r) * exp(-a * r);
    }
    }
    return NAN;
}

/* dF/dr. */
double orc_dF(int kernel, double param, double r) {
    switch (kernel) {
    case ORC_GAUSSIAN: return -r / (param * param) * exp(-r * r / (2.0 * param * param));
    case ORC_LAPLACIAN: return -param * exp(-param * r);
    case ORC_NEGDIST: return -1.0;
    case ORC_MATERN32: {
        double a = sqrt(3.0) / param;
        return -a * a * r * exp(-a * r);
    }
    }
    return NAN;
}

static inline void neumaier_add(double* s, double* c, double v) {
    double t = *s + v;
    if (fabs(*s) >= fabs(v)) *c += (*s - t) + v;
    else *c += (v - t) + *s;
    *s = t;
}

/*
 * Double-double arithmetic (value = hi + lo, ~106-bit significand) built from
 * the error-free transformations TwoSum (Knuth) and TwoProd (via fma).  The
 * power series below alternate in sign with terms far larger than their sum
 * (largest term ~ exp(sqrt(d) x / sigma) for the Gaussian), so they are summed
 * in double-double; the returned error bound accounts for what is left.
 */
typedef struct { double hi, lo; } dd;

static inline dd two_sum(double a, double b) {
    double s = a + b, bb = s - a;
    dd r = {s, (a - (s - bb)) + (b - bb)};
    return r;
}
static inline dd quick_two_sum(double a, double b) {
    double s = a + b;
    dd r = {s, b - (s - a)};
    return r;
}
static inline dd dd_add(dd a, dd b) {
    dd s = two_sum(a.hi, b.hi), t = two_sum(a.lo, b.lo);
    s.lo += t.hi;
    s = quick_two_sum(s.hi, s.lo);
    s.lo += t.lo;
    return quick_two_sum(s.hi, s.lo);
}
static inline dd dd_mul(dd a, dd b) {
    double p = a.hi * b.hi;
    double e = fma(a.hi, b.hi, -p);
    e += a.hi * b.lo + a.lo * b.hi;
    return quick_two_sum(p, e);
}
static inline dd dd_mul_d(dd a, double b) {
    double p = a.hi * b;
    double e = fma(a.hi, b, -p) + a.lo * b;
    return quick_two_sum(p, e);
}
static inline dd dd_div_d(dd a, double b) {
    double q1 = a.hi / b;
    dd p = dd_mul_d((dd){q1, 0.0}, b);
    dd r = dd_add(a, (dd){-p.hi, -p.lo});
    double q2 = r.hi / b;
    return quick_two_sum(q1, q2);
}
static inline dd dd_from(double a) { dd r = {a, 0.0}; return r; }

/*
 * c_d = sqrt(pi) Gamma((d+1)/2) / Gamma(d/2)  (Section 3.2, negative-distance row
 * of Table 1), in double-double from Gamma(z+1) = z Gamma(z):
 *   c_1 = 1,  c_2 = pi/2,  c_{d+2} = c_d (d+1)/d.
 */
static dd cd_dd(int d) {
    static _Thread_local int cached_d = -1;
    static _Thread_local dd cached;
    if (d == cached_d) return cached;
    dd c = (d % 2) ? dd_from(1.0) : (dd){1.5707963267948966, 6.123233995736766e-17};
    for (int k = (d % 2) ? 1 : 2; k + 2 <= d; k += 2) c = dd_div_d(dd_mul_d(c, (double)(k + 1)), (double)k);
    cached_d = d;
    cached = c;
    return c;
}
double orc_cd(int d) {
    dd c = cd_dd(d);
    return c.hi + c.lo;
}

/*
 * Gaussian 1-D counterpart, Table 1:
 *   f(x) = 1F1(d/2; 1/2; -x^2/(2 sigma^2))
 *        = sum_n (-1)^n sqrt(pi) Gamma(n + d/2) / (2^n sigma^{2n} n! Gamma(d/2) Gamma(n + 1/2)) x^{2n}.
 * Term n+1 over term n is  -u (n + d/2) / ((n + 1/2)(n + 1)),  u = x^2/(2 sigma^2).
 * f'(x) = sum_n 2n t_n / x.
 * *err receives a bound on the rounding error: (largest |term|) * (#terms) * 2^-100 + eps |f|.
 */
static double f_gauss_dd(int d, double sigma, double x, double* df, double* err) {
    dd u = dd_div_d(dd_mul(dd_from(x), dd_from(x)), 2.0);
    u = dd_div_d(dd_div_d(u, sigma), sigma);
    double a = 0.5 * d;
    dd term = dd_from(1.0), s = dd_from(1.0), ds = dd_from(0.0);
    double tmax = 1.0;
    int n;
    for (n = 0; n < 200000; ++n) {
        term = dd_div_d(dd_mul_d(dd_mul(term, u), -(n + a)), (n + 0.5) * (n + 1.0));
        s = dd_add(s, term);
        ds = dd_add(ds, dd_mul_d(term, 2.0 * (n + 1.0)));
        if (fabs(term.hi) > tmax) tmax = fabs(term.hi);
        /* past the largest term (ratio < 1) and negligible */
        if (u.hi * (n + 1 + a) < (n + 1.5) * (n + 2.0) && fabs(term.hi) < 1e-34 * tmax) break;
        if (term.hi == 0.0) break;
    }
    if (df) *df = (x != 0.0) ? (ds.hi + ds.lo) / x : 0.0;
    if (err) *err = tmax * (n + 2) * ldexp(1.0, -100) + fabs(s.hi) * DBL_EPSILON;
    return s.hi + s.lo;
}

/*
 * Laplacian 1-D counterpart, Table 1 (paper convention F = exp(-alpha r)):
 *   f(x) = sum_n (-1)^n alpha^n sqrt(pi) Gamma((n+d)/2) / (n! Gamma(d/2) Gamma((n+1)/2)) x^n.
 * b_0 = 1, b_1 = -alpha c_d, and b_{n+2} = b_n alpha^2 (n+d) / ((n+1)^2 (n+2)),
 * so even and odd terms follow two separate recurrences (the even terms are all
 * positive, the odd ones all negative: the sum cancels, hence double-double).
 */
static double f_laplace_dd(int d, double alpha, double x, double* df, double* err) {
    dd ax = dd_mul(dd_from(alpha), dd_from(x));
    dd ax2 = dd_mul(ax, ax);
    dd cdd = cd_dd(d);
    double cd = cdd.hi + cdd.lo;
    dd s = dd_from(0.0), ds = dd_from(0.0);
    double tmax = 0.0;
    int nterms = 0;
    for (int parity = 0; parity < 2; ++parity) {
        dd term = parity == 0 ? dd_from(1.0) : dd_mul(ax, (dd){-cdd.hi, -cdd.lo});
        int n = parity;
        for (int j = 0; j < 200000; ++j) {
            s = dd_add(s, term);
            ds = dd_add(ds, dd_mul_d(term, (double)n));
            if (fabs(term.hi) > tmax) tmax = fabs(term.hi);
            ++nterms;
            double den = (n + 1.0) * (n + 1.0) * (n + 2.0);
            if (ax2.hi * (n + d) < den && fabs(term.hi) < 1e-34 * (tmax > 0 ? tmax : 1.0)) break;
            term = dd_div_d(dd_mul_d(dd_mul(term, ax2), (double)(n + d)), den);
            n += 2;
            if (term.hi == 0.0) break;
        }
    }
    if (df) *df = (x != 0.0) ? (ds.hi + ds.lo) / x : -cd * alpha;
    if (err) *err = tmax * (nterms + 2) * ldexp(1.0, -100) + fabs(s.hi) * DBL_EPSILON;
    return s.hi + s.lo;
}

/*
 * The same two series summed in plain double precision.  Used when their own
 * rounding bound (largest term x #terms x 4 eps) is below 1e-12; otherwise the
 * double-double versions above are used.
 */
static double f_gauss_d(int d, double sigma, double x, double* df, double* err) {
    double u = x * x / (2.0 * sigma * sigma), a = 0.5 * d;
    double term = 1.0, s = 1.0, ds = 0.0, tmax = 1.0;
    int n;
    for (n = 0; n < 200000; ++n) {
        term *= -u * (n + a) / ((n + 0.5) * (n + 1.0));
        s += term;
        ds += 2.0 * (n + 1.0) * term;
        if (fabs(term) > tmax) tmax = fabs(term);
        if (u * (n + 1 + a) < (n + 1.5) * (n + 2.0) && fabs(term) < 1e-18 * tmax) break;
        if (term == 0.0) break;
    }
    *df = (x != 0.0) ? ds / x : 0.0;
    *err = tmax * (n + 2) * 4.0 * DBL_EPSILON;
    return s;
}

static double f_laplace_d(int d, double alpha, double x, double* df, double* err) {
    double ax2 = (alpha * x) * (alpha * x), cd = orc_cd(d);
    double s = 0.0, ds = 0.0, tmax = 0.0;
    int nterms = 0;
    for (int parity = 0; parity < 2; ++parity) {
        double term = parity == 0 ? 1.0 : -cd * alpha * x;
        int n = parity;
        for (int j = 0; j < 200000; ++j) {
            s += term;
            ds += n * term;
            if (fabs(term) > tmax) tmax = fabs(term);
            ++nterms;
            double den = (n + 1.0) * (n + 1.0) * (n + 2.0);
            if (ax2 * (n + d) < den && fabs(term) < 1e-18 * (tmax > 0 ? tmax : 1.0)) break;
            term *= ax2 * (n + d) / den;
            n += 2;
            if (term == 0.0) break;
        }
    }
    *df = (x != 0.0) ? ds / x : -cd * alpha;
    *err = tmax * (nterms + 2) * 4.0 * DBL_EPSILON;
    return s;
}

/*
 * Matern nu = 3/2 1-D counterpart.  F(r) = (1 + a r) exp(-a r) = G(r) - r G'(r) for the
 * Laplacian G(r) = exp(-a r), so its power-series coefficients are G's times (1 - n);
 * Theorem 2.3 maps every power r^n to a multiple of x^n, hence
 *   f(x) = sum_n (1 - n) b_n x^n,  b_n the Laplacian coefficients above (alpha = a),
 * with the same two recurrences (the n = 1 term vanishes: f is C^1 at 0).
 */
static double f_matern_dd(int d, double a, double x, double* df, double* err) {
    dd ax = dd_mul(dd_from(a), dd_from(x));
    dd ax2 = dd_mul(ax, ax);
    dd cdd = cd_dd(d);
    dd s = dd_from(0.0), ds = dd_from(0.0);
    double tmax = 0.0;
    int nterms = 0;
    for (int parity = 0; parity < 2; ++parity) {
        dd term = parity == 0 ? dd_from(1.0) : dd_mul(ax, (dd){-cdd.hi, -cdd.lo});
        int n = parity;
        for (int j = 0; j < 200000; ++j) {
            dd t = dd_mul_d(term, 1.0 - n);
            s = dd_add(s, t);
            ds = dd_add(ds, dd_mul_d(t, (double)n));
            if (fabs(t.hi) > tmax) tmax = fabs(t.hi);
            ++nterms;
            double den = (n + 1.0) * (n + 1.0) * (n + 2.0);
            if (ax2.hi * (n + d) < den && n > 1 && fabs(t.hi) < 1e-34 * (tmax > 0 ? tmax : 1.0)) break;
            term = dd_div_d(dd_mul_d(dd_mul(term, ax2), (double)(n + d)), den);
            n += 2;
            if (term.hi == 0.0) break;
        }
    }
    if (df) *df = (x != 0.0) ? (ds.hi + ds.lo) / x : 0.0;
    if (err) *err = tmax * (nterms + 2) * ldexp(1.0, -100) + fabs(s.hi) * DBL_EPSILON;
    return s.hi + s.lo;
}

static double f_matern_d(int d, double a, double x, double* df, double* err) {
    double ax2 = (a * x) * (a * x), cd = orc_cd(d);
    double s = 0.0, ds = 0.0, tmax = 0.0;
    int nterms = 0;
    for (int parity = 0; parity < 2; ++parity) {
        double term = parity == 0 ? 1.0 : -cd * a * x;
        int n = parity;
        for (int j = 0; j < 200000; ++j) {
            double t = (1.0 - n) * term;
            s += t;
            ds += n * t;
            if (fabs(t) > tmax) tmax = fabs(t);
            ++nterms;
            double den = (n + 1.0) * (n + 1.0) * (n + 2.0);
            if (ax2 * (n + d) < den && n > 1 && fabs(t) < 1e-18 * (tmax > 0 ? tmax : 1.0)) break;
            term *= ax2 * (n + d) / den;
            n += 2;
            if (term == 0.0) break;
        }
    }
    *df = (x != 0.0) ? ds / x : 0.0;
    *err = tmax * (nterms + 2) * 4.0 * DBL_EPSILON;
    return s;
}

static double f_matern(int d, double beta, double x, double* df, double* err) {
    double a = sqrt(3.0) / beta;
    double v = f_matern_d(d, a, x, df, err);
    if (*err <= 1e-12) return v;
    return f_matern_dd(d, a, x, df, err);
}

static double f_gauss(int d, double sigma, double x, double* df, double* err) {
    double v = f_gauss_d(d, sigma, x, df, err);
    if (*err <= 1e-12) return v;
    return f_gauss_dd(d, sigma, x, df, err);
}

static double f_laplace(int d, double alpha, double x, double* df, double* err) {
    double v = f_laplace_d(d, alpha, x, df, err);
    if (*err <= 1e-12) return v;
    return f_laplace_dd(d, alpha, x, df, err);
}

/* Negative distance: f(x) = -c_d x (Table 1, Section 3.2). */
static double f_negdist(int d, double x, double* df, double* err) {
    double cd = orc_cd(d);
    if (df) *df = -cd;
    if (err) *err = cd * fabs(x) * DBL_EPSILON;
    return -cd * x;
}

/*
 * Gauss-Legendre nodes/weights on [-1, 1] (Newton iteration on the Legendre
 * recurrence), computed once.
 */
#define GL_N 16
static double gl_x[GL_N], gl_w[GL_N];
static int gl_ready = 0;
static void gl_init(void) {
    if (gl_ready) return;
    for (int i = 0; i < GL_N; ++i) {
        double z = cos(M_PI * (i + 0.75) / (GL_N + 0.5)), dp = 1.0;
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = z;
            for (int k = 2; k <= GL_N; ++k) {
                double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
                p0 = p1;
                p1 = p2;
            }
            dp = GL_N * (z * p1 - p0) / (z * z - 1.0);
            double dz = p1 / dp;
            z -= dz;
            if (fabs(dz) < 1e-16) break;
        }
        gl_x[i] = z;
        gl_w[i] = 2.0 / ((1.0 - z * z) * dp * dp);
    }
    gl_ready = 1;
}

double orc_fhat_gauss(int d, double sigma, double omega);

/*
 * Gaussian counterpart by Fourier inversion of Lemma 2.6 (second, independent
 * route, used where the alternating series loses accuracy):
 *   f(x)  =  2 int_0^inf fhat(w) cos(2 pi w x) dw,
 *   f'(x) = -2 int_0^inf fhat(w) 2 pi w sin(2 pi w x) dw.
 * fhat ~ exp(-u) u^((d-1)/2) with u = 2 pi^2 sigma^2 w^2 is integrated over the
 * band where it exceeds e^-45 of its peak, composite 16-point Gauss-Legendre
 * with >= 4 panels per period of the cosine.  Rounding bound (*err; the integral of
 * |fhat| is 1/2, so a relative error e of every fhat value costs at most e): fhat is
 * evaluated in log space, where the terms of the exponent reach L = |log(d pi sigma)|
 * + u_max + ((d-1)/2) |log u_max| + lgamma((d+2)/2), each rounded to eps relative, and the
 * cosine's argument reaches 2 pi w_max x; together 4 eps (L + 2 pi w_max x + 4).
 */
static double f_gauss_fourier(int d, double sigma, double x, double* df, double* err) {
    gl_init();
    double a = 0.5 * (d - 1);
    double umax = a + 55.0 + 12.0 * sqrt(a + 1.0);
    double umin = d > 1 ? a - 12.0 * sqrt(a + 1.0) - 10.0 : 0.0;
    if (umin < 0.0) umin = 0.0;
    double c = 2.0 * M_PI * M_PI * sigma * sigma;
    double wlo = sqrt(umin / c), whi = sqrt(umax / c);
    long panels = (long)ceil((whi - wlo) * fabs(x) * 4.0) + 200;
    if (panels > 200000) panels = 200000;
    double h = (whi - wlo) / panels, s = 0.0, cs = 0.0, ds = 0.0, dcs = 0.0;
    for (long k = 0; k < panels; ++k) {
        double mid = wlo + (k + 0.5) * h;
        for (int i = 0; i < GL_N; ++i) {
            double w = mid + 0.5 * h * gl_x[i];
            double fw = orc_fhat_gauss(d, sigma, w) * 0.5 * h * gl_w[i];
            neumaier_add(&s, &cs, fw * cos(2.0 * M_PI * w * x));
            neumaier_add(&ds, &dcs, -fw * 2.0 * M_PI * w * sin(2.0 * M_PI * w * x));
        }
    }
    if (df) *df = 2.0 * (ds + dcs);
    if (err) {
        const double L = fabs(log(d * M_PI * sigma)) + umax + a * fabs(log(umax)) + lgamma(0.5 * (d + 2));
        *err = 4.0 * DBL_EPSILON * (L + 2.0 * M_PI * whi * fabs(x) + 4.0);
    }
    return 2.0 * (s + cs);
}

/* f(x) for x >= 0 and f'(x); returns f, writes f' and a rounding bound. */
double orc_f(int kernel, int d, double param, double x, double* df, double* err) {
    double dummy_df, dummy_err;
    if (!df) df = &dummy_df;
    if (!err) err = &dummy_err;
    switch (kernel) {
    case ORC_GAUSSIAN: {
        double v = f_gauss(d, param, x, df, err);
        if (*err > 1e-12) v = f_gauss_fourier(d, param, x, df, err);
        return v;
    }
    case ORC_LAPLACIAN: return f_laplace(d, param, x, df, err);
    case ORC_NEGDIST: return f_negdist(d, x, df, err);
    case ORC_MATERN32: return f_matern(d, param, x, df, err);
    }
    return NAN;
}

/* Vectorised f / f' for the tests.  Returns the largest rounding bound. */
double orc_f_vec(int kernel, int d, double param, const double* x, int64_t n, double* f, double* df) {
    double emax = 0.0;
    gl_init();
    for (int64_t i = 0; i < n; ++i) {
        double e = 0.0, g = 0.0;
        f[i] = orc_f(kernel, d, param, fabs(x[i]), &g, &e);
        if (df) df[i] = g;
        if (e > emax) emax = e;
    }
    return emax;
}

/*
 * Lemma 2.6: Fourier transform of the Gaussian counterpart,
 *   fhat(w) = d pi sigma exp(-2 pi^2 sigma^2 w^2) (2 pi^2 sigma^2 w^2)^((d-1)/2) / (sqrt(2) Gamma((d+2)/2)),
 * evaluated in log space.
 */
double orc_fhat_gauss(int d, double sigma, double omega) {
    double u = 2.0 * M_PI * M_PI * sigma * sigma * omega * omega;
    if (u == 0.0) return d == 1 ? sigma * sqrt(2.0 * M_PI) : 0.0;
    double lg = log(d * M_PI * sigma) - u + 0.5 * (d - 1) * log(u) - 0.5 * log(2.0) - lgamma(0.5 * (d + 2));
    return exp(lg);
}

/*
 * O-direct: s_m = sum_n w_n F(|x_n - y_m|); X is N x d, Y is M x d, row-major.
 * With grad != NULL also writes the d-dimensional gradient of s_m w.r.t. y_m
 * (sum_n w_n F'(r) (y_m - x_n)/r, zero term at r = 0).
 */
void orc_direct_sum(int kernel, double param, int d, const double* X, int64_t N, const double* Y, int64_t M,
                    const double* w, double* s, double* grad) {
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t m = 0; m < M; ++m) {
        const double* y = Y + m * (int64_t)d;
        double acc = 0.0, comp = 0.0;
        for (int64_t n = 0; n < N; ++n) {
            const double* x = X + n * (int64_t)d;
            double r2 = 0.0;
            for (int i = 0; i < d; ++i) {
                double t = y[i] - x[i];
                r2 += t * t;
            }
            neumaier_add(&acc, &comp, w[n] * orc_F(kernel, param, sqrt(r2)));
        }
        s[m] = acc + comp;
        if (grad) {
            double* g = grad + m * (int64_t)d;
            for (int i = 0; i < d; ++i) g[i] = 0.0;
            for (int64_t n = 0; n < N; ++n) {
                const double* x = X + n * (int64_t)d;
                double r2 = 0.0;
                for (int i = 0; i < d; ++i) {
                    double t = y[i] - x[i];
                    r2 += t * t;
                }
                double r = sqrt(r2);
                if (r == 0.0) continue;
                double coef = w[n] * orc_dF(kernel, param, r) / r;
                for (int i = 0; i < d; ++i) g[i] += coef * (y[i] - x[i]);
            }
        }
    }
}

/*
 * O-sliced partial sums over one chunk of sources.  Zx is n x P (row n holds
 * <xi_p, x_n> for all p), Zy is M x P.  For every (m, p) this adds
 *     sum_n w_n f(|Zy[m,p] - Zx[n,p]|)                 into S[m*P+p] (+ SC compensation)
 *     sum_n w_n f'(|d|) sign(d),  d = Zy[m,p]-Zx[n,p]  into G[m*P+p] (if G != NULL)
 * Returns the largest rounding bound met by the f evaluations.
 */
double orc_sliced_accumulate(int kernel, int d, double param, const double* Zx, int64_t n, const double* w,
                             const double* Zy, int64_t M, int P, double* S, double* SC, double* G, double* GC) {
    double emax = 0.0;
    int64_t tasks = M * (int64_t)P;
    gl_init(); /* before the parallel region: the tables are then read-only */
#pragma omp parallel for schedule(dynamic, 16) reduction(max : emax)
    for (int64_t t = 0; t < tasks; ++t) {
        int64_t m = t / P;
        int p = (int)(t % P);
        double zy = Zy[m * P + p];
        double s = S[t], c = SC[t];
        double g = G ? G[t] : 0.0, gc = G ? GC[t] : 0.0;
        for (int64_t k = 0; k < n; ++k) {
            double delta = zy - Zx[k * P + p];
            double df = 0.0, e = 0.0;
            double fv = orc_f(kernel, d, param, fabs(delta), &df, &e);
            if (e > emax) emax = e;
            neumaier_add(&s, &c, w[k] * fv);
            if (G) {
                double sg = delta > 0.0 ? 1.0 : (delta < 0.0 ? -1.0 : 0.0);
                neumaier_add(&g, &gc, w[k] * df * sg);
            }
        }
        S[t] = s;
        SC[t] = c;
        if (G) {
            G[t] = g;
            GC[t] = gc;
        }
    }
    return emax;
}
