// Plan-time parameter selection for the Fourier summations (host, FP64).
//
// Gaussian (Section 2.2, Lemma 2.6, Eq. (Fourier_cutoff)): after rescaling by a
// period L the periodic kernel has coefficients c_k = fhat(k / L) / L with
//     fhat(w) = d pi sigma exp(-2 pi^2 sigma^2 w^2) (2 pi^2 sigma^2 w^2)^((d-1)/2) / (sqrt 2 Gamma((d+2)/2)).
// The paper leaves the period and the cut-offs (T, eps, K_max) as hand-tuned
// hyperparameters; here they are chosen so that two certified errors stay
// below the target:
//   periodisation  sup_{|u| <= 2R} sum_{j != 0} |f(u + j L)|,
//   truncation     sum_{k not in C} |c_k|,
// where R bounds every projected point (sources and targets).  f for the
// periodisation bound is evaluated by Gauss-Legendre quadrature of the
// Fourier inversion integral (f is even, fhat explicit).
//
// NFFT window: "exponential of semicircle" psi(s) = exp(beta (sqrt(1 - (2s/m)^2) - 1))
// on |s| <= m/2 cells, beta = 2.30 m for twofold oversampling; its Fourier
// transform Psi is computed by quadrature (substitution s = (m/2) sin(theta)),
// and the aliasing ratio sum_{r != 0} Psi(k/n + r) / Psi(k/n) bounds the
// window error.
//
// Laplacian smooth part (Section 3.3): k1(x) = f_lap(|x|) + alpha c_d |x| (the
// 1-D counterpart of exp(-alpha r) + alpha r; the series of Table 1 without its
// n = 1 term).  The paper does not say how this linearly growing function is
// made periodic; here (see the design notes) it is kept exactly on the data
// range |u| <= rho (rescaled), continued by its cubic Taylor polynomial and
// blended smoothly to a constant towards |u| = 1/2, then sampled on a fine
// grid and transformed by a host FFT.
#include <algorithm>
#include <cmath>
#include <complex>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "params.cuh"

namespace slk {

namespace {

constexpr double PI = 3.14159265358979323846;

// ------------------------------------------------------------ quadrature nodes

struct GL {
    std::vector<double> x, w;
    explicit GL(int n) : x(n), w(n) {
        for (int i = 0; i < n; ++i) {
            double z = std::cos(PI * (i + 0.75) / (n + 0.5)), dp = 1.0;
            for (int it = 0; it < 100; ++it) {
                double p0 = 1.0, p1 = z;
                for (int k = 2; k <= n; ++k) {
                    double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
                    p0 = p1;
                    p1 = p2;
                }
                dp = n * (z * p1 - p0) / (z * z - 1.0);
                double dz = p1 / dp;
                z -= dz;
                if (std::fabs(dz) < 1e-16) break;
            }
            x[i] = z;
            w[i] = 2.0 / ((1.0 - z * z) * dp * dp);
        }
    }
};

const GL& gl20() {
    static GL g(20);
    return g;
}

// ------------------------------------------------------------ Gaussian

double log_fhat_gauss(double sigma, int d, double omega) {
    double u = 2.0 * PI * PI * sigma * sigma * omega * omega;
    if (u == 0.0) return d == 1 ? std::log(sigma * std::sqrt(2.0 * PI)) : -INFINITY;
    return std::log(d * PI * sigma) - u + 0.5 * (d - 1) * std::log(u) - 0.5 * std::log(2.0) - std::lgamma(0.5 * (d + 2));
}

// band [w_lo, w_hi] outside which fhat < exp(-60) * peak
void gauss_band(double sigma, int d, double* wlo, double* whi) {
    double a = 0.5 * (d - 1);
    double c = 2.0 * PI * PI * sigma * sigma;
    double umax = a + 70.0 + 14.0 * std::sqrt(a + 1.0);
    double umin = d > 1 ? std::max(0.0, a - 14.0 * std::sqrt(a + 1.0) - 10.0) : 0.0;
    *wlo = std::sqrt(umin / c);
    *whi = std::sqrt(umax / c);
}

// f(x) = 2 int_0^inf fhat(w) cos(2 pi w x) dw  (composite 20-point Gauss-Legendre)
double f_gauss_host(double sigma, int d, double x) {
    double wlo, whi;
    gauss_band(sigma, d, &wlo, &whi);
    const GL& g = gl20();
    long panels = static_cast<long>(std::ceil((whi - wlo) * std::fabs(x) * 2.0)) + 48;
    panels = std::min(panels, 400000L);
    double h = (whi - wlo) / panels, s = 0.0;
    for (long k = 0; k < panels; ++k) {
        double mid = wlo + (k + 0.5) * h;
        for (size_t i = 0; i < g.x.size(); ++i) {
            double w = mid + 0.5 * h * g.x[i];
            s += g.w[i] * 0.5 * h * std::exp(log_fhat_gauss(sigma, d, w)) * std::cos(2.0 * PI * w * x);
        }
    }
    return 2.0 * s;
}

// sup over |u| <= D of sum_{j != 0} |f(u + j L)|  (sampled)
double gauss_periodisation(double sigma, int d, double D, double L) {
    double worst = 0.0;
    const int NU = 12;
    for (int i = 0; i <= NU; ++i) {
        double u = D * i / NU;
        double s = 0.0;
        for (int j = 1; j <= 4; ++j) s += std::fabs(f_gauss_host(sigma, d, j * L + u)) + std::fabs(f_gauss_host(sigma, d, j * L - u));
        worst = std::max(worst, s);
    }
    return worst;
}

// ------------------------------------------------------------ window

// Psi(nu) = int psi(s) exp(-2 pi i s nu) ds, via s = (m/2) sin(t)
double es_Psi(double nu, int m, double beta) {
    const GL& g = gl20();
    const int panels = 64;
    double a = -0.5 * PI, h = PI / panels, s = 0.0;
    for (int k = 0; k < panels; ++k) {
        double mid = a + (k + 0.5) * h;
        for (size_t i = 0; i < g.x.size(); ++i) {
            double t = mid + 0.5 * h * g.x[i];
            double sv = 0.5 * m * std::sin(t);
            s += g.w[i] * 0.5 * h * std::exp(beta * (std::cos(t) - 1.0)) * std::cos(2.0 * PI * sv * nu) * 0.5 * m *
                 std::cos(t);
        }
    }
    return s;
}

// window error estimate for width m, grid n_g, |k| < kmax
double window_error(int m, double beta, int n_g, int kmax) {
    double worst = 0.0;
    for (int k = 0; k < kmax; k += std::max(1, kmax / 16)) {
        double nu = static_cast<double>(k) / n_g;
        double P0 = es_Psi(nu, m, beta);
        double al = 0.0;
        for (int r = 1; r <= 3; ++r) al += std::fabs(es_Psi(nu + r, m, beta)) + std::fabs(es_Psi(nu - r, m, beta));
        worst = std::max(worst, al / P0);
    }
    // spreading and interpolation each alias once; the truncated window leaves
    // a jump of exp(-beta) relative to psi(0) = 1
    return 2.0 * worst + 2.0 * m * std::exp(-beta);
}

// psi(s) in FP64, in the cancellation-free form exp(-beta x^2 / (1 + sqrt(1 - x^2)))
double es_psi_host(double s, int m, double beta) {
    const double x = 2.0 * s / m, q = 1.0 - x * x;
    return q >= 0.0 ? std::exp(-beta * x * x / (1.0 + std::sqrt(q))) : 0.0;
}

// The window's taps as polynomials for the FP32 kernels: a point whose first cell lies at
// s0 = g + 1/2 - m/2 (g in [-1/2, 1/2)) weights cell t < m by psi(s0 + t); per tap, the
// degree-kWinPolyDeg interpolant at the (symmetric) Chebyshev points of g, written in powers of g
// (a Vandermonde solve in FP64 by Gaussian elimination with partial pivoting; on this
// interval the coefficients stay below about one).  Its largest error on a 2001-point grid
// goes to wpoly_err: about 2e-9 for m >= 9 and below exp(-beta) otherwise (the square-root
// branch point of psi at the window's edge, where psi = exp(-beta), limits it).
void fit_window_poly(FourierHost* fp) {
    constexpr int D = kWinPolyDeg, n = kWinPolyDeg + 1;
    const int m = fp->m;
    fp->wpoly.assign(static_cast<size_t>(m) * n, 0.0);
    double worst = 0.0;
    for (int t = 0; t < m; ++t) {
        double A[n][n + 1];
        for (int j = 0; j < n; ++j) {
            const double g = 0.5 * std::cos(PI * (j + 0.5) / n);
            double pw = 1.0;
            for (int k = 0; k < n; ++k, pw *= g) A[j][k] = pw;
            A[j][n] = es_psi_host(g + 0.5 + t - 0.5 * m, m, fp->beta);
        }
        for (int c = 0; c < n; ++c) {
            int piv = c;
            for (int r = c + 1; r < n; ++r)
                if (std::fabs(A[r][c]) > std::fabs(A[piv][c])) piv = r;
            for (int k = 0; k <= n; ++k) std::swap(A[c][k], A[piv][k]);
            for (int r = 0; r < n; ++r) {
                if (r == c) continue;
                const double f = A[r][c] / A[c][c];
                for (int k = c; k <= n; ++k) A[r][k] -= f * A[c][k];
            }
        }
        double* a = fp->wpoly.data() + static_cast<size_t>(t) * n;
        for (int k = 0; k < n; ++k) a[k] = A[k][n] / A[k][k];
    }
    // the kernels evaluate tap t >= ceil(m / 2) as P_{m-1-t}(-g) (psi is even): measure that
    for (int t = 0; t < m; ++t) {
        const bool mirror = t >= (m + 1) / 2;
        const double* a = fp->wpoly.data() + static_cast<size_t>(mirror ? m - 1 - t : t) * n;
        for (int i = 0; i <= 2000; ++i) {
            const double g = -0.5 + i / 2000.0, x = mirror ? -g : g;
            double v = a[D];
            for (int k = D - 1; k >= 0; --k) v = v * x + a[k];
            worst = std::max(worst, std::fabs(v - es_psi_host(g + 0.5 + t - 0.5 * m, m, fp->beta)));
        }
    }
    fp->wpoly_err = worst;
}

void choose_window(FourierHost* fp, double tol_w) {
    const int kmax = fp->n_coeff / 2;
    for (int m = 4; m <= 16; ++m) {
        double beta = 2.30 * m;
        double e = window_error(m, beta, fp->n_g, kmax);
        if (e <= tol_w || m == 16) {
            fp->m = m;
            fp->beta = beta;
            fp->window_err = e;
            break;
        }
    }
    fp->psi.resize(kmax);
    for (int k = 0; k < kmax; ++k) fp->psi[k] = es_Psi(static_cast<double>(k) / fp->n_g, fp->m, fp->beta);
    fit_window_poly(fp);
}


void set_active_window(FourierHost* fp) {
    double umax = fp->R * fp->n_g / fp->L;
    int base = static_cast<int>(std::ceil(-umax - 0.5 * fp->m)) - 1;
    int last = static_cast<int>(std::ceil(umax - 0.5 * fp->m)) + fp->m;  // exclusive
    fp->win_base = base;
    fp->W = last - base + 1;
}

int next_pow2(int v) {
    int p = 1;
    while (p < v) p <<= 1;
    return p;
}

// ------------------------------------------------------------ Laplacian

// Double-double numbers (hi + lo) from the error-free TwoSum and fma-based
// TwoProd; the alternating Laplacian series below has terms up to ~1e8 times
// its value at the data ranges of interest, so it is summed with ~106 bits.
struct DD {
    double hi, lo;
};
inline DD dd_two_sum(double a, double b) {
    double s = a + b, v = s - a;
    return {s, (a - (s - v)) + (b - v)};
}
inline DD dd_norm(double s, double e) {
    double t = s + e;
    return {t, e - (t - s)};
}
inline DD dd_add(DD a, DD b) {
    DD s = dd_two_sum(a.hi, b.hi), t = dd_two_sum(a.lo, b.lo);
    s.lo += t.hi;
    s = dd_norm(s.hi, s.lo);
    s.lo += t.lo;
    return dd_norm(s.hi, s.lo);
}
inline DD dd_mul(DD a, DD b) {
    double p = a.hi * b.hi;
    double e = std::fma(a.hi, b.hi, -p) + (a.hi * b.lo + a.lo * b.hi);
    return dd_norm(p, e);
}
inline DD dd_scale(DD a, double b) {
    double p = a.hi * b;
    return dd_norm(p, std::fma(a.hi, b, -p) + a.lo * b);
}
inline DD dd_div(DD a, double b) {
    double q = a.hi / b;
    DD r = dd_add(a, dd_scale({-q, 0.0}, b));
    return dd_norm(q, r.hi / b);
}

// k1(x) = sum_{n != 1} b_n x^n, x >= 0 (Table 1 Laplacian series without the
// alpha c_d |x| term) and its first three derivatives, from the term-wise
// derivatives of the series, in double-double.  Returns k1; der[q] receives
// the q-th derivative (q = 0..3) when der != NULL; *err receives a rounding
// bound.  cd must carry c_d to double-double accuracy.
double k1_laplace(double alpha, int d, DD cd, double x, double* der, double* err, bool matern = false) {
    DD ax = dd_mul({alpha, 0.0}, {x, 0.0});
    DD ax2 = dd_mul(ax, ax);
    DD s[4] = {{0, 0}, {0, 0}, {0, 0}, {0, 0}};
    double tmax = 0.0;
    int terms = 0;
    for (int parity = 0; parity < 2; ++parity) {
        DD term = parity == 0 ? DD{1.0, 0.0} : dd_mul(ax, {-cd.hi, -cd.lo});
        int n = parity;
        for (int j = 0; j < 100000; ++j) {
            // the Matern nu = 3/2 series weighs the x^n term by 1 - n (which also drops n = 1)
            const DD tw = matern ? dd_scale(term, 1.0 - n) : term;
            if (n != 1 && x != 0.0) {
                // d^q/dx^q x^n = n (n-1) ... (n-q+1) x^(n-q)
                DD f = tw;
                for (int q = 0; q < 4; ++q) {
                    s[q] = dd_add(s[q], f);
                    f = dd_div(dd_scale(f, static_cast<double>(n - q)), x);
                }
            } else if (n == 0) {
                s[0] = dd_add(s[0], tw);
            }
            tmax = std::max(tmax, std::fabs(tw.hi));
            ++terms;
            double den = (n + 1.0) * (n + 1.0) * (n + 2.0);
            if (ax2.hi * (n + d) < den && n > 1 && std::fabs(tw.hi) < 1e-34 * std::max(tmax, 1e-300)) break;
            term = dd_div(dd_scale(dd_mul(term, ax2), static_cast<double>(n + d)), den);
            n += 2;
            if (term.hi == 0.0) break;
        }
    }
    if (der)
        for (int q = 0; q < 4; ++q) der[q] = s[q].hi + s[q].lo;
    *err = tmax * terms * std::ldexp(1.0, -100) + std::fabs(s[0].hi) * 2.220446049250313e-16;
    return s[0].hi + s[0].lo;
}

// c_d in double-double: c_1 = 1, c_2 = pi/2, c_{d+2} = c_d (d+1)/d
DD cd_dd(int d) {
    DD c = (d % 2) ? DD{1.0, 0.0} : DD{1.5707963267948966, 6.123233995736766e-17};
    for (int k = (d % 2) ? 1 : 2; k + 2 <= d; k += 2) c = dd_div(dd_scale(c, static_cast<double>(k + 1)), k);
    return c;
}

// smooth step: 0 for t <= 0, 1 for t >= 1, C-infinity
double smooth_step(double t) {
    if (t <= 0.0) return 0.0;
    if (t >= 1.0) return 1.0;
    double a = std::exp(-1.0 / t), b = std::exp(-1.0 / (1.0 - t));
    return a / (a + b);
}

void fft_inplace(std::vector<std::complex<double>>& a, int sign) {
    const size_t n = a.size();
    for (size_t i = 1, j = 0; i < n; ++i) {
        size_t bit = n >> 1;
        for (; j & bit; bit >>= 1) j ^= bit;
        j ^= bit;
        if (i < j) std::swap(a[i], a[j]);
    }
    for (size_t len = 2; len <= n; len <<= 1) {
        double ang = sign * 2.0 * PI / static_cast<double>(len);
        for (size_t i = 0; i < n; i += len)
            for (size_t k = 0; k < len / 2; ++k) {
                std::complex<double> wk(std::cos(ang * k), std::sin(ang * k));
                std::complex<double> u = a[i + k], v = a[i + k + len / 2] * wk;
                a[i + k] = u + v;
                a[i + k + len / 2] = u - v;
            }
    }
}

// J_0(x) .. J_nmax(x) for x >= 0 by Miller's backward recurrence
// J_{n-1} = (2n/x) J_n - J_{n+1}, normalised with J_0 + 2 sum_k J_{2k} = 1.
void bessel_j_all(double x, int nmax, std::vector<double>& out) {
    out.assign(nmax + 1, 0.0);
    if (x == 0.0) {
        out[0] = 1.0;
        return;
    }
    int start = std::max(nmax, static_cast<int>(x)) + 40 + static_cast<int>(std::sqrt(40.0 * std::max(nmax, 1)));
    if (start % 2) ++start;
    double jp1 = 0.0, j = 1e-300, norm = 0.0;
    std::vector<double> tmp(start + 1, 0.0);
    for (int n = start; n >= 1; --n) {
        const double jm1 = (2.0 * n / x) * j - jp1;
        jp1 = j;
        j = jm1;
        tmp[n - 1] = j;
        if (std::fabs(j) > 1e250) {  // rescale to stay in range
            for (int q = n - 1; q <= start; ++q) tmp[q] *= 1e-250;
            jp1 *= 1e-250;
            j *= 1e-250;
        }
    }
    tmp[start] = 0.0;
    // recompute the normalisation over the stored values: J_0 + 2 sum J_{2k}
    norm = tmp[0];
    for (int n = 2; n <= start; n += 2) norm += 2.0 * tmp[n];
    for (int n = 0; n <= nmax; ++n) out[n] = tmp[n] / norm;
}

// Chebyshev evaluation of the truncated Fourier sum on [-R, R] (Jacobi-Anger expansion):
// with u = z / R and w_k = 2 pi k R / L,
//   exp(+-i w u) = sum_j eps_j (+-i)^j J_j(w) T_j(u),   eps_0 = 1, eps_j = 2,
// so  t(v) = c_0 w^_0 + 2 Re sum_{k>0} c_k w^_k e^{i w_k v} = sum_l beta_l T_l(v),  beta = M mu,
//   mu_j = sum_n w_n T_j(u_n),
//   M_lj = 2 eps_l eps_j cos(pi (l - j) / 2) sum_{k>0} c_k J_l(w_k) J_j(w_k)  (+ c_0 at l = j = 0).
// Truncating the expansion at q terms changes t by at most 4 sum|w| sum_k c_k tau_k,
// tau_k = 2 sum_{j >= q} |J_j(w_k)|; q is the smallest value keeping that below tol_c.
void choose_chebyshev(FourierHost* fp, double tol_c) {
    const int K = fp->k_hi - fp->k_lo + 1;
    const double wmax = 2.0 * PI * fp->k_hi * fp->R / fp->L;
    const int qcap = 96;
    std::vector<std::vector<double>> J(K);
    for (int i = 0; i < K; ++i) bessel_j_all(2.0 * PI * (fp->k_lo + i) * fp->R / fp->L, qcap + 64, J[i]);
    int q = 0;
    double err = 0.0;
    for (int cand = 4; cand <= qcap; ++cand) {
        double e = 0.0;
        for (int i = 0; i < K; ++i) {
            double tau = 0.0;
            for (int j = cand; j <= qcap + 64; ++j) tau += 2.0 * std::fabs(J[i][j]);
            e += 4.0 * fp->coef[i] * tau;
        }
        if (e <= tol_c) {
            q = cand;
            err = e;
            break;
        }
    }
    (void)wmax;
    if (!q) {
        fp->cheb_q = fp->cheb_qp = 0;
        return;
    }
    int qp = 96;
    for (int b : {8, 10, 12, 16, 24, 32, 48, 64, 96})
        if (q <= b) {
            qp = b;
            break;
        }
    fp->cheb_q = q;
    fp->cheb_qp = qp;
    fp->cheb_err = err;
    fp->cheb_M.assign(static_cast<size_t>(qp) * qp, 0.0);
    for (int l = 0; l < q; ++l)
        for (int j = 0; j < q; ++j) {
            const int e = l - j;
            if (e % 2) continue;
            const double sgn = ((e / 2) % 2) ? -1.0 : 1.0;
            const double el = l ? 2.0 : 1.0, ej = j ? 2.0 : 1.0;
            double acc = 0.0;
            for (int i = 0; i < K; ++i) acc += fp->coef[i] * J[i][l] * J[i][j];
            fp->cheb_M[static_cast<size_t>(l) * qp + j] = 2.0 * el * ej * sgn * acc;
        }
    if (fp->has_k0) fp->cheb_M[0] += fp->coef[K];  // c_0 w^_0, w^_0 = mu_0
}

std::mutex cache_mu;
std::map<std::tuple<int, double, int, double, double, int, int>, FourierHost> cache;

}  // namespace

void add_window_poly_error(FourierHost* fp) {
    if (fp->method != SLK_FOURIER_NFFT) return;
    // the polynomial taps' error enters spreading and interpolation once each, over the m
    // cells of a window
    const double e = 2.0 * fp->m * fp->wpoly_err;
    fp->window_err += e;
    fp->model_err += e;
}

double cd_host(int d) { return std::sqrt(PI) * std::exp(std::lgamma(0.5 * (d + 1)) - std::lgamma(0.5 * d)); }

FourierHost choose_gaussian(double sigma, int d, double R, int n_coeff_req, int method, double tol) {
    const int method_req = method;
    {
        std::lock_guard<std::mutex> g(cache_mu);
        auto it = cache.find({0, sigma, d, R, tol, n_coeff_req, method});
        if (it != cache.end()) return it->second;
    }
    FourierHost fp;
    fp.R = R;
    const double D = 2.0 * R;
    const double tol_p = 0.25 * tol, tol_t = 0.25 * tol;
    // periodisation: smallest L (coarse search) with error <= tol_p
    double gap = 2.0 * sigma * std::sqrt(std::log(1.0 / tol_p));
    double L = D + gap;
    double e = gauss_periodisation(sigma, d, D, L);
    int guard = 0;
    while (e > tol_p && guard++ < 40) {
        gap *= 1.25;
        L = D + gap;
        e = gauss_periodisation(sigma, d, D, L);
    }
    if (e > tol_p) fail(SLK_ERR_ACCURACY, "no period meets the periodisation target %.3g", tol_p);
    // shrink while it still holds
    for (int it = 0; it < 12; ++it) {
        double L2 = D + gap * 0.9;
        double e2 = gauss_periodisation(sigma, d, D, L2);
        if (e2 > tol_p) break;
        gap *= 0.9;
        L = L2;
        e = e2;
    }
    fp.L = L;
    fp.period_err = e;
    // coefficients c_k = fhat(k/L)/L, k >= 0
    auto ck = [&](int k) { return std::exp(log_fhat_gauss(sigma, d, static_cast<double>(k) / L)) / L; };
    double wlo, whi;
    gauss_band(sigma, d, &wlo, &whi);
    const int kcap = static_cast<int>(std::ceil(whi * L)) + 2;
    // truncation to |k| < N_c/2
    int Nc = n_coeff_req;
    if (Nc <= 0) {
        // smallest even N_c whose tail is below tol_t
        double tail = 0.0;
        int k = kcap;
        while (k > 0 && tail + 2.0 * ck(k - 1) <= tol_t) {
            tail += 2.0 * ck(k - 1);
            --k;
        }
        Nc = std::max(16, 2 * k + 2);
    }
    double trunc = 0.0;
    for (int k = Nc / 2; k <= kcap + 8; ++k) trunc += 2.0 * ck(k);
    if (trunc > tol_t)
        fail(SLK_ERR_ACCURACY, "%d Fourier coefficients leave a truncation error %.3g above %.3g (period %.4g)", Nc, trunc,
             tol_t, L);
    fp.n_coeff = Nc;
    fp.trunc_err = trunc;
    // NDFT band: drop coefficients from both ends while the dropped mass stays small
    int klo = 1, khi = Nc / 2 - 1;
    double dropped = 0.0;
    for (;;) {
        double a = klo <= khi ? 2.0 * ck(klo) : INFINITY, b = klo <= khi ? 2.0 * ck(khi) : INFINITY;
        double c = std::min(a, b);
        if (klo > khi || dropped + c > 0.5 * tol_t) break;
        dropped += c;
        if (a <= b) ++klo;
        else --khi;
    }
    fp.has_k0 = ck(0) > 0.0 && ck(0) > 0.5 * tol_t * 1e-3 ? 1 : 0;
    if (d == 1) {
        klo = 1;
        fp.has_k0 = 1;
    }
    fp.k_lo = klo;
    fp.k_hi = std::max(khi, klo);
    fp.ndft_drop = dropped;
    fp.coef.clear();
    for (int k = fp.k_lo; k <= fp.k_hi; ++k) fp.coef.push_back(ck(k));
    fp.coef.push_back(fp.has_k0 ? ck(0) : 0.0);
    // NFFT grid and window
    fp.n_g = next_pow2(2 * Nc);
    choose_window(&fp, 0.25 * tol);
    set_active_window(&fp);
    fp.mult.resize(Nc / 2);
    for (int k = 0; k < Nc / 2; ++k) fp.mult[k] = ck(k) / (fp.psi[k] * fp.psi[k]);
    // method (the NDFT kernels take bands of at most 64 coefficients; the Chebyshev
    // evaluation needs at most 96 terms)
    const int K = fp.k_hi - fp.k_lo + 1;
    if (method == SLK_FOURIER_NDFT && K > 64)
        fail(SLK_ERR_UNSUPPORTED, "the NDFT band has %d coefficients (at most 64); use the NFFT", K);
    if (method == SLK_FOURIER_CHEB || method == SLK_FOURIER_AUTO) choose_chebyshev(&fp, 0.25 * tol);
    if (method == SLK_FOURIER_CHEB && fp.cheb_q == 0)
        fail(SLK_ERR_UNSUPPORTED, "the Chebyshev evaluation would need more than 96 terms; use the NFFT");
    if (method == SLK_FOURIER_AUTO)
        method = fp.cheb_q ? SLK_FOURIER_CHEB : ((K <= 2 * fp.m && K <= 64) ? SLK_FOURIER_NDFT : SLK_FOURIER_NFFT);
    if (method == SLK_FOURIER_NFFT && fp.W > fp.n_g) {
        if (K > 64) fail(SLK_ERR_ACCURACY, "neither the NFFT window nor the NDFT band fits");
        method = SLK_FOURIER_NDFT;
    }
    fp.method = method;
    fp.model_err = fp.period_err + trunc +
                   (method == SLK_FOURIER_NDFT ? dropped : (method == SLK_FOURIER_CHEB ? dropped + fp.cheb_err : fp.window_err));
    {
        std::lock_guard<std::mutex> g(cache_mu);
        cache[{0, sigma, d, R, tol, n_coeff_req, method_req}] = fp;
    }
    return fp;
}

FourierHost choose_laplace_smooth(double alpha, int d, double R, int n_coeff_req, double tol, int max_nc,
                                  bool matern) {
    const int key = matern ? 2 : 1;
    {
        std::lock_guard<std::mutex> g(cache_mu);
        auto it = cache.find({key, alpha, d, R, tol, n_coeff_req, max_nc});
        if (it != cache.end()) return it->second;
    }
    const double D = 2.0 * R;
    const DD cd = cd_dd(d);
    const double tol_t = 0.25 * tol;
    FourierHost best;
    bool have = false;
    for (double rho : {0.25, 0.3, 0.35, 0.4}) {
        FourierHost fp;
        fp.R = R;
        fp.L = D / rho;
        const int nf = 1 << 16;
        std::vector<std::complex<double>> a(nf);
        double emax = 0.0;
        // beyond the data range |u| > rho the function continues as the cubic
        // Taylor polynomial T of k1 at x0 = rho L (C^3 junction), blended by a
        // C-infinity step B to the constant k1(x0) at |u| = 1/2:
        //     phi1 = B T + (1 - B) k1(x0)
        const double x0 = rho * fp.L;
        double t0[4];
        k1_laplace(alpha, d, cd, x0, t0, &emax, matern);
        for (int j = 0; j < nf; ++j) {
            double u = (j < nf / 2 ? j : j - nf) / static_cast<double>(nf);  // in [-1/2, 1/2)
            double au = std::fabs(u), e = 0.0;
            double v;
            if (au <= rho) {
                v = k1_laplace(alpha, d, cd, au * fp.L, nullptr, &e, matern);
            } else {
                double h = (au - rho) * fp.L;
                double T = t0[0] + h * (t0[1] + h * (0.5 * t0[2] + h * t0[3] / 6.0));
                double B = smooth_step((0.5 - au) / (0.5 - rho));
                v = B * T + (1.0 - B) * t0[0];
            }
            emax = std::max(emax, e);
            a[j] = v;
        }
        if (emax > 0.05 * tol) continue;  // series too ill-conditioned at this scale
        fft_inplace(a, -1);
        std::vector<double> c(nf / 2);
        for (int k = 0; k < nf / 2; ++k) c[k] = a[k].real() / nf;
        // smallest power-of-two N_c with tail <= tol_t
        int Nc = n_coeff_req;
        auto tail_of = [&](int nc) {
            double t = 0.0;
            for (int k = nc / 2; k < nf / 2; ++k) t += 2.0 * std::fabs(c[k]);
            return t;
        };
        if (Nc <= 0) {
            Nc = 16;
            while (Nc < max_nc && tail_of(Nc) > tol_t) Nc <<= 1;
        }
        double trunc = tail_of(Nc);
        if (trunc > tol_t) continue;
        fp.n_coeff = Nc;
        fp.trunc_err = trunc + emax;
        fp.period_err = 0.0;  // k1 is reproduced exactly on |u| <= 2R by construction
        fp.n_g = next_pow2(2 * Nc);
        fp.coef.assign(c.begin(), c.begin() + Nc / 2);
        if (!have || fp.n_coeff < best.n_coeff) {
            best = fp;
            have = true;
        }
    }
    if (!have)
        fail(SLK_ERR_ACCURACY, "%s: no grid of at most %d coefficients meets %.3g (alpha*R = %.3g)",
             matern ? "Matern kernel" : "Laplacian smooth part", max_nc, tol_t, alpha * R);
    choose_window(&best, 0.25 * tol);
    set_active_window(&best);
    best.mult.resize(best.n_coeff / 2);
    for (int k = 0; k < best.n_coeff / 2; ++k) best.mult[k] = best.coef[k] / (best.psi[k] * best.psi[k]);
    best.method = SLK_FOURIER_NFFT;
    best.k_lo = 1;
    best.k_hi = 1;
    best.has_k0 = 0;
    best.model_err = best.trunc_err + best.window_err;
    {
        std::lock_guard<std::mutex> g(cache_mu);
        cache[{key, alpha, d, R, tol, n_coeff_req, max_nc}] = best;
    }
    return best;
}

}  // namespace slk
