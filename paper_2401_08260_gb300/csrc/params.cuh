// Plan-time Fourier parameters (host side).
#pragma once

#include <vector>

#include "common.cuh"

namespace slk {

struct FourierHost {
    int method = 0;          // SLK_FOURIER_NDFT or SLK_FOURIER_NFFT
    double L = 0.0;          // period in projected units
    double R = 0.0;          // certified window half-width
    int n_coeff = 0;         // N_c: coefficients k with |k| < N_c / 2
    int k_lo = 1, k_hi = 1;  // NDFT band (k > 0)
    int has_k0 = 0;
    std::vector<double> coef;  // NDFT: c_{k_lo..k_hi}, then c_0; Laplacian: c_0..c_{N_c/2-1}
    int n_g = 0, m = 0, W = 0, win_base = 0;
    double beta = 0.0;
    // the window's m taps as degree-kWinPolyDeg polynomials in g in [-1/2, 1/2) (see
    // fit_window_poly): wpoly[t * (kWinPolyDeg + 1) + k], and their largest error
    std::vector<double> wpoly;
    double wpoly_err = 0.0;
    std::vector<double> psi;   // Psi(k / n_g), k < N_c / 2
    std::vector<double> mult;  // c_k / Psi(k / n_g)^2, k < N_c / 2
    // Chebyshev evaluation (Jacobi-Anger): q terms, certified error; the device works with
    // qp >= q terms (qp one of 8, 10, 12, 16, 24, 32, 48, 64, 96, so its loops have fixed
    // length), M is qp x qp (row-major) and zero outside the leading q x q block
    int cheb_q = 0, cheb_qp = 0;
    std::vector<double> cheb_M;
    double cheb_err = 0.0;
    double period_err = 0.0, trunc_err = 0.0, window_err = 0.0, ndft_drop = 0.0, model_err = 0.0;
};

double cd_host(int d);
// The FP32 kernels evaluate the NFFT window's taps as polynomials: add their fitted error
// (wpoly_err, over spreading and interpolation) to the certified window and model errors of
// an NFFT choice.  FP64 plans evaluate the window itself and skip this.
void add_window_poly_error(FourierHost* fp);
FourierHost choose_gaussian(double sigma, int d, double R, int n_coeff_req, int method, double tol);
// max_nc: largest N_c whose grid (2 N_c complex values) fits one block's shared memory
// Fourier coefficients of a Laplacian-type counterpart on the window: the Laplacian's
// smooth part k1 = f_lap + alpha c_d |x| (matern = false), or, with matern, the whole
// Matern nu = 3/2 counterpart (its series is the Laplacian one, alpha = sqrt(3) / beta,
// with the x^n term scaled by 1 - n; no |x| term).
FourierHost choose_laplace_smooth(double alpha, int d, double R, int n_coeff_req, double tol, int max_nc,
                                  bool matern = false);

}  // namespace slk
