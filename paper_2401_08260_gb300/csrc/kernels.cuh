// Launchers of the library's kernels (one declaration per kernel family).
#pragma once

#include "common.cuh"

namespace slk {

// ------------------------------------------------------------ k_util.cu
// Draw P directions uniform on S^{d-1} (Algorithm 1, first step): Philox4x32-10
// counter-based generator (Salmon et al. 2011), Box-Muller, row normalisation.
// rows p0 .. p0 + P - 1 of the direction sequence of `seed` (Philox4x32-10, Box-Muller, normalised)
void launch_draw_directions(double* xi, int P, int d, uint64_t seed, int p0, cudaStream_t st);
// Row-normalise a P x d FP64 matrix in place.
void launch_normalize_rows(double* xi, int P, int d, cudaStream_t st);
// mu[k] = mean over up to 4096 evenly strided rows of x (the centre subtracted
// before projecting; exact in exact arithmetic by translation invariance).
template <class T>
void launch_sample_mean(const T* x, int64_t N, int d, int64_t ldx, double* mu, cudaStream_t st);
// dst[i] = (T) src[i].
template <class T>
void launch_convert(const double* src, T* dst, int64_t n, cudaStream_t st);
// *out = max(*out, max |Z[p][i]|) over P rows of n entries (row stride ldz).
template <class T>
void launch_absmax(const T* Z, int P, int64_t n, int64_t ldz, float* out, cudaStream_t st);
// s[i] = (T)(acc[i] * scale).
template <class T>
void launch_finalize(const double* acc, T* s, int64_t n, double scale, cudaStream_t st);


// ------------------------------------------------------------ k_project.cu
// Z[p][i] = sum_k xi[p][k] (x[i][k] - mu[k]),  p < P, i < n  (SIMT, FP32 or FP64).
template <class T>
void launch_project_simt(const T* xi, int P, const T* x, int64_t n, int d, int64_t ldx, const T* mu, T* Z,
                         int64_t ldz, cudaStream_t st);
// gy[i][k] = scale * gs[i] * sum_p G[p * ldG + i] xi[p][k]   (gs may be NULL = ones;
// G slice-major, P rows of M derivatives).
template <class T>
void launch_grad_gemm(const T* G, int64_t ldG, int64_t M, int P, const T* xi, int d, const T* gs, double scale, T* gy,
                      int64_t ldg, cudaStream_t st);

// ------------------------------------------------------------ k_tcgen05.cu
// Row pitch (elements) of the 16-bit operands of the tensor-core projection.
int64_t umma_operand_ld(int d);
// out[i][k] = 16-bit (x[i][k] - mu[k]) (BF16, or FP16 hi plus scaled FP16 lo when split);
// label names the launch in the timing registry; max_blocks > 0 caps the grid.
void launch_center_cast(const float* x, int64_t n, int d, int64_t ldx, const float* mu, void* out, void* out_lo,
                        int split, cudaStream_t st, const char* label = "center_cast", int max_blocks = 0);
// out[s][k] = x[s * N / S][k] (the strided sample of S rows the centre is estimated from).
void launch_gather_rows(const float* x, int64_t N, int d, int64_t ldx, int64_t S, float* out, cudaStream_t st);
// Streaming multiprocessors of the current device.
int device_sm_count();
// Z[p][i] = sum_k xi[p][k] xc[i][k] on tensor cores (tcgen05, TMA), FP32 accumulate;
// *absmax = max(*absmax, max |Z|) when absmax != NULL; timeouts set bits 8/16/32 of *err.
void launch_project_umma(const void* xa, const void* xa_lo, int64_t n, const void* xib, const void* xib_lo, int P,
                         int d, int split, float* Z, int64_t ldz, float* absmax, unsigned* err, cudaStream_t st);

// Fused target side of the Chebyshev evaluation: BF16 tensor-core projection of n
// centred targets (xa) onto the P directions (xib) with, in the epilogue, the
// sum t_p = sum_l coef[p][l] T_l(z/R) (Clenshaw; or sum_l coef[p][l] (z/R)^l by Horner
// when horner) accumulated over the slices of each tile; part receives
// umma_cheb_parts(P) rows of n FP64 partial sums, row stride ldp (no projection is
// stored).  Targets outside [-R, R] set bit 4 of *err.
int64_t umma_cheb_parts(int P);
bool umma_cheb_fits(int P, int q);
void launch_umma_cheb_target(const void* xa, int64_t n, const void* xib, int P, int d, const float* coef, int q,
                             int horner, double R, double* part, int64_t ldp, unsigned* err, cudaStream_t st);
// The same with the FP32 targets y (row stride ldy) read directly: the kernel centres
// them (y - mu) and rounds them to BF16 in shared memory, bit for bit the operand that
// launch_center_cast followed by launch_umma_cheb_target uses.  Needs
// umma_f32_operand_ok(y, ldy).
bool umma_f32_operand_ok(const float* x, int64_t ld);
void launch_umma_cheb_target_f32(const float* y, int64_t ldy, const float* mu, int64_t n, const void* xib, int P, int d,
                                 const float* coef, int q, int horner, double R, double* part, int64_t ldp,
                                 unsigned* err, cudaStream_t st);
// Fused source side of the Chebyshev evaluation (BF16 tensor cores): projections of n
// centred points (xa, BF16) onto the P directions (xib) with the moments
// mu_j = sum_n w_n T_j(z / R), j < q, accumulated in the epilogue (double-float per thread,
// no projection stored); mom receives umma_moments_chunks(P) x P x q FP64 partials
// (mom[(c * P + p) * q + j]), *absmax the largest |z| over the points.  q is 8, 10, 12 or 16.
bool umma_moments_fit(int q);
int64_t umma_moments_chunks(int P);
void launch_umma_moments(const void* xa, int64_t n, const void* xib, int P, int d, const float* w, int q, double R,
                         double* mom, float* absmax, unsigned* err, cudaStream_t st);

// ------------------------------------------------------------ k_pair.cu
// The two fused Chebyshev sides on CTA pairs (tcgen05 cta_group::2, M = 256) reading the
// FP32 points directly (centred and rounded to BF16 in shared memory, the same operand as
// the single-CTA kernels); work items of 256 points x 256 slices, P <= 512.
//   target side: part receives pair_cheb_parts(P) rows of n FP64 partial row sums (row
//                stride ldp);
//   source side: mom receives pair_moments_chunks(P) x P x q FP64 partials, *absmax the
//                largest |z| over the points.
// Both need umma_f32_operand_ok on the points; q is 8, 10, 12 or 16.
bool pair_cheb_fits(int P, int q, int d);
int64_t pair_cheb_parts(int P);
void launch_pair_cheb_target(const float* y, int64_t ldy, const float* mu, int64_t n, const void* xib, int P, int d,
                             const float* coef, int q, int horner, double R, double* part, int64_t ldp, unsigned* err,
                             cudaStream_t st);
int64_t pair_moments_chunks(int P);
void launch_pair_moments(const float* x, int64_t ldx, const float* mu, int64_t n, const void* xib, int P, int d,
                         const float* w, int q, double R, double* mom, float* absmax, unsigned* err, cudaStream_t st);
// The FP16 hi/lo (FP32-accurate) projection of launch_project_umma(split = 1) on CTA pairs:
// 256-point x 256-slice tiles, M = 256 and N = 256 pair MMAs, each CTA loading its own 128
// point rows and 128 direction rows (hi and lo) per K stage; same operands, same promotion of
// every 16-wide K step, same output (Z slice-major with row stride ldz, absmax if not NULL).
void launch_pair_project_x3(const void* xa, const void* xa_lo, int64_t n, const void* xib, const void* xib_lo, int P,
                            int d, float* Z, int64_t ldz, float* absmax, unsigned* err, cudaStream_t st);

// ------------------------------------------------------------ k_rff.cu
// Random Fourier features (Section 4.3, comparison system).  feat: D x (d + 1) FP64 rows
// (v_p, b_p) drawn from the kernel's spectral measure (Gaussian: N(0, param^-2 I); Laplacian:
// multivariate Cauchy of scale param) and U[0, 2 pi) phases, Philox4x32-10 keyed by seed.
void launch_rff_draw(double* feat, int D, int d, int laplacian, double param, uint64_t seed, cudaStream_t st);
// V (D x d) and b (D) in the working precision from feat.
template <class T>
void launch_rff_split(const double* feat, int D, int d, T* V, T* b, cudaStream_t st);
// cs[p] = (C_p, S_p) from the projections Z (D x n, row stride n) of the sources.
template <class T>
void launch_rff_source(const T* Z, int D, int64_t n, const T* w, const T* b, int variant, double2* cs, cudaStream_t st);
// s (m targets) from their projections Z (D x m) and cs.
template <class T>
void launch_rff_target(const T* Z, int D, int64_t m, const T* b, const double2* cs, int variant, T* s, cudaStream_t st);

// s[i] = scale * sum_{r < parts} part[r * n + i] (fixed order).
template <class T>
void launch_sum_parts(const double* part, int parts, int64_t n, double scale, T* s, cudaStream_t st);
// acc[i] = (first ? 0 : acc[i]) + a * t[i] in FP64 (the slice batches of a one-shot sum)
template <class T>
void launch_accumulate_scaled(double* acc, const T* t, double a, int64_t n, bool first, cudaStream_t st);
// dst[c][r] = BF16(src[r][c]) (rows x cols FP32 in; cols x ld16(rows) out, zero padded).
void launch_transpose_bf16(const float* src, int rows, int cols, void* dst, cudaStream_t st);
// The backward product's A operand: g16[m][p] = BF16(G[p * ldG + m]) for the slice-major
// derivatives G (P rows of M), M rows of pitch ld16(P) out, zero padded; tiled through
// shared memory so that both sides are coalesced.
void launch_derivs_bf16(const float* G, int P, int64_t M, int64_t ldG, void* g16, cudaStream_t st);
// Backward product on tensor cores: gy[m][k] = scale * gs[m] * sum_p G[m][p] xi[p][k] with G (M x P)
// and xi^T (d x P) in BF16 (row pitch ld16(P)); gs may be NULL (ones).
void launch_grad_umma(const void* g16, int64_t M, int P, const void* xit16, int d, const float* gs, double scale,
                      float* gy, int64_t ldg, unsigned* err, cudaStream_t st);

// ------------------------------------------------------------ k_fourier.cu
// The NFFT window's taps as polynomials (FP32 plans): a point whose first window cell lies at
// offset s0 = g + 1/2 - m/2 cells (g in [-1/2, 1/2)) gives tap t < m the weight psi(s0 + t),
// a degree-8 polynomial P_t(g).  psi is even, so P_{m-1-t}(g) = P_t(-g): with h = g^2,
// P_t = E_t(h) + g O_t(h) and P_{m-1-t} = E_t(h) - g O_t(h), and likewise for the derivatives
// P_t' = D_t(h) + g Q_t(h), P_{m-1-t}' = g Q_t(h) - D_t(h); stored for t < ceil(m / 2).
// Passed to the kernels by value (uniform operands of their multiply-adds).
constexpr int kWinPolyHalf = (kWinPolyMaxM + 1) / 2;
struct WinPoly {
    float ev[kWinPolyHalf][5];  // E_t: coefficients of h^0 .. h^4
    float od[kWinPolyHalf][4];  // O_t: h^0 .. h^3
    float de[kWinPolyHalf][4];  // D_t: h^0 .. h^3
    float dq[kWinPolyHalf][4];  // Q_t: h^0 .. h^3
};

struct FourierDev {
    // geometry of the periodic 1-D problem (Section 3.1 with the rescaling of
    // the paragraph "Rescaling"): x~ = z / L, period 1 in x~
    double L;
    // NDFT: positive band [k_lo, k_hi] (+ k = 0 if has_k0), coefficients c_k
    int k_lo, k_hi, has_k0;
    // NFFT: grid n_g, window width m (cells), ES shape beta, active window
    // [win_base, win_base + W) in grid cells
    int n_g, m, W, win_base;
    double beta;
    // certified window: every projected target lies in [-R, R]
    double R;
    // Chebyshev evaluation: number of terms (padded); horner = 1 when the monomial
    // coefficients mono (T, P x q) may replace Clenshaw on the target side
    int q;
    int horner;
    const void* mono;
    // NFFT window taps as polynomials (used by the FP32 kernels)
    WinPoly wp;
    // FP32 NFFT plans: the interpolant tabulated per grid cell (launch_interp_table), or NULL
    const void* itab;
};

// FP32 NFFT plans: per slice and grid cell r < W - m + 1, the coefficients of the interpolant
// sum_t h[p][r + t] psi(s0 + t) as a polynomial in g (s0 = g + 1/2 - m/2), 16 floats per cell
// (9 used); launch_nfft_target<float> reads it when fd.itab is set.
int64_t interp_table_floats(int P, const FourierDev& fd);
void launch_interp_table(const float* h, int P, const FourierDev& fd, float* tab, cudaStream_t st);

// Chebyshev evaluation of the truncated Fourier sum (Jacobi-Anger expansion on [-R, R]):
// source side beta[p][l] = sum_j M[l][j] sum_n w_n T_j(z_{p,n}/R) (M is q x q, FP64);
// target side acc[m] += sum_p sum_l beta[p][l] T_l(z_{p,m}/R), or the z-derivative into
// G[m][p]; targets outside [-R, R] set bit 4 of *err.
// With mono != nullptr (q <= 16) the source side also writes the same polynomials in the
// monomial basis, mono[p][k] = sum_l beta[p][l] [u^k] T_l(u) (converted in FP64), and sets
// *mono_bad when for some slice sum_k |mono| > mono_ratio sum_l |beta|.  Only otherwise is
// Horner's rule (one FMA per term, rounding bound gamma_2q sum_k |mono_k|) used on the
// target side.
template <class T>
void launch_cheb_source(const T* Z, int P, int64_t n, int64_t ldz, const T* w, const FourierDev& fd,
                        const double* M, T* beta, T* mono, unsigned* mono_bad, double mono_ratio, T* scratch,
                        int64_t scratch_elems, cudaStream_t st);
int64_t cheb_source_scratch(int P, int64_t n, const FourierDev& fd);
// beta (and the monomial form, as launch_cheb_source) from FP64 moment partials
// partial[(c * P + p) * q + j], c < nchunk, summed in a fixed order.
void launch_cheb_reduce_f64(const double* partial, int nchunk, int P, const FourierDev& fd, const double* M,
                            float* beta, float* mono, unsigned* mono_bad, double mono_ratio, cudaStream_t st);
template <class T>
void launch_cheb_target(const T* Z, int P, int64_t n, int64_t ldz, const FourierDev& fd, const T* beta, double* acc,
                        T* G, int64_t ldg, unsigned* err, cudaStream_t st);

// NDFT, source side: cw[p][j] = c_{k_lo+j} * sum_n w_n exp(-2 pi i k z_{p,n} / L),
// j = 0..K-1 (and cw0[p] = c_0 sum_n w_n if has_k0).  coef holds c_k (FP64).
template <class T>
void launch_ndft_source(const T* Z, int P, int64_t n, int64_t ldz, const T* w, const FourierDev& fd,
                        const double* coef, Cplx<T>* cw, T* cw0, T* scratch, int64_t scratch_elems, cudaStream_t st);
// NDFT, target side: with acc != NULL, acc[m] += sum_p t_p(z_{p,m}); with G != NULL,
// G[p * ldg + m] = dt_p/dz (the per-slice derivatives of the gradient, slice-major); either
// or both.  Targets outside [-R, R] set bit 4 of *err.  The other target launchers
// (Chebyshev, NFFT) take acc and G the same way.
template <class T>
void launch_ndft_target(const T* Z, int P, int64_t n, int64_t ldz, const FourierDev& fd, const Cplx<T>* cw,
                        const T* cw0, double* acc, T* G, int64_t ldg, unsigned* err, cudaStream_t st);
// NFFT, source side: spread w onto the grid window of every slice (partial
// sums per point chunk, then a fixed-order reduction), FFT, multiply by
// mult[k] = c_k / Psi(k/n_g)^2 for |k| < n_coeff/2, inverse FFT; h is P x W.  With
// pairs != NULL the sources are read from the sorting route's (key, w) pairs instead of
// (Z, w): P x n pairs grouped by key bucket (launch_sort_pairs), which the spreading
// exploits to add most window taps in registers.
template <class T>
void launch_nfft_source(const T* Z, int P, int64_t n, int64_t ldz, const T* w, const T* pairs, const FourierDev& fd,
                        int n_coeff, const double* mult, T* h, T* scratch, int64_t scratch_elems, unsigned* err,
                        cudaStream_t st);
// Scratch elements launch_nfft_source needs.
int64_t nfft_source_scratch(int P, int64_t n, const FourierDev& fd);
int64_t ndft_source_scratch(int P, int64_t n, const FourierDev& fd);
// NFFT, target side: acc[m] += sum_p sum_j h[p][j] psi(n_g z/L - j) and / or the
// derivative dt_p/dz into G[p * ldg + m].  Targets outside [-R, R] set bit 4 of *err.
template <class T>
void launch_nfft_target(const T* Z, int P, int64_t n, int64_t ldz, const FourierDev& fd, const T* h, double* acc,
                        T* G, int64_t ldg, unsigned* err, cudaStream_t st);

// ------------------------------------------------------------ k_sort.cu
// Per slice p < P, the n sources ordered by their projection z[p * ldz + i] into (key, w)
// pairs (kw, P x n), w the source weights, by a segmented stable LSD radix sort with 8-bit
// digits carrying the weight as payload.  NB > 0: the digits are those of the equal-width
// bucket index bucket_of(z; kmin[p], kscale[p], NB) (one pass per byte of NB - 1), so the
// pairs come out grouped by bucket in ascending bucket order, in source order within a
// bucket; NB = 0: the digits are the order-preserving bits of z (a full sort).
template <class T>
void launch_sort_pairs(const T* z, int P, int64_t n, int64_t ldz, const T* w, void* kw, void* scratch,
                       size_t scratch_bytes, const float* kmin, const float* kscale, int NB, cudaStream_t st);
// kmin[p] = the smallest of the n projections of slice p, kscale[p] = NB / (largest - smallest)
// (0 if they are all equal): the bucket geometry of the grouping above.
template <class T>
void launch_slice_minmax(const T* Z, int P, int64_t n, int64_t ldz, int NB, float* kmin, float* kscale,
                         cudaStream_t st);
template <class T>
size_t sort_pairs_scratch(int P, int64_t n);
// Bytes of the sorted (key, w) pairs of P segments of n sources, plus kPairPadBytes after
// them (the target lookups read FP32 pairs in aligned 32-byte chunks of four).
constexpr int64_t kPairPadBytes = 32;
template <class T>
int64_t sorted_pairs_bytes(int P, int64_t n);
// From pairs grouped by bucket: one 32-byte record per bucket b <= NB, rec[p][b]: the
// exclusive prefix sums of w and w*key at the bucket's first index (16 bytes: two doubles for
// FP64 data, double-float pairs (hi, lo) for FP32 data), that index and the first index of
// the next bucket (a target's lookup reads one record); rec[p][NB] holds the totals.
// have_geometry: kmin / kscale already hold the buckets the pairs were grouped by;
// otherwise the pairs are fully sorted and the geometry is set from their first and last keys.
constexpr int64_t kBucketRecordBytes = 32;
template <class T>
void launch_bucket_tables(int P, int64_t n, const void* kw, int NB, float* kmin, float* kscale, void* rec,
                          bool have_geometry, cudaStream_t st);
// Negative-distance 1-D sums at the targets (Section 3.2 in the range-free
// form t = -c_d [z (2 A_< - W) - (2 B_< - S)]): with acc != NULL summed over slices into
// acc[m], times `scale`; with G != NULL the derivative g = scale c_d (W - A_< - A_<=)
// (sign(0) = 0) written to G[p * ldg + m] (added to it if accumulate_G); both from one
// lookup per slice-point when both are given.  Slices are processed in batches whose
// pairs and bucket records fit in L2.
template <class T>
void launch_negdist_target(const T* Z, int P, int64_t n, int64_t ldz, const void* kw, int64_t nx, const void* rec,
                           int NB, const float* kmin, const float* kscale, double cd, double scale, double* acc, T* G,
                           int64_t ldg, int accumulate_G, cudaStream_t st);

}  // namespace slk
