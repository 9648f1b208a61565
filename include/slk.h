/*
 * slk.h -- C ABI of the sliced fast kernel summation library (GB300, sm_103a).
 *
 * The library computes kernel sums
 *
 *     s_m = sum_{n=1..N} w_n F(|x_n - y_m|),   m = 1..M,   x_n, y_m in R^d,
 *
 * (the problem statement of Section 3 of "Fast Kernel Summation in High
 * Dimensions via Slicing and Fourier Transforms") for the radial kernels
 *
 *     Gaussian            F(r) = exp(-r^2 / (2 sigma^2))      (Table 1, Sec. 2.2)
 *     Laplacian           F(r) = exp(-alpha r)                (Table 1, Sec. 3.3)
 *     negative distance   F(r) = -r                           (Table 1, Sec. 3.2)
 *
 * by slicing (Algorithm 1): project onto P unit directions xi_p, run a 1-D
 * summation of the 1-D counterpart f of Table 1 on every slice, and average:
 *
 *     s_m ~ (1/P) sum_p sum_n w_n f(|<xi_p, x_n - y_m>|).
 *
 * The 1-D summation is a fast Fourier summation (Section 3.1: NDFT, or the NFFT
 * of the remark that follows it: window spreading, FFT, multiplication by the
 * Fourier coefficients, inverse FFT, interpolation) for the Gaussian, the
 * sorting algorithm of Section 3.2 (Algorithm 2) for the negative distance
 * kernel, and both combined (Section 3.3) for the Laplacian.
 *
 * Conventions shared by every call:
 *   - Points are row-major: point i occupies elements [i*ld, i*ld + d) of its
 *     array (ld >= d, in elements).  Directions are row-major P x d, FP64.
 *   - Element type of x, y, w, s and the gradient: double for
 *     SLK_PREC_F64, float for every other precision.
 *   - Pointers may be device pointers (memory of the plan's device, or
 *     managed memory) or host pointers (pageable or pinned).  Host arrays are
 *     staged through device memory inside the call, on the given stream.
 *   - `stream` is a cudaStream_t (NULL = the legacy default stream).  Every
 *     call enqueues its work on that stream and returns without waiting,
 *     except when an output is a host pointer (the call then synchronises the
 *     stream before returning) or when noted.
 *   - Every call returns a status and never aborts or throws.  The detail
 *     of the last failure on the calling thread is in slk_last_error().
 *   - Ownership: the caller owns x, y, w, s and gradients.  A plan owns its
 *     directions, its cached per-slice x-side data and its workspace; it
 *     keeps no pointer to x or w after slk_plan_create returns.
 */
#ifndef SLK_H
#define SLK_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define SLK_VERSION_MAJOR 0
#define SLK_VERSION_MINOR 1

typedef enum {
    SLK_OK = 0,
    SLK_ERR_INVALID = 1,      /* a bad argument or descriptor field */
    SLK_ERR_OOM = 2,          /* device allocation failed or over the memory budget */
    SLK_ERR_CUDA = 3,         /* a CUDA runtime error (kernel launch, copy, ...) */
    SLK_ERR_ACCURACY = 4,     /* the requested accuracy cannot be certified */
    SLK_ERR_TIMEOUT = 5,      /* a bounded wait ran out */
    SLK_ERR_BUSY = 6,         /* no slot or memory free right now; retry later */
    SLK_ERR_UNSUPPORTED = 7,  /* valid request the library does not implement */
    SLK_ERR_NOT_FOUND = 8     /* unknown request id */
} slk_status;

typedef enum {
    SLK_GAUSSIAN = 0,         /* param = sigma > 0 */
    SLK_LAPLACIAN = 1,        /* param = alpha > 0 (F = exp(-alpha r)) */
    SLK_NEGDIST = 2,          /* param ignored */
    SLK_MATERN32 = 3          /* Matern nu = 3/2, param = beta > 0:
                                 F = (1 + sqrt(3) r / beta) exp(-sqrt(3) r / beta) */
} slk_kernel;

typedef enum {
    SLK_PREC_F64 = 0,         /* FP64 storage and arithmetic (SIMT) */
    SLK_PREC_F32 = 1,         /* FP32 storage; FP32 SIMT projection */
    SLK_PREC_BF16 = 2,        /* FP32 storage; BF16 tensor-core projection, FP32 accumulate */
    SLK_PREC_F16X3 = 3        /* FP32 storage; tensor-core projection with FP16 hi/lo split
                                 (three products), about FP32 accuracy */
} slk_precision;

typedef enum {
    SLK_FOURIER_AUTO = 0,     /* the fastest method that meets the target (Chebyshev, NDFT or NFFT) */
    SLK_FOURIER_NFFT = 1,     /* spread + FFT + multiply + inverse FFT + interpolate */
    SLK_FOURIER_NDFT = 2,     /* direct sums over the significant coefficients */
    SLK_FOURIER_CHEB = 3      /* the NDFT's exponentials expanded in Chebyshev polynomials on the
                                 certified window (Jacobi-Anger): moments at the sources, a
                                 Chebyshev series at the targets (Gaussian kernel) */
} slk_fourier_method;

/* Plan descriptor.  Zero-initialise, then set the fields you need. */
typedef struct {
    int32_t kernel;           /* slk_kernel */
    int32_t precision;        /* slk_precision */
    double param;             /* sigma (Gaussian) or alpha (Laplacian) */
    int32_t d;                /* dimension, >= 1 */
    int32_t P;                /* number of slices (directions), >= 1 */
    int32_t n_coeff;          /* Fourier coefficients N_c: k in (-N_c/2, N_c/2); 0 = automatic */
    int32_t method;           /* slk_fourier_method (Gaussian and Laplacian smooth part) */
    uint64_t seed;            /* seed of the library's direction draw (when directions == NULL) */
    const double* directions; /* optional P x d row-major unit directions (host or device);
                                 NULL = draw them (Philox4x32-10 + Box-Muller, normalised) */
    double tol;               /* target model error (truncation + periodisation + window),
                                 relative to sum|w|; 0 = default for the precision */
    double radius;            /* half-width R of the certified window: every projected
                                 target must satisfy |<xi_p, y - mu>| <= R (mu = the plan's
                                 centre); 0 = automatic: 1.25 x the largest projected source,
                                 except on the BF16 Gaussian path with the Chebyshev
                                 evaluation, where the window is fixed before the sources are
                                 projected: 1.5 x the largest projection over the sample of
                                 (at most 4096) sources the centre is estimated from, or the
                                 first rule when a source falls outside that */
    int32_t slice_batch;      /* slk_kernel_sum only: build and run plans of at most slice_batch
                                 slices one after another and combine their sums, so that the
                                 working memory is one batch's plan (Sec. 5.4, remark on
                                 memory and batching); 0 = all at once.  A plan from
                                 slk_plan_create holds every slice and ignores the field. */
    int32_t slice_offset;     /* first slice of the library's draw: the plan draws the rows
                                 slice_offset .. slice_offset + P - 1 of the direction sequence
                                 of `seed`, so that plans over disjoint slice ranges (GPUs of a
                                 sharded sum, batches) together use the same directions as one
                                 plan over all slices; >= 0, slice_offset + P <= 2^31 - 1;
                                 ignored when directions != NULL */
    int32_t reserved[6];
} slk_plan_desc;

/* What a plan chose (filled by slk_plan_get_info). */
typedef struct {
    int32_t kernel, precision, d, P;
    int64_t N;
    int32_t method;           /* slk_fourier_method actually used (0 if none) */
    int32_t n_coeff;          /* N_c */
    int32_t n_grid;           /* NFFT grid size (2 N_c) */
    int32_t window;           /* NFFT window width in grid cells */
    int32_t k_lo, k_hi;       /* NDFT band of significant k > 0 (inclusive) */
    int32_t cheb_terms;       /* Chebyshev terms q (SLK_FOURIER_CHEB) */
    int32_t cheb_horner;      /* 1: targets evaluate the Chebyshev sum by Horner's rule on its
                                 monomial coefficients (chosen only where that rounding bound is
                                 within twice Clenshaw's), 0: Clenshaw's recurrence */
    int32_t sort_buckets;     /* sorting route: equal-width key buckets per slice (NB; 0 if none) */
    double period;            /* L: period of the Fourier summation in projected units */
    double radius;            /* certified window half-width R */
    double model_error;       /* certified bound: truncation + periodisation + window (per unit sum|w|) */
    double c_d;               /* sqrt(pi) Gamma((d+1)/2) / Gamma(d/2) */
    int64_t device_bytes;     /* device memory held by the plan */
} slk_plan_info;

typedef struct slk_plan_s* slk_plan;

/* Library version and the status text (static strings). */
int32_t slk_version(void);
const char* slk_status_string(slk_status status);
/* Detail of the last failure on this thread ("" if none); valid until the next call. */
const char* slk_last_error(void);

/*
 * Build a plan: draw or copy the directions, project the sources x (N x d,
 * row stride ldx) onto them and precompute the x-side of every slice
 * (Algorithm 1, first step, and the source half of the 1-D method:
 * Fourier coefficients w_hat or Chebyshev moments (Sec. 3.1), or the sorted
 * (key, w) pairs with per-bucket prefix sums of w and w * key (Sec. 3.2),
 * kept exact as double-float values with FP64 totals per chunk and bucket).
 * w holds N weights.  N >= 1.
 * Errors: SLK_ERR_INVALID (bad descriptor, N < 1, ldx < d), SLK_ERR_OOM,
 * SLK_ERR_ACCURACY (no Fourier parameters meet desc->tol), SLK_ERR_CUDA.
 */
slk_status slk_plan_create(slk_plan* plan, const slk_plan_desc* desc, const void* x, int64_t N, int64_t ldx,
                           const void* w, void* stream);

/*
 * Kernel sums at M targets y (M x d, row stride ldy) into s (M values):
 * project the targets, evaluate every slice's 1-D sum and average (Algorithm 1).
 * M == 0 is a no-op.  Errors: SLK_ERR_INVALID, SLK_ERR_ACCURACY (a projected
 * target lies outside the certified window), SLK_ERR_OOM, SLK_ERR_CUDA.
 */
slk_status slk_sum(slk_plan plan, const void* y, int64_t M, int64_t ldy, void* s, void* stream);

/*
 * Gradient of sum_m gs_m s_m with respect to the targets: for every m,
 *     gy_m = gs_m (1/P) sum_p xi_p  sum_n w_n f'(|d|) sign(d),  d = <xi_p, y_m - x_n>,
 * with sign(0) = 0 (the derivative of the sliced estimator).  gs may be NULL
 * (all ones).  gy is M x d with row stride ldg.  Errors as slk_sum.
 */
slk_status slk_grad(slk_plan plan, const void* y, int64_t M, int64_t ldy, const void* gs, void* gy, int64_t ldg,
                    void* stream);

/*
 * Sums and per-slice derivatives in one pass: s as slk_sum, and, from the same
 * projection of the targets and the same evaluation of every slice's 1-D sum,
 *     g[p * ldd + m] = t_p'(z),  z = <xi_p, y_m - mu>,
 * the derivative of slice p's 1-D sum at target m (Section 3.2's sorting sums:
 * c_d (W - A_<(z) - A_<=(z)) with sign(0) = 0; Sections 3.1 and 3.3: the derivative
 * of the evaluated Fourier or Chebyshev sum; the Laplacian adds both), in the units
 * of s, so that the gradient of sum_m gs_m s_m is gs_m (1/P) sum_p g[p][m] xi_p
 * (slk_grad_derivs).  This is the forward pass of a training step: the backward pass
 * then needs neither the targets nor a second evaluation.
 * g: P rows of M values, row stride ldd >= M (slice-major), float for F32 / BF16 /
 * F16X3 plans and double for F64, caller-owned device or host memory; M < 2^31.
 * Errors as slk_sum.
 */
slk_status slk_sum_derivs(slk_plan plan, const void* y, int64_t M, int64_t ldy, void* s, void* g, int64_t ldd,
                          void* stream);

/*
 * Gradient from saved derivatives: gy_m = gs_m (1/P) sum_p g[p * ldd + m] xi_p for the
 * g that slk_sum_derivs wrote (the backward product of slk_grad without projecting or
 * evaluating the targets again).  gs may be NULL (all ones); gy is M x d with row stride
 * ldgy.  Errors: SLK_ERR_INVALID, SLK_ERR_OOM, SLK_ERR_CUDA.
 */
slk_status slk_grad_derivs(slk_plan plan, const void* g, int64_t M, int64_t ldd, const void* gs, void* gy,
                           int64_t ldgy, void* stream);

/*
 * Projections of n points onto the plan's directions (Algorithm 1, the inner
 * products <xi_p, x_i>), centred by the plan's centre mu:
 *     Z[p * ldz + i] = <xi_p, x_i - mu>,   p < P, i < n,
 * computed on the plan's projection path (SIMT FP64/FP32, or tensor cores for
 * SLK_PREC_BF16 / SLK_PREC_F16X3).  x is n x d (row stride ldx); Z holds
 * P x ldz elements of the plan's element type (ldz >= n).  Host or device.
 */
slk_status slk_plan_project(slk_plan plan, const void* x, int64_t n, int64_t ldx, void* Z, int64_t ldz, void* stream);

/* The plan's centre mu (d values, FP64) into host memory. */
slk_status slk_plan_get_center(slk_plan plan, double* mu_host);

/*
 * Wait for the plan's outstanding work and return the device-side status of
 * its last call: SLK_ERR_ACCURACY when a projected target fell outside the
 * certified window [-R, R] of a Fourier plan (sums with device outputs are
 * asynchronous, so this status is otherwise reported by the next call).
 */
slk_status slk_plan_sync(slk_plan plan);

/* Copy the plan's directions (P x d row-major FP64) to host memory xi_host. */
slk_status slk_plan_get_directions(slk_plan plan, double* xi_host);

/* Report the parameters the plan chose.  Synchronises the plan's stream. */
slk_status slk_plan_get_info(slk_plan plan, slk_plan_info* info);

/* Release the plan.  Does not wait: its device memory is freed in stream order
 * after the plan's last call (on that call's stream), so the caller must not
 * use the plan's results on another stream without ordering that stream after
 * it.  A device-side status of the last call that was not yet collected (by
 * slk_plan_sync or a later call) is dropped. */
slk_status slk_plan_destroy(slk_plan plan);

/*
 * Host-only: the Fourier parameters a plan with this descriptor would choose
 * when every projected point lies in [-radius, radius] (radius > 0).  Fills the
 * Fourier fields of *info (method, n_coeff, n_grid, window, k_lo, k_hi, period,
 * radius, model_error, c_d).  Needs no GPU.  Errors: SLK_ERR_INVALID,
 * SLK_ERR_ACCURACY, SLK_ERR_UNSUPPORTED (negative distance: no Fourier part).
 */
slk_status slk_fourier_params(const slk_plan_desc* desc, double radius, slk_plan_info* info);

/*
 * One-shot convenience: plan, sum and destroy in one call (same arguments and
 * errors as the three calls).  With 0 < desc->slice_batch < desc->P the P
 * slices are processed in batches of at most slice_batch (Sec. 5.4, remark on
 * memory and batching): batch b covers the slices [p0, p0 + P_b) of the draw
 * (slice_offset + p0 onwards) or the rows p0 .. p0 + P_b - 1 of
 * desc->directions, is planned and summed on its own, and the result is
 * s = sum_b (P_b / P) s_b, accumulated in FP64 on the device; the device
 * memory held at once is one batch's plan plus 12 M bytes (20 M for FP64).
 * Each batch chooses its own window and Fourier parameters from its slices.
 */
slk_status slk_kernel_sum(const slk_plan_desc* desc, const void* x, int64_t N, int64_t ldx, const void* w,
                          const void* y, int64_t M, int64_t ldy, void* s, void* stream);

/*
 * Kernel sums like slk_sum, without allocating device memory (the paper has no
 * counterpart; this is a service of this library).
 *
 * For callers that must not allocate device memory on the call path: for
 * example a serving loop that has reserved the GPU's memory for its own pool
 * up front, or code running where the CUDA allocator may not be called.
 * slk_sum allocates its working buffers (projections of the targets and an
 * FP64 accumulator) from the stream-ordered pool; this variant instead uses
 * one fixed 64 MiB array in device memory that the library reserves on every
 * GPU that loads it (held until the process exits).
 *
 *  - y (M x d, row stride ldy) and s (M values) must be device pointers.
 *  - Working memory per call: align256(P*M*e) + align256(8*M), plus, for the
 *    tensor-core precisions, align256(2*M*ld16) (twice for SLK_PREC_F16X3),
 *    e = 8 for SLK_PREC_F64 and 4 otherwise, ld16 = d rounded up to a multiple
 *    of 8; calls needing more than 64 MiB return SLK_ERR_INVALID (split the
 *    targets).
 *  - The first call on a device looks up the array's device address (once
 *    per device, cached); make that first call before any stream capture.
 *  - Every call uses the same array, which keeps the last call's contents
 *    (the accumulator is cleared at the start of each call).  Calls whose work
 *    overlaps on the GPU (other streams, other threads, several plans on the
 *    same device) race on the array: order them on one stream or synchronise.
 *  - Results agree with slk_sum's to rounding: the same projections and 1-D
 *    method, run as separate projection and target kernels (on the BF16
 *    Chebyshev path slk_sum evaluates inside the projection kernel instead,
 *    summing in another order); errors as slk_sum, plus SLK_ERR_INVALID for
 *    host pointers or sizes beyond the array.
 */
slk_status slk_sum_noalloc(slk_plan plan, const void* y, int64_t M, int64_t ldy, void* s, void* stream);

/*
 * Random Fourier features (Section 4.3): the comparison system of the paper's Table 2,
 * for shift-invariant positive definite kernels with K(x, y) = E_{v ~ mu} cos<x - y, v>
 * (Bochner's theorem).  D samples v_p of the spectral measure mu -- Gaussian
 * F = exp(-r^2 / (2 sigma^2)): mu = N(0, sigma^-2 I); Laplacian F = exp(-alpha r): the
 * multivariate Cauchy law of scale alpha, sampled as alpha g / |h| with g ~ N(0, I_d),
 * h ~ N(0, 1) -- and phases b_p ~ U[0, 2 pi) give
 *   variant 1 (RFF-1): s_m = (2 / D) sum_p cos(<y_m, v_p> + b_p) sum_n w_n cos(<x_n, v_p> + b_p)
 *   variant 2 (RFF-2): s_m = (1 / D) sum_p [cos<y_m, v_p> C_p + sin<y_m, v_p> S_p],
 *                      C_p = sum_n w_n cos<x_n, v_p>,  S_p = sum_n w_n sin<x_n, v_p>
 * (the paper prints the sums over p without the 1 / D of the sample average).
 */
typedef struct {
    int32_t kernel;           /* SLK_GAUSSIAN (param = sigma) or SLK_LAPLACIAN (param = alpha) */
    int32_t precision;        /* SLK_PREC_F64 or SLK_PREC_F32 (storage and arithmetic) */
    double param;
    int32_t d;                /* dimension >= 1 */
    int32_t D;                /* number of features, 1 .. 65535 */
    int32_t variant;          /* 1 (RFF-1) or 2 (RFF-2) */
    int32_t reserved0;
    uint64_t seed;            /* seed of the library's feature draw (when features == NULL) */
    const double* features;   /* optional D x (d + 1) row-major FP64 rows (v_p, b_p), host or
                                 device; NULL = draw them (Philox4x32-10 keyed by seed) */
    int32_t reserved[4];
} slk_rff_desc;

/*
 * s[m] (M values, host or device, the precision's type) = the RFF estimate of the kernel
 * sums of the N sources x (row stride ldx, weights w) at the M targets y (row stride ldy);
 * inputs host or device.  Synchronous on stream when any pointer is on the host.
 * Errors: SLK_ERR_INVALID (kernel not Gaussian or Laplacian, precision not F64/F32,
 * D or d out of range, NULL pointers, N < 1, strides below d), SLK_ERR_OOM, SLK_ERR_CUDA.
 */
slk_status slk_rff_sum(const slk_rff_desc* desc, const void* x, int64_t N, int64_t ldx, const void* w,
                       const void* y, int64_t M, int64_t ldy, void* s, void* stream);
/* The features the library draws for desc (seed, kernel, param, d, D) into the host array
 * features (D x (d + 1) doubles: v_p then b_p per row). */
slk_status slk_rff_features(const slk_rff_desc* desc, double* features);

/*
 * Profiling support (not part of the paper's method).  Every kernel launch of
 * the library is counted; while timing is enabled, each launch is also
 * bracketed by CUDA events recorded on the stream it is launched on.
 *   slk_launch_count   kernels launched by this process so far.
 *   slk_device_alloc_count  device allocations the library has made in this
 *                      process so far (stream-ordered allocations of plans,
 *                      workspaces and staging buffers).
 *   slk_timing_enable  on != 0 starts recording events for later launches.
 *   slk_timing_read    waits for the recorded events and writes, per kernel
 *                      name in first-launch order, the launch count and the
 *                      summed device time in milliseconds into out[0..cap);
 *                      *count receives the number of names (may exceed cap).
 *   slk_timing_reset   drops the recorded events.
 */
typedef struct {
    char name[48];
    int64_t launches;
    double total_ms;
} slk_kernel_time;

int64_t slk_launch_count(void);
int64_t slk_device_alloc_count(void);
slk_status slk_timing_enable(int32_t on);
slk_status slk_timing_read(slk_kernel_time* out, int32_t cap, int32_t* count);
slk_status slk_timing_reset(void);

#ifdef __cplusplus
}
#endif

#endif /* SLK_H */
