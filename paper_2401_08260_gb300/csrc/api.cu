// C ABI: plans, sums and gradients (Algorithm 1 with the 1-D methods of Section 3).
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdarg>
#include <cstring>
#include <memory>
#include <mutex>
#include <string>
#include <vector>

#include "kernels.cuh"
#include "params.cuh"

// ------------------------------------------------------------ errors / memory

namespace slk {

static thread_local std::string g_last_error;

void set_last_error(const std::string& msg) { g_last_error = msg; }

void fail(slk_status st, const char* fmt, ...) {
    char buf[1024];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    throw Error{st, std::string(buf)};
}

std::atomic<int64_t> g_dev_allocs{0};

void* dev_alloc(size_t bytes, cudaStream_t st) {
    g_dev_allocs.fetch_add(1, std::memory_order_relaxed);
    void* p = nullptr;
    cudaError_t e = cudaMallocAsync(&p, bytes, st);
    if (e != cudaSuccess) {
        cudaGetLastError();
        fail(SLK_ERR_OOM, "device allocation of %zu bytes failed: %s", bytes, cudaGetErrorString(e));
    }
    return p;
}

void dev_free(void* p, cudaStream_t st) {
    if (p) cudaFreeAsync(p, st);
}

bool is_device_pointer(const void* p) {
    if (!p) return false;
    cudaPointerAttributes a;
    cudaError_t e = cudaPointerGetAttributes(&a, p);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// Keep freed blocks in the device's default pool so that repeated plans and
// calls reuse memory instead of returning it to the driver.
static void configure_pool(int device) {
    static bool done[64] = {};
    if (device < 0 || device >= 64 || done[device]) return;
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, device) == cudaSuccess) {
        uint64_t thr = UINT64_MAX;
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
    }
    cudaGetLastError();
    done[device] = true;
}

}  // namespace slk

using namespace slk;

// ------------------------------------------------------------ plan object

// Pinned host words that receive the plans' deferred device status.  They are handed out
// from blocks of 256 (never returned to the driver) and come back through a host callback
// queued on the plan's last stream, so a word is reused only after the last copy into it
// has landed; creating and destroying a plan thus neither allocates nor frees pinned
// memory, which would synchronise the device.
struct PinnedWords {
    std::mutex mu;
    std::vector<unsigned*> free;
    unsigned* get() {
        std::lock_guard<std::mutex> g(mu);
        if (free.empty()) {
            unsigned* blk = nullptr;
            SLK_CHECK_CUDA(cudaHostAlloc(reinterpret_cast<void**>(&blk), 256 * sizeof(unsigned), cudaHostAllocPortable));
            for (int i = 0; i < 256; ++i) free.push_back(blk + i);
        }
        unsigned* p = free.back();
        free.pop_back();
        return p;
    }
    void put(unsigned* p) {
        std::lock_guard<std::mutex> g(mu);
        free.push_back(p);
    }
};
PinnedWords& pinned_words() {
    static PinnedWords* w = new PinnedWords();  // outlives every plan (host callbacks may run late)
    return *w;
}
void CUDART_CB return_pinned_word(void* p) { pinned_words().put(static_cast<unsigned*>(p)); }

struct slk_plan_s {
    slk_plan_desc desc{};
    int device = 0;
    bool f64 = false;
    int64_t N = 0;
    int d = 0, P = 0;
    double cd = 0.0;
    double R = 0.0;
    cudaStream_t stream = nullptr;  // stream of the last call (frees are ordered on it)

    DevBuf<double> xi64;  // P x d
    DevBuf<float> xi32;   // P x d (FP32 storage paths)
    DevBuf<double> mu64;  // d
    DevBuf<float> mu32;   // d
    // tensor-core projection (BF16, or FP16 hi/lo split): 16-bit directions P x ldo
    int tc = 0;  // 0 SIMT, 1 BF16, 2 FP16 x3
    DevBuf<unsigned char> xib, xib_lo;
    DevBuf<unsigned char> xit16;  // xi^T in BF16 (d x ld16(P)) for the tensor-core backward product

    // Fourier side (Gaussian, Laplacian smooth part)
    bool fourier = false;
    FourierHost fh;
    FourierDev fd{};
    DevBuf<double> coef, mult, chebM;
    DevBuf<unsigned char> beta;  // T P x q (Chebyshev)
    DevBuf<unsigned char> mono;  // T P x q (the same polynomials in powers of z / R)
    DevBuf<unsigned char> cw;   // Cplx<T> P x K
    DevBuf<unsigned char> cw0;  // T P
    DevBuf<unsigned char> hgrid;  // T P x W (FP32: then the interpolant per grid cell, launch_interp_table)

    // sorting side (negative distance, Laplacian non-smooth part)
    bool sorting = false;
    double sort_scale = 1.0;
    DevBuf<unsigned char> kw;  // sorted (key, w) pairs, P x N
    DevBuf<unsigned char> rec;  // bucket records (prefix sums of w and w*key, pair range), P x (NB + 1) x 32 B
    DevBuf<float> kmin, kscale;
    int NB = 0;

    // deferred device-side status
    DevBuf<unsigned> err_dev;
    unsigned* err_host = nullptr;
    cudaEvent_t done = nullptr;
    bool pending = false;

    // Releases in stream order after the last call (stream): every device buffer is freed
    // on that stream, the event is destroyed (its resources go once it completes) and the
    // status word returns to the pool through a host callback on the same stream.
    ~slk_plan_s() {
        for (DevBuf<double>* b : {&xi64, &mu64, &coef, &mult, &chebM}) b->stream = stream;
        for (DevBuf<float>* b : {&xi32, &mu32, &kmin, &kscale}) b->stream = stream;
        for (DevBuf<unsigned char>* b : {&xib, &xib_lo, &xit16, &beta, &mono, &cw, &cw0, &hgrid, &kw, &rec})
            b->stream = stream;
        err_dev.stream = stream;
        if (done) cudaEventDestroy(done);
        if (err_host && cudaLaunchHostFunc(stream, return_pinned_word, err_host) != cudaSuccess)
            cudaGetLastError();  // the word is then not reused
    }
    int64_t device_bytes() const {
        return static_cast<int64_t>(xi64.bytes() + xi32.bytes() + mu64.bytes() + mu32.bytes() + xib.bytes() +
                                    xib_lo.bytes() + xit16.bytes() + coef.bytes() +
                                    mult.bytes() + chebM.bytes() + beta.bytes() + mono.bytes() + cw.bytes() + cw0.bytes() + hgrid.bytes() + kw.bytes() +
                                    rec.bytes() + kmin.bytes() + kscale.bytes());
    }
};

namespace {

// Coefficients for the NFFT kernels: the Laplacian's smooth part (alpha = param) or the
// Matern nu = 3/2 counterpart (a = sqrt(3) / beta, beta = param).
FourierHost fourier_smooth(const slk_plan_desc& desc, int d, double R, double tol) {
    const int max_nc = desc.precision == SLK_PREC_F64 ? 4096 : 8192;
    if (desc.kernel == SLK_MATERN32)
        return choose_laplace_smooth(std::sqrt(3.0) / desc.param, d, R, desc.n_coeff, tol, max_nc, true);
    return choose_laplace_smooth(desc.param, d, R, desc.n_coeff, tol, max_nc);
}

// Default model-error target per precision, well below the accuracy bar of the
// arithmetic (FP64 1e-12 for the Gaussian).  The Laplacian's smooth part has
// coefficients decaying only like k^-4 (its |x|^3 term at 0), so it asks for
// 1e-7 (FP64) and 2e-6 (FP32) to keep the grid at a few thousand coefficients; so does the
// Matern nu = 3/2 counterpart (also an |x|^3 term).
double default_tol(int kernel, int precision) {
    if (kernel == SLK_LAPLACIAN || kernel == SLK_MATERN32) return precision == SLK_PREC_F64 ? 1e-7 : 2e-6;
    if (precision == SLK_PREC_F64) return 1e-12;
    if (precision == SLK_PREC_BF16) return 1e-5;
    return 2e-7;
}

template <class Fn>
slk_status guarded(Fn&& fn) {
    try {
        fn();
        return SLK_OK;
    } catch (const Error& e) {
        set_last_error(e.msg);
        return e.status;
    } catch (const std::bad_alloc&) {
        set_last_error("host allocation failed");
        return SLK_ERR_OOM;
    } catch (...) {
        set_last_error("unexpected exception");
        return SLK_ERR_CUDA;
    }
}

// Device-side status of the previous call on the plan (non-blocking unless wait).
slk_status collect(slk_plan plan, bool wait) {
    if (!plan->pending) return SLK_OK;
    if (!wait) {
        cudaError_t q = cudaEventQuery(plan->done);
        if (q == cudaErrorNotReady) {
            cudaGetLastError();
            return SLK_OK;
        }
    } else {
        SLK_CHECK_CUDA(cudaEventSynchronize(plan->done));
    }
    plan->pending = false;
    unsigned e = *plan->err_host;
    *plan->err_host = 0;
    if (e & 4u) {
        set_last_error("a projected target lies outside the certified window [-R, R]; rebuild the plan with a larger radius");
        return SLK_ERR_ACCURACY;
    }
    if (e & 3u) {
        set_last_error("a projected point fell outside the NFFT grid window");
        return SLK_ERR_ACCURACY;
    }
    if (e & 56u) {
        set_last_error("a bounded wait in the tensor-core projection ran out");
        return SLK_ERR_TIMEOUT;
    }
    return SLK_OK;
}

void finish_call(slk_plan plan, cudaStream_t st) {
    SLK_CHECK_CUDA(cudaMemcpyAsync(plan->err_host, plan->err_dev.get(), sizeof(unsigned), cudaMemcpyDeviceToHost, st));
    SLK_CHECK_CUDA(cudaMemsetAsync(plan->err_dev.get(), 0, sizeof(unsigned), st));
    SLK_CHECK_CUDA(cudaEventRecord(plan->done, st));
    plan->pending = true;
}

// Device view of a user array of n rows x d columns (row stride ld): either the
// user's pointer or a compact staged copy.
template <class T>
struct InView {
    const T* ptr = nullptr;
    int64_t ld = 0;
    DevBuf<T> staged;
    InView(const void* user, int64_t n, int d, int64_t ld_user, cudaStream_t st) {
        if (is_device_pointer(user) || n == 0) {
            ptr = static_cast<const T*>(user);
            ld = ld_user;
        } else {
            staged.alloc(static_cast<size_t>(n) * d, st);
            // contiguous rows: one linear copy (a pitched copy of n rows runs far below the
            // link's bandwidth)
            if (ld_user == d)
                SLK_CHECK_CUDA(cudaMemcpyAsync(staged.get(), user, sizeof(T) * static_cast<size_t>(n) * d,
                                               cudaMemcpyHostToDevice, st));
            else
                SLK_CHECK_CUDA(cudaMemcpy2DAsync(staged.get(), sizeof(T) * d, user, sizeof(T) * ld_user,
                                                 sizeof(T) * d, n, cudaMemcpyHostToDevice, st));
            ptr = staged.get();
            ld = d;
        }
    }
};

template <class T>
const T* xi_of(slk_plan plan) {
    if constexpr (sizeof(T) == 8) return plan->xi64.get();
    else return plan->xi32.get();
}
template <class T>
const T* mu_of(slk_plan plan) {
    if constexpr (sizeof(T) == 8) return plan->mu64.get();
    else return plan->mu32.get();
}

// Centre and cast n FP32 points to the 16-bit tensor-core operand in one pass, then run
// tc_kernel(xa, xa_lo, row0 = 0, n, st) on it.  (Running the two in L2-sized chunks was
// measured slower: the shorter launches lose more than the L2 reuse of the copy gains.)
template <class F>
void cast_and_run(slk_plan plan, const float* x, int64_t n, int64_t ldx, cudaStream_t st, F&& tc_kernel) {
    const int split = plan->tc == 2;
    const size_t bytes = static_cast<size_t>(n) * umma_operand_ld(plan->d) * 2;
    DevBuf<unsigned char> xa(bytes, st), xl(split ? bytes : 0, st);
    launch_center_cast(x, n, plan->d, ldx, plan->mu32.get(), xa.get(), xl.get(), split, st);
    tc_kernel(static_cast<const void*>(xa.get()), static_cast<const void*>(xl.get()), int64_t(0), n, st);
}

// Z (P x n, ldz = n) = projections of n points onto the plan's directions, centred;
// *absmax = max |Z| when absmax != NULL.
template <class T>
void project(slk_plan plan, const T* x, int64_t n, int64_t ldx, T* Z, float* absmax, cudaStream_t st) {
    if constexpr (sizeof(T) == 4) {
        if (plan->tc) {
            cast_and_run(plan, x, n, ldx, st,
                         [&](const void* xa, const void* xl, int64_t r0, int64_t rows, cudaStream_t s) {
                             launch_project_umma(xa, xl, rows, plan->xib.get(), plan->xib_lo.get(), plan->P, plan->d,
                                                 plan->tc == 2, Z + r0, n, absmax, plan->err_dev.get(), s);
                         });
            return;
        }
    }
    launch_project_simt<T>(xi_of<T>(plan), plan->P, x, n, plan->d, ldx, mu_of<T>(plan), Z, n, st);
    if (absmax) launch_absmax<T>(Z, plan->P, n, n, absmax, st);
}

// Device copy of the chosen Fourier parameters (plan->fh, plan->R) and the tables the
// source side needs.
template <class T>
void fourier_setup(slk_plan plan, cudaStream_t st) {
    const int P = plan->P;
    FourierHost& fh = plan->fh;
    FourierDev& fd = plan->fd;
    fd.L = fh.L;
    fd.k_lo = fh.k_lo;
    fd.k_hi = fh.k_hi;
    fd.has_k0 = fh.has_k0;
    fd.n_g = fh.n_g;
    fd.m = fh.m;
    fd.W = fh.W;
    fd.win_base = fh.win_base;
    fd.beta = fh.beta;
    std::memset(&fd.wp, 0, sizeof(fd.wp));
    static_assert(kWinPolyDeg == 8, "the even/odd tap polynomials have degree 8");
    if (fh.m > 0 && fh.m <= kWinPolyMaxM && fh.wpoly.size() == static_cast<size_t>(fh.m) * (kWinPolyDeg + 1)) {
        for (int t = 0; t < (fh.m + 1) / 2; ++t) {
            const double* a = fh.wpoly.data() + static_cast<size_t>(t) * (kWinPolyDeg + 1);
            for (int j = 0; j <= 4; ++j) fd.wp.ev[t][j] = static_cast<float>(a[2 * j]);
            for (int j = 0; j <= 3; ++j) {
                fd.wp.od[t][j] = static_cast<float>(a[2 * j + 1]);
                fd.wp.de[t][j] = static_cast<float>((2 * j + 1) * a[2 * j + 1]);
                fd.wp.dq[t][j] = static_cast<float>((2 * j + 2) * a[2 * j + 2]);
            }
        }
    }
    fd.R = plan->R;
    fd.q = fh.cheb_qp;
    fd.horner = 0;
    fd.mono = nullptr;
    fd.itab = nullptr;
    if (fh.method == SLK_FOURIER_CHEB) {
        plan->chebM.alloc(fh.cheb_M.size(), st);
        SLK_CHECK_CUDA(cudaMemcpyAsync(plan->chebM.get(), fh.cheb_M.data(), sizeof(double) * fh.cheb_M.size(),
                                       cudaMemcpyHostToDevice, st));
        plan->beta.alloc(sizeof(T) * P * fh.cheb_qp, st);
        if (fh.cheb_qp <= 16) plan->mono.alloc(sizeof(T) * P * fh.cheb_qp, st);
    } else if (fh.method == SLK_FOURIER_NDFT) {
        const int K = fh.k_hi - fh.k_lo + 1;
        plan->coef.alloc(fh.coef.size(), st);
        SLK_CHECK_CUDA(cudaMemcpyAsync(plan->coef.get(), fh.coef.data(), sizeof(double) * fh.coef.size(),
                                       cudaMemcpyHostToDevice, st));
        plan->cw.alloc(sizeof(Cplx<T>) * P * K, st);
        plan->cw0.alloc(sizeof(T) * P, st);
    } else {
        plan->mult.alloc(fh.mult.size(), st);
        SLK_CHECK_CUDA(cudaMemcpyAsync(plan->mult.get(), fh.mult.data(), sizeof(double) * fh.mult.size(),
                                       cudaMemcpyHostToDevice, st));
        // FP32: the interpolant table follows the grid window in the same buffer (64-byte aligned)
        const size_t grid_bytes = (sizeof(T) * P * fh.W + 63) & ~size_t(63);
        plan->hgrid.alloc(grid_bytes + (sizeof(T) == 4 ? sizeof(float) * interp_table_floats(P, fd) : 0), st);
    }
}

// Horner's rounding bound gamma_2q sum|a| against Clenshaw's scale sum|beta|: at most twice it
// for FP32 / FP64 evaluation; for BF16 projections (whose input rounding, 2^-9 of each
// coordinate, dominates) up to 8x, i.e. below 2^-16 sum|beta| for q <= 16.
double mono_ratio_of(slk_plan plan) { return plan->tc == 1 ? 8.0 : 2.0; }

// Reads the Horner check of the Chebyshev source side; also waits for the table uploads.
void cheb_finish(slk_plan plan, const unsigned* bad_dev, cudaStream_t st) {
    unsigned bad_host = 1;
    SLK_CHECK_CUDA(cudaMemcpyAsync(&bad_host, bad_dev, sizeof(unsigned), cudaMemcpyDeviceToHost, st));
    SLK_CHECK_CUDA(cudaStreamSynchronize(st));
    plan->fd.horner = plan->fh.cheb_qp <= 16 && bad_host == 0;
    plan->fd.mono = plan->fd.horner ? plan->mono.get() : nullptr;
}

template <class T>
void plan_fourier_source(slk_plan plan, const T* Zx, const T* w, cudaStream_t st) {
    const int P = plan->P;
    const int64_t N = plan->N;
    FourierHost& fh = plan->fh;
    FourierDev& fd = plan->fd;
    fourier_setup<T>(plan, st);
    if (fh.method == SLK_FOURIER_CHEB) {
        DevBuf<unsigned> bad(1, st);
        SLK_CHECK_CUDA(cudaMemsetAsync(bad.get(), 0, sizeof(unsigned), st));
        int64_t ne = cheb_source_scratch(P, N, fd);
        DevBuf<T> scratch(ne, st);
        launch_cheb_source<T>(Zx, P, N, N, w, fd, plan->chebM.get(), reinterpret_cast<T*>(plan->beta.get()),
                              fh.cheb_qp <= 16 ? reinterpret_cast<T*>(plan->mono.get()) : nullptr, bad.get(),
                              mono_ratio_of(plan), scratch.get(), ne, st);
        cheb_finish(plan, bad.get(), st);
    } else if (fh.method == SLK_FOURIER_NDFT) {
        int64_t ne = ndft_source_scratch(P, N, fd);
        DevBuf<T> scratch(ne, st);
        launch_ndft_source<T>(Zx, P, N, N, w, fd, plan->coef.get(), reinterpret_cast<Cplx<T>*>(plan->cw.get()),
                              reinterpret_cast<T*>(plan->cw0.get()), scratch.get(), ne, st);
    } else {
        int64_t ne = nfft_source_scratch(P, N, fd);
        DevBuf<T> scratch(ne, st);
        // the sorting route's pairs (Laplacian), when built, feed a spreading in key order
        const T* pairs = plan->sorting ? reinterpret_cast<const T*>(plan->kw.get()) : nullptr;
        launch_nfft_source<T>(Zx, P, N, N, w, pairs, fd, fh.n_coeff, plan->mult.get(),
                              reinterpret_cast<T*>(plan->hgrid.get()), scratch.get(), ne, plan->err_dev.get(), st);
        if constexpr (sizeof(T) == 4) {
            // FP32: the target side reads the interpolant tabulated per grid cell
            float* tab = reinterpret_cast<float*>(plan->hgrid.get() + ((sizeof(T) * P * fh.W + 63) & ~size_t(63)));
            launch_interp_table(reinterpret_cast<const float*>(plan->hgrid.get()), P, fd, tab, st);
            fd.itab = tab;
        }
    }
    // the host copies of the coefficient tables must outlive the async copies
    SLK_CHECK_CUDA(cudaStreamSynchronize(st));
}

// Largest |projection| over a sample of min(N, 4096) strided source rows (the rows the
// centre is estimated from), on the BF16 tensor-core path: launched here, the value is copied
// into the pinned word *out and ev is recorded after the copy (read it once ev completes).
void sample_projection_max_async(slk_plan plan, const float* x, int64_t N, int64_t ldx, float* out, cudaEvent_t ev,
                                 cudaStream_t st) {
    const int d = plan->d, P = plan->P;
    const int64_t S = N < 4096 ? N : 4096;
    DevBuf<float> xs(static_cast<size_t>(S) * d, st);
    launch_gather_rows(x, N, d, ldx, S, xs.get(), st);
    DevBuf<float> zs(static_cast<size_t>(P) * S, st);
    DevBuf<float> mx(1, st);
    SLK_CHECK_CUDA(cudaMemsetAsync(mx.get(), 0, sizeof(float), st));
    cast_and_run(plan, xs.get(), S, d, st, [&](const void* xa, const void*, int64_t, int64_t rows, cudaStream_t s) {
        launch_project_umma(xa, nullptr, rows, plan->xib.get(), nullptr, P, d, 0, zs.get(), S, mx.get(),
                            plan->err_dev.get(), s);
    });
    SLK_CHECK_CUDA(cudaMemcpyAsync(out, mx.get(), sizeof(float), cudaMemcpyDeviceToHost, st));
    SLK_CHECK_CUDA(cudaEventRecord(ev, st));
}

struct EventGuard {
    cudaEvent_t ev = nullptr;
    EventGuard() { SLK_CHECK_CUDA(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming)); }
    ~EventGuard() { cudaEventDestroy(ev); }
};
// A pinned word for one readback; back to the pool only once the copy into it (recorded
// by `after`) has landed, also when an error leaves the call early.
struct PinnedWordGuard {
    unsigned* w = pinned_words().get();
    cudaEvent_t after = nullptr;
    ~PinnedWordGuard() {
        if (after && cudaEventSynchronize(after) != cudaSuccess) {
            cudaGetLastError();
            return;  // not reused
        }
        pinned_words().put(w);
    }
};

// Source side of the Chebyshev evaluation fused into the projection (BF16 path): the
// Fourier parameters are chosen for a radius fixed before the projection (the caller's, or
// 1.5 x the largest projection over the sample of sources), the moments come out of the
// projection kernel itself and no projection is stored.  The centring cast of the sources
// does not depend on the radius, so it is queued before the host waits for the sample's
// largest projection and keeps the GPU busy meanwhile.  Returns false, with nothing kept,
// when the method is not the Chebyshev one, its term count is not supported by the fused
// kernel, or a projected source lies outside the radius (the caller then takes the two-pass
// route, which sets the radius from all sources).
bool fused_cheb_source(slk_plan plan, const float* x, int64_t ldx, const float* w, cudaStream_t st) {
    const int P = plan->P, d = plan->d;
    const int64_t N = plan->N;
    const int m = plan->desc.method;
    if (m != SLK_FOURIER_AUTO && m != SLK_FOURIER_CHEB) return false;
    const bool user_radius = plan->desc.radius > 0.0;
    EventGuard sample_done;
    PinnedWordGuard sample_max;
    if (!user_radius) {
        sample_projection_max_async(plan, x, N, ldx, reinterpret_cast<float*>(sample_max.w), sample_done.ev, st);
        sample_max.after = sample_done.ev;
    }
    // CTA-pair route: the moments kernel reads the FP32 sources itself (no cast)
    const bool pair = P <= 512 && umma_f32_operand_ok(x, ldx);
    DevBuf<unsigned char> xa;
    if (!pair) {
        xa.alloc(static_cast<size_t>(N) * umma_operand_ld(d) * 2, st);
        launch_center_cast(x, N, d, ldx, plan->mu32.get(), xa.get(), nullptr, 0, st);
    }
    double R = plan->desc.radius;
    if (!user_radius) {
        SLK_CHECK_CUDA(cudaEventSynchronize(sample_done.ev));
        const float ms = *reinterpret_cast<const float*>(sample_max.w);
        if (!std::isfinite(ms)) fail(SLK_ERR_INVALID, "non-finite projected sources");
        R = 1.5 * ms + 1e-6;
    }
    double tol = plan->desc.tol;
    if (tol <= 0.0) tol = default_tol(SLK_GAUSSIAN, plan->desc.precision);
    FourierHost fh = choose_gaussian(plan->desc.param, d, R, plan->desc.n_coeff, plan->desc.method, tol);
    if (fh.method != SLK_FOURIER_CHEB || !umma_moments_fit(fh.cheb_qp) || (pair && !pair_cheb_fits(P, fh.cheb_qp, d)))
        return false;
    plan->fh = fh;
    plan->R = R;
    fourier_setup<float>(plan, st);
    const int64_t nchunk = pair ? pair_moments_chunks(P) : umma_moments_chunks(P);
    DevBuf<double> mom(static_cast<size_t>(nchunk) * P * fh.cheb_qp, st);
    DevBuf<float> mx(1, st);
    SLK_CHECK_CUDA(cudaMemsetAsync(mx.get(), 0, sizeof(float), st));
    if (pair)
        launch_pair_moments(x, ldx, plan->mu32.get(), N, plan->xib.get(), P, d, w, fh.cheb_qp, R, mom.get(), mx.get(),
                            plan->err_dev.get(), st);
    else
        launch_umma_moments(xa.get(), N, plan->xib.get(), P, d, w, fh.cheb_qp, R, mom.get(), mx.get(),
                            plan->err_dev.get(), st);
    // the reduction runs before the range check, so one wait covers both; its output is
    // discarded when a source lies outside the radius
    DevBuf<unsigned> bad(1, st);
    SLK_CHECK_CUDA(cudaMemsetAsync(bad.get(), 0, sizeof(unsigned), st));
    launch_cheb_reduce_f64(mom.get(), static_cast<int>(nchunk), P, plan->fd, plan->chebM.get(),
                           reinterpret_cast<float*>(plan->beta.get()),
                           fh.cheb_qp <= 16 ? reinterpret_cast<float*>(plan->mono.get()) : nullptr, bad.get(),
                           mono_ratio_of(plan), st);
    float rx = 0.0f;
    SLK_CHECK_CUDA(cudaMemcpyAsync(&rx, mx.get(), sizeof(float), cudaMemcpyDeviceToHost, st));
    cheb_finish(plan, bad.get(), st);
    if (!std::isfinite(rx)) fail(SLK_ERR_INVALID, "non-finite projected sources");
    if (rx > R) {
        if (user_radius)
            fail(SLK_ERR_INVALID, "radius %.6g is smaller than the largest projected source %.6g", R, rx);
        return false;
    }
    plan->fourier = true;
    return true;
}

template <class T>
void plan_sort_source(slk_plan plan, const T* Zx, const T* w, cudaStream_t st) {
    const int P = plan->P;
    const int64_t N = plan->N;
    // buckets of about 4 sources (a target scans its bucket's sources in any order), or of
    // about 8 when the records of all slices would exceed 4 GB
    int nb = 1;
    while (static_cast<int64_t>(nb) * 4 < N && nb < (1 << 22)) nb <<= 1;
    if (nb > 1 && static_cast<int64_t>(P) * (nb + 1) * kBucketRecordBytes > (int64_t(4) << 30)) nb >>= 1;
    plan->NB = nb;
    plan->kw.alloc(sorted_pairs_bytes<T>(P, N), st);
    plan->kmin.alloc(P, st);
    plan->kscale.alloc(P, st);
    // the sources grouped by equal-width bucket (Section 3.2 needs only the prefix sums at
    // bucket starts plus the sources of a target's own bucket, in any order)
    launch_slice_minmax<T>(Zx, P, N, N, nb, plan->kmin.get(), plan->kscale.get(), st);
    {
        const size_t sb = sort_pairs_scratch<T>(P, N);
        DevBuf<unsigned char> scratch(sb, st);
        launch_sort_pairs<T>(Zx, P, N, N, w, plan->kw.get(), scratch.get(), sb, plan->kmin.get(), plan->kscale.get(),
                             nb, st);
    }
    plan->rec.alloc(static_cast<size_t>(P) * (nb + 1) * kBucketRecordBytes, st);
    launch_bucket_tables<T>(P, N, plan->kw.get(), nb, plan->kmin.get(), plan->kscale.get(), plan->rec.get(), true, st);
}

template <class T>
void create_impl(slk_plan plan, const void* x_user, int64_t ldx, const void* w_user, cudaStream_t st) {
    const int64_t N = plan->N;
    const int d = plan->d, P = plan->P;
    InView<T> xv(x_user, N, d, ldx, st);
    InView<T> wv(w_user, N, 1, 1, st);
    // directions (Algorithm 1, first step)
    plan->xi64.alloc(static_cast<size_t>(P) * d, st);
    if (plan->desc.directions) {
        SLK_CHECK_CUDA(cudaMemcpyAsync(plan->xi64.get(), plan->desc.directions, sizeof(double) * P * d,
                                       cudaMemcpyDefault, st));
        // the caller may free a host copy after we return; a device copy is ordered on st
        if (!is_device_pointer(plan->desc.directions)) SLK_CHECK_CUDA(cudaStreamSynchronize(st));
    } else {
        launch_draw_directions(plan->xi64.get(), P, d, plan->desc.seed, plan->desc.slice_offset, st);
    }
    plan->mu64.alloc(d, st);
    launch_sample_mean<T>(xv.ptr, N, d, xv.ld, plan->mu64.get(), st);
    if constexpr (sizeof(T) == 4) {
        plan->xi32.alloc(static_cast<size_t>(P) * d, st);
        launch_convert<float>(plan->xi64.get(), plan->xi32.get(), static_cast<int64_t>(P) * d, st);
        plan->mu32.alloc(d, st);
        launch_convert<float>(plan->mu64.get(), plan->mu32.get(), d, st);
        if (plan->desc.precision == SLK_PREC_BF16 || plan->desc.precision == SLK_PREC_F16X3) {
            plan->tc = plan->desc.precision == SLK_PREC_BF16 ? 1 : 2;
            const size_t bytes = static_cast<size_t>(P) * umma_operand_ld(d) * 2;
            plan->xib.alloc(bytes, st);
            if (plan->tc == 2) plan->xib_lo.alloc(bytes, st);
            launch_center_cast(plan->xi32.get(), P, d, d, nullptr, plan->xib.get(), plan->xib_lo.get(), plan->tc == 2,
                               st, "cast_directions");
            plan->xit16.alloc(static_cast<size_t>(d) * umma_operand_ld(P) * 2, st);
            launch_transpose_bf16(plan->xi32.get(), P, d, plan->xit16.get(), st);
        }
    }
    // project the sources (and find the largest |z| for the Fourier window)
    const int kernel = plan->desc.kernel;
    if constexpr (sizeof(T) == 4) {
        if (plan->tc == 1 && kernel == SLK_GAUSSIAN && fused_cheb_source(plan, xv.ptr, xv.ld, wv.ptr, st)) return;
    }
    const bool need_fourier = kernel != SLK_NEGDIST;
    DevBuf<T> Zx(static_cast<size_t>(P) * N, st);
    DevBuf<float> mx(1, st);
    SLK_CHECK_CUDA(cudaMemsetAsync(mx.get(), 0, sizeof(float), st));
    project<T>(plan, xv.ptr, N, xv.ld, Zx.get(), need_fourier ? mx.get() : nullptr, st);
    if (need_fourier) {
        float rx = 0.0f;
        SLK_CHECK_CUDA(cudaMemcpyAsync(&rx, mx.get(), sizeof(float), cudaMemcpyDeviceToHost, st));
        SLK_CHECK_CUDA(cudaStreamSynchronize(st));
        if (!std::isfinite(rx)) fail(SLK_ERR_INVALID, "non-finite projected sources");
        double R = plan->desc.radius > 0.0 ? plan->desc.radius : 1.25 * static_cast<double>(rx) + 1e-6;
        if (R < rx) fail(SLK_ERR_INVALID, "radius %.6g is smaller than the largest projected source %.6g", R, rx);
        plan->R = R;
        double tol = plan->desc.tol;
        if (tol <= 0.0) tol = default_tol(kernel, plan->desc.precision);
        if (kernel == SLK_GAUSSIAN) plan->fh = choose_gaussian(plan->desc.param, d, R, plan->desc.n_coeff, plan->desc.method, tol);
        else plan->fh = fourier_smooth(plan->desc, d, R, tol);
        if (!plan->f64) add_window_poly_error(&plan->fh);
    }
    // the sorting route first: its pairs, grouped by key, also feed the Laplacian's spreading
    if (kernel == SLK_NEGDIST || kernel == SLK_LAPLACIAN) {
        plan->sorting = true;
        plan->sort_scale = kernel == SLK_LAPLACIAN ? plan->desc.param : 1.0;
        plan_sort_source<T>(plan, Zx.get(), wv.ptr, st);
    }
    if (need_fourier) {
        plan->fourier = true;
        plan_fourier_source<T>(plan, Zx.get(), wv.ptr, st);
    }
}

// Gaussian sums on the BF16 tensor-core path with the Chebyshev evaluation take the
// fused route: the targets' projections stay in TMEM and only per-tile row sums reach HBM.
template <class T>
bool sum_fused_cheb(slk_plan plan, const T* y, int64_t M, int64_t ldy, void* s_user, cudaStream_t st) {
    if constexpr (sizeof(T) == 4) {
        if (plan->tc != 1 || !plan->fourier || plan->sorting || plan->fh.method != SLK_FOURIER_CHEB ||
            !umma_cheb_fits(plan->P, plan->fh.cheb_qp) || M >= (int64_t(1) << 31))
            return false;
        const void* coef = plan->fd.horner ? plan->fd.mono : plan->beta.get();
        // aligned FP32 rows and P <= 512: the CTA-pair kernel, all slices of a tile at once
        const bool pair = umma_f32_operand_ok(y, ldy) && pair_cheb_fits(plan->P, plan->fh.cheb_qp, plan->d);
        const int parts = static_cast<int>(pair ? pair_cheb_parts(plan->P) : umma_cheb_parts(plan->P));
        DevBuf<double> part(static_cast<size_t>(parts) * M, st);
        if (pair)
            launch_pair_cheb_target(y, ldy, plan->mu32.get(), M, plan->xib.get(), plan->P, plan->d,
                                    static_cast<const float*>(coef), plan->fh.cheb_qp, plan->fd.horner, plan->R,
                                    part.get(), M, plan->err_dev.get(), st);
        else if (umma_f32_operand_ok(y, ldy))  // aligned FP32 rows: centred and rounded in the kernel
            launch_umma_cheb_target_f32(y, ldy, plan->mu32.get(), M, plan->xib.get(), plan->P, plan->d,
                                        static_cast<const float*>(coef), plan->fh.cheb_qp, plan->fd.horner, plan->R,
                                        part.get(), M, plan->err_dev.get(), st);
        else
            cast_and_run(plan, y, M, ldy, st,
                         [&](const void* ya, const void*, int64_t r0, int64_t rows, cudaStream_t s) {
                             launch_umma_cheb_target(ya, rows, plan->xib.get(), plan->P, plan->d,
                                                     static_cast<const float*>(coef), plan->fh.cheb_qp,
                                                     plan->fd.horner, plan->R, part.get() + r0, M,
                                                     plan->err_dev.get(), s);
                         });
        if (is_device_pointer(s_user)) {
            launch_sum_parts<T>(part.get(), parts, M, 1.0 / plan->P, static_cast<T*>(s_user), st);
        } else {
            DevBuf<T> s(M, st);
            launch_sum_parts<T>(part.get(), parts, M, 1.0 / plan->P, s.get(), st);
            SLK_CHECK_CUDA(cudaMemcpyAsync(s_user, s.get(), sizeof(T) * M, cudaMemcpyDeviceToHost, st));
            SLK_CHECK_CUDA(cudaStreamSynchronize(st));
        }
        return true;
    }
    return false;
}

// The target side of every slice at the projected targets Zy (P x M, row stride M): with
// acc, the 1-D sums summed over slices into acc[m]; with G, their derivatives dt_p/dz into
// G[p * ldg + m] (slice-major); either or both (Algorithm 1; Sections 3.1-3.3 and their
// derivatives).  For the Laplacian the sorting part adds its derivative to the Fourier part's.
template <class T>
void target_side(slk_plan plan, const T* Zy, int64_t M, double* acc, T* G, int64_t ldg, cudaStream_t st) {
    const int P = plan->P;
    if (plan->fourier) {
        if (plan->fh.method == SLK_FOURIER_CHEB)
            launch_cheb_target<T>(Zy, P, M, M, plan->fd, reinterpret_cast<const T*>(plan->beta.get()), acc, G, ldg,
                                  plan->err_dev.get(), st);
        else if (plan->fh.method == SLK_FOURIER_NDFT)
            launch_ndft_target<T>(Zy, P, M, M, plan->fd, reinterpret_cast<const Cplx<T>*>(plan->cw.get()),
                                  reinterpret_cast<const T*>(plan->cw0.get()), acc, G, ldg, plan->err_dev.get(), st);
        else
            launch_nfft_target<T>(Zy, P, M, M, plan->fd, reinterpret_cast<const T*>(plan->hgrid.get()), acc, G, ldg,
                                  plan->err_dev.get(), st);
    }
    if (plan->sorting)
        launch_negdist_target<T>(Zy, P, M, M, plan->kw.get(), plan->N, plan->rec.get(), plan->NB, plan->kmin.get(),
                                 plan->kscale.get(), plan->cd, plan->sort_scale, acc, G, ldg, plan->fourier ? 1 : 0, st);
}

// s = acc / P into the caller's s (device or host)
template <class T>
void finish_sum(const double* acc, int64_t M, int P, void* s_user, cudaStream_t st) {
    if (is_device_pointer(s_user)) {
        launch_finalize<T>(acc, static_cast<T*>(s_user), M, 1.0 / P, st);
    } else {
        DevBuf<T> s(M, st);
        launch_finalize<T>(acc, s.get(), M, 1.0 / P, st);
        SLK_CHECK_CUDA(cudaMemcpyAsync(s_user, s.get(), sizeof(T) * M, cudaMemcpyDeviceToHost, st));
        SLK_CHECK_CUDA(cudaStreamSynchronize(st));
    }
}

template <class T>
void sum_impl(slk_plan plan, const void* y_user, int64_t M, int64_t ldy, void* s_user, cudaStream_t st) {
    const int P = plan->P, d = plan->d;
    InView<T> yv(y_user, M, d, ldy, st);
    if (sum_fused_cheb<T>(plan, yv.ptr, M, yv.ld, s_user, st)) return;
    DevBuf<T> Zy(static_cast<size_t>(P) * M, st);
    project<T>(plan, yv.ptr, M, yv.ld, Zy.get(), nullptr, st);
    DevBuf<double> acc(M, st);
    SLK_CHECK_CUDA(cudaMemsetAsync(acc.get(), 0, sizeof(double) * M, st));
    target_side<T>(plan, Zy.get(), M, acc.get(), static_cast<T*>(nullptr), 0, st);
    finish_sum<T>(acc.get(), M, P, s_user, st);
}

template <class T>
void project_impl(slk_plan plan, const void* x_user, int64_t n, int64_t ldx, void* Z_user, int64_t ldz,
                  cudaStream_t st) {
    InView<T> xv(x_user, n, plan->d, ldx, st);
    DevBuf<T> Z(static_cast<size_t>(plan->P) * n, st);
    project<T>(plan, xv.ptr, n, xv.ld, Z.get(), nullptr, st);
    SLK_CHECK_CUDA(cudaMemcpy2DAsync(Z_user, sizeof(T) * ldz, Z.get(), sizeof(T) * n, sizeof(T) * n, plan->P,
                                     cudaMemcpyDefault, st));
    if (!is_device_pointer(Z_user)) SLK_CHECK_CUDA(cudaStreamSynchronize(st));
}

// Backward product (Algorithm 1 differentiated): gy_m = gs_m (1/P) sum_p G[p * ldG + m] xi_p
// into the caller's gy (M x d, row stride ldgy, device or host); gs device memory or NULL.
template <class T>
void backward_product(slk_plan plan, const T* G, int64_t ldG, int64_t M, const T* gs, void* gy_user, int64_t ldgy,
                      cudaStream_t st) {
    const int P = plan->P, d = plan->d;
    const bool g_dev = is_device_pointer(gy_user);
    DevBuf<T> gy_tmp(g_dev ? 0 : static_cast<size_t>(M) * d, st);
    T* out = g_dev ? static_cast<T*>(gy_user) : gy_tmp.get();
    const int64_t ldo = g_dev ? ldgy : d;
    bool done = false;
    if constexpr (sizeof(T) == 4) {
        if (plan->tc) {
            // on tensor cores: BF16 operands (the derivatives transposed to M x P), FP32 accumulate
            DevBuf<unsigned char> g16(static_cast<size_t>(M) * umma_operand_ld(P) * 2, st);
            launch_derivs_bf16(G, P, M, ldG, g16.get(), st);
            launch_grad_umma(g16.get(), M, P, plan->xit16.get(), d, gs, 1.0 / P, out, ldo, plan->err_dev.get(), st);
            done = true;
        }
    }
    if (!done) launch_grad_gemm<T>(G, ldG, M, P, xi_of<T>(plan), d, gs, 1.0 / P, out, ldo, st);
    if (!g_dev) {
        SLK_CHECK_CUDA(cudaMemcpy2DAsync(gy_user, sizeof(T) * ldgy, out, sizeof(T) * d, sizeof(T) * d, M,
                                         cudaMemcpyDeviceToHost, st));
        SLK_CHECK_CUDA(cudaStreamSynchronize(st));
    }
}

template <class T>
void grad_impl(slk_plan plan, const void* y_user, int64_t M, int64_t ldy, const void* gs_user, void* gy_user,
               int64_t ldg, cudaStream_t st) {
    const int P = plan->P, d = plan->d;
    InView<T> yv(y_user, M, d, ldy, st);
    DevBuf<T> Zy(static_cast<size_t>(P) * M, st);
    project<T>(plan, yv.ptr, M, yv.ld, Zy.get(), nullptr, st);
    DevBuf<T> G(static_cast<size_t>(P) * M, st);
    target_side<T>(plan, Zy.get(), M, nullptr, G.get(), M, st);
    InView<T> gsv(gs_user, gs_user ? M : 0, 1, 1, st);
    backward_product<T>(plan, G.get(), M, M, gs_user ? gsv.ptr : nullptr, gy_user, ldg, st);
}

// Sums and the per-slice derivatives from one projection of the targets and one evaluation
// of the target side (the sorting route's lookup serves both).
template <class T>
void sum_derivs_impl(slk_plan plan, const void* y_user, int64_t M, int64_t ldy, void* s_user, void* g_user,
                     int64_t ldd, cudaStream_t st) {
    const int P = plan->P, d = plan->d;
    InView<T> yv(y_user, M, d, ldy, st);
    DevBuf<T> Zy(static_cast<size_t>(P) * M, st);
    project<T>(plan, yv.ptr, M, yv.ld, Zy.get(), nullptr, st);
    DevBuf<double> acc(M, st);
    SLK_CHECK_CUDA(cudaMemsetAsync(acc.get(), 0, sizeof(double) * M, st));
    const bool g_dev = is_device_pointer(g_user);
    DevBuf<T> gtmp(g_dev ? 0 : static_cast<size_t>(P) * M, st);
    T* G = g_dev ? static_cast<T*>(g_user) : gtmp.get();
    const int64_t ldG = g_dev ? ldd : M;
    target_side<T>(plan, Zy.get(), M, acc.get(), G, ldG, st);
    finish_sum<T>(acc.get(), M, P, s_user, st);
    if (!g_dev) {
        SLK_CHECK_CUDA(cudaMemcpy2DAsync(g_user, sizeof(T) * ldd, G, sizeof(T) * M, sizeof(T) * M, P,
                                         cudaMemcpyDeviceToHost, st));
        SLK_CHECK_CUDA(cudaStreamSynchronize(st));
    }
}

template <class T>
void grad_derivs_impl(slk_plan plan, const void* g_user, int64_t M, int64_t ldd, const void* gs_user, void* gy_user,
                      int64_t ldgy, cudaStream_t st) {
    InView<T> gv(g_user, plan->P, static_cast<int>(M), ldd, st);
    InView<T> gsv(gs_user, gs_user ? M : 0, 1, 1, st);
    backward_product<T>(plan, gv.ptr, gv.ld, M, gs_user ? gsv.ptr : nullptr, gy_user, ldgy, st);
}

void validate_desc(const slk_plan_desc* desc) {
    SLK_REQUIRE(desc, "descriptor is NULL");
    SLK_REQUIRE(desc->kernel >= SLK_GAUSSIAN && desc->kernel <= SLK_MATERN32, "unknown kernel %d", desc->kernel);
    SLK_REQUIRE(desc->precision >= SLK_PREC_F64 && desc->precision <= SLK_PREC_F16X3, "unknown precision %d",
                desc->precision);
    SLK_REQUIRE(desc->d >= 1, "d must be >= 1");
    SLK_REQUIRE(desc->P >= 1 && desc->P <= 65535, "P must be in [1, 65535]");
    SLK_REQUIRE(desc->method >= SLK_FOURIER_AUTO && desc->method <= SLK_FOURIER_CHEB, "unknown Fourier method");
    if ((desc->kernel == SLK_LAPLACIAN || desc->kernel == SLK_MATERN32) && desc->method != SLK_FOURIER_AUTO &&
        desc->method != SLK_FOURIER_NFFT)
        fail(SLK_ERR_UNSUPPORTED, "the Laplacian and Matern kernels use the NFFT (their coefficients decay like k^-4)");
    SLK_REQUIRE(desc->n_coeff >= 0 && desc->n_coeff <= (1 << 14) && desc->n_coeff % 2 == 0,
                "n_coeff must be even and in [0, 16384]");
    if (desc->kernel != SLK_NEGDIST)
        SLK_REQUIRE(desc->param > 0.0 && std::isfinite(desc->param), "kernel parameter must be positive");
    SLK_REQUIRE(desc->tol >= 0.0 && desc->radius >= 0.0, "tol and radius must be >= 0");
    SLK_REQUIRE(desc->slice_batch >= 0, "slice_batch must be >= 0");
    SLK_REQUIRE(desc->slice_offset >= 0 && desc->slice_offset <= INT32_MAX - desc->P,
                "slice_offset must be in [0, 2^31 - 1 - P]");
}

// slk_kernel_sum over slice batches (Sec. 5.4, remark on memory and batching): batch b plans
// the slices [p0, p0 + P_b) on its own, sums into a device buffer, and adds (P_b / P) times that
// into an FP64 accumulator; one batch's plan is alive at a time.
template <class T>
void batched_kernel_sum(const slk_plan_desc& desc, const void* x, int64_t N, int64_t ldx, const void* w,
                        const void* y, int64_t M, int64_t ldy, void* s, cudaStream_t st);

}  // namespace

// ------------------------------------------------------------ exported calls

extern "C" {

int32_t slk_version(void) { return SLK_VERSION_MAJOR * 100 + SLK_VERSION_MINOR; }

const char* slk_status_string(slk_status status) {
    switch (status) {
    case SLK_OK: return "ok";
    case SLK_ERR_INVALID: return "invalid argument";
    case SLK_ERR_OOM: return "out of device memory";
    case SLK_ERR_CUDA: return "CUDA error";
    case SLK_ERR_ACCURACY: return "accuracy target cannot be met";
    case SLK_ERR_TIMEOUT: return "timed out";
    case SLK_ERR_BUSY: return "busy";
    case SLK_ERR_UNSUPPORTED: return "unsupported";
    case SLK_ERR_NOT_FOUND: return "not found";
    }
    return "unknown status";
}

const char* slk_last_error(void) { return g_last_error.c_str(); }

slk_status slk_plan_create(slk_plan* out, const slk_plan_desc* desc, const void* x, int64_t N, int64_t ldx,
                           const void* w, void* stream) {
    set_last_error("");
    return guarded([&] {
        SLK_REQUIRE(out, "plan output pointer is NULL");
        *out = nullptr;
        validate_desc(desc);
        SLK_REQUIRE(x && w, "x and w must not be NULL");
        SLK_REQUIRE(N >= 1 && N < (int64_t(1) << 31), "N must be in [1, 2^31)");
        SLK_REQUIRE(ldx >= desc->d, "ldx must be >= d");
        cudaStream_t st = static_cast<cudaStream_t>(stream);
        std::unique_ptr<slk_plan_s> plan(new slk_plan_s());
        plan->desc = *desc;
        SLK_CHECK_CUDA(cudaGetDevice(&plan->device));
        configure_pool(plan->device);
        plan->f64 = desc->precision == SLK_PREC_F64;
        plan->N = N;
        plan->d = desc->d;
        plan->P = desc->P;
        plan->cd = cd_host(desc->d);
        plan->stream = st;
        plan->err_dev.alloc(1, st);
        SLK_CHECK_CUDA(cudaMemsetAsync(plan->err_dev.get(), 0, sizeof(unsigned), st));
        plan->err_host = pinned_words().get();
        *plan->err_host = 0;
        SLK_CHECK_CUDA(cudaEventCreateWithFlags(&plan->done, cudaEventDisableTiming));
        if (plan->f64) create_impl<double>(plan.get(), x, ldx, w, st);
        else create_impl<float>(plan.get(), x, ldx, w, st);
        finish_call(plan.get(), st);
        slk_status s = collect(plan.get(), true);
        if (s != SLK_OK) throw Error{s, slk_last_error()};
        SLK_CHECK_LAUNCH();
        *out = plan.release();
    });
}

slk_status slk_sum(slk_plan plan, const void* y, int64_t M, int64_t ldy, void* s, void* stream) {
    set_last_error("");
    return guarded([&] {
        SLK_REQUIRE(plan, "plan is NULL");
        slk_status prev = collect(plan, false);
        if (prev != SLK_OK) throw Error{prev, slk_last_error()};
        SLK_REQUIRE(M >= 0, "M must be >= 0");
        if (M == 0) return;
        SLK_REQUIRE(y && s, "y and s must not be NULL");
        SLK_REQUIRE(ldy >= plan->d, "ldy must be >= d");
        cudaStream_t st = static_cast<cudaStream_t>(stream);
        if (plan->f64) sum_impl<double>(plan, y, M, ldy, s, st);
        else sum_impl<float>(plan, y, M, ldy, s, st);
        finish_call(plan, st);
        plan->stream = st;
        if (!is_device_pointer(s)) {
            slk_status e = collect(plan, true);
            if (e != SLK_OK) throw Error{e, slk_last_error()};
        }
    });
}

slk_status slk_grad(slk_plan plan, const void* y, int64_t M, int64_t ldy, const void* gs, void* gy, int64_t ldg,
                    void* stream) {
    set_last_error("");
    return guarded([&] {
        SLK_REQUIRE(plan, "plan is NULL");
        slk_status prev = collect(plan, false);
        if (prev != SLK_OK) throw Error{prev, slk_last_error()};
        SLK_REQUIRE(M >= 0, "M must be >= 0");
        if (M == 0) return;
        SLK_REQUIRE(y && gy, "y and gy must not be NULL");
        SLK_REQUIRE(ldy >= plan->d && ldg >= plan->d, "ldy and ldg must be >= d");
        cudaStream_t st = static_cast<cudaStream_t>(stream);
        if (plan->f64) grad_impl<double>(plan, y, M, ldy, gs, gy, ldg, st);
        else grad_impl<float>(plan, y, M, ldy, gs, gy, ldg, st);
        finish_call(plan, st);
        plan->stream = st;
        if (!is_device_pointer(gy)) {
            slk_status e = collect(plan, true);
            if (e != SLK_OK) throw Error{e, slk_last_error()};
        }
    });
}

slk_status slk_sum_derivs(slk_plan plan, const void* y, int64_t M, int64_t ldy, void* s, void* g, int64_t ldd,
                          void* stream) {
    set_last_error("");
    return guarded([&] {
        SLK_REQUIRE(plan, "plan is NULL");
        slk_status prev = collect(plan, false);
        if (prev != SLK_OK) throw Error{prev, slk_last_error()};
        SLK_REQUIRE(M >= 0, "M must be >= 0");
        if (M == 0) return;
        SLK_REQUIRE(y && s && g, "y, s and g must not be NULL");
        SLK_REQUIRE(ldy >= plan->d, "ldy must be >= d");
        SLK_REQUIRE(ldd >= M, "ldd must be >= M");
        SLK_REQUIRE(M <= INT32_MAX, "M must be < 2^31");
        cudaStream_t st = static_cast<cudaStream_t>(stream);
        if (plan->f64) sum_derivs_impl<double>(plan, y, M, ldy, s, g, ldd, st);
        else sum_derivs_impl<float>(plan, y, M, ldy, s, g, ldd, st);
        finish_call(plan, st);
        plan->stream = st;
        if (!is_device_pointer(s) || !is_device_pointer(g)) {
            slk_status e = collect(plan, true);
            if (e != SLK_OK) throw Error{e, slk_last_error()};
        }
    });
}

slk_status slk_grad_derivs(slk_plan plan, const void* g, int64_t M, int64_t ldd, const void* gs, void* gy,
                           int64_t ldgy, void* stream) {
    set_last_error("");
    return guarded([&] {
        SLK_REQUIRE(plan, "plan is NULL");
        slk_status prev = collect(plan, false);
        if (prev != SLK_OK) throw Error{prev, slk_last_error()};
        SLK_REQUIRE(M >= 0, "M must be >= 0");
        if (M == 0) return;
        SLK_REQUIRE(g && gy, "g and gy must not be NULL");
        SLK_REQUIRE(ldd >= M && ldgy >= plan->d, "ldd must be >= M and ldgy >= d");
        SLK_REQUIRE(M <= INT32_MAX, "M must be < 2^31");
        cudaStream_t st = static_cast<cudaStream_t>(stream);
        if (plan->f64) grad_derivs_impl<double>(plan, g, M, ldd, gs, gy, ldgy, st);
        else grad_derivs_impl<float>(plan, g, M, ldd, gs, gy, ldgy, st);
        finish_call(plan, st);
        plan->stream = st;
        if (!is_device_pointer(gy)) {
            slk_status e = collect(plan, true);
            if (e != SLK_OK) throw Error{e, slk_last_error()};
        }
    });
}

slk_status slk_plan_project(slk_plan plan, const void* x, int64_t n, int64_t ldx, void* Z, int64_t ldz, void* stream) {
    set_last_error("");
    return guarded([&] {
        SLK_REQUIRE(plan, "plan is NULL");
        slk_status prev = collect(plan, false);
        if (prev != SLK_OK) throw Error{prev, slk_last_error()};
        SLK_REQUIRE(n >= 0, "n must be >= 0");
        if (n == 0) return;
        SLK_REQUIRE(x && Z, "x and Z must not be NULL");
        SLK_REQUIRE(ldx >= plan->d && ldz >= n, "ldx must be >= d and ldz >= n");
        cudaStream_t st = static_cast<cudaStream_t>(stream);
        if (plan->f64) project_impl<double>(plan, x, n, ldx, Z, ldz, st);
        else project_impl<float>(plan, x, n, ldx, Z, ldz, st);
        finish_call(plan, st);
        plan->stream = st;
        if (!is_device_pointer(Z)) {
            slk_status e = collect(plan, true);
            if (e != SLK_OK) throw Error{e, slk_last_error()};
        }
    });
}

slk_status slk_plan_get_center(slk_plan plan, double* mu_host) {
    set_last_error("");
    return guarded([&] {
        SLK_REQUIRE(plan && mu_host, "plan and mu_host must not be NULL");
        SLK_CHECK_CUDA(cudaMemcpyAsync(mu_host, plan->mu64.get(), sizeof(double) * plan->d, cudaMemcpyDeviceToHost,
                                       plan->stream));
        SLK_CHECK_CUDA(cudaStreamSynchronize(plan->stream));
    });
}

slk_status slk_plan_sync(slk_plan plan) {
    set_last_error("");
    return guarded([&] {
        SLK_REQUIRE(plan, "plan is NULL");
        slk_status e = collect(plan, true);
        if (e != SLK_OK) throw Error{e, slk_last_error()};
    });
}

slk_status slk_plan_get_directions(slk_plan plan, double* xi_host) {
    set_last_error("");
    return guarded([&] {
        SLK_REQUIRE(plan && xi_host, "plan and xi_host must not be NULL");
        SLK_CHECK_CUDA(cudaMemcpyAsync(xi_host, plan->xi64.get(), sizeof(double) * plan->P * plan->d,
                                       cudaMemcpyDeviceToHost, plan->stream));
        SLK_CHECK_CUDA(cudaStreamSynchronize(plan->stream));
    });
}

slk_status slk_plan_get_info(slk_plan plan, slk_plan_info* info) {
    set_last_error("");
    return guarded([&] {
        SLK_REQUIRE(plan && info, "plan and info must not be NULL");
        SLK_CHECK_CUDA(cudaStreamSynchronize(plan->stream));
        std::memset(info, 0, sizeof(*info));
        info->kernel = plan->desc.kernel;
        info->precision = plan->desc.precision;
        info->d = plan->d;
        info->P = plan->P;
        info->N = plan->N;
        info->c_d = plan->cd;
        info->device_bytes = plan->device_bytes();
        info->sort_buckets = plan->NB;
        if (plan->fourier) {
            info->method = plan->fh.method;
            info->n_coeff = plan->fh.n_coeff;
            info->n_grid = plan->fh.n_g;
            info->window = plan->fh.m;
            info->k_lo = plan->fh.k_lo;
            info->k_hi = plan->fh.k_hi;
            info->cheb_terms = plan->fh.cheb_q;
            info->cheb_horner = plan->fd.horner;
            info->period = plan->fh.L;
            info->radius = plan->R;
            info->model_error = plan->fh.model_err;
        }
    });
}

slk_status slk_plan_destroy(slk_plan plan) {
    set_last_error("");
    return guarded([&] {
        if (!plan) return;
        delete plan;  // stream-ordered release after the plan's last call (no wait)
    });
}

slk_status slk_fourier_params(const slk_plan_desc* desc, double radius, slk_plan_info* info) {
    set_last_error("");
    return guarded([&] {
        validate_desc(desc);
        SLK_REQUIRE(info && radius > 0.0 && std::isfinite(radius), "info must not be NULL and radius > 0");
        if (desc->kernel == SLK_NEGDIST) fail(SLK_ERR_UNSUPPORTED, "the negative distance kernel has no Fourier part");
        const bool f64 = desc->precision == SLK_PREC_F64;
        double tol = desc->tol;
        if (tol <= 0.0) tol = default_tol(desc->kernel, desc->precision);
        FourierHost fh = desc->kernel == SLK_GAUSSIAN
                             ? choose_gaussian(desc->param, desc->d, radius, desc->n_coeff, desc->method, tol)
                             : fourier_smooth(*desc, desc->d, radius, tol);
        if (!f64) add_window_poly_error(&fh);
        std::memset(info, 0, sizeof(*info));
        info->kernel = desc->kernel;
        info->precision = desc->precision;
        info->d = desc->d;
        info->P = desc->P;
        info->method = fh.method;
        info->n_coeff = fh.n_coeff;
        info->n_grid = fh.n_g;
        info->window = fh.m;
        info->k_lo = fh.k_lo;
        info->k_hi = fh.k_hi;
        info->cheb_terms = fh.cheb_q;
        info->period = fh.L;
        info->radius = radius;
        info->model_error = fh.model_err;
        info->c_d = cd_host(desc->d);
    });
}

slk_status slk_kernel_sum(const slk_plan_desc* desc, const void* x, int64_t N, int64_t ldx, const void* w,
                          const void* y, int64_t M, int64_t ldy, void* s, void* stream) {
    if (desc && desc->slice_batch > 0 && desc->slice_batch < desc->P) {
        set_last_error("");
        return guarded([&] {
            validate_desc(desc);
            SLK_REQUIRE(M >= 0, "M must be >= 0");
            if (M == 0) return;
            SLK_REQUIRE(y && s, "y and s must not be NULL");
            cudaStream_t st = static_cast<cudaStream_t>(stream);
            if (desc->precision == SLK_PREC_F64) batched_kernel_sum<double>(*desc, x, N, ldx, w, y, M, ldy, s, st);
            else batched_kernel_sum<float>(*desc, x, N, ldx, w, y, M, ldy, s, st);
        });
    }
    slk_plan plan = nullptr;
    slk_status st = slk_plan_create(&plan, desc, x, N, ldx, w, stream);
    if (st != SLK_OK) return st;
    st = slk_sum(plan, y, M, ldy, s, stream);
    if (st == SLK_OK) st = slk_plan_sync(plan);
    std::string keep = slk_last_error();
    slk_status d = slk_plan_destroy(plan);
    if (st != SLK_OK) {
        set_last_error(keep);
        return st;
    }
    return d;
}

}  // extern "C"

// ------------------------------------------------------------ random Fourier features

namespace {

void validate_rff(const slk_rff_desc* desc) {
    SLK_REQUIRE(desc, "desc is NULL");
    SLK_REQUIRE(desc->kernel == SLK_GAUSSIAN || desc->kernel == SLK_LAPLACIAN,
                "random Fourier features need a positive definite kernel (Gaussian or Laplacian)");
    SLK_REQUIRE(desc->precision == SLK_PREC_F64 || desc->precision == SLK_PREC_F32, "precision must be F64 or F32");
    SLK_REQUIRE(desc->param > 0.0 && std::isfinite(desc->param), "param must be > 0");
    SLK_REQUIRE(desc->d >= 1, "d must be >= 1");
    SLK_REQUIRE(desc->D >= 1 && desc->D <= 65535, "D must be in 1 .. 65535");
    SLK_REQUIRE(desc->variant == 1 || desc->variant == 2, "variant must be 1 or 2");
}

// The features on the device (D x (d + 1) FP64): the caller's, or the library's draw.
DevBuf<double> rff_features_dev(const slk_rff_desc* desc, cudaStream_t st) {
    const size_t n = static_cast<size_t>(desc->D) * (desc->d + 1);
    DevBuf<double> feat(n, st);
    if (desc->features) {
        SLK_CHECK_CUDA(cudaMemcpyAsync(feat.get(), desc->features, sizeof(double) * n, cudaMemcpyDefault, st));
        if (!is_device_pointer(desc->features)) SLK_CHECK_CUDA(cudaStreamSynchronize(st));
    } else {
        launch_rff_draw(feat.get(), desc->D, desc->d, desc->kernel == SLK_LAPLACIAN, desc->param, desc->seed, st);
    }
    return feat;
}

template <class T>
void rff_impl(const slk_rff_desc* desc, const void* x, int64_t N, int64_t ldx, const void* w, const void* y, int64_t M,
              int64_t ldy, void* s_user, cudaStream_t st) {
    const int D = desc->D, d = desc->d;
    InView<T> xv(x, N, d, ldx, st), yv(y, M, d, ldy, st), wv(w, N, 1, 1, st);
    DevBuf<double> feat = rff_features_dev(desc, st);
    DevBuf<T> V(static_cast<size_t>(D) * d, st), b(D, st);
    launch_rff_split<T>(feat.get(), D, d, V.get(), b.get(), st);
    DevBuf<double2> cs(D, st);
    {
        DevBuf<T> Zx(static_cast<size_t>(D) * N, st);
        launch_project_simt<T>(V.get(), D, xv.ptr, N, d, xv.ld, nullptr, Zx.get(), N, st);
        launch_rff_source<T>(Zx.get(), D, N, wv.ptr, b.get(), desc->variant, cs.get(), st);
    }
    DevBuf<T> Zy(static_cast<size_t>(D) * M, st);
    launch_project_simt<T>(V.get(), D, yv.ptr, M, d, yv.ld, nullptr, Zy.get(), M, st);
    if (is_device_pointer(s_user)) {
        launch_rff_target<T>(Zy.get(), D, M, b.get(), cs.get(), desc->variant, static_cast<T*>(s_user), st);
    } else {
        DevBuf<T> s(M, st);
        launch_rff_target<T>(Zy.get(), D, M, b.get(), cs.get(), desc->variant, s.get(), st);
        SLK_CHECK_CUDA(cudaMemcpyAsync(s_user, s.get(), sizeof(T) * M, cudaMemcpyDeviceToHost, st));
        SLK_CHECK_CUDA(cudaStreamSynchronize(st));
    }
}

}  // namespace

extern "C" slk_status slk_rff_sum(const slk_rff_desc* desc, const void* x, int64_t N, int64_t ldx, const void* w,
                                  const void* y, int64_t M, int64_t ldy, void* s, void* stream) {
    set_last_error("");
    return guarded([&] {
        validate_rff(desc);
        SLK_REQUIRE(x && w, "x and w must not be NULL");
        SLK_REQUIRE(N >= 1 && M >= 0, "N must be >= 1 and M >= 0");
        SLK_REQUIRE(ldx >= desc->d && (M == 0 || ldy >= desc->d), "row strides must be >= d");
        if (M == 0) return;
        SLK_REQUIRE(y && s, "y and s must not be NULL");
        cudaStream_t st = static_cast<cudaStream_t>(stream);
        if (desc->precision == SLK_PREC_F64) rff_impl<double>(desc, x, N, ldx, w, y, M, ldy, s, st);
        else rff_impl<float>(desc, x, N, ldx, w, y, M, ldy, s, st);
        SLK_CHECK_CUDA(cudaGetLastError());
    });
}

extern "C" slk_status slk_rff_features(const slk_rff_desc* desc, double* features) {
    set_last_error("");
    return guarded([&] {
        validate_rff(desc);
        SLK_REQUIRE(features, "features must not be NULL");
        cudaStream_t st = nullptr;
        slk_rff_desc own = *desc;
        own.features = nullptr;
        DevBuf<double> feat = rff_features_dev(&own, st);
        SLK_CHECK_CUDA(cudaMemcpyAsync(features, feat.get(), sizeof(double) * own.D * (own.d + 1),
                                       cudaMemcpyDeviceToHost, st));
        SLK_CHECK_CUDA(cudaStreamSynchronize(st));
    });
}

namespace {

template <class T>
void batched_kernel_sum(const slk_plan_desc& desc, const void* x, int64_t N, int64_t ldx, const void* w,
                        const void* y, int64_t M, int64_t ldy, void* s, cudaStream_t st) {
    const int P = desc.P, B = desc.slice_batch, d = desc.d;
    DevBuf<T> sb(static_cast<size_t>(M), st);
    DevBuf<double> acc(static_cast<size_t>(M), st);
    for (int p0 = 0; p0 < P; p0 += B) {
        slk_plan_desc b = desc;
        b.P = std::min(B, P - p0);
        b.slice_batch = 0;
        if (desc.directions) b.directions = desc.directions + static_cast<size_t>(p0) * d;
        else b.slice_offset = desc.slice_offset + p0;
        slk_plan plan = nullptr;
        slk_status r = slk_plan_create(&plan, &b, x, N, ldx, w, st);
        if (r != SLK_OK) throw Error{r, slk_last_error()};
        r = slk_sum(plan, y, M, ldy, sb.get(), st);
        if (r == SLK_OK) r = slk_plan_sync(plan);
        std::string keep = slk_last_error();
        slk_plan_destroy(plan);
        if (r != SLK_OK) throw Error{r, keep};
        launch_accumulate_scaled<T>(acc.get(), sb.get(), static_cast<double>(b.P) / P, M, p0 == 0, st);
    }
    T* out = is_device_pointer(s) ? static_cast<T*>(s) : sb.get();
    launch_sum_parts<T>(acc.get(), 1, M, 1.0, out, st);
    if (out != s)
        SLK_CHECK_CUDA(cudaMemcpyAsync(s, out, sizeof(T) * static_cast<size_t>(M), cudaMemcpyDeviceToHost, st));
    SLK_CHECK_CUDA(cudaStreamSynchronize(st));
}

}  // namespace

// ------------------------------------------------------------ sums without device allocation
//
// slk_sum_noalloc: the same target-side computation as slk_sum, for callers
// that must not allocate device memory while they run (see include/slk.h).
// Its working memory is one file-scope device array shared by every call.

namespace {

constexpr size_t kNoAllocScratchBytes = size_t(64) << 20;  // 64 MiB per device

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

std::mutex g_noalloc_mu;
void* g_noalloc_addr[128] = {};

// Device address of the scratch array on the current device.  The name
// g_noalloc_scratch is only a host-side stand-in; the address is looked up
// once per device (the first call on that device) and cached.
unsigned char* noalloc_scratch(int device) {
    SLK_REQUIRE(device >= 0 && device < 128, "device index out of range");
    std::lock_guard<std::mutex> g(g_noalloc_mu);
    if (!g_noalloc_addr[device]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) {
            cudaGetLastError();
            fail(SLK_ERR_CUDA, "cudaGetSymbolAddress of the scratch array failed: %s", cudaGetErrorString(e));
        }
        g_noalloc_addr[device] = p;
    }
    return static_cast<unsigned char*>(g_noalloc_addr[device]);
}

size_t align256(size_t b) { return (b + 255) & ~size_t(255); }

template <class T>
size_t noalloc_bytes(slk_plan plan, int64_t M) {
    size_t b = align256(sizeof(T) * static_cast<size_t>(plan->P) * M) + align256(sizeof(double) * M);
    if (plan->tc) b += align256(static_cast<size_t>(M) * umma_operand_ld(plan->d) * 2) * (plan->tc == 2 ? 2 : 1);
    return b;
}

template <class T>
void sum_noalloc_impl(slk_plan plan, const T* y, int64_t M, int64_t ldy, T* s, unsigned char* scratch,
                      cudaStream_t st) {
    const int P = plan->P, d = plan->d;
    unsigned char* cur = scratch;
    T* Zy = reinterpret_cast<T*>(cur);
    cur += align256(sizeof(T) * static_cast<size_t>(P) * M);
    double* acc = reinterpret_cast<double*>(cur);
    cur += align256(sizeof(double) * M);
    bool projected = false;
    if constexpr (sizeof(T) == 4) {
        if (plan->tc) {
            const int split = plan->tc == 2;
            const size_t b16 = align256(static_cast<size_t>(M) * umma_operand_ld(d) * 2);
            unsigned char* xa = cur;
            unsigned char* xl = split ? cur + b16 : nullptr;
            launch_center_cast(y, M, d, ldy, plan->mu32.get(), xa, xl, split, st);
            launch_project_umma(xa, xl, M, plan->xib.get(), plan->xib_lo.get(), P, d, split, Zy, M, nullptr,
                                plan->err_dev.get(), st);
            projected = true;
        }
    }
    if (!projected) launch_project_simt<T>(xi_of<T>(plan), P, y, M, d, ldy, mu_of<T>(plan), Zy, M, st);
    // the array keeps the previous call's contents: the accumulator must start at zero
    SLK_CHECK_CUDA(cudaMemsetAsync(acc, 0, sizeof(double) * M, st));
    target_side<T>(plan, Zy, M, acc, static_cast<T*>(nullptr), 0, st);
    launch_finalize<T>(acc, s, M, 1.0 / P, st);
}

}  // namespace

extern "C" slk_status slk_sum_noalloc(slk_plan plan, const void* y, int64_t M, int64_t ldy, void* s, void* stream) {
    set_last_error("");
    return guarded([&] {
        SLK_REQUIRE(plan, "plan is NULL");
        slk_status prev = collect(plan, false);
        if (prev != SLK_OK) throw Error{prev, slk_last_error()};
        SLK_REQUIRE(M >= 0, "M must be >= 0");
        if (M == 0) return;
        SLK_REQUIRE(y && s, "y and s must not be NULL");
        SLK_REQUIRE(ldy >= plan->d, "ldy must be >= d");
        SLK_REQUIRE(is_device_pointer(y) && is_device_pointer(s),
                    "slk_sum_noalloc needs device pointers for y and s (host arrays would need staging buffers)");
        const size_t need = plan->f64 ? noalloc_bytes<double>(plan, M) : noalloc_bytes<float>(plan, M);
        if (need > kNoAllocScratchBytes)
            fail(SLK_ERR_INVALID,
                 "slk_sum_noalloc: %lld targets x %d slices need %zu bytes of working memory, more than the %zu-byte "
                 "scratch array; split the targets into smaller calls",
                 static_cast<long long>(M), plan->P, need, kNoAllocScratchBytes);
        int dev = 0;
        SLK_CHECK_CUDA(cudaGetDevice(&dev));
        SLK_REQUIRE(dev == plan->device, "the current device is not the plan's device");
        unsigned char* scratch = noalloc_scratch(dev);
        cudaStream_t st = static_cast<cudaStream_t>(stream);
        if (plan->f64)
            sum_noalloc_impl<double>(plan, static_cast<const double*>(y), M, ldy, static_cast<double*>(s), scratch, st);
        else
            sum_noalloc_impl<float>(plan, static_cast<const float*>(y), M, ldy, static_cast<float*>(s), scratch, st);
        finish_call(plan, st);
        plan->stream = st;
    });
}

extern "C" int64_t slk_device_alloc_count(void) { return slk::g_dev_allocs.load(); }
