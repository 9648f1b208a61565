// Fast Fourier summation on every slice (Section 3.1).
//
// Notation: a projected point z (source or target) of slice p is rescaled to
// x~ = z / L in the periodic cell [-1/2, 1/2) (paragraph "Rescaling" of
// Section 3.1, read as x~ = (z - c) / L with the centre c = 0 after the
// projections were centred).  The 1-D sum on a slice is
//     t(y~) = sum_{k in C} c_k w^_k exp(2 pi i k y~),   w^_k = sum_n w_n exp(-2 pi i k x~_n).
//
// NDFT ("plain" method): w^_k directly for the significant band of k.
// NFFT (remark on the non-equispaced FFT): spread the weights onto an
// oversampled grid of n_g cells with the "exponential of semicircle" window
//     psi(s) = exp(beta (sqrt(1 - (2 s / m)^2) - 1)),  |s| <= m/2  (s in cells),
// FFT, multiply by c_k / Psi(k/n_g)^2 (Psi = Fourier transform of psi), inverse
// FFT, then interpolate with the same window.
//
// Because the projected data occupy only |z| <= R << L/2, only the grid cells
// [win_base, win_base + W) that a window can touch are stored.
#include <type_traits>

#include "kernels.cuh"

namespace slk {

namespace {

constexpr int NDFT_KC = 16;       // k values accumulated per pass (registers)
constexpr int NDFT_CHUNK = 32768;  // sources per block in the NDFT reduction
constexpr int NDFT_KMAX = 64;     // largest band the NDFT kernels take
constexpr int SPREAD_NARROW_W = 64;
constexpr int SPREAD_WARPS = 8;
constexpr int SPREAD_CHUNK = 4096;  // sources per warp in the narrow spread

// psi(s) = exp(beta (sqrt(1 - x^2) - 1)) = exp(-beta x^2 / (1 + sqrt(1 - x^2))), x = 2 s / m,
// and 0 for |x| > 1.  The second form has no cancellation near x = 0 (where the first loses
// beta times the rounding of the square root); FP32 takes the square root as q rsqrt(q) and
// the exponential as exp2 of the exponent times log2(e).
__device__ inline float es_window(float s, float two_over_m, float beta) {
    const float x = s * two_over_m;
    const float x2 = x * x;
    const float q = 1.0f - x2;
    if (!(q >= 0.0f)) return 0.0f;
    const float r = q > 0.0f ? q * rsqrtf(q) : 0.0f;
    return exp2f((-beta * 1.44269504088896341f) * __fdividef(x2, 1.0f + r));
}
__device__ inline double es_window(double s, double two_over_m, double beta) {
    const double x = s * two_over_m;
    const double x2 = x * x;
    const double q = 1.0 - x2;
    if (!(q >= 0.0)) return 0.0;
    return exp(-beta * x2 / (1.0 + sqrt(q)));
}

// derivative of psi with respect to s
template <class T>
__device__ inline T es_window_deriv(T s, T two_over_m, T beta) {
    T x = s * two_over_m;
    T q = T(1) - x * x;
    if (q <= T(1e-6)) return T(0);
    T r = sqrt(q);
    return exp(beta * (r - T(1))) * beta * (-x * two_over_m) / r;
}

// The weights of all MM taps of a point whose first window cell lies at s0 (FP32: g =
// s0 + (MM - 1) / 2 in [-1/2, 1/2), the plan's even/odd tap polynomials, two taps from one
// evaluation of E_t and O_t; FP64: psi itself).  DERIV: the derivatives d psi / ds instead.
template <int MM, bool DERIV>
__device__ __forceinline__ void window_taps(const WinPoly& wp, float s0, float, float, float (&wt)[MM]) {
    const float g = s0 + 0.5f * static_cast<float>(MM - 1), h = g * g;
#pragma unroll
    for (int t = 0; t < (MM + 1) / 2; ++t) {
        float e, o;
        if (DERIV) {
            e = fmaf(fmaf(fmaf(wp.de[t][3], h, wp.de[t][2]), h, wp.de[t][1]), h, wp.de[t][0]);
            o = fmaf(fmaf(fmaf(wp.dq[t][3], h, wp.dq[t][2]), h, wp.dq[t][1]), h, wp.dq[t][0]);
        } else {
            e = fmaf(fmaf(fmaf(fmaf(wp.ev[t][4], h, wp.ev[t][3]), h, wp.ev[t][2]), h, wp.ev[t][1]), h, wp.ev[t][0]);
            o = fmaf(fmaf(fmaf(wp.od[t][3], h, wp.od[t][2]), h, wp.od[t][1]), h, wp.od[t][0]);
        }
        const float go = g * o;
        wt[t] = e + go;
        if (MM - 1 - t != t) wt[MM - 1 - t] = DERIV ? go - e : e - go;
    }
}
// One tap at a time by Horner's rule on the same polynomials (tap t >= ceil(MM / 2) as the
// mirrored tap at -g): more multiply-adds than window_taps, but each tap's chain interleaves
// with the use of its weight (the interpolation reads a grid value per tap).
template <int MM, bool DERIV>
__device__ __forceinline__ float window_tap(const WinPoly& wp, int t, float g) {
    const bool mirror = t >= (MM + 1) / 2;
    const int u = mirror ? MM - 1 - t : t;
    const float x = mirror ? -g : g;
    float v;
    if (DERIV) {
        v = wp.dq[u][3];
        v = fmaf(v, x, wp.de[u][3]);
        v = fmaf(v, x, wp.dq[u][2]);
        v = fmaf(v, x, wp.de[u][2]);
        v = fmaf(v, x, wp.dq[u][1]);
        v = fmaf(v, x, wp.de[u][1]);
        v = fmaf(v, x, wp.dq[u][0]);
        v = fmaf(v, x, wp.de[u][0]);
        return mirror ? -v : v;
    }
    v = wp.ev[u][4];
    v = fmaf(v, x, wp.od[u][3]);
    v = fmaf(v, x, wp.ev[u][3]);
    v = fmaf(v, x, wp.od[u][2]);
    v = fmaf(v, x, wp.ev[u][2]);
    v = fmaf(v, x, wp.od[u][1]);
    v = fmaf(v, x, wp.ev[u][1]);
    v = fmaf(v, x, wp.od[u][0]);
    return fmaf(v, x, wp.ev[u][0]);
}
template <int MM, bool DERIV>
__device__ __forceinline__ double window_tap(const WinPoly&, int t, double s0, double two_over_m, double beta) {
    return DERIV ? es_window_deriv(s0 + double(t), two_over_m, beta) : es_window(s0 + double(t), two_over_m, beta);
}

// tap t's weight (or derivative) for a point whose first window cell lies at s0
template <int MM, bool DERIV>
__device__ __forceinline__ float tap_value(const WinPoly& wp, int t, float s0, float, float) {
    return window_tap<MM, DERIV>(wp, t, s0 + 0.5f * static_cast<float>(MM - 1));
}
template <int MM, bool DERIV>
__device__ __forceinline__ double tap_value(const WinPoly& wp, int t, double s0, double two_over_m, double beta) {
    return window_tap<MM, DERIV>(wp, t, s0, two_over_m, beta);
}

template <int MM, bool DERIV>
__device__ __forceinline__ void window_taps(const WinPoly&, double s0, double two_over_m, double beta,
                                            double (&wt)[MM]) {
#pragma unroll
    for (int t = 0; t < MM; ++t)
        wt[t] = DERIV ? es_window_deriv(s0 + double(t), two_over_m, beta) : es_window(s0 + double(t), two_over_m, beta);
}

template <class T>
__device__ inline T warp_sum(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// fixed-order sum of one value per thread of a 256-thread block; result valid in thread 0
template <class T>
__device__ inline T block_sum_256(T v, T* red) {
    v = warp_sum(v);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    T r = T(0);
    if (threadIdx.x == 0)
        for (int i = 0; i < 8; ++i) r += red[i];
    return r;
}

// compensated (Kahan) accumulation for the FP32 slice average
struct KahanF {
    float s = 0.f, c = 0.f;
    __device__ void add(float v) {
        float y = v - c;
        float t = s + y;
        c = (t - s) - y;
        s = t;
    }
    __device__ double value() const { return static_cast<double>(s) - static_cast<double>(c); }
};
struct KahanD {
    double s = 0.0;
    __device__ void add(double v) { s += v; }
    __device__ double value() const { return s; }
};
template <class T> struct Acc;
template <> struct Acc<float> { using type = KahanF; };
template <> struct Acc<double> { using type = KahanD; };

// ------------------------------------------------------------ NDFT source

// Phases in units of pi: with s = 2 z / L, exp(-2 pi i k z / L) = cospi(k s) - i sinpi(k s)
// (exact argument reduction); consecutive k by the recurrence e^{-i(k+1)th} = e^{-ik th} e^{-i th}.
__device__ inline void sincospi_t(float x, float* s, float* c) { sincospif(x, s, c); }
__device__ inline void sincospi_t(double x, double* s, double* c) { sincospi(x, s, c); }

// One block: slice p, sources [chunk * NDFT_CHUNK, ...).  Each thread accumulates the K band
// sums (and sum w for k = 0) in registers; warp shuffles, then one shared-memory pass.
template <class T, int KMAX>
__global__ void __launch_bounds__(256) k_ndft_source(const T* __restrict__ Z, int64_t n, int64_t ldz,
                                                     const T* __restrict__ w, T two_over_L, int k_lo, int K,
                                                     int has_k0, T* __restrict__ partial, int P) {
    __shared__ T red[8][2 * KMAX + 1];
    const int p = blockIdx.y;
    const int64_t i0 = static_cast<int64_t>(blockIdx.x) * NDFT_CHUNK;
    const int64_t i1 = (i0 + NDFT_CHUNK < n) ? i0 + NDFT_CHUNK : n;
    const T* zr = Z + static_cast<int64_t>(p) * ldz;
    T re[KMAX], im[KMAX], a0 = T(0);
#pragma unroll
    for (int j = 0; j < KMAX; ++j) re[j] = im[j] = T(0);
    for (int64_t i = i0 + threadIdx.x; i < i1; i += 256) {
        const T wv = w[i];
        const T s = zr[i] * two_over_L;
        T sb, cb, s1, c1;
        sincospi_t(T(k_lo) * s, &sb, &cb);
        sincospi_t(s, &s1, &c1);
        T cr = cb, ci = -sb;
#pragma unroll
        for (int j = 0; j < KMAX; ++j) {
            if (j < K) {
                re[j] = fma(wv, cr, re[j]);
                im[j] = fma(wv, ci, im[j]);
                const T nr = cr * c1 + ci * s1;
                const T ni = ci * c1 - cr * s1;
                cr = nr;
                ci = ni;
            }
        }
        a0 += wv;
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int j = 0; j < KMAX; ++j) {
        if (j < K) {
            const T r = warp_sum(re[j]), m = warp_sum(im[j]);
            if (lane == 0) {
                red[warp][2 * j] = r;
                red[warp][2 * j + 1] = m;
            }
        }
    }
    {
        const T a = warp_sum(a0);
        if (lane == 0) red[warp][2 * KMAX] = a;
    }
    __syncthreads();
    const int stride = 2 * K + 1;
    T* out = partial + (static_cast<int64_t>(blockIdx.x) * P + p) * stride;
    for (int v = threadIdx.x; v < stride; v += blockDim.x) {
        const int src = v < 2 * K ? v : 2 * KMAX;
        T acc = T(0);
        for (int q = 0; q < 8; ++q) acc += red[q][src];
        out[v] = has_k0 || v < 2 * K ? acc : T(0);
    }
}

// cw[p][j] = c_{k_lo + j} * sum over chunks (fixed order); cw0[p] = c_0 sum w
template <class T>
__global__ void k_ndft_reduce(const T* __restrict__ partial, int nchunk, int P, int K, int has_k0,
                              const double* __restrict__ coef, Cplx<T>* __restrict__ cw, T* __restrict__ cw0) {
    const int stride = 2 * K + 1;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < P * (K + 1); t += gridDim.x * blockDim.x) {
        int p = t / (K + 1), j = t % (K + 1);
        if (j == K) {
            double a = 0.0;
            for (int c = 0; c < nchunk; ++c) a += static_cast<double>(partial[(static_cast<int64_t>(c) * P + p) * stride + 2 * K]);
            cw0[p] = has_k0 ? static_cast<T>(coef[K] * a) : T(0);
        } else {
            double r = 0.0, m = 0.0;
            for (int c = 0; c < nchunk; ++c) {
                const T* q = partial + (static_cast<int64_t>(c) * P + p) * stride;
                r += static_cast<double>(q[2 * j]);
                m += static_cast<double>(q[2 * j + 1]);
            }
            cw[static_cast<int64_t>(p) * K + j] = Cplx<T>{static_cast<T>(coef[j] * r), static_cast<T>(coef[j] * m)};
        }
    }
}

// ------------------------------------------------------------ NDFT target

// One thread per target: t_p(z) = 2 Re sum_j cw[p][j] e^{+i (k_lo + j) th} + cw0[p] for every
// slice, averaged into acc[m]; GRAD writes dt_p/dz into G[p * ldg + m] instead.
template <class T, int KMAX, bool GRAD>
__global__ void __launch_bounds__(256) k_ndft_target(const T* __restrict__ Z, int P, int64_t n, int64_t ldz,
                                                     T two_over_L, int k_lo, int K, const Cplx<T>* __restrict__ cw,
                                                     const T* __restrict__ cw0, int slice_chunk, T R,
                                                     double* __restrict__ acc, T* __restrict__ G, int64_t ldg,
                                                     unsigned* __restrict__ err) {
    extern __shared__ unsigned char smem_raw[];
    Cplx<T>* scw = reinterpret_cast<Cplx<T>*>(smem_raw);
    T* scw0 = reinterpret_cast<T*>(scw + static_cast<size_t>(slice_chunk) * K);
    const int64_t m = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    const T two_pi_over_L = two_over_L * T(3.141592653589793238462643383279);
    typename Acc<T>::type sum;
    bool bad = false;
    for (int p0 = 0; p0 < P; p0 += slice_chunk) {
        const int pc = (P - p0 < slice_chunk) ? P - p0 : slice_chunk;
        __syncthreads();
        for (int e = threadIdx.x; e < pc * K; e += blockDim.x) scw[e] = cw[static_cast<int64_t>(p0) * K + e];
        for (int e = threadIdx.x; e < pc; e += blockDim.x) scw0[e] = cw0[p0 + e];
        __syncthreads();
        if (m >= n) continue;
        for (int q = 0; q < pc; ++q) {
            const int p = p0 + q;
            const T z = Z[static_cast<int64_t>(p) * ldz + m];
            if (!(z <= R && z >= -R)) bad = true;  // outside the certified window (or NaN)
            const T s = z * two_over_L;
            T sb, cb, s1, c1;
            sincospi_t(T(k_lo) * s, &sb, &cb);
            sincospi_t(s, &s1, &c1);
            T cr = cb, ci = sb;  // e^{+i k th}
            T t = T(0), dt = T(0);
            const Cplx<T>* row = scw + static_cast<size_t>(q) * K;
#pragma unroll
            for (int j = 0; j < KMAX; ++j) {
                if (j < K) {
                    const Cplx<T> a = row[j];
                    if (GRAD) dt -= T(k_lo + j) * (a.re * ci + a.im * cr);  // d/dth Re(a e^{ik th})
                    else t += a.re * cr - a.im * ci;                        // Re(a e^{ik th})
                    const T nr = cr * c1 - ci * s1;
                    const T ni = ci * c1 + cr * s1;
                    cr = nr;
                    ci = ni;
                }
            }
            // th = 2 pi z / L: dt_p/dz = 2 * dt * 2 pi / L
            if (GRAD) G[p * ldg + m] = T(2) * dt * two_pi_over_L;
            else sum.add(T(2) * t + scw0[q]);
        }
    }
    if (bad) atomicOr(err, 4u);
    if (!GRAD && m < n) acc[m] += sum.value();
}

// The same evaluation for few targets, where one thread per target would occupy only a
// handful of SMs: one warp per target, lane l taking the slices p = l, l + 32, ...; each
// lane sums its slices (compensated for FP32), then the 32 lane sums are added in a fixed
// butterfly order, so the result does not depend on scheduling.
template <class T, int KMAX, bool GRAD>
__global__ void __launch_bounds__(256) k_ndft_target_warp(const T* __restrict__ Z, int P, int64_t n, int64_t ldz,
                                                          T two_over_L, int k_lo, int K,
                                                          const Cplx<T>* __restrict__ cw, const T* __restrict__ cw0,
                                                          T R, double* __restrict__ acc, T* __restrict__ G, int64_t ldg,
                                                          unsigned* __restrict__ err) {
    const int lane = threadIdx.x & 31;
    const int64_t m = (static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
    if (m >= n) return;  // m is the same for the whole warp
    const T two_pi_over_L = two_over_L * T(3.141592653589793238462643383279);
    typename Acc<T>::type sum;
    bool bad = false;
    for (int p = lane; p < P; p += 32) {
        const T z = Z[static_cast<int64_t>(p) * ldz + m];
        if (!(z <= R && z >= -R)) bad = true;  // outside the certified window (or NaN)
        const T s = z * two_over_L;
        T sb, cb, s1, c1;
        sincospi_t(T(k_lo) * s, &sb, &cb);
        sincospi_t(s, &s1, &c1);
        T cr = cb, ci = sb;  // e^{+i k th}
        T t = T(0), dt = T(0);
        const Cplx<T>* row = cw + static_cast<int64_t>(p) * K;
#pragma unroll
        for (int j = 0; j < KMAX; ++j) {
            if (j < K) {
                const Cplx<T> a = row[j];
                if (GRAD) dt -= T(k_lo + j) * (a.re * ci + a.im * cr);
                else t += a.re * cr - a.im * ci;
                const T nr = cr * c1 - ci * s1;
                const T ni = ci * c1 + cr * s1;
                cr = nr;
                ci = ni;
            }
        }
        if (GRAD) G[p * ldg + m] = T(2) * dt * two_pi_over_L;
        else sum.add(T(2) * t + cw0[p]);
    }
    if (bad) atomicOr(err, 4u);
    if (!GRAD) {
        double v = sum.value();
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0) acc[m] += v;
    }
}

// ------------------------------------------------------------ Chebyshev evaluation

// One source's contribution w T_j(u), j < QMAX, to the moments (Chebyshev recurrence
// T_{j+1} = 2u T_j - T_{j-1}).
template <class T, int QMAX>
__device__ __forceinline__ void cheb_accumulate(T (&mu)[QMAX], T wv, T u) {
    const T u2 = u + u;
    T tm1 = T(1), t = u;  // T_0, T_1
    mu[0] += wv;
#pragma unroll
    for (int j = 1; j < QMAX; ++j) {
        mu[j] = fma(wv, t, mu[j]);
        const T tn = fma(u2, t, -tm1);
        tm1 = t;
        t = tn;
    }
}

// Source side: mu[p][j] = sum_n w_n T_j(z_{p,n} / R), j < q; per-thread registers, warp
// shuffles, one shared pass.  VEC: FP32 rows 16-byte aligned, read four sources per load.
template <class T, int QMAX, bool VEC>
__global__ void __launch_bounds__(256) k_cheb_moments(const T* __restrict__ Z, int64_t n, int64_t ldz,
                                                      const T* __restrict__ w, T inv_R, int q, T* __restrict__ partial,
                                                      int P) {
    __shared__ T red[8][QMAX];
    const int p = blockIdx.y;
    const int64_t i0 = static_cast<int64_t>(blockIdx.x) * NDFT_CHUNK;
    const int64_t i1 = (i0 + NDFT_CHUNK < n) ? i0 + NDFT_CHUNK : n;
    const T* zr = Z + static_cast<int64_t>(p) * ldz;
    T mu[QMAX];
#pragma unroll
    for (int j = 0; j < QMAX; ++j) mu[j] = T(0);
    int64_t rest = i0;  // first source left for the scalar loop
    if constexpr (VEC && sizeof(T) == 4) {
        // two float4 groups per step: eight sources whose loads are issued together
        const int64_t nv = (i1 - i0) >> 2;
        const float4* z4 = reinterpret_cast<const float4*>(zr + i0);
        const float4* w4 = reinterpret_cast<const float4*>(w + i0);
        for (int64_t g = threadIdx.x; g < nv; g += 512) {
            float4 zz[2], ww[2];
#pragma unroll
            for (int r = 0; r < 2; ++r) {
                const int64_t gi = g + r * 256;
                zz[r] = gi < nv ? z4[gi] : make_float4(0.f, 0.f, 0.f, 0.f);
                ww[r] = gi < nv ? w4[gi] : make_float4(0.f, 0.f, 0.f, 0.f);
            }
#pragma unroll
            for (int r = 0; r < 2; ++r) {
                cheb_accumulate<T, QMAX>(mu, ww[r].x, zz[r].x * inv_R);
                cheb_accumulate<T, QMAX>(mu, ww[r].y, zz[r].y * inv_R);
                cheb_accumulate<T, QMAX>(mu, ww[r].z, zz[r].z * inv_R);
                cheb_accumulate<T, QMAX>(mu, ww[r].w, zz[r].w * inv_R);
            }
        }
        rest = i0 + 4 * nv;
    }
    // four sources per step: their loads are issued together (memory-level parallelism)
    constexpr int U = 4;
    for (int64_t ib = rest + threadIdx.x; ib < i1; ib += 256 * U) {
        T wv[U], u[U];
#pragma unroll
        for (int r = 0; r < U; ++r) {
            const int64_t i = ib + static_cast<int64_t>(r) * 256;
            wv[r] = i < i1 ? w[i] : T(0);
            u[r] = i < i1 ? zr[i] * inv_R : T(0);
        }
#pragma unroll
        for (int r = 0; r < U; ++r) cheb_accumulate<T, QMAX>(mu, wv[r], u[r]);
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int j = 0; j < QMAX; ++j) {
        const T v = warp_sum(mu[j]);
        if (lane == 0) red[warp][j] = v;
    }
    __syncthreads();
    for (int j = threadIdx.x; j < q; j += blockDim.x) {
        T acc = T(0);
        for (int r = 0; r < 8; ++r) acc += red[r][j];
        partial[(static_cast<int64_t>(blockIdx.x) * P + p) * q + j] = acc;
    }
}

// beta[p][l] = sum_j M[l][j] mu[p][j], mu summed over chunks in a fixed order (FP64);
// optionally the monomial form of the same polynomial (q <= 16, see launch_cheb_source).
template <class T, class TP = T>
__global__ void k_cheb_reduce(const TP* __restrict__ partial, int nchunk, int P, int q, const double* __restrict__ M,
                              T* __restrict__ beta, T* __restrict__ mono, unsigned* __restrict__ mono_bad,
                              double mono_ratio) {
    extern __shared__ double smu[];  // mu[q], then beta[q]
    double* sbeta = smu + q;
    const int p = blockIdx.x;
    for (int j = threadIdx.x; j < q; j += blockDim.x) {
        double a = 0.0;
        for (int c = 0; c < nchunk; ++c) a += static_cast<double>(partial[(static_cast<int64_t>(c) * P + p) * q + j]);
        smu[j] = a;
    }
    __syncthreads();
    for (int l = threadIdx.x; l < q; l += blockDim.x) {
        double a = 0.0;
        for (int j = 0; j < q; ++j) a += M[static_cast<int64_t>(l) * q + j] * smu[j];
        sbeta[l] = a;
        beta[static_cast<int64_t>(p) * q + l] = static_cast<T>(a);
    }
    if (mono == nullptr) return;
    __syncthreads();
    if (threadIdx.x == 0) {
        // coefficients of T_l in powers of u from T_{l+1} = 2u T_l - T_{l-1} (integers, exact)
        double a[16], tm[16], tc[16], tn[16];
        double sb = 0.0;
        for (int k = 0; k < 16; ++k) a[k] = tm[k] = tc[k] = 0.0;
        tm[0] = 1.0;  // T_0
        tc[1] = 1.0;  // T_1
        for (int l = 0; l < q && l < 16; ++l) {
            const double* t = l == 0 ? tm : tc;
            if (l >= 2) {
                for (int k = 0; k < 16; ++k) tn[k] = (k ? 2.0 * tc[k - 1] : 0.0) - tm[k];
                for (int k = 0; k < 16; ++k) {
                    tm[k] = tc[k];
                    tc[k] = tn[k];
                }
                t = tc;
            }
            for (int k = 0; k <= l; ++k) a[k] += sbeta[l] * t[k];
            sb += fabs(sbeta[l]);
        }
        double sa = 0.0;
        for (int k = 0; k < q && k < 16; ++k) {
            sa += fabs(a[k]);
            mono[static_cast<int64_t>(p) * q + k] = static_cast<T>(a[k]);
        }
        if (q > 16 || !(sa <= mono_ratio * sb)) atomicOr(mono_bad, 1u);
    }
}

// Target side: t_p(z) = sum_l beta[p][l] T_l(z / R) by Clenshaw's recurrence, summed over
// slices into acc[m]; GRAD writes dt_p/dz = (1/R) sum_l l beta_l U_{l-1}(v) into G[p * ldg + m].
template <class T, int QMAX, bool GRAD, bool HORNER>
__global__ void __launch_bounds__(256) k_cheb_target(const T* __restrict__ Z, int P, int64_t n, int64_t ldz, T inv_R,
                                                     int q, const T* __restrict__ beta, int slice_chunk, T R,
                                                     double* __restrict__ acc, T* __restrict__ G, int64_t ldg,
                                                     unsigned* __restrict__ err) {
    extern __shared__ unsigned char smem_raw[];
    T* sb = reinterpret_cast<T*>(smem_raw);
    const int64_t m = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    typename Acc<T>::type sum;
    bool bad = false;
    for (int p0 = 0; p0 < P; p0 += slice_chunk) {
        const int pc = (P - p0 < slice_chunk) ? P - p0 : slice_chunk;
        __syncthreads();
        for (int e = threadIdx.x; e < pc * q; e += blockDim.x) sb[e] = beta[static_cast<int64_t>(p0) * q + e];
        __syncthreads();
        if (m >= n) continue;
        // four slices per step: their loads are issued together (memory-level parallelism)
        constexpr int U = 4;
        for (int s0 = 0; s0 < pc; s0 += U) {
        T zz[U];
#pragma unroll
        for (int r = 0; r < U; ++r) zz[r] = s0 + r < pc ? Z[static_cast<int64_t>(p0 + s0 + r) * ldz + m] : T(0);
#pragma unroll
        for (int r = 0; r < U; ++r) {
            const int s = s0 + r;
            if (s >= pc) break;
            const int p = p0 + s;
            const T z = zz[r];
            if (!(z <= R && z >= -R)) bad = true;  // outside the certified window (or NaN)
            const T v = z * inv_R, v2 = v + v;
            const T* b = sb + static_cast<size_t>(s) * q;
            T b1 = T(0), b2 = T(0);
            if (GRAD) {
                // sum_{n < q-1} (n+1) beta_{n+1} U_n(v):  Clenshaw for U (result b_0)
#pragma unroll
                for (int k = QMAX - 2; k >= 0; --k) {
                    const T bk = fma(v2, b1, T(k + 1) * b[k + 1] - b2);
                    b2 = b1;
                    b1 = bk;
                }
                G[p * ldg + m] = b1 * inv_R;
            } else if (HORNER) {
                // b holds the monomial coefficients
                T r = b[QMAX - 1];
#pragma unroll
                for (int k = QMAX - 2; k >= 0; --k) r = fma(r, v, b[k]);
                sum.add(r);
            } else {
#pragma unroll
                for (int k = QMAX - 1; k >= 1; --k) {
                    const T bk = fma(v2, b1, b[k] - b2);
                    b2 = b1;
                    b1 = bk;
                }
                sum.add(fma(v, b1, b[0] - b2));
            }
        }
        }
    }
    if (bad) atomicOr(err, 4u);
    if (!GRAD && m < n) acc[m] += sum.value();
}

// ------------------------------------------------------------ NFFT spread

// Narrow window (W <= 64): lane = slice, every lane keeps a private window in
// shared memory laid out [cell][lane] (conflict-free), warps split the sources.
template <class T>
__global__ void __launch_bounds__(256) k_spread_narrow(const T* __restrict__ Z, int P, int64_t n, int64_t ldz,
                                                       const T* __restrict__ w, T scale_u, int m, T two_over_m, T beta,
                                                       int W, int win_base, T* __restrict__ partial,
                                                       unsigned* __restrict__ err) {
    extern __shared__ unsigned char smem_raw[];
    T* win = reinterpret_cast<T*>(smem_raw);  // [SPREAD_WARPS][W][32]
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int p = blockIdx.y * 32 + lane;
    T* mine = win + static_cast<size_t>(warp) * W * 32;
    for (int r = 0; r < W; ++r) mine[r * 32 + lane] = T(0);
    const int64_t i0 = (static_cast<int64_t>(blockIdx.x) * SPREAD_WARPS + warp) * SPREAD_CHUNK;
    const int64_t i1 = (i0 + SPREAD_CHUNK < n) ? i0 + SPREAD_CHUNK : n;
    const T half_m = T(0.5) * T(m);
    bool bad = false;
    if (p < P) {
        const T* zr = Z + static_cast<int64_t>(p) * ldz;
        for (int64_t i = i0; i < i1; ++i) {
            const T u = zr[i] * scale_u;  // grid coordinate n_g z / L
            const T wv = w[i];
            const T c0 = ceil(u - half_m);
            const int r0 = static_cast<int>(c0) - win_base;
            if (r0 < 0 || r0 + m > W) {
                bad = true;
                continue;
            }
            T s = c0 - u;
            for (int t = 0; t < m; ++t, s += T(1)) mine[(r0 + t) * 32 + lane] += wv * es_window(s, two_over_m, beta);
        }
    }
    if (bad) atomicOr(err, 1u);
    __syncthreads();
    // fixed-order reduction over the warps of the block
    for (int e = threadIdx.x; e < W * 32; e += blockDim.x) {
        T v = T(0);
        for (int q = 0; q < SPREAD_WARPS; ++q) v += win[static_cast<size_t>(q) * W * 32 + e];
        const int r = e / 32, l = e % 32;
        const int pp = blockIdx.y * 32 + l;
        if (pp < P) partial[(static_cast<int64_t>(blockIdx.x) * P + pp) * W + r] = v;
    }
}

// Wide window: one slice per block row, a block-shared window with shared
// atomics (sources spread over many cells, little contention).
template <class T, int MMAX>
__global__ void __launch_bounds__(256) k_spread_wide(const T* __restrict__ Z, int P, int64_t n, int64_t ldz,
                                                     const T* __restrict__ w, T scale_u, int m, T two_over_m, T beta, const WinPoly wp,
                                                     int W, int win_base, int64_t chunk, T* __restrict__ partial,
                                                     unsigned* __restrict__ err) {
    extern __shared__ unsigned char smem_raw[];
    T* win = reinterpret_cast<T*>(smem_raw);
    const int p = blockIdx.y;
    for (int r = threadIdx.x; r < W; r += blockDim.x) win[r] = T(0);
    __syncthreads();
    const int64_t i0 = static_cast<int64_t>(blockIdx.x) * chunk;
    const int64_t i1 = (i0 + chunk < n) ? i0 + chunk : n;
    const T* zr = Z + static_cast<int64_t>(p) * ldz;
    const T half_m = T(0.5) * T(m);
    bool bad = false;
    for (int64_t i = i0 + threadIdx.x; i < i1; i += blockDim.x) {
        const T u = zr[i] * scale_u;
        const T wv = w[i];
        const T c0 = ceil(u - half_m);
        const int r0 = static_cast<int>(c0) - win_base;
        if (r0 < 0 || r0 + m > W) {
            bad = true;
            continue;
        }
        T wt[MMAX];
        window_taps<MMAX, false>(wp, c0 - u, two_over_m, beta, wt);
#pragma unroll
        for (int t = 0; t < MMAX; ++t)
            if (t < m) atomicAdd(&win[r0 + t], wv * wt[t]);
    }
    if (bad) atomicOr(err, 1u);
    __syncthreads();
    for (int r = threadIdx.x; r < W; r += blockDim.x)
        partial[(static_cast<int64_t>(blockIdx.x) * P + p) * W + r] = win[r];
}

// Spreading from sources grouped by key bucket (the sorting route's pairs: (key, w)
// interleaved, slice p's n pairs at pairs + 2 p n, buckets much narrower than a grid cell,
// so the pairs ascend in grid cell).  Each lane walks its warp's share of the block's chunk
// with stride 32 (coalesced loads); its points then stay in one window position for long
// runs, so it accumulates the m taps in registers and adds them to the block's shared window
// only when the position changes (and at the end).  Any order is correct; the grouping only
// makes the shared-memory additions rare.
template <class T, int MMAX>
__global__ void __launch_bounds__(256) k_spread_sorted(const T* __restrict__ pairs, int64_t n, T scale_u, int m,
                                                       T two_over_m, T beta, const WinPoly wp, int W, int win_base,
                                                       int64_t chunk, T* __restrict__ partial,
                                                       unsigned* __restrict__ err) {
    extern __shared__ unsigned char smem_raw[];
    T* win = reinterpret_cast<T*>(smem_raw);
    const int p = blockIdx.y, P = gridDim.y;
    for (int r = threadIdx.x; r < W; r += blockDim.x) win[r] = T(0);
    __syncthreads();
    const int64_t i0 = static_cast<int64_t>(blockIdx.x) * chunk;
    const int64_t i1 = (i0 + chunk < n) ? i0 + chunk : n;
    const T* kw = pairs + 2 * static_cast<int64_t>(p) * n;
    const T half_m = T(0.5) * T(m);
    T acc[MMAX];
#pragma unroll
    for (int t = 0; t < MMAX; ++t) acc[t] = T(0);
    int cur = -1;
    bool bad = false;
    // warp w takes the w-th eighth of the chunk, its lanes every 32nd pair of it: loads stay
    // coalesced and a lane's successive points are only 32 apart in key order
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t per_warp = chunk / (blockDim.x >> 5);
    const int64_t w0 = i0 + warp * per_warp;
    const int64_t w1 = (w0 + per_warp < i1) ? w0 + per_warp : i1;
    for (int64_t i = w0 + lane; i < w1; i += 32) {
        const T key = kw[2 * i], wv = kw[2 * i + 1];
        const T u = key * scale_u;
        const T c0 = ceil(u - half_m);
        const int r0 = static_cast<int>(c0) - win_base;
        if (r0 < 0 || r0 + m > W) {
            bad = true;
            continue;
        }
        if (r0 != cur) {
            if (cur >= 0) {
#pragma unroll
                for (int t = 0; t < MMAX; ++t)
                    if (t < m) atomicAdd(&win[cur + t], acc[t]);
            }
#pragma unroll
            for (int t = 0; t < MMAX; ++t) acc[t] = T(0);
            cur = r0;
        }
        T wt[MMAX];
        window_taps<MMAX, false>(wp, c0 - u, two_over_m, beta, wt);
#pragma unroll
        for (int t = 0; t < MMAX; ++t)
            if (t < m) acc[t] = fma(wv, wt[t], acc[t]);
    }
    if (cur >= 0) {
#pragma unroll
        for (int t = 0; t < MMAX; ++t)
            if (t < m) atomicAdd(&win[cur + t], acc[t]);
    }
    if (bad) atomicOr(err, 1u);
    __syncthreads();
    for (int r = threadIdx.x; r < W; r += blockDim.x)
        partial[(static_cast<int64_t>(blockIdx.x) * P + p) * W + r] = win[r];
}

template <class T>
__global__ void k_window_reduce(const T* __restrict__ partial, int nchunk, int P, int W, T* __restrict__ g) {
    for (int64_t e = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; e < static_cast<int64_t>(P) * W;
         e += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        T v = T(0);
        for (int c = 0; c < nchunk; ++c) v += partial[static_cast<int64_t>(c) * P * W + e];
        g[e] = v;
    }
}

// ------------------------------------------------------------ FFT * multiply * IFFT

// In-place radix-2 FFT of n = 2^logn complex values in shared memory
// (bit-reversal permutation, then log2(n) butterfly stages); sign = -1 forward.
template <class T>
__device__ void smem_fft(Cplx<T>* a, int n, int logn, int sign) {
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        int j = __brev(static_cast<unsigned>(i)) >> (32 - logn);
        if (j > i) {
            Cplx<T> t = a[i];
            a[i] = a[j];
            a[j] = t;
        }
    }
    __syncthreads();
    for (int len = 2; len <= n; len <<= 1) {
        const int half = len >> 1;
        for (int b = threadIdx.x; b < (n >> 1); b += blockDim.x) {
            const int grp = b / half, pos = b % half;
            const int i = grp * len + pos, j = i + half;
            T s, c;
            // twiddle exp(sign 2 pi i pos / len)
            if constexpr (sizeof(T) == 4) sincospif(T(2) * T(pos) / T(len), &s, &c);
            else sincospi(T(2) * T(pos) / T(len), &s, &c);
            s *= T(sign);
            const Cplx<T> u = a[i], v = a[j];
            const T vr = v.re * c - v.im * s, vi = v.re * s + v.im * c;
            a[i] = Cplx<T>{u.re + vr, u.im + vi};
            a[j] = Cplx<T>{u.re - vr, u.im - vi};
        }
        __syncthreads();
    }
}

template <class T>
__global__ void __launch_bounds__(512) k_fft_multiply(const T* __restrict__ g, int P, int n_g, int logn, int W,
                                                      int win_base, int kmax, const double* __restrict__ mult,
                                                      T* __restrict__ h) {
    extern __shared__ unsigned char smem_raw[];
    Cplx<T>* a = reinterpret_cast<Cplx<T>*>(smem_raw);
    const int p = blockIdx.x;
    for (int j = threadIdx.x; j < n_g; j += blockDim.x) a[j] = Cplx<T>{T(0), T(0)};
    __syncthreads();
    for (int r = threadIdx.x; r < W; r += blockDim.x) {
        int j = (win_base + r) % n_g;
        if (j < 0) j += n_g;
        // several window cells can alias onto one grid cell only if W > n_g (excluded)
        a[j].re = g[static_cast<int64_t>(p) * W + r];
    }
    __syncthreads();
    smem_fft(a, n_g, logn, -1);
    for (int j = threadIdx.x; j < n_g; j += blockDim.x) {
        const int k = j < n_g / 2 ? j : j - n_g;
        const int ak = k < 0 ? -k : k;
        const T f = ak < kmax ? static_cast<T>(mult[ak]) : T(0);
        a[j].re *= f;
        a[j].im *= f;
    }
    __syncthreads();
    smem_fft(a, n_g, logn, +1);
    for (int r = threadIdx.x; r < W; r += blockDim.x) {
        int j = (win_base + r) % n_g;
        if (j < 0) j += n_g;
        h[static_cast<int64_t>(p) * W + r] = a[j].re;
    }
}

// ------------------------------------------------------------ NFFT interpolation

template <class T, int MMAX>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? 8 : 4) k_nfft_target(const T* __restrict__ Z, int P, int64_t n, int64_t ldz, T scale_u,
                                                     int m, T two_over_m, T beta, const WinPoly wp, int W, int win_base,
                                                     const T* __restrict__ h, int slice_chunk, T R,
                                                     double* __restrict__ acc, T* __restrict__ G, int64_t ldg,
                                                     unsigned* __restrict__ err) {
    extern __shared__ unsigned char smem_raw[];
    T* sh = reinterpret_cast<T*>(smem_raw);
    const int64_t mi = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    const T half_m = T(0.5) * T(m);
    typename Acc<T>::type sum;
    bool bad = false;
    for (int p0 = 0; p0 < P; p0 += slice_chunk) {
        const int pc = (P - p0 < slice_chunk) ? P - p0 : slice_chunk;
        __syncthreads();
        for (int e = threadIdx.x; e < pc * W; e += blockDim.x) sh[e] = h[static_cast<int64_t>(p0) * W + e];
        __syncthreads();
        if (mi >= n) continue;
        constexpr int U = 4;  // projections of four slices loaded together (memory-level parallelism)
        T zq[U];
        for (int q = 0; q < pc; ++q) {
            const int p = p0 + q;
            if (q % U == 0) {
#pragma unroll
                for (int r = 0; r < U; ++r) zq[r] = q + r < pc ? Z[static_cast<int64_t>(p + r) * ldz + mi] : T(0);
            }
            T z = zq[0];
#pragma unroll
            for (int r = 1; r < U; ++r)
                if (q % U == r) z = zq[r];
            if (!(z <= R && z >= -R)) bad = true;  // outside the certified window (or NaN)
            const T u = z * scale_u;
            const T c0 = ceil(u - half_m);
            const int r0 = static_cast<int>(c0) - win_base;
            if (r0 < 0 || r0 + m > W) {
                bad = true;
                continue;
            }
            const T* row = sh + static_cast<size_t>(q) * W + r0;
            const T s0 = c0 - u;
            T t = T(0);
            if (G) {
                // d/du sum_j h_j psi(u - j) = -sum_j h_j psi'(j - u)
#pragma unroll
                for (int k = 0; k < MMAX; ++k)
                    if (k < m) t -= row[k] * tap_value<MMAX, true>(wp, k, s0, two_over_m, beta);
                G[p * ldg + mi] = t * scale_u;
            } else {
#pragma unroll
                for (int k = 0; k < MMAX; ++k)
                    if (k < m) t = fma(row[k], tap_value<MMAX, false>(wp, k, s0, two_over_m, beta), t);
                sum.add(t);
            }
        }
    }
    if (bad) atomicOr(err, 4u);
    if (!G && mi < n) acc[mi] += sum.value();
}

// ------------------------------------------------------------ NFFT interpolation from a table

// FP32 plans: the interpolant sum_t h[r + t] P_t(g) on grid cell r (the window's first cell
// r + win_base) is itself a polynomial of degree kWinPolyDeg in g, with coefficients
// C[r][k] = sum_t h[r + t] a_t[k] (a_t the tap polynomials of WinPoly, the mirrored taps as
// a_{m-1-t}[k] = (-1)^k a_t[k]); one block per slice writes its ncell = W - m + 1 cells, 16
// floats per cell (9 used, 64-byte rows for aligned vector loads), summed in FP64.
constexpr int TAB_STRIDE = 16;

__global__ void __launch_bounds__(256) k_interp_table(const float* __restrict__ h, int W, int m, const WinPoly wp,
                                                      int ncell, float* __restrict__ tab) {
    const int p = blockIdx.x;
    const float* hp = h + static_cast<int64_t>(p) * W;
    float* tp = tab + static_cast<int64_t>(p) * ncell * TAB_STRIDE;
    for (int r = threadIdx.x; r < ncell; r += blockDim.x) {
        double c[kWinPolyDeg + 1];
#pragma unroll
        for (int k = 0; k <= kWinPolyDeg; ++k) c[k] = 0.0;
        for (int t = 0; t < m; ++t) {
            const bool mirror = t >= (m + 1) / 2;
            const int u = mirror ? m - 1 - t : t;
            const double hv = static_cast<double>(hp[r + t]);
#pragma unroll
            for (int j = 0; j <= 4; ++j) c[2 * j] += hv * static_cast<double>(wp.ev[u][j]);
#pragma unroll
            for (int j = 0; j <= 3; ++j) c[2 * j + 1] += (mirror ? -hv : hv) * static_cast<double>(wp.od[u][j]);
        }
#pragma unroll
        for (int k = 0; k < TAB_STRIDE; ++k) tp[static_cast<int64_t>(r) * TAB_STRIDE + k] = k <= kWinPolyDeg ? static_cast<float>(c[k]) : 0.0f;
    }
}

// Target side from the table: one thread per target walks every slice (the slices in the same
// order everywhere, so that the threads of an SM read one slice's 64-byte cells at a time from
// L1); per slice one 48-byte read of the cell's coefficients and Horner's rule (and its
// derivative for the gradient).  Same window check and Kahan slice sum as k_nfft_target.
template <bool GRAD>
__global__ void __launch_bounds__(256) k_nfft_target_tab(const float* __restrict__ Z, int P, int64_t n, int64_t ldz,
                                                         float scale_u, int m, int win_base, int ncell,
                                                         const float* __restrict__ tab, float R,
                                                         double* __restrict__ acc, float* __restrict__ G, int64_t ldg,
                                                         unsigned* __restrict__ err) {
    const int64_t mi = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (mi >= n) return;
    const float half_m = 0.5f * static_cast<float>(m), gofs = 0.5f * static_cast<float>(m - 1);
    KahanF sum;
    bool bad = false;
    constexpr int U = 4;  // projections of four slices loaded together
    for (int p0 = 0; p0 < P; p0 += U) {
        float zq[U];
#pragma unroll
        for (int r = 0; r < U; ++r) zq[r] = p0 + r < P ? Z[static_cast<int64_t>(p0 + r) * ldz + mi] : 0.0f;
#pragma unroll
        for (int r = 0; r < U; ++r) {
            const int p = p0 + r;
            if (p >= P) break;
            const float z = zq[r];
            if (!(z <= R && z >= -R)) bad = true;  // outside the certified window (or NaN)
            const float u = z * scale_u;
            const float c0 = ceilf(u - half_m);
            const int r0 = static_cast<int>(c0) - win_base;
            if (r0 < 0 || r0 >= ncell) {
                bad = true;
                continue;
            }
            const float g = c0 - u + gofs;
            const float4* cp = reinterpret_cast<const float4*>(tab + (static_cast<int64_t>(p) * ncell + r0) * TAB_STRIDE);
            const float4 a = __ldg(cp), b = __ldg(cp + 1), c = __ldg(cp + 2);
            if (GRAD) {
                // d/du sum_j h_j psi(u - j) = -d/dg of the cell polynomial (g = c0 - u + const)
                float dv = 8.0f * c.x;
                dv = fmaf(dv, g, 7.0f * b.w);
                dv = fmaf(dv, g, 6.0f * b.z);
                dv = fmaf(dv, g, 5.0f * b.y);
                dv = fmaf(dv, g, 4.0f * b.x);
                dv = fmaf(dv, g, 3.0f * a.w);
                dv = fmaf(dv, g, 2.0f * a.z);
                dv = fmaf(dv, g, a.y);
                G[static_cast<int64_t>(p) * ldg + mi] = -dv * scale_u;
            } else {
                float v = c.x;
                v = fmaf(v, g, b.w);
                v = fmaf(v, g, b.z);
                v = fmaf(v, g, b.y);
                v = fmaf(v, g, b.x);
                v = fmaf(v, g, a.w);
                v = fmaf(v, g, a.z);
                v = fmaf(v, g, a.y);
                v = fmaf(v, g, a.x);
                sum.add(v);
            }
        }
    }
    if (bad) atomicOr(err, 4u);
    if (!GRAD) acc[mi] += sum.value();
}

}  // namespace

// ------------------------------------------------------------ launchers

// Calls f(std::integral_constant<int, MM>{}) with MM >= m taps: the window's exact width for
// the FP32 kernels (their taps unrolled with no idle ones), 8, 12 or 16 for FP64.
template <class T, class F>
void tap_dispatch(int m, F&& f) {
    SLK_REQUIRE(m >= 4 && m <= kWinPolyMaxM, "NFFT window of %d cells", m);
    if constexpr (sizeof(T) == 4) {
        switch (m) {
            case 4: f(std::integral_constant<int, 4>{}); break;
            case 5: f(std::integral_constant<int, 5>{}); break;
            case 6: f(std::integral_constant<int, 6>{}); break;
            case 7: f(std::integral_constant<int, 7>{}); break;
            case 8: f(std::integral_constant<int, 8>{}); break;
            case 9: f(std::integral_constant<int, 9>{}); break;
            case 10: f(std::integral_constant<int, 10>{}); break;
            case 11: f(std::integral_constant<int, 11>{}); break;
            case 12: f(std::integral_constant<int, 12>{}); break;
            case 13: f(std::integral_constant<int, 13>{}); break;
            case 14: f(std::integral_constant<int, 14>{}); break;
            case 15: f(std::integral_constant<int, 15>{}); break;
            default: f(std::integral_constant<int, 16>{}); break;
        }
    } else {
        if (m <= 8) f(std::integral_constant<int, 8>{});
        else if (m <= 12) f(std::integral_constant<int, 12>{});
        else f(std::integral_constant<int, 16>{});
    }
}


int64_t ndft_source_scratch(int P, int64_t n, const FourierDev& fd) {
    int K = fd.k_hi - fd.k_lo + 1;
    return ceil_div(n, NDFT_CHUNK) * static_cast<int64_t>(P) * (2 * K + 1);
}

#define SLK_NDFT_DISPATCH(KV, ...)                                                        \
    do {                                                                                  \
        if ((KV) <= 4) { constexpr int KM = 4; __VA_ARGS__; }                             \
        else if ((KV) <= 8) { constexpr int KM = 8; __VA_ARGS__; }                        \
        else if ((KV) <= 12) { constexpr int KM = 12; __VA_ARGS__; }                      \
        else if ((KV) <= 16) { constexpr int KM = 16; __VA_ARGS__; }                      \
        else if ((KV) <= 24) { constexpr int KM = 24; __VA_ARGS__; }                      \
        else if ((KV) <= 32) { constexpr int KM = 32; __VA_ARGS__; }                      \
        else if ((KV) <= 48) { constexpr int KM = 48; __VA_ARGS__; }                      \
        else { constexpr int KM = 64; __VA_ARGS__; }                                      \
    } while (0)

template <class T>
void launch_ndft_source(const T* Z, int P, int64_t n, int64_t ldz, const T* w, const FourierDev& fd,
                        const double* coef, Cplx<T>* cw, T* cw0, T* scratch, int64_t scratch_elems, cudaStream_t st) {
    const int K = fd.k_hi - fd.k_lo + 1;
    SLK_REQUIRE(K >= 1 && K <= NDFT_KMAX, "NDFT band of %d coefficients exceeds %d", K, NDFT_KMAX);
    const int64_t nchunk = ceil_div(n, NDFT_CHUNK);
    SLK_REQUIRE(scratch_elems >= ndft_source_scratch(P, n, fd), "NDFT scratch too small");
    SLK_REQUIRE(nchunk <= 2147483647 && P <= 65535, "NDFT launch too large");
    dim3 grid(static_cast<unsigned>(nchunk), P);
    const T two_over_L = static_cast<T>(2.0 / fd.L);
    {
        SLK_TIMED("ndft_source", st);
        SLK_NDFT_DISPATCH(K, k_ndft_source<T, KM><<<grid, 256, 0, st>>>(Z, n, ldz, w, two_over_L, fd.k_lo, K,
                                                                        fd.has_k0, scratch, P));
    }
    SLK_CHECK_LAUNCH();
    int total = P * (K + 1);
    {
        SLK_TIMED("ndft_reduce", st);
        k_ndft_reduce<T><<<static_cast<unsigned>(ceil_div(total, 256)), 256, 0, st>>>(
            scratch, static_cast<int>(nchunk), P, K, fd.has_k0, coef, cw, cw0);
    }
    SLK_CHECK_LAUNCH();
}

// Below this many targets the NDFT target side runs one warp per target (see k_ndft_target_warp).
constexpr int64_t kNdftWarpTargets = 32768;

template <class T>
void launch_ndft_target(const T* Z, int P, int64_t n, int64_t ldz, const FourierDev& fd, const Cplx<T>* cw,
                        const T* cw0, double* acc, T* G, int64_t ldg, unsigned* err, cudaStream_t st) {
    if (acc && G) {
        launch_ndft_target<T>(Z, P, n, ldz, fd, cw, cw0, acc, nullptr, 0, err, st);
        launch_ndft_target<T>(Z, P, n, ldz, fd, cw, cw0, nullptr, G, ldg, err, st);
        return;
    }
    if (n <= 0) return;
    const int K = fd.k_hi - fd.k_lo + 1;
    SLK_REQUIRE(K >= 1 && K <= NDFT_KMAX, "NDFT band of %d coefficients exceeds %d", K, NDFT_KMAX);
    const size_t per_slice = sizeof(Cplx<T>) * K + sizeof(T);
    int chunk = static_cast<int>((96 * 1024) / per_slice);
    if (chunk > P) chunk = P;
    if (chunk < 1) chunk = 1;
    const size_t smem = per_slice * chunk + 16;
    const T two_over_L = static_cast<T>(2.0 / fd.L);
    const unsigned blocks = static_cast<unsigned>(ceil_div(n, 256));
    SLK_TIMED(G ? "ndft_target_grad" : "ndft_target", st);
    if (n < kNdftWarpTargets) {
        // few targets: one warp per target (eight per block) keeps every SM busy
        const unsigned wblocks = static_cast<unsigned>(ceil_div(n, 8));
        if (G)
            SLK_NDFT_DISPATCH(K, (k_ndft_target_warp<T, KM, true><<<wblocks, 256, 0, st>>>(
                                     Z, P, n, ldz, two_over_L, fd.k_lo, K, cw, cw0, static_cast<T>(fd.R), acc, G, ldg, err)));
        else
            SLK_NDFT_DISPATCH(K, (k_ndft_target_warp<T, KM, false><<<wblocks, 256, 0, st>>>(
                                     Z, P, n, ldz, two_over_L, fd.k_lo, K, cw, cw0, static_cast<T>(fd.R), acc, G, ldg, err)));
        SLK_CHECK_LAUNCH();
        return;
    }
    if (G) {
        SLK_NDFT_DISPATCH(K, {
            cudaFuncSetAttribute(k_ndft_target<T, KM, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, 100 * 1024);
            k_ndft_target<T, KM, true><<<blocks, 256, smem, st>>>(Z, P, n, ldz, two_over_L, fd.k_lo, K, cw, cw0, chunk,
                                                                 static_cast<T>(fd.R), acc, G, ldg, err);
        });
    } else {
        SLK_NDFT_DISPATCH(K, {
            cudaFuncSetAttribute(k_ndft_target<T, KM, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, 100 * 1024);
            k_ndft_target<T, KM, false><<<blocks, 256, smem, st>>>(Z, P, n, ldz, two_over_L, fd.k_lo, K, cw, cw0,
                                                                  chunk, static_cast<T>(fd.R), acc, G, ldg, err);
        });
    }
    SLK_CHECK_LAUNCH();
}

// The term count is padded on the host to one of these (zero coefficients beyond the
// certified q), so every loop over the terms has a compile-time length.
#define SLK_CHEB_DISPATCH(QV, ...)                                                        \
    do {                                                                                  \
        switch (QV) {                                                                     \
            case 8: { constexpr int QM = 8; __VA_ARGS__; } break;                         \
            case 10: { constexpr int QM = 10; __VA_ARGS__; } break;                       \
            case 12: { constexpr int QM = 12; __VA_ARGS__; } break;                       \
            case 16: { constexpr int QM = 16; __VA_ARGS__; } break;                       \
            case 24: { constexpr int QM = 24; __VA_ARGS__; } break;                       \
            case 32: { constexpr int QM = 32; __VA_ARGS__; } break;                       \
            case 48: { constexpr int QM = 48; __VA_ARGS__; } break;                       \
            case 64: { constexpr int QM = 64; __VA_ARGS__; } break;                       \
            case 96: { constexpr int QM = 96; __VA_ARGS__; } break;                       \
            default: fail(SLK_ERR_INVALID, "Chebyshev term count %d is not a padded size", QV); \
        }                                                                                 \
    } while (0)

int64_t cheb_source_scratch(int P, int64_t n, const FourierDev& fd) {
    return ceil_div(n, NDFT_CHUNK) * static_cast<int64_t>(P) * fd.q;
}

template <class T>
void launch_cheb_source(const T* Z, int P, int64_t n, int64_t ldz, const T* w, const FourierDev& fd,
                        const double* M, T* beta, T* mono, unsigned* mono_bad, double mono_ratio, T* scratch,
                        int64_t scratch_elems, cudaStream_t st) {
    const int q = fd.q;
    SLK_REQUIRE(q >= 1 && q <= 96, "Chebyshev terms out of range");
    const int64_t nchunk = ceil_div(n, NDFT_CHUNK);
    SLK_REQUIRE(scratch_elems >= cheb_source_scratch(P, n, fd), "Chebyshev scratch too small");
    SLK_REQUIRE(nchunk <= 2147483647 && P <= 65535, "Chebyshev launch too large");
    dim3 grid(static_cast<unsigned>(nchunk), P);
    const T inv_R = static_cast<T>(1.0 / fd.R);
    {
        SLK_TIMED("cheb_moments", st);
        const bool vec = sizeof(T) == 4 && ldz % 4 == 0 && reinterpret_cast<uintptr_t>(Z) % 16 == 0 &&
                         reinterpret_cast<uintptr_t>(w) % 16 == 0;
        if (vec)
            SLK_CHEB_DISPATCH(q, (k_cheb_moments<T, QM, true><<<grid, 256, 0, st>>>(Z, n, ldz, w, inv_R, q, scratch, P)));
        else
            SLK_CHEB_DISPATCH(q, (k_cheb_moments<T, QM, false><<<grid, 256, 0, st>>>(Z, n, ldz, w, inv_R, q, scratch, P)));
    }
    SLK_CHECK_LAUNCH();
    {
        SLK_TIMED("cheb_reduce", st);
        k_cheb_reduce<T><<<P, 128, 2 * sizeof(double) * q, st>>>(scratch, static_cast<int>(nchunk), P, q, M, beta,
                                                                  q <= 16 ? mono : nullptr, mono_bad, mono_ratio);
    }
    SLK_CHECK_LAUNCH();
}

void launch_cheb_reduce_f64(const double* partial, int nchunk, int P, const FourierDev& fd, const double* M,
                            float* beta, float* mono, unsigned* mono_bad, double mono_ratio, cudaStream_t st) {
    const int q = fd.q;
    SLK_TIMED("cheb_reduce", st);
    k_cheb_reduce<float, double><<<P, 128, 2 * sizeof(double) * q, st>>>(partial, nchunk, P, q, M, beta,
                                                                         q <= 16 ? mono : nullptr, mono_bad, mono_ratio);
    SLK_CHECK_LAUNCH();
}

template <class T>
void launch_cheb_target(const T* Z, int P, int64_t n, int64_t ldz, const FourierDev& fd, const T* beta, double* acc,
                        T* G, int64_t ldg, unsigned* err, cudaStream_t st) {
    if (acc && G) {
        launch_cheb_target<T>(Z, P, n, ldz, fd, beta, acc, nullptr, 0, err, st);
        launch_cheb_target<T>(Z, P, n, ldz, fd, beta, nullptr, G, ldg, err, st);
        return;
    }
    if (n <= 0) return;
    const int q = fd.q;
    int chunk = static_cast<int>((48 * 1024) / (sizeof(T) * q));
    if (chunk > P) chunk = P;
    if (chunk < 1) chunk = 1;
    const size_t smem = sizeof(T) * q * chunk;
    const T inv_R = static_cast<T>(1.0 / fd.R);
    const unsigned blocks = static_cast<unsigned>(ceil_div(n, 256));
    SLK_TIMED(G ? "cheb_target_grad" : "cheb_target", st);
    if (G) {
        SLK_CHEB_DISPATCH(q, (k_cheb_target<T, QM, true, false><<<blocks, 256, smem, st>>>(
                                 Z, P, n, ldz, inv_R, q, beta, chunk, static_cast<T>(fd.R), acc, G, ldg, err)));
    } else if (fd.horner && fd.mono) {
        const T* mono = static_cast<const T*>(fd.mono);
        SLK_CHEB_DISPATCH(q, (k_cheb_target<T, QM, false, true><<<blocks, 256, smem, st>>>(
                                 Z, P, n, ldz, inv_R, q, mono, chunk, static_cast<T>(fd.R), acc, G, ldg, err)));
    } else {
        SLK_CHEB_DISPATCH(q, (k_cheb_target<T, QM, false, false><<<blocks, 256, smem, st>>>(
                                 Z, P, n, ldz, inv_R, q, beta, chunk, static_cast<T>(fd.R), acc, G, ldg, err)));
    }
    SLK_CHECK_LAUNCH();
}

template void launch_cheb_source<float>(const float*, int, int64_t, int64_t, const float*, const FourierDev&,
                                        const double*, float*, float*, unsigned*, double, float*, int64_t, cudaStream_t);
template void launch_cheb_source<double>(const double*, int, int64_t, int64_t, const double*, const FourierDev&,
                                         const double*, double*, double*, unsigned*, double, double*, int64_t, cudaStream_t);
template void launch_cheb_target<float>(const float*, int, int64_t, int64_t, const FourierDev&, const float*, double*,
                                        float*, int64_t, unsigned*, cudaStream_t);
template void launch_cheb_target<double>(const double*, int, int64_t, int64_t, const FourierDev&, const double*,
                                         double*, double*, int64_t, unsigned*, cudaStream_t);

int64_t nfft_source_scratch(int P, int64_t n, const FourierDev& fd) {
    int64_t nchunk;
    if (fd.W <= SPREAD_NARROW_W) nchunk = ceil_div(n, static_cast<int64_t>(SPREAD_WARPS) * SPREAD_CHUNK);
    else nchunk = ceil_div(n, 65536);
    return (nchunk + 1) * static_cast<int64_t>(P) * fd.W;
}

template <class T>
void launch_nfft_source(const T* Z, int P, int64_t n, int64_t ldz, const T* w, const T* pairs, const FourierDev& fd,
                        int n_coeff, const double* mult, T* h, T* scratch, int64_t scratch_elems, unsigned* err,
                        cudaStream_t st) {
    SLK_REQUIRE(scratch_elems >= nfft_source_scratch(P, n, fd), "NFFT scratch too small");
    SLK_REQUIRE(fd.W <= fd.n_g, "NFFT window wider than the grid");
    SLK_REQUIRE(fd.m >= 1 && fd.m <= 16, "NFFT window of %d cells", fd.m);
    const T scale_u = static_cast<T>(fd.n_g / fd.L);
    const T two_over_m = static_cast<T>(2.0 / fd.m);
    const T beta = static_cast<T>(fd.beta);
    // scratch layout: [partials nchunk x P x W] [reduced grid P x W]
    T* partial = scratch;
    int64_t nchunk;
    if (pairs) {
        // sources grouped by key: taps accumulated in registers along each thread's run
        const int64_t chunk = 65536;
        nchunk = ceil_div(n, chunk);
        const size_t smem = sizeof(T) * fd.W;
        SLK_REQUIRE(smem <= 200 * 1024, "NFFT window too wide");
        dim3 grid(static_cast<unsigned>(nchunk), P);
        SLK_TIMED("spread_sorted", st);
        tap_dispatch<T>(fd.m, [&](auto mm) {
            constexpr int MM = decltype(mm)::value;
            SLK_CHECK_CUDA(cudaFuncSetAttribute(k_spread_sorted<T, MM>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                200 * 1024));
            k_spread_sorted<T, MM><<<grid, 256, smem, st>>>(pairs, n, scale_u, fd.m, two_over_m, beta, fd.wp, fd.W,
                                                           fd.win_base, chunk, partial, err);
        });
    } else if (fd.W <= SPREAD_NARROW_W) {
        nchunk = ceil_div(n, static_cast<int64_t>(SPREAD_WARPS) * SPREAD_CHUNK);
        size_t smem = sizeof(T) * SPREAD_WARPS * fd.W * 32;
        static bool attr_set[2] = {false, false};
        if (!attr_set[sizeof(T) == 8]) {
            SLK_CHECK_CUDA(cudaFuncSetAttribute(k_spread_narrow<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                sizeof(T) * SPREAD_WARPS * SPREAD_NARROW_W * 32));
            attr_set[sizeof(T) == 8] = true;
        }
        dim3 grid(static_cast<unsigned>(nchunk), static_cast<unsigned>(ceil_div(P, 32)));
        {
            SLK_TIMED("spread_narrow", st);
            k_spread_narrow<T><<<grid, 256, smem, st>>>(Z, P, n, ldz, w, scale_u, fd.m, two_over_m, beta, fd.W,
                                                         fd.win_base, partial, err);
        }
    } else {
        const int64_t chunk = 65536;
        nchunk = ceil_div(n, chunk);
        size_t smem = sizeof(T) * fd.W;
        SLK_REQUIRE(smem <= 200 * 1024, "NFFT window too wide");
        static bool attr_set[2] = {false, false};
        if (!attr_set[sizeof(T) == 8]) {
            attr_set[sizeof(T) == 8] = true;
        }
        dim3 grid(static_cast<unsigned>(nchunk), P);
        {
            SLK_TIMED("spread_wide", st);
            tap_dispatch<T>(fd.m, [&](auto mm) {
                constexpr int MM = decltype(mm)::value;
                SLK_CHECK_CUDA(
                    cudaFuncSetAttribute(k_spread_wide<T, MM>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
                k_spread_wide<T, MM><<<grid, 256, smem, st>>>(Z, P, n, ldz, w, scale_u, fd.m, two_over_m, beta, fd.wp,
                                                              fd.W, fd.win_base, chunk, partial, err);
            });
        }
    }
    SLK_CHECK_LAUNCH();
    T* g = partial + nchunk * static_cast<int64_t>(P) * fd.W;
    int64_t tot = static_cast<int64_t>(P) * fd.W;
    {
        SLK_TIMED("window_reduce", st);
        k_window_reduce<T><<<static_cast<unsigned>(ceil_div(tot, 256) < 8192 ? ceil_div(tot, 256) : 8192), 256, 0, st>>>(
            partial, static_cast<int>(nchunk), P, fd.W, g);
    }
    SLK_CHECK_LAUNCH();
    int logn = 0;
    while ((1 << logn) < fd.n_g) ++logn;
    SLK_REQUIRE((1 << logn) == fd.n_g, "NFFT grid must be a power of two");
    size_t smem = sizeof(Cplx<T>) * fd.n_g;
    SLK_REQUIRE(smem <= 200 * 1024, "NFFT grid too large for one block");
    static bool attr_fft[2] = {false, false};
    if (!attr_fft[sizeof(T) == 8]) {
        SLK_CHECK_CUDA(cudaFuncSetAttribute(k_fft_multiply<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
        attr_fft[sizeof(T) == 8] = true;
    }
    {
        SLK_TIMED("fft_multiply", st);
        k_fft_multiply<T><<<P, 512, smem, st>>>(g, P, fd.n_g, logn, fd.W, fd.win_base, n_coeff / 2, mult, h);
    }
    SLK_CHECK_LAUNCH();
}

int64_t interp_table_floats(int P, const FourierDev& fd) {
    return static_cast<int64_t>(P) * (fd.W - fd.m + 1) * TAB_STRIDE;
}

void launch_interp_table(const float* h, int P, const FourierDev& fd, float* tab, cudaStream_t st) {
    SLK_REQUIRE(fd.W >= fd.m && fd.m >= 1 && fd.m <= kWinPolyMaxM, "NFFT window of %d cells over %d", fd.m, fd.W);
    {
        SLK_TIMED("interp_table", st);
        k_interp_table<<<P, 256, 0, st>>>(h, fd.W, fd.m, fd.wp, fd.W - fd.m + 1, tab);
    }
    SLK_CHECK_LAUNCH();
}

template <class T>
void launch_nfft_target(const T* Z, int P, int64_t n, int64_t ldz, const FourierDev& fd, const T* h, double* acc,
                        T* G, int64_t ldg, unsigned* err, cudaStream_t st) {
    if (acc && G) {
        launch_nfft_target<T>(Z, P, n, ldz, fd, h, acc, nullptr, 0, err, st);
        launch_nfft_target<T>(Z, P, n, ldz, fd, h, nullptr, G, ldg, err, st);
        return;
    }
    if (n <= 0) return;
    if constexpr (sizeof(T) == 4) {
        if (fd.itab) {
            const unsigned blocks = static_cast<unsigned>(ceil_div(n, 256));
            const int ncell = fd.W - fd.m + 1;
            const float* tab = static_cast<const float*>(fd.itab);
            SLK_TIMED(G ? "nfft_target_grad" : "nfft_target", st);
            if (G)
                k_nfft_target_tab<true><<<blocks, 256, 0, st>>>(Z, P, n, ldz, static_cast<float>(fd.n_g / fd.L), fd.m,
                                                               fd.win_base, ncell, tab, static_cast<float>(fd.R), acc, G,
                                                               ldg, err);
            else
                k_nfft_target_tab<false><<<blocks, 256, 0, st>>>(Z, P, n, ldz, static_cast<float>(fd.n_g / fd.L), fd.m,
                                                                fd.win_base, ncell, tab, static_cast<float>(fd.R), acc,
                                                                G, ldg, err);
            SLK_CHECK_LAUNCH();
            return;
        }
    }
    // slices whose grid windows a block holds at once: about 24 KB, so that several blocks share
    // an SM (the loop over slices is latency-bound; occupancy hides it)
    int chunk = static_cast<int>((24 * 1024) / (sizeof(T) * fd.W));
    if (chunk > P) chunk = P;
    if (chunk < 1) chunk = 1;
    size_t smem = sizeof(T) * fd.W * chunk;
    SLK_REQUIRE(smem <= 100 * 1024, "NFFT window too wide for the interpolation");
    {
        SLK_TIMED("nfft_target", st);
        const unsigned blocks = static_cast<unsigned>(ceil_div(n, 256));
        tap_dispatch<T>(fd.m, [&](auto mm) {
            constexpr int MM = decltype(mm)::value;
            SLK_CHECK_CUDA(
                cudaFuncSetAttribute(k_nfft_target<T, MM>, cudaFuncAttributeMaxDynamicSharedMemorySize, 100 * 1024));
            k_nfft_target<T, MM><<<blocks, 256, smem, st>>>(
                Z, P, n, ldz, static_cast<T>(fd.n_g / fd.L), fd.m, static_cast<T>(2.0 / fd.m), static_cast<T>(fd.beta),
                fd.wp, fd.W, fd.win_base, h, chunk, static_cast<T>(fd.R), acc, G, ldg, err);
        });
    }
    SLK_CHECK_LAUNCH();
}

template void launch_ndft_source<float>(const float*, int, int64_t, int64_t, const float*, const FourierDev&,
                                        const double*, Cplx<float>*, float*, float*, int64_t, cudaStream_t);
template void launch_ndft_source<double>(const double*, int, int64_t, int64_t, const double*, const FourierDev&,
                                         const double*, Cplx<double>*, double*, double*, int64_t, cudaStream_t);
template void launch_ndft_target<float>(const float*, int, int64_t, int64_t, const FourierDev&, const Cplx<float>*,
                                        const float*, double*, float*, int64_t, unsigned*, cudaStream_t);
template void launch_ndft_target<double>(const double*, int, int64_t, int64_t, const FourierDev&,
                                         const Cplx<double>*, const double*, double*, double*, int64_t, unsigned*,
                                         cudaStream_t);
template void launch_nfft_source<float>(const float*, int, int64_t, int64_t, const float*, const float*,
                                        const FourierDev&, int, const double*, float*, float*, int64_t, unsigned*,
                                        cudaStream_t);
template void launch_nfft_source<double>(const double*, int, int64_t, int64_t, const double*, const double*,
                                         const FourierDev&, int, const double*, double*, double*, int64_t, unsigned*,
                                         cudaStream_t);
template void launch_nfft_target<float>(const float*, int, int64_t, int64_t, const FourierDev&, const float*, double*,
                                        float*, int64_t, unsigned*, cudaStream_t);
template void launch_nfft_target<double>(const double*, int, int64_t, int64_t, const FourierDev&, const double*,
                                         double*, double*, int64_t, unsigned*, cudaStream_t);

}  // namespace slk
