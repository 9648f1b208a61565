// Random Fourier features (Section 4.3): the comparison system of the paper's Table 2.
//
// K(x, y) = E_{v ~ mu} cos<x - y, v> for the spectral measure mu of the kernel (Bochner);
// with D samples v_p and phases b_p ~ U[0, 2 pi):
//   RFF-1:  s_m = (2 / D) sum_p cos(<y_m, v_p> + b_p) C_p,   C_p = sum_n w_n cos(<x_n, v_p> + b_p)
//   RFF-2:  s_m = (1 / D) sum_p [cos<y_m, v_p> C_p + sin<y_m, v_p> S_p],
//           C_p = sum_n w_n cos<x_n, v_p>,  S_p = sum_n w_n sin<x_n, v_p>.
// The projections <x_n, v_p> come from the SIMT projection (FP32 or FP64, uncentred);
// the kernels here draw the features, form C_p, S_p (FP64 per chunk of points, summed in a
// fixed order) and evaluate the targets.
#include "kernels.cuh"
#include "philox.cuh"

namespace slk {

namespace {

// counters: (index, feature, stream tag, 0) under the key of the seed, a stream of the
// same generator as the direction draw
constexpr uint32_t kTagV = 0x72666631u, kTagB = 0x72666632u;

// feat row p = (v_p (d values), b_p): Gaussian v = g / sigma, Laplacian v = alpha g / |h|
// (multivariate Cauchy), g ~ N(0, I_d) by Box-Muller pairs, h ~ N(0, 1), b = 2 pi u.
__global__ void k_rff_draw(double* __restrict__ feat, int D, int d, int laplacian, double param, uint32_t k0,
                           uint32_t k1) {
    const int p = blockIdx.y;
    double scale;
    {
        uint32_t c[4] = {0u, static_cast<uint32_t>(p), kTagB, 0u};
        philox4x32_10(c, k0, k1);
        if (laplacian) {
            const double r = sqrt(-2.0 * log(u01(c[0], c[1])));
            double sn, cs;
            sincospi(2.0 * u01(c[2], c[3]), &sn, &cs);
            scale = param / fabs(r * cs);
        } else {
            scale = 1.0 / param;
        }
        if (blockIdx.x == 0 && threadIdx.x == 0) {
            uint32_t e[4] = {1u, static_cast<uint32_t>(p), kTagB, 0u};
            philox4x32_10(e, k0, k1);
            feat[static_cast<int64_t>(p) * (d + 1) + d] = 2.0 * 3.14159265358979323846 * u01(e[0], e[1]);
        }
    }
    const int pairs = (d + 1) / 2;
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < pairs; j += gridDim.x * blockDim.x) {
        uint32_t c[4] = {static_cast<uint32_t>(j), static_cast<uint32_t>(p), kTagV, 0u};
        philox4x32_10(c, k0, k1);
        const double r = sqrt(-2.0 * log(u01(c[0], c[1])));
        double sn, cs;
        sincospi(2.0 * u01(c[2], c[3]), &sn, &cs);
        double* row = feat + static_cast<int64_t>(p) * (d + 1);
        row[2 * j] = scale * r * cs;
        if (2 * j + 1 < d) row[2 * j + 1] = scale * r * sn;
    }
}

// V[p][k] = feat[p][k], b[p] = feat[p][d] in the working precision
template <class T>
__global__ void k_rff_split(const double* __restrict__ feat, int D, int d, T* __restrict__ V, T* __restrict__ b) {
    const int64_t total = static_cast<int64_t>(D) * (d + 1);
    for (int64_t e = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; e < total;
         e += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const int p = static_cast<int>(e / (d + 1)), k = static_cast<int>(e % (d + 1));
        if (k < d) V[static_cast<int64_t>(p) * d + k] = static_cast<T>(feat[e]);
        else b[p] = static_cast<T>(feat[e]);
    }
}

__device__ inline void sin_cos(float a, float* s, float* c) { sincosf(a, s, c); }
__device__ inline void sin_cos(double a, double* s, double* c) { sincos(a, s, c); }

constexpr int RFF_THREADS = 256, RFF_CHUNK = 8192;

// part[(p * nchunk + chunk) * 2 + {0, 1}] = sums over the chunk's points of
// w cos(z + b) and 0 (RFF-1), or w cos z and w sin z (RFF-2); block reduction in FP64.
template <class T, int VARIANT>
__global__ void __launch_bounds__(RFF_THREADS) k_rff_source(const T* __restrict__ Z, int64_t n, const T* __restrict__ w,
                                                           const T* __restrict__ b, int nchunk,
                                                           double* __restrict__ part) {
    const int p = blockIdx.y, chunk = blockIdx.x;
    const int64_t i0 = static_cast<int64_t>(chunk) * RFF_CHUNK;
    const int64_t i1 = i0 + RFF_CHUNK < n ? i0 + RFF_CHUNK : n;
    const T bp = VARIANT == 1 ? b[p] : T(0);
    const T* row = Z + static_cast<int64_t>(p) * n;
    double c = 0.0, s = 0.0;
    for (int64_t i = i0 + threadIdx.x; i < i1; i += RFF_THREADS) {
        T sn, cs;
        sin_cos(row[i] + bp, &sn, &cs);
        c += static_cast<double>(w[i] * cs);
        if (VARIANT == 2) s += static_cast<double>(w[i] * sn);
    }
    __shared__ double rc[RFF_THREADS / 32], rs[RFF_THREADS / 32];
    for (int o = 16; o > 0; o >>= 1) {
        c += __shfl_xor_sync(0xffffffffu, c, o);
        s += __shfl_xor_sync(0xffffffffu, s, o);
    }
    if ((threadIdx.x & 31) == 0) {
        rc[threadIdx.x >> 5] = c;
        rs[threadIdx.x >> 5] = s;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double tc = 0.0, ts = 0.0;
        for (int k = 0; k < RFF_THREADS / 32; ++k) {
            tc += rc[k];
            ts += rs[k];
        }
        part[(static_cast<int64_t>(p) * nchunk + chunk) * 2] = tc;
        part[(static_cast<int64_t>(p) * nchunk + chunk) * 2 + 1] = ts;
    }
}

// cs[p] = (C_p, S_p): the chunk partials of slice p summed in chunk order
__global__ void k_rff_reduce(const double* __restrict__ part, int D, int nchunk, double2* __restrict__ cs) {
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < D; p += gridDim.x * blockDim.x) {
        double c = 0.0, s = 0.0;
        for (int k = 0; k < nchunk; ++k) {
            c += part[(static_cast<int64_t>(p) * nchunk + k) * 2];
            s += part[(static_cast<int64_t>(p) * nchunk + k) * 2 + 1];
        }
        cs[p] = make_double2(c, s);
    }
}

// s[i] = scale * sum_p [cos(z + b_p) C_p (RFF-1) | cos z C_p + sin z S_p (RFF-2)], one
// thread per target, feature terms summed with Kahan compensation in the working precision
template <class T, int VARIANT>
__global__ void __launch_bounds__(RFF_THREADS) k_rff_target(const T* __restrict__ Z, int64_t m, int D,
                                                           const T* __restrict__ b, const double2* __restrict__ cs,
                                                           double scale, T* __restrict__ s) {
    const int64_t i = blockIdx.x * static_cast<int64_t>(RFF_THREADS) + threadIdx.x;
    if (i >= m) return;
    T acc = T(0), comp = T(0);
    for (int p = 0; p < D; ++p) {
        const double2 q = cs[p];
        T sn, c;
        sin_cos(Z[static_cast<int64_t>(p) * m + i] + (VARIANT == 1 ? b[p] : T(0)), &sn, &c);
        const T t = VARIANT == 1 ? c * static_cast<T>(q.x) : c * static_cast<T>(q.x) + sn * static_cast<T>(q.y);
        const T y = t - comp;
        const T tt = acc + y;
        comp = (tt - acc) - y;
        acc = tt;
    }
    s[i] = static_cast<T>(scale * (static_cast<double>(acc) - static_cast<double>(comp)));
}

}  // namespace

void launch_rff_draw(double* feat, int D, int d, int laplacian, double param, uint64_t seed, cudaStream_t st) {
    dim3 grid(static_cast<unsigned>(ceil_div((d + 1) / 2, 256) < 64 ? ceil_div((d + 1) / 2, 256) : 64),
              static_cast<unsigned>(D));
    SLK_REQUIRE(D <= 65535, "too many features for one draw");
    {
        SLK_TIMED("rff_draw", st);
        k_rff_draw<<<grid, 256, 0, st>>>(feat, D, d, laplacian, param, static_cast<uint32_t>(seed),
                                         static_cast<uint32_t>(seed >> 32));
    }
    SLK_CHECK_LAUNCH();
}

template <class T>
void launch_rff_split(const double* feat, int D, int d, T* V, T* b, cudaStream_t st) {
    const int64_t total = static_cast<int64_t>(D) * (d + 1);
    {
        SLK_TIMED("rff_split", st);
        k_rff_split<T><<<static_cast<unsigned>(ceil_div(total, 256) < 4096 ? ceil_div(total, 256) : 4096), 256, 0, st>>>(
            feat, D, d, V, b);
    }
    SLK_CHECK_LAUNCH();
}

template <class T>
void launch_rff_source(const T* Z, int D, int64_t n, const T* w, const T* b, int variant, double2* cs, cudaStream_t st) {
    const int nchunk = static_cast<int>(ceil_div(n, RFF_CHUNK));
    SLK_REQUIRE(D <= 65535, "too many features for one launch");
    DevBuf<double> part(static_cast<size_t>(D) * nchunk * 2, st);
    dim3 grid(static_cast<unsigned>(nchunk), static_cast<unsigned>(D));
    {
        SLK_TIMED("rff_source", st);
        if (variant == 1) k_rff_source<T, 1><<<grid, RFF_THREADS, 0, st>>>(Z, n, w, b, nchunk, part.get());
        else k_rff_source<T, 2><<<grid, RFF_THREADS, 0, st>>>(Z, n, w, b, nchunk, part.get());
    }
    SLK_CHECK_LAUNCH();
    {
        SLK_TIMED("rff_reduce", st);
        k_rff_reduce<<<static_cast<unsigned>(ceil_div(D, 128)), 128, 0, st>>>(part.get(), D, nchunk, cs);
    }
    SLK_CHECK_LAUNCH();
}

template <class T>
void launch_rff_target(const T* Z, int D, int64_t m, const T* b, const double2* cs, int variant, T* s, cudaStream_t st) {
    if (m <= 0) return;
    const double scale = variant == 1 ? 2.0 / D : 1.0 / D;
    const unsigned grid = static_cast<unsigned>(ceil_div(m, RFF_THREADS));
    {
        SLK_TIMED("rff_target", st);
        if (variant == 1) k_rff_target<T, 1><<<grid, RFF_THREADS, 0, st>>>(Z, m, D, b, cs, scale, s);
        else k_rff_target<T, 2><<<grid, RFF_THREADS, 0, st>>>(Z, m, D, b, cs, scale, s);
    }
    SLK_CHECK_LAUNCH();
}

#define SLK_INST(T)                                                                                         \
    template void launch_rff_split<T>(const double*, int, int, T*, T*, cudaStream_t);                        \
    template void launch_rff_source<T>(const T*, int, int64_t, const T*, const T*, int, double2*, cudaStream_t); \
    template void launch_rff_target<T>(const T*, int, int64_t, const T*, const double2*, int, T*, cudaStream_t);
SLK_INST(float)
SLK_INST(double)
#undef SLK_INST

}  // namespace slk
