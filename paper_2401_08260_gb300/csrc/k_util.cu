// Directions, centring, conversions, range reduction and the final scaling.
#include "kernels.cuh"
#include "philox.cuh"

namespace slk {

// ------------------------------------------------------------ directions

// Row p of xi is row p0 + p of the seed's sequence: the counter holds the global slice index,
// so plans over disjoint slice ranges reproduce the rows of one plan over all of them.
__global__ void k_draw_directions(double* xi, int P, int d, uint32_t p0, uint32_t k0, uint32_t k1) {
    int p = blockIdx.y;
    int pairs = (d + 1) / 2;
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < pairs; j += gridDim.x * blockDim.x) {
        uint32_t c[4] = {static_cast<uint32_t>(j), p0 + static_cast<uint32_t>(p), 0x736c6b31u, 0u};
        philox4x32_10(c, k0, k1);
        double u1 = u01(c[0], c[1]), u2 = u01(c[2], c[3]);
        double r = sqrt(-2.0 * log(u1));
        double s, co;
        sincospi(2.0 * u2, &s, &co);
        xi[static_cast<int64_t>(p) * d + 2 * j] = r * co;
        if (2 * j + 1 < d) xi[static_cast<int64_t>(p) * d + 2 * j + 1] = r * s;
    }
}

__global__ void k_normalize_rows(double* xi, int d) {
    double* row = xi + static_cast<int64_t>(blockIdx.x) * d;
    double acc = 0.0;
    for (int k = threadIdx.x; k < d; k += blockDim.x) acc += row[k] * row[k];
    __shared__ double red[32];
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x < 32) {
        double v = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (threadIdx.x == 0) red[0] = v;
    }
    __syncthreads();
    double inv = 1.0 / sqrt(red[0]);
    for (int k = threadIdx.x; k < d; k += blockDim.x) row[k] *= inv;
}

void launch_draw_directions(double* xi, int P, int d, uint64_t seed, int p0, cudaStream_t st) {
    int pairs = (d + 1) / 2;
    dim3 grid(static_cast<unsigned>(ceil_div(pairs, 256)), P);
    {
        SLK_TIMED("draw_directions", st);
        k_draw_directions<<<grid, 256, 0, st>>>(xi, P, d, static_cast<uint32_t>(p0), static_cast<uint32_t>(seed),
                                                static_cast<uint32_t>(seed >> 32));
    }
    SLK_CHECK_LAUNCH();
    launch_normalize_rows(xi, P, d, st);
}

void launch_normalize_rows(double* xi, int P, int d, cudaStream_t st) {
    {
        SLK_TIMED("normalize_rows", st);
        k_normalize_rows<<<P, 256, 0, st>>>(xi, d);
    }
    SLK_CHECK_LAUNCH();
}

// ------------------------------------------------------------ centre

// partial[c][k] = sum of column k over the c-th group of sampled rows
template <class T>
__global__ void k_sample_mean_partial(const T* x, int64_t N, int d, int64_t ldx, int S, int groups, double* partial) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    const int g = blockIdx.y;
    if (k >= d) return;
    double acc = 0.0;
    for (int s = g; s < S; s += groups) {
        int64_t row = (static_cast<int64_t>(s) * N) / S;
        acc += static_cast<double>(x[row * ldx + k]);
    }
    partial[static_cast<int64_t>(g) * d + k] = acc;
}

__global__ void k_sample_mean_final(const double* partial, int d, int S, int groups, double* mu) {
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < d; k += gridDim.x * blockDim.x) {
        double acc = 0.0;
        for (int g = 0; g < groups; ++g) acc += partial[static_cast<int64_t>(g) * d + k];
        mu[k] = acc / S;
    }
}

template <class T>
void launch_sample_mean(const T* x, int64_t N, int d, int64_t ldx, double* mu, cudaStream_t st) {
    const int S = static_cast<int>(N < 4096 ? N : 4096);
    const int groups = S < 64 ? S : 64;
    DevBuf<double> partial(static_cast<size_t>(groups) * d, st);
    {
        SLK_TIMED("sample_mean_partial", st);
        dim3 grid(static_cast<unsigned>(ceil_div(d, 128)), groups);
        k_sample_mean_partial<T><<<grid, 128, 0, st>>>(x, N, d, ldx, S, groups, partial.get());
    }
    SLK_CHECK_LAUNCH();
    {
        SLK_TIMED("sample_mean_final", st);
        k_sample_mean_final<<<static_cast<unsigned>(ceil_div(d, 128)), 128, 0, st>>>(partial.get(), d, S, groups, mu);
    }
    SLK_CHECK_LAUNCH();
}

template <class T>
__global__ void k_convert(const double* src, T* dst, int64_t n) {
    for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x)
        dst[i] = static_cast<T>(src[i]);
}

template <class T>
void launch_convert(const double* src, T* dst, int64_t n, cudaStream_t st) {
    if (n <= 0) return;
    int64_t blocks = ceil_div(n, 256);
    {
        SLK_TIMED("convert", st);
        k_convert<T><<<static_cast<unsigned>(blocks < 4096 ? blocks : 4096), 256, 0, st>>>(src, dst, n);
    }
    SLK_CHECK_LAUNCH();
}

// ------------------------------------------------------------ range

template <class T>
__global__ void k_absmax(const T* Z, int64_t n, int64_t ldz, float* out) {
    const T* row = Z + static_cast<int64_t>(blockIdx.y) * ldz;
    float m = 0.0f;
    for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        float v = fabsf(static_cast<float>(row[i]));
        m = v > m ? v : m;  // NaN never wins; caught by the window checks downstream
    }
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    // non-negative floats order like their bit patterns: an integer max is exact
    if ((threadIdx.x & 31) == 0) atomicMax(reinterpret_cast<unsigned int*>(out), __float_as_uint(m));
}

template <class T>
void launch_absmax(const T* Z, int P, int64_t n, int64_t ldz, float* out, cudaStream_t st) {
    if (n <= 0 || P <= 0) return;
    int64_t bx = ceil_div(n, 256);
    dim3 grid(static_cast<unsigned>(bx < 64 ? bx : 64), P);
    {
        SLK_TIMED("absmax", st);
        k_absmax<T><<<grid, 256, 0, st>>>(Z, n, ldz, out);
    }
    SLK_CHECK_LAUNCH();
}

template <class T>
__global__ void k_finalize(const double* acc, T* s, int64_t n, double scale) {
    for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x)
        s[i] = static_cast<T>(acc[i] * scale);
}

template <class T>
void launch_finalize(const double* acc, T* s, int64_t n, double scale, cudaStream_t st) {
    if (n <= 0) return;
    int64_t blocks = ceil_div(n, 256);
    {
        SLK_TIMED("finalize", st);
        k_finalize<T><<<static_cast<unsigned>(blocks < 8192 ? blocks : 8192), 256, 0, st>>>(acc, s, n, scale);
    }
    SLK_CHECK_LAUNCH();
}

template <class T>
__global__ void k_sum_parts(const double* part, int parts, int64_t n, double scale, T* s) {
    for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        double a = 0.0;
        for (int r = 0; r < parts; ++r) a += part[r * n + i];
        s[i] = static_cast<T>(a * scale);
    }
}

template <class T>
void launch_sum_parts(const double* part, int parts, int64_t n, double scale, T* s, cudaStream_t st) {
    if (n <= 0) return;
    const int64_t blocks = ceil_div(n, 256);
    SLK_TIMED("sum_parts", st);
    k_sum_parts<T><<<static_cast<unsigned>(blocks < 8192 ? blocks : 8192), 256, 0, st>>>(part, parts, n, scale, s);
    SLK_CHECK_LAUNCH();
}

template void launch_sum_parts<float>(const double*, int, int64_t, double, float*, cudaStream_t);
template void launch_sum_parts<double>(const double*, int, int64_t, double, double*, cudaStream_t);
// acc = (first ? 0 : acc) + a t: one batch's sums weighted by its share of the slices
template <class T>
__global__ void k_accumulate_scaled(double* __restrict__ acc, const T* __restrict__ t, double a, int64_t n,
                                    int first) {
    for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const double v = a * static_cast<double>(t[i]);
        acc[i] = first ? v : acc[i] + v;
    }
}

template <class T>
void launch_accumulate_scaled(double* acc, const T* t, double a, int64_t n, bool first, cudaStream_t st) {
    if (n <= 0) return;
    const int64_t blocks = ceil_div(n, 256);
    SLK_TIMED("accumulate_scaled", st);
    k_accumulate_scaled<T><<<static_cast<unsigned>(blocks < 8192 ? blocks : 8192), 256, 0, st>>>(acc, t, a, n,
                                                                                                 first ? 1 : 0);
    SLK_CHECK_LAUNCH();
}

template void launch_accumulate_scaled<float>(double*, const float*, double, int64_t, bool, cudaStream_t);
template void launch_accumulate_scaled<double>(double*, const double*, double, int64_t, bool, cudaStream_t);

__global__ void k_gather_rows(const float* __restrict__ x, int64_t N, int d, int64_t ldx, int64_t S,
                              float* __restrict__ out) {
    for (int64_t e = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; e < S * d;
         e += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const int64_t s = e / d;
        const int k = static_cast<int>(e - s * d);
        out[e] = x[((s * N) / S) * ldx + k];
    }
}

void launch_gather_rows(const float* x, int64_t N, int d, int64_t ldx, int64_t S, float* out, cudaStream_t st) {
    if (S <= 0) return;
    const int64_t blocks = ceil_div(S * d, 256);
    SLK_TIMED("gather_rows", st);
    k_gather_rows<<<static_cast<unsigned>(blocks < 4096 ? blocks : 4096), 256, 0, st>>>(x, N, d, ldx, S, out);
    SLK_CHECK_LAUNCH();
}

template void launch_sample_mean<float>(const float*, int64_t, int, int64_t, double*, cudaStream_t);
template void launch_sample_mean<double>(const double*, int64_t, int, int64_t, double*, cudaStream_t);
template void launch_convert<float>(const double*, float*, int64_t, cudaStream_t);
template void launch_convert<double>(const double*, double*, int64_t, cudaStream_t);
template void launch_absmax<float>(const float*, int, int64_t, int64_t, float*, cudaStream_t);
template void launch_absmax<double>(const double*, int, int64_t, int64_t, float*, cudaStream_t);
template void launch_finalize<float>(const double*, float*, int64_t, double, cudaStream_t);
template void launch_finalize<double>(const double*, double*, int64_t, double, cudaStream_t);

}  // namespace slk
