// Sorting route of Section 3.2 (negative distance kernel; the non-smooth part
// of the Laplacian in Section 3.3).
//
// Per slice the sources are sorted by their projection (segmented LSD radix
// sort on order-preserving key bits, 8-bit digits, stable, with the source
// index as payload) and stored as (key, w) pairs in sorted order.  The sorted
// range of each slice is cut into NB buckets of equal key width; FP64
// exclusive prefix sums of w and w z are kept only at bucket starts:
//     A_b = sum over sources in buckets < b of w,   B_b = same of w z.
// A target z in bucket b then has
//     A_< = A_b + sum_{sources of bucket b with key < z} w,   B_< likewise,
// (a short scan of the sorted bucket, stopped at the insertion point) and
//     t(z) = -c_d sum_n w_n |z - x_n| = -c_d [ z (2 A_< - W) - (2 B_< - S) ],
// W, S the totals.  This is Algorithm 2 regrouped: splitting the sum at z gives
//     sum_{x<z} w (z - x) + sum_{x>=z} w (x - z) = z (2 A_< - W) - (2 B_< - S),
// the same value without the joint sort of sources and targets.
#include "kernels.cuh"

namespace slk {

namespace {

constexpr int RS_THREADS = 256, RS_ITEMS = 16, RS_TILE = RS_THREADS * RS_ITEMS, RS_BINS = 256;

template <class T> struct KeyOf;
template <> struct KeyOf<float> { using U = uint32_t; static constexpr int passes = 4; };
template <> struct KeyOf<double> { using U = unsigned long long; static constexpr int passes = 8; };

__device__ inline float key_from_bits(uint32_t u) {
    return __uint_as_float((u & 0x80000000u) ? (u & 0x7fffffffu) : ~u);
}
__device__ inline double key_from_bits(unsigned long long u) {
    return __longlong_as_double(static_cast<long long>((u & 0x8000000000000000ull) ? (u & 0x7fffffffffffffffull) : ~u));
}

template <class T, class U>
__global__ void k_to_bits(const T* __restrict__ in, int64_t n, int64_t ld, U* __restrict__ out, int32_t* __restrict__ idx) {
    const int p = blockIdx.y;
    for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        out[static_cast<int64_t>(p) * n + i] = key_bits(in[static_cast<int64_t>(p) * ld + i]);
        idx[static_cast<int64_t>(p) * n + i] = static_cast<int32_t>(i);
    }
}

template <class T, class U>
__global__ void k_from_bits(const U* __restrict__ in, int64_t total, T* __restrict__ out) {
    for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < total;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x)
        out[i] = key_from_bits(in[i]);
}

// digit histogram of one tile: hist[(p * 256 + digit) * tiles + tile]
template <class U>
__global__ void __launch_bounds__(RS_THREADS) k_radix_hist(const U* __restrict__ keys, int64_t n, int shift, int tiles,
                                                          int32_t* __restrict__ hist) {
    __shared__ int32_t h[RS_BINS];
    const int p = blockIdx.y, tile = blockIdx.x;
    h[threadIdx.x] = 0;
    __syncthreads();
    const U* seg = keys + static_cast<int64_t>(p) * n;
    const int64_t base = static_cast<int64_t>(tile) * RS_TILE;
#pragma unroll
    for (int r = 0; r < RS_ITEMS; ++r) {
        int64_t i = base + r * RS_THREADS + threadIdx.x;
        if (i < n) atomicAdd(&h[static_cast<int>((seg[i] >> shift) & 0xffu)], 1);
    }
    __syncthreads();
    hist[(static_cast<int64_t>(p) * RS_BINS + threadIdx.x) * tiles + tile] = h[threadIdx.x];
}

// exclusive scan of one segment's 256 x tiles counts (digit-major), in place
__global__ void __launch_bounds__(1024) k_radix_scan(int32_t* __restrict__ hist, int tiles) {
    __shared__ int32_t warp_tot[32];
    __shared__ int32_t carry_s;
    int32_t* h = hist + static_cast<int64_t>(blockIdx.x) * RS_BINS * tiles;
    const int64_t total = static_cast<int64_t>(RS_BINS) * tiles;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (threadIdx.x == 0) carry_s = 0;
    __syncthreads();
    for (int64_t b = 0; b < total; b += 1024) {
        int64_t i = b + threadIdx.x;
        int32_t v = i < total ? h[i] : 0;
        int32_t x = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int32_t y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) warp_tot[warp] = x;
        __syncthreads();
        if (warp == 0) {
            int32_t t = warp_tot[lane];
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                int32_t y = __shfl_up_sync(0xffffffffu, t, o);
                if (lane >= o) t += y;
            }
            warp_tot[lane] = t;  // inclusive
        }
        __syncthreads();
        int32_t carry = carry_s;
        int32_t excl = carry + (warp ? warp_tot[warp - 1] : 0) + x - v;
        if (i < total) h[i] = excl;
        __syncthreads();
        if (threadIdx.x == 1023) carry_s = excl + v;
        __syncthreads();
    }
}

// stable scatter of one tile by the digit at `shift`
template <class U>
__global__ void __launch_bounds__(RS_THREADS) k_radix_scatter(const U* __restrict__ kin, const int32_t* __restrict__ vin,
                                                             int64_t n, int shift, int tiles,
                                                             const int32_t* __restrict__ hist, U* __restrict__ kout,
                                                             int32_t* __restrict__ vout) {
    __shared__ int32_t off[RS_BINS];
    __shared__ int32_t cnt[RS_THREADS / 32][RS_BINS];
    __shared__ int32_t round_tot[RS_BINS];
    const int p = blockIdx.y, tile = blockIdx.x;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t seg = static_cast<int64_t>(p) * n;
    off[threadIdx.x] = hist[(static_cast<int64_t>(p) * RS_BINS + threadIdx.x) * tiles + tile];
    for (int w = 0; w < RS_THREADS / 32; ++w) cnt[w][threadIdx.x] = 0;
    const unsigned lt_mask = (1u << lane) - 1u;
    const int64_t base = static_cast<int64_t>(tile) * RS_TILE;
    __syncthreads();
    for (int r = 0; r < RS_ITEMS; ++r) {
        const int64_t i = base + r * RS_THREADS + threadIdx.x;
        const bool valid = i < n;
        U key = valid ? kin[seg + i] : U(0);
        int32_t val = valid ? vin[seg + i] : 0;
        const int digit = valid ? static_cast<int>((key >> shift) & 0xffu) : RS_BINS + lane;
        const unsigned peers = __match_any_sync(0xffffffffu, digit);
        const int rank = __popc(peers & lt_mask);
        if (valid && rank == 0) cnt[warp][digit] = __popc(peers);
        __syncthreads();
        {  // per digit: exclusive prefix over warps (warp order = stable order)
            int32_t run = 0;
            for (int w = 0; w < RS_THREADS / 32; ++w) {
                int32_t c = cnt[w][threadIdx.x];
                cnt[w][threadIdx.x] = run;
                run += c;
            }
            round_tot[threadIdx.x] = run;
        }
        __syncthreads();
        if (valid) {
            const int32_t pos = off[digit] + cnt[warp][digit] + rank;
            kout[seg + pos] = key;
            vout[seg + pos] = val;
        }
        __syncthreads();
        off[threadIdx.x] += round_tot[threadIdx.x];
        for (int w = 0; w < RS_THREADS / 32; ++w) cnt[w][threadIdx.x] = 0;
        __syncthreads();
    }
}

// ------------------------------------------------------------ sorted pairs and bucket sums

template <class T>
struct KW {
    T key, w;
};

template <class T>
__global__ void k_gather_pairs(const T* __restrict__ keys, const int32_t* __restrict__ idx, const T* __restrict__ w,
                               int64_t total, int64_t n, KW<T>* __restrict__ kw) {
    for (int64_t e = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; e < total;
         e += static_cast<int64_t>(gridDim.x) * blockDim.x)
        kw[e] = KW<T>{keys[e], w[idx[e]]};
}

__device__ inline int bucket_of(float z, float kmin, float kscale, int NB) {
    float f = (z - kmin) * kscale;
    int b = f < 0.0f ? 0 : (f >= static_cast<float>(NB) ? NB - 1 : static_cast<int>(f));
    return b;
}

template <class T>
__global__ void k_bucket_minmax(const KW<T>* __restrict__ kw, int P, int64_t n, int NB, float* kmin, float* kscale) {
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < P; p += gridDim.x * blockDim.x) {
        float lo = static_cast<float>(kw[static_cast<int64_t>(p) * n].key);
        float hi = static_cast<float>(kw[static_cast<int64_t>(p) * n + n - 1].key);
        kmin[p] = lo;
        kscale[p] = hi > lo ? static_cast<float>(NB) / (hi - lo) : 0.0f;
    }
}

// tab[p][b] = first sorted index whose bucket is >= b (b = 0..NB)
template <class T>
__global__ void k_bucket_tab(const KW<T>* __restrict__ kw, int64_t n, int NB, const float* __restrict__ kmin,
                             const float* __restrict__ kscale, int32_t* __restrict__ tab) {
    const int p = blockIdx.y;
    const KW<T>* ks = kw + static_cast<int64_t>(p) * n;
    int32_t* tb = tab + static_cast<int64_t>(p) * (NB + 1);
    const float lo = kmin[p], sc = kscale[p];
    for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const int b = bucket_of(static_cast<float>(ks[i].key), lo, sc, NB);
        const int bp = i > 0 ? bucket_of(static_cast<float>(ks[i - 1].key), lo, sc, NB) : -1;
        for (int q = bp + 1; q <= b; ++q) tb[q] = static_cast<int32_t>(i);
        if (i == n - 1)
            for (int q = b + 1; q <= NB; ++q) tb[q] = static_cast<int32_t>(n);
    }
}

// per bucket sums of w and w z in FP64 (fixed order: the sorted order)
template <class T>
__global__ void k_bucket_sums(const KW<T>* __restrict__ kw, int64_t n, int NB, const int32_t* __restrict__ tab,
                              double2* __restrict__ AB) {
    const int p = blockIdx.y;
    for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < NB; b += gridDim.x * blockDim.x) {
        const int32_t* tb = tab + static_cast<int64_t>(p) * (NB + 1);
        const KW<T>* ks = kw + static_cast<int64_t>(p) * n;
        double a = 0.0, c = 0.0;
        for (int32_t i = tb[b]; i < tb[b + 1]; ++i) {
            const double wv = static_cast<double>(ks[i].w);
            a += wv;
            c += wv * static_cast<double>(ks[i].key);
        }
        AB[static_cast<int64_t>(p) * (NB + 1) + b] = make_double2(a, c);
    }
}

// exclusive FP64 scan of the bucket sums of one slice, in place; AB[NB] = totals
__global__ void __launch_bounds__(1024) k_bucket_prefix(double2* __restrict__ AB, int NB) {
    __shared__ double wa[32], wb[32];
    __shared__ double ca_s, cb_s;
    double2* row = AB + static_cast<int64_t>(blockIdx.x) * (NB + 1);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (threadIdx.x == 0) {
        ca_s = 0.0;
        cb_s = 0.0;
    }
    __syncthreads();
    for (int base = 0; base < NB; base += 1024) {
        const int b = base + threadIdx.x;
        const double2 v = b < NB ? row[b] : make_double2(0.0, 0.0);
        double xa = v.x, xb = v.y;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const double ya = __shfl_up_sync(0xffffffffu, xa, o), yb = __shfl_up_sync(0xffffffffu, xb, o);
            if (lane >= o) {
                xa += ya;
                xb += yb;
            }
        }
        if (lane == 31) {
            wa[warp] = xa;
            wb[warp] = xb;
        }
        __syncthreads();
        if (warp == 0) {
            double sa = wa[lane], sb = wb[lane];
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const double ya = __shfl_up_sync(0xffffffffu, sa, o), yb = __shfl_up_sync(0xffffffffu, sb, o);
                if (lane >= o) {
                    sa += ya;
                    sb += yb;
                }
            }
            wa[lane] = sa;
            wb[lane] = sb;
        }
        __syncthreads();
        const double ca = ca_s, cb = cb_s;
        const double ea = ca + (warp ? wa[warp - 1] : 0.0) + xa - v.x;
        const double eb = cb + (warp ? wb[warp - 1] : 0.0) + xb - v.y;
        if (b < NB) row[b] = make_double2(ea, eb);
        __syncthreads();
        if (threadIdx.x == 1023) {
            ca_s = ea + v.x;
            cb_s = eb + v.y;
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) row[NB] = make_double2(ca_s, cb_s);
}

// ------------------------------------------------------------ targets

// Slices [p0, p1): for target m, bucket b of z; A_< and B_< from the bucket's FP64
// prefix plus the sorted pairs of bucket b below z (and A_<= for the gradient).
template <class T>
__global__ void __launch_bounds__(256) k_negdist_target(const T* __restrict__ Z, int P, int p0, int p1, int64_t n,
                                                       int64_t ldz, const KW<T>* __restrict__ kw, int64_t nx,
                                                       const double2* __restrict__ AB, int NB,
                                                       const float* __restrict__ kmin, const float* __restrict__ kscale,
                                                       const int32_t* __restrict__ tab, double cd, double scale,
                                                       double* __restrict__ acc, T* __restrict__ G, int accumulate_G) {
    const int64_t m = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (m >= n) return;
    double sum = 0.0;
    for (int p = p0; p < p1; ++p) {
        const T z = Z[static_cast<int64_t>(p) * ldz + m];
        const KW<T>* ks = kw + static_cast<int64_t>(p) * nx;
        const int32_t* tb = tab + static_cast<int64_t>(p) * (NB + 1);
        const double2* ab = AB + static_cast<int64_t>(p) * (NB + 1);
        const int b = bucket_of(static_cast<float>(z), kmin[p], kscale[p], NB);
        const int32_t hi = tb[b + 1];
        int32_t i = tb[b];
        T a = T(0), bz = T(0);
        for (; i < hi; ++i) {
            const KW<T> e = ks[i];
            if (!(e.key < z)) break;
            a += e.w;
            bz += e.w * e.key;
        }
        const double2 base = ab[b], tot = ab[NB];
        const double Al = base.x + static_cast<double>(a);
        if (G) {
            T aeq = T(0);
            for (; i < hi; ++i) {
                const KW<T> e = ks[i];
                if (e.key != z) break;
                aeq += e.w;
            }
            const double g = scale * cd * (tot.x - 2.0 * Al - static_cast<double>(aeq));
            T* gp = G + m * P + p;
            *gp = accumulate_G ? static_cast<T>(static_cast<double>(*gp) + g) : static_cast<T>(g);
        } else {
            const double Bl = base.y + static_cast<double>(bz);
            const double zd = static_cast<double>(z);
            sum += -cd * (zd * (2.0 * Al - tot.x) - (2.0 * Bl - tot.y));
        }
    }
    if (!G) acc[m] += scale * sum;
}

}  // namespace

// ------------------------------------------------------------ launchers

template <class T>
size_t segmented_sort_scratch(int P, int64_t n) {
    using U = typename KeyOf<T>::U;
    int64_t tiles = ceil_div(n, RS_TILE);
    size_t total = static_cast<size_t>(P) * n;
    return 2 * total * sizeof(U) + total * sizeof(int32_t) + static_cast<size_t>(P) * RS_BINS * tiles * sizeof(int32_t) +
           1024;
}

template <class T>
void launch_segmented_sort(const T* keys_in, int P, int64_t n, int64_t ldk, T* keys_out, int32_t* idx_out,
                           void* scratch, size_t scratch_bytes, cudaStream_t st) {
    using U = typename KeyOf<T>::U;
    SLK_REQUIRE(n < (int64_t(1) << 31), "segments longer than 2^31 are not supported");
    SLK_REQUIRE(scratch_bytes >= segmented_sort_scratch<T>(P, n), "sort scratch too small");
    SLK_REQUIRE(P <= 65535, "too many segments for one sort launch");
    const int tiles = static_cast<int>(ceil_div(n, RS_TILE));
    const size_t total = static_cast<size_t>(P) * n;
    unsigned char* s = static_cast<unsigned char*>(scratch);
    U* kb0 = reinterpret_cast<U*>(s);
    U* kb1 = kb0 + total;
    int32_t* v1 = reinterpret_cast<int32_t*>(kb1 + total);
    int32_t* hist = v1 + total;
    int32_t* v0 = idx_out;
    dim3 g1(static_cast<unsigned>(ceil_div(n, 256) < 1024 ? ceil_div(n, 256) : 1024), P);
    {
        SLK_TIMED("to_bits", st);
        k_to_bits<T, U><<<g1, 256, 0, st>>>(keys_in, n, ldk, kb0, v0);
    }
    SLK_CHECK_LAUNCH();
    dim3 gt(tiles, P);
    U* kin = kb0;
    U* kout = kb1;
    int32_t* vin = v0;
    int32_t* vout = v1;
    for (int pass = 0; pass < KeyOf<T>::passes; ++pass) {
        const int shift = 8 * pass;
        {
            SLK_TIMED("radix_hist", st);
            k_radix_hist<U><<<gt, RS_THREADS, 0, st>>>(kin, n, shift, tiles, hist);
        }
        SLK_CHECK_LAUNCH();
        {
            SLK_TIMED("radix_scan", st);
            k_radix_scan<<<P, 1024, 0, st>>>(hist, tiles);
        }
        SLK_CHECK_LAUNCH();
        {
            SLK_TIMED("radix_scatter", st);
            k_radix_scatter<U><<<gt, RS_THREADS, 0, st>>>(kin, vin, n, shift, tiles, hist, kout, vout);
        }
        SLK_CHECK_LAUNCH();
        U* tk = kin;
        kin = kout;
        kout = tk;
        int32_t* tv = vin;
        vin = vout;
        vout = tv;
    }
    // an even number of passes leaves keys in kb0 and payload in idx_out
    int64_t tot = static_cast<int64_t>(total);
    {
        SLK_TIMED("from_bits", st);
        k_from_bits<T, U><<<static_cast<unsigned>(ceil_div(tot, 256) < 16384 ? ceil_div(tot, 256) : 16384), 256, 0, st>>>(
            kin, tot, keys_out);
    }
    SLK_CHECK_LAUNCH();
}

template <class T>
int64_t sorted_pairs_bytes(int P, int64_t n) {
    return static_cast<int64_t>(sizeof(KW<T>)) * P * n;
}

template <class T>
void launch_sorted_pairs(const T* keys, const int32_t* idx, const T* w, int P, int64_t n, void* kw, int NB,
                         float* kmin, float* kscale, int32_t* tab, double2* AB, cudaStream_t st) {
    const int64_t total = static_cast<int64_t>(P) * n;
    KW<T>* pairs = static_cast<KW<T>*>(kw);
    {
        SLK_TIMED("gather_pairs", st);
        k_gather_pairs<T><<<static_cast<unsigned>(ceil_div(total, 256) < 16384 ? ceil_div(total, 256) : 16384), 256, 0,
                            st>>>(keys, idx, w, total, n, pairs);
    }
    SLK_CHECK_LAUNCH();
    {
        SLK_TIMED("bucket_minmax", st);
        k_bucket_minmax<T><<<static_cast<unsigned>(ceil_div(P, 128)), 128, 0, st>>>(pairs, P, n, NB, kmin, kscale);
    }
    SLK_CHECK_LAUNCH();
    {
        SLK_TIMED("bucket_tab", st);
        dim3 g(static_cast<unsigned>(ceil_div(n, 256) < 1024 ? ceil_div(n, 256) : 1024), P);
        k_bucket_tab<T><<<g, 256, 0, st>>>(pairs, n, NB, kmin, kscale, tab);
    }
    SLK_CHECK_LAUNCH();
    {
        SLK_TIMED("bucket_sums", st);
        dim3 g(static_cast<unsigned>(ceil_div(NB, 256)), P);
        k_bucket_sums<T><<<g, 256, 0, st>>>(pairs, n, NB, tab, AB);
    }
    SLK_CHECK_LAUNCH();
    {
        SLK_TIMED("bucket_prefix", st);
        k_bucket_prefix<<<P, 1024, 0, st>>>(AB, NB);
    }
    SLK_CHECK_LAUNCH();
}

template <class T>
void launch_negdist_target(const T* Z, int P, int64_t n, int64_t ldz, const void* kw, int64_t nx, const double2* AB,
                           int NB, const float* kmin, const float* kscale, const int32_t* tab, double cd, double scale,
                           double* acc, T* G, int accumulate_G, cudaStream_t st) {
    if (n <= 0) return;
    // slices per launch: keep one batch's pairs (the randomly accessed state) within ~64 MB of L2
    const int64_t per_slice = static_cast<int64_t>(sizeof(KW<T>)) * nx + static_cast<int64_t>(NB + 1) * 20;
    int batch = static_cast<int>((int64_t(64) << 20) / (per_slice > 0 ? per_slice : 1));
    if (batch < 1) batch = 1;
    if (batch > P) batch = P;
    for (int p0 = 0; p0 < P; p0 += batch) {
        const int p1 = p0 + batch < P ? p0 + batch : P;
        SLK_TIMED(G ? "negdist_target_grad" : "negdist_target", st);
        k_negdist_target<T><<<static_cast<unsigned>(ceil_div(n, 256)), 256, 0, st>>>(
            Z, P, p0, p1, n, ldz, static_cast<const KW<T>*>(kw), nx, AB, NB, kmin, kscale, tab, cd, scale, acc, G,
            accumulate_G);
        SLK_CHECK_LAUNCH();
    }
}

#define SLK_INST(T)                                                                                                   \
    template size_t segmented_sort_scratch<T>(int, int64_t);                                                          \
    template void launch_segmented_sort<T>(const T*, int, int64_t, int64_t, T*, int32_t*, void*, size_t, cudaStream_t); \
    template int64_t sorted_pairs_bytes<T>(int, int64_t);                                                             \
    template void launch_sorted_pairs<T>(const T*, const int32_t*, const T*, int, int64_t, void*, int, float*, float*, \
                                         int32_t*, double2*, cudaStream_t);                                           \
    template void launch_negdist_target<T>(const T*, int, int64_t, int64_t, const void*, int64_t, const double2*, int, \
                                           const float*, const float*, const int32_t*, double, double, double*, T*,   \
                                           int, cudaStream_t);
SLK_INST(float)
SLK_INST(double)
#undef SLK_INST

}  // namespace slk
