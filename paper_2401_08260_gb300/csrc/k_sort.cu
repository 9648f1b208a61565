// Sorting route of Section 3.2 (negative distance kernel; the non-smooth part
// of the Laplacian in Section 3.3).
//
// Per slice the key range [min z, max z] of the sources is cut into NB buckets of equal
// width, and the sources are grouped by bucket (a segmented stable LSD radix sort on the
// digits of the bucket index, one 8-bit pass per byte of NB - 1, carrying the weight) into
// (key, w) pairs, ascending by bucket and in source order within a bucket.  Exclusive
// prefix sums of w and w z are kept only at bucket starts:
//     A_b = sum over sources in buckets < b of w,   B_b = same of w z.
// A target z in bucket b then has
//     A_< = A_b + sum_{sources of bucket b with key < z} w,   B_< likewise,
// (a scan of bucket b's few sources, in any order) and
//     t(z) = -c_d sum_n w_n |z - x_n| = -c_d [ z (2 A_< - W) - (2 B_< - S) ],
// W, S the totals.  This is Algorithm 2 regrouped: splitting the sum at z gives
//     sum_{x<z} w (z - x) + sum_{x>=z} w (x - z) = z (2 A_< - W) - (2 B_< - S),
// the same value without the joint sort of sources and targets.
#include "kernels.cuh"

namespace slk {

namespace {

constexpr int RS_THREADS = 256, RS_ITEMS = 8, RS_TILE = RS_THREADS * RS_ITEMS, RS_BINS = 256;

template <class T> struct KeyOf;
template <> struct KeyOf<float> { using U = uint32_t; static constexpr int passes = 4; };
template <> struct KeyOf<double> { using U = unsigned long long; static constexpr int passes = 8; };

__device__ inline float key_from_bits(uint32_t u) {
    return __uint_as_float((u & 0x80000000u) ? (u & 0x7fffffffu) : ~u);
}
__device__ inline double key_from_bits(unsigned long long u) {
    return __longlong_as_double(static_cast<long long>((u & 0x8000000000000000ull) ? (u & 0x7fffffffffffffffull) : ~u));
}

template <class T>
struct KW {
    T key, w;
};

// Equal-width key buckets of a slice: b = floor((z - kmin) * kscale) clamped to [0, NB).
__device__ inline int bucket_of(float z, float kmin, float kscale, int NB) {
    float f = (z - kmin) * kscale;
    int b = f < 0.0f ? 0 : (f >= static_cast<float>(NB) ? NB - 1 : static_cast<int>(f));
    return b;
}

// Radix digit of a key: its own bits (a full sort), or the bits of its slice's bucket index
// (BUCKETED: the keys end up grouped by bucket, in source order within a bucket).
struct Buckets {
    const float* kmin;
    const float* kscale;
    int NB;
    int mask;  // digit mask of a pass (digits of dbits <= 8 bits)
};
// The digit function of a slice, its bucket geometry read once per thread (read through the
// Buckets pointers at every use it would be reloaded after each global store)
template <bool BUCKETED>
struct DigitOf {
    float lo = 0.0f, sc = 0.0f;
    int NB = 0, mask = 0xff;
    __device__ __forceinline__ DigitOf(const Buckets& bk, int p) {
        if (BUCKETED) {
            lo = bk.kmin[p];
            sc = bk.kscale[p];
            NB = bk.NB;
            mask = bk.mask;
        }
    }
    template <class U>
    __device__ __forceinline__ int operator()(U k, int shift) const {
        if constexpr (BUCKETED)
            return (bucket_of(static_cast<float>(key_from_bits(k)), lo, sc, NB) >> shift) & mask;
        else
            return static_cast<int>((k >> shift) & 0xffu);
    }
};

// Key bits and payload of the intermediate passes, interleaved (one store per key)
template <class U, class T>
struct alignas(sizeof(U) + sizeof(T)) KV {
    U k;
    T v;
};

// Digit histogram of one tile: hist[(p * 256 + digit) * tiles + tile].  FIRST: the keys are
// the order-preserving bits of the projections z (row stride ldz), otherwise the bits array.
template <class T, class U, bool FIRST, bool BUCKETED>
__global__ void __launch_bounds__(RS_THREADS) k_radix_hist(const T* __restrict__ z, int64_t ldz,
                                                          const KV<U, T>* __restrict__ keys, int64_t n, int shift,
                                                          int tiles, int32_t* __restrict__ hist, Buckets bk) {
    __shared__ int32_t h[RS_BINS];
    const int p = blockIdx.y, tile = blockIdx.x;
    h[threadIdx.x] = 0;
    __syncthreads();
    const int64_t base = static_cast<int64_t>(tile) * RS_TILE;
    // all loads first (they are independent), then the shared-memory counts
    U k[RS_ITEMS];
#pragma unroll
    for (int r = 0; r < RS_ITEMS; ++r) {
        const int64_t i = base + r * RS_THREADS + threadIdx.x;
        if (i < n) k[r] = FIRST ? key_bits(z[static_cast<int64_t>(p) * ldz + i]) : keys[static_cast<int64_t>(p) * n + i].k;
    }
    const DigitOf<BUCKETED> digit_of(bk, p);
#pragma unroll
    for (int r = 0; r < RS_ITEMS; ++r) {
        const int64_t i = base + r * RS_THREADS + threadIdx.x;
        if (i < n) atomicAdd(&h[digit_of(k[r], shift)], 1);
    }
    __syncthreads();
    hist[(static_cast<int64_t>(p) * RS_BINS + threadIdx.x) * tiles + tile] = h[threadIdx.x];
}

// Exclusive scan of one (slice, digit) row of per-tile counts, in place; the row total
// goes to rt[p * 256 + digit].  Rows are independent (P x 256 blocks); each block walks its
// row in coalesced 256-wide chunks, carrying the running total.
__global__ void __launch_bounds__(256) k_radix_scan_rows(int32_t* __restrict__ hist, int tiles, int32_t* __restrict__ rt) {
    __shared__ int32_t warp_tot[8];
    const int row = blockIdx.y * RS_BINS + blockIdx.x;
    int32_t* h = hist + static_cast<int64_t>(row) * tiles;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int32_t carry = 0;
    for (int base = 0; base < tiles; base += 256) {
        const int j = base + threadIdx.x;
        const int32_t v = j < tiles ? h[j] : 0;
        int32_t x = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int32_t y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) warp_tot[warp] = x;
        __syncthreads();
        int32_t before = carry, chunk = 0;
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const int32_t t = warp_tot[q];
            if (q < warp) before += t;
            chunk += t;
        }
        if (j < tiles) h[j] = before + x - v;
        carry += chunk;
        __syncthreads();
    }
    if (threadIdx.x == 0) rt[row] = carry;
}

// Exclusive scan of the 256 digit totals of each slice, in place (digit bases).
__global__ void __launch_bounds__(256) k_radix_scan_digits(int32_t* __restrict__ rt) {
    __shared__ int32_t warp_tot[8];
    int32_t* r = rt + static_cast<int64_t>(blockIdx.x) * RS_BINS;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int32_t v = r[threadIdx.x];
    int32_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) warp_tot[warp] = x;
    __syncthreads();
    int32_t base = 0;
    for (int q = 0; q < warp; ++q) base += warp_tot[q];
    r[threadIdx.x] = base + x - v;
}

constexpr int RS_WARPS = RS_THREADS / 32;

template <class T, class U>
constexpr size_t radix_pass_smem() {
    return static_cast<size_t>(RS_TILE) * (sizeof(U) + sizeof(T)) + (RS_WARPS + 2) * RS_BINS * sizeof(int32_t);
}

// One stable LSD pass over a tile of RS_TILE keys with their payload (the source weight).
// Each warp ranks a contiguous run of RS_TILE / RS_WARPS keys with warp-private digit
// counters (match_any per 32 keys); per-digit prefixes over the warps and over the digits
// give every key its place in the tile's digit-sorted order, the tile is reordered in shared
// memory, and each digit's run is written to its global offset (from the scanned histogram)
// in contiguous stores.  FIRST reads the projections and the weights (source index order);
// LAST writes (key, w) pairs instead of the interleaved bits and payload.
template <class T, class U, bool FIRST, bool LAST, bool BUCKETED>
__global__ void __launch_bounds__(RS_THREADS, 5) k_radix_pass(const T* __restrict__ z, int64_t ldz, const T* __restrict__ w,
                                                          const KV<U, T>* __restrict__ kvin, int64_t n, int shift,
                                                          int tiles, const int32_t* __restrict__ hist,
                                                          const int32_t* __restrict__ dbase,
                                                          KV<U, T>* __restrict__ kvout, KW<T>* __restrict__ pout,
                                                          Buckets bk) {
    extern __shared__ __align__(16) unsigned char rs_smem[];
    U* sk = reinterpret_cast<U*>(rs_smem);
    T* sv = reinterpret_cast<T*>(sk + RS_TILE);
    int32_t* wcnt = reinterpret_cast<int32_t*>(sv + RS_TILE);  // [warp][digit]
    int32_t* loc = wcnt + RS_WARPS * RS_BINS;                   // tile-local start of each digit
    int32_t* glob = loc + RS_BINS;                              // global start of each digit for this tile
    const int p = blockIdx.y, tile = blockIdx.x;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t seg = static_cast<int64_t>(p) * n;
    const int64_t base = static_cast<int64_t>(tile) * RS_TILE;
    for (int i = threadIdx.x; i < RS_WARPS * RS_BINS; i += RS_THREADS) wcnt[i] = 0;
    glob[threadIdx.x] = hist[(static_cast<int64_t>(p) * RS_BINS + threadIdx.x) * tiles + tile] +
                        dbase[p * RS_BINS + threadIdx.x];
    __syncthreads();

    constexpr int RUN = RS_TILE / RS_WARPS;  // keys per warp
    U key[RS_ITEMS];
    T val[RS_ITEMS];
    int rank[RS_ITEMS];
    int32_t* mycnt = wcnt + warp * RS_BINS;
    const unsigned lt_mask = (1u << lane) - 1u;
#pragma unroll
    for (int r = 0; r < RS_ITEMS; ++r) {
        const int64_t e = base + warp * RUN + r * 32 + lane;
        const bool valid = e < n;
        if (FIRST) {
            key[r] = valid ? key_bits(z[static_cast<int64_t>(p) * ldz + e]) : U(0);
            val[r] = valid ? w[e] : T(0);
        } else {
            const KV<U, T> kv = valid ? kvin[seg + e] : KV<U, T>{U(0), T(0)};
            key[r] = kv.k;
            val[r] = kv.v;
        }
    }
    const DigitOf<BUCKETED> digit_of(bk, p);
#pragma unroll
    for (int r = 0; r < RS_ITEMS; ++r) {
        const int64_t e = base + warp * RUN + r * 32 + lane;
        const bool valid = e < n;
        const int digit = valid ? digit_of(key[r], shift) : RS_BINS + lane;
        const unsigned peers = __match_any_sync(0xffffffffu, digit);
        const int before = valid ? mycnt[digit] : 0;
        rank[r] = before + __popc(peers & lt_mask);
        __syncwarp();
        if (valid && (peers & lt_mask) == 0u) mycnt[digit] = before + __popc(peers);
        __syncwarp();
    }
    __syncthreads();
    // per digit: exclusive prefix over the warps (warp order = input order), tile total
    const int t = threadIdx.x;
    int32_t run = 0;
#pragma unroll
    for (int q = 0; q < RS_WARPS; ++q) {
        const int32_t c = wcnt[q * RS_BINS + t];
        wcnt[q * RS_BINS + t] = run;
        run += c;
    }
    // exclusive scan of the digit totals over the 256 digits
    {
        int32_t x = run;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int32_t y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        __shared__ int32_t wt[RS_WARPS];
        if (lane == 31) wt[warp] = x;
        __syncthreads();
        int32_t off = 0;
        for (int q = 0; q < warp; ++q) off += wt[q];
        loc[t] = off + x - run;
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < RS_ITEMS; ++r) {
        const int64_t e = base + warp * RUN + r * 32 + lane;
        if (e < n) {
            const int digit = digit_of(key[r], shift);
            const int pos = loc[digit] + wcnt[warp * RS_BINS + digit] + rank[r];
            sk[pos] = key[r];
            sv[pos] = val[r];
        }
    }
    __syncthreads();
    const int cnt = static_cast<int>(n - base < RS_TILE ? n - base : RS_TILE);
    for (int j = threadIdx.x; j < cnt; j += RS_THREADS) {
        const U k = sk[j];
        const int digit = digit_of(k, shift);
        const int64_t g = seg + glob[digit] + (j - loc[digit]);
        if (LAST) pout[g] = KW<T>{key_from_bits(k), sv[j]};
        else kvout[g] = KV<U, T>{k, sv[j]};
    }
}

// ------------------------------------------------------------ sorted pairs and bucket sums


// Bucket geometry of every slice from its projections (one block per slice): kmin = the
// smallest key, kscale = NB / (largest - smallest) (0 when all keys are equal), in the same
// float arithmetic as bucket_of.
template <class T>
__global__ void __launch_bounds__(256) k_slice_minmax(const T* __restrict__ Z, int64_t n, int64_t ldz, int NB,
                                                     float* __restrict__ kmin, float* __restrict__ kscale) {
    const int p = blockIdx.x;
    const T* row = Z + static_cast<int64_t>(p) * ldz;
    float lo = INFINITY, hi = -INFINITY;
    for (int64_t i = threadIdx.x; i < n; i += 256) {
        const float v = static_cast<float>(row[i]);
        lo = fminf(lo, v);
        hi = fmaxf(hi, v);
    }
    __shared__ float slo[8], shi[8];
    for (int o = 16; o > 0; o >>= 1) {
        lo = fminf(lo, __shfl_xor_sync(0xffffffffu, lo, o));
        hi = fmaxf(hi, __shfl_xor_sync(0xffffffffu, hi, o));
    }
    if ((threadIdx.x & 31) == 0) {
        slo[threadIdx.x >> 5] = lo;
        shi[threadIdx.x >> 5] = hi;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int k = 1; k < 8; ++k) {
            lo = fminf(lo, slo[k]);
            hi = fmaxf(hi, shi[k]);
        }
        lo = fminf(lo, slo[0]);
        hi = fmaxf(hi, shi[0]);
        kmin[p] = lo;
        kscale[p] = hi > lo ? static_cast<float>(NB) / (hi - lo) : 0.0f;
    }
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

// Exact-enough sums without FP64 arithmetic in the hot loops (FP64 runs at a small
// fraction of the FP32 rate on this GPU): a value is an unevaluated pair hi + lo of floats
// ("double-float", about 44 significant bits).  TwoSum (Knuth) adds without rounding loss,
// and a product w key is split exactly into p + e with an FMA, e = fma(w, key, -p).
struct DF {
    float hi, lo;
};
__device__ __forceinline__ DF df_norm(float hi, float lo) {
    const float s = hi + lo;
    return DF{s, lo - (s - hi)};
}
__device__ __forceinline__ DF df_add(DF a, DF b) {
    const float s = a.hi + b.hi, v = s - a.hi;
    const float e = (a.hi - (s - v)) + (b.hi - v) + a.lo + b.lo;
    return df_norm(s, e);
}
__device__ __forceinline__ DF df_shfl_up(DF a, int o) {
    return DF{__shfl_up_sync(0xffffffffu, a.hi, o), __shfl_up_sync(0xffffffffu, a.lo, o)};
}
__device__ __forceinline__ DF df_shfl_down(DF a, int o) {
    return DF{__shfl_down_sync(0xffffffffu, a.hi, o), __shfl_down_sync(0xffffffffu, a.lo, o)};
}
__device__ __forceinline__ DF df_from(double d) {
    const float hi = static_cast<float>(d);
    return DF{hi, static_cast<float>(d - static_cast<double>(hi))};
}
__device__ __forceinline__ double df_value(DF a) { return static_cast<double>(a.hi) + static_cast<double>(a.lo); }

// Prefix entry at a bucket start: sums of w and w key before it.  FP32 data: double-float
// pairs (no FP64 arithmetic on the target side); FP64 data: doubles.  16 bytes either way.
template <class T>
struct Pre;
template <>
struct Pre<float> {
    float ahi, alo, bhi, blo;
};
template <>
struct Pre<double> {
    double a, b;
};

// One bucket of one slice: the prefix entry at its first sorted index, that index and the
// first index of the next bucket, in one 32-byte (one-sector) record.
template <class T>
struct alignas(32) BucketRec {
    Pre<T> e;
    int32_t start, end;
    int32_t pad[2];
};
static_assert(sizeof(BucketRec<float>) == kBucketRecordBytes && sizeof(BucketRec<double>) == kBucketRecordBytes,
              "bucket records are 32 bytes");

// Running sums (w, w key) over sorted pairs, and their scan arithmetic.
template <class T>
struct PairSum;
template <>
struct PairSum<float> {
    DF a{0.0f, 0.0f}, b{0.0f, 0.0f};
    __device__ __forceinline__ void add(float w, float key) {
        // TwoSum into (hi, lo) without renormalising every step
        float s = a.hi + w, bp = s - a.hi;
        a.lo += (a.hi - (s - bp)) + (w - bp);
        a.hi = s;
        const float pr = w * key;
        s = b.hi + pr;
        bp = s - b.hi;
        b.lo += (b.hi - (s - bp)) + (pr - bp) + fmaf(w, key, -pr);
        b.hi = s;
    }
    __device__ __forceinline__ void norm() {
        a = df_norm(a.hi, a.lo);
        b = df_norm(b.hi, b.lo);
    }
    __device__ __forceinline__ void plus(const PairSum& o) {
        a = df_add(a, o.a);
        b = df_add(b, o.b);
    }
    __device__ __forceinline__ PairSum shfl_up(int o) const {
        PairSum r;
        r.a = df_shfl_up(a, o);
        r.b = df_shfl_up(b, o);
        return r;
    }
    __device__ __forceinline__ PairSum shfl_down(int o) const {
        PairSum r;
        r.a = df_shfl_down(a, o);
        r.b = df_shfl_down(b, o);
        return r;
    }
    __device__ __forceinline__ double2 to_double2() const { return make_double2(df_value(a), df_value(b)); }
    __device__ static PairSum from_double2(double2 v) {
        PairSum r;
        r.a = df_from(v.x);
        r.b = df_from(v.y);
        return r;
    }
    __device__ __forceinline__ Pre<float> entry() const { return Pre<float>{a.hi, a.lo, b.hi, b.lo}; }
    __device__ static PairSum from_pair(float sa, float sb) {
        PairSum r;
        r.a = DF{sa, 0.0f};
        r.b = DF{sb, 0.0f};
        return r;
    }
};
template <>
struct PairSum<double> {
    double a = 0.0, b = 0.0;
    __device__ __forceinline__ void add(double w, double key) {
        a += w;
        b = fma(w, key, b);
    }
    __device__ __forceinline__ void norm() {}
    __device__ __forceinline__ void plus(const PairSum& o) {
        a += o.a;
        b += o.b;
    }
    __device__ __forceinline__ PairSum shfl_up(int o) const {
        PairSum r;
        r.a = __shfl_up_sync(0xffffffffu, a, o);
        r.b = __shfl_up_sync(0xffffffffu, b, o);
        return r;
    }
    __device__ __forceinline__ PairSum shfl_down(int o) const {
        PairSum r;
        r.a = __shfl_down_sync(0xffffffffu, a, o);
        r.b = __shfl_down_sync(0xffffffffu, b, o);
        return r;
    }
    __device__ __forceinline__ double2 to_double2() const { return make_double2(a, b); }
    __device__ static PairSum from_double2(double2 v) {
        PairSum r;
        r.a = v.x;
        r.b = v.y;
        return r;
    }
    __device__ __forceinline__ Pre<double> entry() const { return Pre<double>{a, b}; }
    __device__ static PairSum from_pair(double sa, double sb) {
        PairSum r;
        r.a = sa;
        r.b = sb;
        return r;
    }
};

constexpr int PS_THREADS = 256, PS_ITEMS = 8, PS_CHUNK = PS_THREADS * PS_ITEMS;

// per chunk of PS_CHUNK sorted pairs: (sum w, sum w key) in FP64; cs[p][c], row length nchunk + 1
template <class T>
__global__ void __launch_bounds__(PS_THREADS) k_pair_chunk_sums(const KW<T>* __restrict__ kw, int64_t n, int nchunk,
                                                               double2* __restrict__ cs) {
    __shared__ PairSum<T> red[PS_THREADS / 32];
    const int p = blockIdx.y, c = blockIdx.x;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const KW<T>* ks = kw + static_cast<int64_t>(p) * n;
    const int64_t i0 = static_cast<int64_t>(c) * PS_CHUNK + threadIdx.x;
    // a thread's PS_ITEMS pairs in plain arithmetic (their rounding is ~2^-24 of a sum of
    // eight terms, negligible against the prefixes); double-float from there on
    T sa = T(0), sb = T(0);
#pragma unroll
    for (int r = 0; r < PS_ITEMS; ++r) {  // coalesced; a fixed order within the chunk
        const int64_t i = i0 + r * PS_THREADS;
        if (i < n) {
            const KW<T> e = ks[i];
            sa += e.w;
            sb = fma(e.w, e.key, sb);
        }
    }
    PairSum<T> acc = PairSum<T>::from_pair(sa, sb);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc.plus(acc.shfl_down(o));
    if (lane == 0) red[warp] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        PairSum<T> t = red[0];
        for (int q = 1; q < PS_THREADS / 32; ++q) t.plus(red[q]);
        cs[static_cast<int64_t>(p) * (nchunk + 1) + c] = t.to_double2();
    }
}

// A prefix entry from lane src of the warp
__device__ __forceinline__ Pre<float> shfl_pre(const Pre<float>& e, int src) {
    return Pre<float>{__shfl_sync(0xffffffffu, e.ahi, src), __shfl_sync(0xffffffffu, e.alo, src),
                      __shfl_sync(0xffffffffu, e.bhi, src), __shfl_sync(0xffffffffu, e.blo, src)};
}
__device__ __forceinline__ Pre<double> shfl_pre(const Pre<double>& e, int src) {
    return Pre<double>{__shfl_sync(0xffffffffu, e.a, src), __shfl_sync(0xffffffffu, e.b, src)};
}

// One whole 32-byte record in one store (a record written in pieces leaves partial sectors,
// which the memory system completes with a read of the sector from DRAM)
template <class T>
__device__ __forceinline__ void store_record(BucketRec<T>* dst, const Pre<T>& e, int32_t start, int32_t end) {
    static_assert(sizeof(Pre<T>) == 16, "prefix entries are 16 bytes");
    uint32_t v[8];
    memcpy(v, &e, sizeof(e));
    v[4] = static_cast<uint32_t>(start);
    v[5] = static_cast<uint32_t>(end);
    v[6] = 0u;
    v[7] = 0u;
    asm volatile("st.global.v8.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};" ::"l"(dst), "r"(v[0]), "r"(v[1]),
                 "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]), "r"(v[7])
                 : "memory");
}

// Bucket records from the sorted pairs and the scanned chunk sums (cs[p][c] = exclusive
// prefix before chunk c): the thread holding the first pair i of bucket b writes record b
// whole (prefix entry before i, start i, end = the first pair of a higher bucket), together
// with the records of the empty buckets just below b (start = end = i); the thread of the
// last pair also writes the records above its bucket (record NB holds the totals).  Each
// thread takes PS_ITEMS consecutive pairs; a bucket's end, when it lies beyond the thread's
// pairs, comes from a block-wide scan of the threads' first bucket starts (and, past the
// block's chunk, from one look-ahead per block).
template <class T>
__global__ void __launch_bounds__(PS_THREADS) k_pair_prefix_tab(const KW<T>* __restrict__ kw, int64_t n, int nchunk,
                                                               const double2* __restrict__ cs, int NB,
                                                               const float* __restrict__ kmin,
                                                               const float* __restrict__ kscale,
                                                               BucketRec<T>* __restrict__ rec) {
    __shared__ PairSum<T> wsum[PS_THREADS / 32];
    __shared__ PairSum<T> chunk_start;
    __shared__ int64_t warp_next[PS_THREADS / 32];
    __shared__ int64_t block_next;
    const int p = blockIdx.y, c = blockIdx.x;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const KW<T>* ks = kw + static_cast<int64_t>(p) * n;
    BucketRec<T>* rb = rec + static_cast<int64_t>(p) * (NB + 1);
    const float lo = kmin[p], sc = kscale[p];
    const int64_t i0 = static_cast<int64_t>(c) * PS_CHUNK + static_cast<int64_t>(threadIdx.x) * PS_ITEMS;
    if (threadIdx.x == 0) chunk_start = PairSum<T>::from_double2(cs[static_cast<int64_t>(p) * (nchunk + 1) + c]);
    KW<T> el[PS_ITEMS];
    T sa = T(0), sb = T(0);  // this thread's PS_ITEMS pairs in plain arithmetic
#pragma unroll
    for (int r = 0; r < PS_ITEMS; ++r) {
        const int64_t i = i0 + r;
        el[r] = i < n ? ks[i] : KW<T>{T(0), T(0)};
        sa += el[r].w;
        sb = fma(el[r].w, el[r].key, sb);
    }
    const PairSum<T> own = PairSum<T>::from_pair(sa, sb);
    // inclusive scan of the thread totals within the warp, then the warps in order
    PairSum<T> x = own;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const PairSum<T> y = x.shfl_up(o);
        if (lane >= o) {
            PairSum<T> t = y;
            t.plus(x);
            x = t;
        }
    }
    if (lane == 31) wsum[warp] = x;
    __syncthreads();
    PairSum<T> start = chunk_start;
    for (int q = 0; q < warp; ++q) start.plus(wsum[q]);
    // exclusive: the warp's inclusive value one lane up (zero in lane 0)
    PairSum<T> prev = x.shfl_up(1);
    if (lane > 0) start.plus(prev);
    start.norm();
    T la = T(0), lb = T(0);  // the run within this thread's pairs, plain arithmetic
    int bprev = i0 == 0 ? -1 : (i0 < n ? bucket_of(static_cast<float>(ks[i0 - 1].key), lo, sc, NB) : NB);
    // bucket of every pair (NB past the end, so that index n starts the sentinel "bucket")
    int bk[PS_ITEMS];
#pragma unroll
    for (int r = 0; r < PS_ITEMS; ++r) bk[r] = i0 + r < n ? bucket_of(static_cast<float>(el[r].key), lo, sc, NB) : NB;
    // first bucket start among this thread's positions (n counts as one), then the first one
    // after this thread: a suffix minimum over the block's threads
    constexpr int64_t kNone = INT64_MAX;
    int64_t first = kNone;
#pragma unroll
    for (int r = PS_ITEMS - 1; r >= 0; --r)
        if (i0 + r <= n && bk[r] > (r ? bk[r - 1] : bprev)) first = i0 + r;
    int64_t after = kNone;  // min of `first` over the later lanes of this warp
    {
        int64_t v = first;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int64_t u = __shfl_down_sync(0xffffffffu, v, o);
            if (lane + o < 32) v = u < v ? u : v;
        }
        // v: min over lanes >= lane; the later lanes' minimum is the next lane's v
        const int64_t nxt = __shfl_down_sync(0xffffffffu, v, 1);
        after = lane < 31 ? nxt : kNone;
        if (lane == 0) warp_next[warp] = v;
    }
    if (threadIdx.x == PS_THREADS - 1) {
        // the first start past the block's chunk: one look-ahead over the last bucket's pairs
        const int64_t e = static_cast<int64_t>(c + 1) * PS_CHUNK;
        if (e >= n) {
            block_next = n;
        } else {
            const int blast = bucket_of(static_cast<float>(ks[e - 1].key), lo, sc, NB);
            int64_t j = e;
            while (j < n && bucket_of(static_cast<float>(ks[j].key), lo, sc, NB) == blast) ++j;
            block_next = j;
        }
    }
    __syncthreads();
    for (int q = warp + 1; q < PS_THREADS / 32; ++q) after = warp_next[q] < after ? warp_next[q] : after;
    if (after == kNone) after = block_next;
#pragma unroll
    for (int r = 0; r < PS_ITEMS; ++r) {
        const int64_t i = i0 + r;
        const int bi = bk[r];
        const bool starts = i < n && bi > bprev;
        Pre<T> e{};
        if (starts) {
            // bucket bi starts here: its whole record
            PairSum<T> pre = start;
            pre.plus(PairSum<T>::from_pair(la, lb));
            e = pre.entry();
            int64_t end = after;
#pragma unroll
            for (int j = PS_ITEMS - 1; j > r; --j)
                if (i0 + j <= n && bk[j] > bk[j - 1]) end = i0 + j;
            store_record(rb + bi, e, static_cast<int32_t>(i), static_cast<int32_t>(end));
        }
        // the empty buckets above bprev start and end here: filled by the whole warp, one
        // lane's run after another (long runs occur in the sparse tails of a slice)
        const int q0 = starts ? bprev + 1 : 0, q1 = starts ? bi : 0;
        unsigned todo = __ballot_sync(0xffffffffu, q1 > q0);
        while (todo) {
            const int src = __ffs(todo) - 1;
            todo &= todo - 1;
            const int a0 = __shfl_sync(0xffffffffu, q0, src), a1 = __shfl_sync(0xffffffffu, q1, src);
            const int32_t at = __shfl_sync(0xffffffffu, static_cast<int32_t>(i), src);
            const Pre<T> es = shfl_pre(e, src);
            for (int q = a0 + lane; q < a1; q += 32) store_record(rb + q, es, at, at);
        }
        if (starts) bprev = bi;
        if (i < n) {
            la += el[r].w;
            lb = fma(el[r].w, el[r].key, lb);
        }
        if (i == n - 1) {
            PairSum<T> tot = start;
            tot.plus(PairSum<T>::from_pair(la, lb));
            const Pre<T> et = tot.entry();
            for (int q = bi + 1; q <= NB; ++q)
                store_record(rb + q, et, static_cast<int32_t>(n), static_cast<int32_t>(n));
        }
    }
}

// exclusive FP64 scan of one row of NB double2 values, in place; row[NB] = the totals
__global__ void __launch_bounds__(1024) k_row_exclusive_scan(double2* __restrict__ AB, int NB) {
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

// 32 bytes (one sector, 32-byte aligned) of read-only data in one load
__device__ __forceinline__ void ld_sector(const void* ptr, float (&r)[8]) {
    asm("ld.global.nc.v8.f32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
        : "=f"(r[0]), "=f"(r[1]), "=f"(r[2]), "=f"(r[3]), "=f"(r[4]), "=f"(r[5]), "=f"(r[6]), "=f"(r[7])
        : "l"(ptr));
}

// ------------------------------------------------------------ targets

// Per-slice value and derivative at z from the prefix entry of z's bucket (e), the totals
// (tot) and the sums over the bucket's sources below z (a_loc = sum w, b_loc = sum w key):
//   t = -c_d [ z (2A_< - W) - (2B_< - S) ],   g = c_d (W - 2A_< - a_eq).
// FP32 data: the differences 2A_< - W and 2B_< - S and the product with z are formed in
// double-float arithmetic (TwoSum / exact FMA products), so the only rounding of size
// 2^-24 is that of the result itself, whatever the cancellation between the terms.
__device__ __forceinline__ DF df_two_sum(float a, float b) {
    const float s = a + b, v = s - a;
    return DF{s, (a - (s - v)) + (b - v)};
}
// 2 (hi + lo + loc) - (thi + tlo) as a double-float
__device__ __forceinline__ DF df_twice_minus(float hi, float lo, float loc, float thi, float tlo) {
    const DF h = df_two_sum(2.0f * hi, -thi);
    const DF l = df_two_sum(2.0f * lo, 2.0f * loc);
    return df_add(h, DF{l.hi, l.lo - tlo});
}
__device__ __forceinline__ float negdist_value(const Pre<float>& e, const Pre<float>& tot, float a_loc, float b_loc,
                                               float z, float cd) {
    const DF u = df_twice_minus(e.ahi, e.alo, a_loc, tot.ahi, tot.alo);  // 2A_< - W
    const DF v = df_twice_minus(e.bhi, e.blo, b_loc, tot.bhi, tot.blo);  // 2B_< - S
    const float p = z * u.hi;
    const DF zu = df_norm(p, fmaf(z, u.hi, -p) + z * u.lo);
    const DF d = df_add(zu, DF{-v.hi, -v.lo});
    return -cd * (d.hi + d.lo);
}
__device__ __forceinline__ double negdist_value(const Pre<double>& e, const Pre<double>& tot, double a_loc,
                                                double b_loc, double z, double cd) {
    const double A = e.a + a_loc, B = e.b + b_loc;
    return -cd * (z * (2.0 * A - tot.a) - (2.0 * B - tot.b));
}
__device__ __forceinline__ float negdist_slope(const Pre<float>& e, const Pre<float>& tot, float a_loc, float a_eq,
                                               float cd) {
    const DF u = df_twice_minus(e.ahi, e.alo, a_loc, tot.ahi, tot.alo);  // 2A_< - W
    return cd * (-(u.hi + (u.lo + a_eq)));
}
__device__ __forceinline__ double negdist_slope(const Pre<double>& e, const Pre<double>& tot, double a_loc,
                                                double a_eq, double cd) {
    return cd * (tot.a - 2.0 * (e.a + a_loc) - a_eq);
}

// Slices [p0, p1): for target m, bucket b of z; A_< and B_< from the bucket's prefix entry
// plus the pairs of bucket b below z (and A_<= for the gradient); VAL: the values by
// negdist_value, summed over the slices with Kahan compensation and added to the FP64
// accumulator once per launch; DER: the derivatives by negdist_slope into G[p * ldg + m]
// (coalesced across the warp).  One lookup serves both.
template <class T, bool VAL, bool DER>
__global__ void __launch_bounds__(256) k_negdist_target(const T* __restrict__ Z, int P, int p0, int p1, int64_t n,
                                                       int64_t ldz, const KW<T>* __restrict__ kw, int64_t nx,
                                                       const BucketRec<T>* __restrict__ rec, int NB,
                                                       const float* __restrict__ kmin, const float* __restrict__ kscale,
                                                       T cd, T scale, double* __restrict__ acc, T* __restrict__ G,
                                                       int64_t ldg, int accumulate_G) {
    const int64_t m = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (m >= n) return;
    T sum = T(0), comp = T(0);  // Kahan
    for (int p = p0; p < p1; ++p) {
        const T z = Z[static_cast<int64_t>(p) * ldz + m];
        const BucketRec<T>* rb = rec + static_cast<int64_t>(p) * (NB + 1);
        const int b = bucket_of(static_cast<float>(z), kmin[p], kscale[p], NB);
        // the bucket's sources in any order: those below z, and (gradient) those equal to z
        T a = T(0), bz = T(0), aeq = T(0);
        Pre<T> eb;
        if constexpr (sizeof(T) == 4) {
            // the record in one 32-byte load, the pairs in aligned 32-byte chunks of four: one
            // sector per load instead of one load per pair (the lanes of a warp read unrelated
            // buckets, so every load is a separate sector access)
            float rr[8];
            ld_sector(rb + b, rr);
            eb = Pre<T>{rr[0], rr[1], rr[2], rr[3]};
            const int64_t base = static_cast<int64_t>(p) * nx;
            const int64_t g0 = base + __float_as_int(rr[4]), g1 = base + __float_as_int(rr[5]);
            for (int64_t g = g0 & ~int64_t(3); g < g1; g += 4) {
                float v[8];
                ld_sector(kw + g, v);
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    if (g + j >= g0 && g + j < g1) {
                        const float key = v[2 * j], wv = v[2 * j + 1];
                        if (key < z) {
                            a += wv;
                            if (VAL) bz = fmaf(wv, key, bz);
                        } else if (DER && key == z) {
                            aeq += wv;
                        }
                    }
                }
            }
        } else {
            const KW<T>* ks = kw + static_cast<int64_t>(p) * nx;
            const BucketRec<T> r = rb[b];  // one sector: prefix entry and the bucket's pair range
            eb = r.e;
            for (int32_t i = r.start; i < r.end; ++i) {
                const KW<T> e = ks[i];
                if (e.key < z) {
                    a += e.w;
                    if (VAL) bz = fma(e.w, e.key, bz);
                } else if (DER && e.key == z) {
                    aeq += e.w;
                }
            }
        }
        const Pre<T> tot = rb[NB].e;
        if (DER) {
            const T g = scale * negdist_slope(eb, tot, a, aeq, cd);
            T* gp = G + static_cast<int64_t>(p) * ldg + m;
            *gp = accumulate_G ? *gp + g : g;
        }
        if (VAL) {
            const T t = negdist_value(eb, tot, a, bz, z, cd);
            const T y = t - comp;
            const T tt = sum + y;
            comp = (tt - sum) - y;
            sum = tt;
        }
    }
    if (VAL) acc[m] += static_cast<double>(scale) * (static_cast<double>(sum) - static_cast<double>(comp));
}

}  // namespace

// ------------------------------------------------------------ launchers

template <class T>
size_t sort_pairs_scratch(int P, int64_t n) {
    using U = typename KeyOf<T>::U;
    const int64_t tiles = ceil_div(n, RS_TILE);
    const size_t total = static_cast<size_t>(P) * n;
    return 2 * total * (sizeof(U) + sizeof(T)) + static_cast<size_t>(P) * RS_BINS * (tiles + 1) * sizeof(int32_t) +
           1024;
}

template <class T, class U, bool FIRST, bool LAST, bool BUCKETED>
void radix_pass(dim3 grid, const T* z, int64_t ldz, const T* w, const KV<U, T>* kvin, int64_t n, int shift, int tiles,
                const int32_t* hist, const int32_t* dbase, KV<U, T>* kvout, KW<T>* pout, const Buckets& bk,
                cudaStream_t st) {
    constexpr size_t smem = radix_pass_smem<T, U>();
    static bool attr = false;
    if (!attr) {
        SLK_CHECK_CUDA(cudaFuncSetAttribute(k_radix_pass<T, U, FIRST, LAST, BUCKETED>,
                                            cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem)));
        attr = true;
    }
    k_radix_pass<T, U, FIRST, LAST, BUCKETED><<<grid, RS_THREADS, smem, st>>>(z, ldz, w, kvin, n, shift, tiles, hist,
                                                                              dbase, kvout, pout, bk);
}

template <class T, class U, bool BUCKETED>
void sort_passes(const T* z, int P, int64_t n, int64_t ldz, const T* w, KW<T>* pairs, unsigned char* s, int passes,
                 int dbits, const Buckets& bk, cudaStream_t st) {
    static_assert(sizeof(KV<U, T>) == sizeof(U) + sizeof(T), "interleaved key and payload");
    const int tiles = static_cast<int>(ceil_div(n, RS_TILE));
    const size_t total = static_cast<size_t>(P) * n;
    KV<U, T>* kv0 = reinterpret_cast<KV<U, T>*>(s);
    KV<U, T>* kv1 = kv0 + total;
    int32_t* hist = reinterpret_cast<int32_t*>(kv1 + total);
    int32_t* dbase = hist + static_cast<size_t>(P) * RS_BINS * tiles;  // P x 256 digit bases
    dim3 gt(tiles, P);
    const KV<U, T>* kvin = nullptr;
    for (int pass = 0; pass < passes; ++pass) {
        const int shift = dbits * pass;
        KV<U, T>* kvout = (pass & 1) ? kv1 : kv0;
        const bool first = pass == 0, last = pass == passes - 1;
        {
            SLK_TIMED("radix_hist", st);
            if (first)
                k_radix_hist<T, U, true, BUCKETED><<<gt, RS_THREADS, 0, st>>>(z, ldz, nullptr, n, shift, tiles, hist, bk);
            else
                k_radix_hist<T, U, false, BUCKETED><<<gt, RS_THREADS, 0, st>>>(nullptr, 0, kvin, n, shift, tiles, hist,
                                                                              bk);
        }
        SLK_CHECK_LAUNCH();
        {
            SLK_TIMED("radix_scan", st);
            k_radix_scan_rows<<<dim3(RS_BINS, P), 256, 0, st>>>(hist, tiles, dbase);
            SLK_CHECK_LAUNCH();
            k_radix_scan_digits<<<P, 256, 0, st>>>(dbase);
        }
        SLK_CHECK_LAUNCH();
        {
            SLK_TIMED("radix_scatter", st);
            if (first && last)
                radix_pass<T, U, true, true, BUCKETED>(gt, z, ldz, w, nullptr, n, shift, tiles, hist, dbase, nullptr,
                                                       pairs, bk, st);
            else if (first)
                radix_pass<T, U, true, false, BUCKETED>(gt, z, ldz, w, nullptr, n, shift, tiles, hist, dbase, kvout,
                                                        nullptr, bk, st);
            else if (last)
                radix_pass<T, U, false, true, BUCKETED>(gt, nullptr, 0, nullptr, kvin, n, shift, tiles, hist, dbase,
                                                        nullptr, pairs, bk, st);
            else
                radix_pass<T, U, false, false, BUCKETED>(gt, nullptr, 0, nullptr, kvin, n, shift, tiles, hist, dbase,
                                                         kvout, nullptr, bk, st);
        }
        SLK_CHECK_LAUNCH();
        kvin = kvout;
    }
}

template <class T>
void launch_sort_pairs(const T* z, int P, int64_t n, int64_t ldz, const T* w, void* kw, void* scratch,
                       size_t scratch_bytes, const float* kmin, const float* kscale, int NB, cudaStream_t st) {
    using U = typename KeyOf<T>::U;
    SLK_REQUIRE(n < (int64_t(1) << 31), "segments longer than 2^31 are not supported");
    SLK_REQUIRE(scratch_bytes >= sort_pairs_scratch<T>(P, n), "sort scratch too small");
    SLK_REQUIRE(P <= 65535, "too many segments for one sort launch");
    if (n <= 0) return;
    unsigned char* s = static_cast<unsigned char*>(scratch);
    KW<T>* pairs = static_cast<KW<T>*>(kw);
    if (NB > 0) {
        // group by bucket only: one 8-bit digit pass per byte of the bucket index
        int bits = 0;
        while ((1 << bits) < NB) ++bits;
        const int passes = bits > 8 ? (bits + 7) / 8 : 1;
        const int dbits = 8;
        sort_passes<T, U, true>(z, P, n, ldz, w, pairs, s, passes, dbits, Buckets{kmin, kscale, NB, (1 << dbits) - 1},
                                st);
    } else {
        sort_passes<T, U, false>(z, P, n, ldz, w, pairs, s, KeyOf<T>::passes, 8, Buckets{nullptr, nullptr, 0, 0xff},
                                 st);
    }
}

template <class T>
void launch_slice_minmax(const T* Z, int P, int64_t n, int64_t ldz, int NB, float* kmin, float* kscale,
                         cudaStream_t st) {
    {
        SLK_TIMED("slice_minmax", st);
        k_slice_minmax<T><<<P, 256, 0, st>>>(Z, n, ldz, NB, kmin, kscale);
    }
    SLK_CHECK_LAUNCH();
}

template <class T>
int64_t sorted_pairs_bytes(int P, int64_t n) {
    return static_cast<int64_t>(sizeof(KW<T>)) * P * n + kPairPadBytes;
}

template <class T>
void launch_bucket_tables(int P, int64_t n, const void* kw, int NB, float* kmin, float* kscale, void* rec,
                          bool have_geometry, cudaStream_t st) {
    const KW<T>* pairs = static_cast<const KW<T>*>(kw);
    SLK_REQUIRE(reinterpret_cast<uintptr_t>(rec) % 32 == 0, "bucket records must be 32-byte aligned");
    if (!have_geometry) {
        // fully sorted pairs: the bucket geometry from the first and last key of each slice
        {
            SLK_TIMED("bucket_minmax", st);
            k_bucket_minmax<T><<<static_cast<unsigned>(ceil_div(P, 128)), 128, 0, st>>>(pairs, P, n, NB, kmin, kscale);
        }
        SLK_CHECK_LAUNCH();
    }
    const int nchunk = static_cast<int>(ceil_div(n, PS_CHUNK));
    DevBuf<double2> cs(static_cast<size_t>(P) * (nchunk + 1), st);
    dim3 g(static_cast<unsigned>(nchunk), P);
    {
        SLK_TIMED("pair_chunk_sums", st);
        k_pair_chunk_sums<T><<<g, PS_THREADS, 0, st>>>(pairs, n, nchunk, cs.get());
    }
    SLK_CHECK_LAUNCH();
    {
        SLK_TIMED("chunk_scan", st);
        k_row_exclusive_scan<<<P, 1024, 0, st>>>(cs.get(), nchunk);
    }
    SLK_CHECK_LAUNCH();
    {
        SLK_TIMED("pair_prefix_tab", st);
        k_pair_prefix_tab<T><<<g, PS_THREADS, 0, st>>>(pairs, n, nchunk, cs.get(), NB, kmin, kscale,
                                                       static_cast<BucketRec<T>*>(rec));
    }
    SLK_CHECK_LAUNCH();
}

template <class T>
void launch_negdist_target(const T* Z, int P, int64_t n, int64_t ldz, const void* kw, int64_t nx, const void* rec,
                           int NB, const float* kmin, const float* kscale, double cd, double scale, double* acc, T* G,
                           int64_t ldg, int accumulate_G, cudaStream_t st) {
    if (n <= 0 || (!acc && !G)) return;
    SLK_REQUIRE(!G || ldg >= n, "derivative rows shorter than the targets");
    // slices per launch: keep one batch's pairs (the randomly accessed state) within ~64 MB of L2
    const int64_t per_slice = static_cast<int64_t>(sizeof(KW<T>)) * nx + static_cast<int64_t>(NB + 1) * kBucketRecordBytes;
    int batch = static_cast<int>((int64_t(64) << 20) / (per_slice > 0 ? per_slice : 1));
    if (batch < 1) batch = 1;
    if (batch > P) batch = P;
    const unsigned blocks = static_cast<unsigned>(ceil_div(n, 256));
    const KW<T>* pairs = static_cast<const KW<T>*>(kw);
    const BucketRec<T>* recs = static_cast<const BucketRec<T>*>(rec);
    // FP32: records and four-pair chunks are read as aligned 32-byte sectors (the pair array
    // carries kPairPadBytes of padding for the last chunk)
    SLK_REQUIRE(reinterpret_cast<uintptr_t>(kw) % 32 == 0 && reinterpret_cast<uintptr_t>(rec) % 32 == 0,
                "sorted pairs and bucket records must be 32-byte aligned");
    const T c = static_cast<T>(cd), sc = static_cast<T>(scale);
    for (int p0 = 0; p0 < P; p0 += batch) {
        const int p1 = p0 + batch < P ? p0 + batch : P;
        SLK_TIMED(acc && G ? "negdist_target_both" : (G ? "negdist_target_grad" : "negdist_target"), st);
        if (acc && G)
            k_negdist_target<T, true, true><<<blocks, 256, 0, st>>>(Z, P, p0, p1, n, ldz, pairs, nx, recs, NB, kmin,
                                                                    kscale, c, sc, acc, G, ldg, accumulate_G);
        else if (G)
            k_negdist_target<T, false, true><<<blocks, 256, 0, st>>>(Z, P, p0, p1, n, ldz, pairs, nx, recs, NB, kmin,
                                                                     kscale, c, sc, acc, G, ldg, accumulate_G);
        else
            k_negdist_target<T, true, false><<<blocks, 256, 0, st>>>(Z, P, p0, p1, n, ldz, pairs, nx, recs, NB, kmin,
                                                                     kscale, c, sc, acc, G, ldg, accumulate_G);
        SLK_CHECK_LAUNCH();
    }
}

#define SLK_INST(T)                                                                                                   \
    template size_t sort_pairs_scratch<T>(int, int64_t);                                                              \
    template void launch_sort_pairs<T>(const T*, int, int64_t, int64_t, const T*, void*, void*, size_t, const float*, \
                                       const float*, int, cudaStream_t);                                               \
    template void launch_slice_minmax<T>(const T*, int, int64_t, int64_t, int, float*, float*, cudaStream_t);         \
    template int64_t sorted_pairs_bytes<T>(int, int64_t);                                                             \
    template void launch_bucket_tables<T>(int, int64_t, const void*, int, float*, float*, void*, bool, cudaStream_t); \
    template void launch_negdist_target<T>(const T*, int, int64_t, int64_t, const void*, int64_t, const void*, int,   \
                                           const float*, const float*, double, double, double*, T*, int64_t, int,    \
                                           cudaStream_t);
SLK_INST(float)
SLK_INST(double)
#undef SLK_INST

}  // namespace slk
