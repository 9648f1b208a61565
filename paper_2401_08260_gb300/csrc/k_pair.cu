// Fused Chebyshev kernels on CTA pairs (tcgen05 cta_group::2, sm_103a).
//
// Both sides of the Chebyshev evaluation of the truncated Fourier sum (Section 3.1,
// with the projection of Algorithm 1 fused in) read the caller's FP32 points directly:
//   target side  t(y) = sum_p sum_l beta[p][l] T_l(<xi_p, y - mu> / R)   (row sums per point)
//   source side  mom[p][j] = sum_n w_n T_j(<xi_p, x_n - mu> / R)          (moments per slice)
// The pair of CTAs of a cluster of two forms one 256-point tile.  Each CTA brings in,
// per 64-wide K stage, its own 128 FP32 point rows (two 32-column TMA boxes, converted
// in place to centred BF16 in the tensor core's 128-byte-swizzled layout by its eight
// worker warps) and its own 128 rows of each 256-direction sub-tile; while it works on a
// tile its producer streams the rows of its next tile into L2, one contiguous chunk per
// stage.  The even CTA
// issues M = 256, N = 256 MMAs (kind::f16, FP32 accumulate) for up to two sub-tiles,
// i.e. all P <= 512 slices of the tile at once, into two 256-column accumulators of each
// CTA's tensor memory:
//   target side: A = points (rows = TMEM lanes), B = directions, D[point][slice];
//   source side: A = directions (rows = slices), B = points, D[slice][point].
// Every point is therefore read once, and each direction once per 256 points (the CTA
// pair shares the tile through the pair MMA, not through any shared load).
//
// Signals between the two CTAs are remote mbarrier arrivals at cluster scope:
//   workers of both CTAs     -> full[s] of the even CTA  (stage converted, 16 arrivals)
//   even CTA's MMA commit    -> its own empty[s]; its producer forwards the release to the
//                               odd CTA's empty[s] when it refills that stage
//   even CTA's MMA commit    -> its own acc_full; one worker thread forwards it
//   workers of both CTAs     -> acc_empty of the even CTA (16 arrivals)
// The worker warps alternate between converting the stages of a tile and reading its
// accumulators back once the MMAs are done (the 512 TMEM columns hold one tile's two
// accumulators); each reads 32 columns at a time, the next load in flight while it
// evaluates the current one.
// Every wait is bounded; on a timeout the CTA records an error bit and skips the rest.
// Before exit each CTA waits for its own TMA fills, the even CTA for its last MMAs, and
// both meet at a cluster barrier before tensor memory is freed.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <type_traits>

#include "cheb_epi.cuh"
#include "kernels.cuh"
#include "umma.cuh"

namespace slk {

namespace {

using namespace umma;

constexpr int QM = 128;                      // rows per CTA (TMEM lanes); pair MMA M = 256
constexpr int QN = 256;                      // MMA N (128 rows of B from each CTA)
constexpr int QK = 64;                       // K elements per stage
constexpr int QSTAGES = 3;
constexpr int QTHREADS = 384;                // warp 0 TMA, 1 MMA, 4-11 workers (convert + epilogue)
constexpr int WORKER0 = 4;                   // first worker warp (TMEM lane quarter = warp % 4)
constexpr int WORKER_WARPS = 8;              // each converts 16 of the 128 rows of a stage
constexpr int CVT_BYTES = QM * QK * 4;       // 128 FP32 rows x 64 (two 32-column boxes)
constexpr int DIR_BYTES = QM * QK * 2;       // 128 BF16 direction rows x 64, one sub-tile
constexpr int QSTAGE_BYTES = CVT_BYTES + 2 * DIR_BYTES;
constexpr int QMAX_P = 2 * QN;               // slices per pass (two accumulators)
constexpr uint32_t QTMEM_COLS = 512;

enum { SIDE_TARGET = 0, SIDE_SOURCE = 1 };

struct PairSmem {
    uint64_t raw[QSTAGES];    // this CTA's TMA bytes of a stage have landed
    uint64_t full[QSTAGES];   // even CTA: both CTAs' converters finished a stage
    uint64_t empty[QSTAGES];  // the stage may be refilled
    uint64_t acc_full;        // the tile's accumulators are complete
    uint64_t acc_empty;       // even CTA: both CTAs' epilogues have read them
    uint64_t drain;           // even CTA: its last MMAs completed
    uint32_t tmem_base;
};

struct PairArgs {
    int n;          // points
    int P;          // slices (<= 512)
    int d;
    int tiles;      // 256-point tiles
    int q;          // Chebyshev terms
    int horner;     // target side: monomial coefficients
    float R, inv_R;
    const float* mu;    // centre (d values)
    const float* beta;  // target side: P x q coefficients
    double* part;       // target side: 2 x ldp FP64 row sums
    int64_t ldp;
    const float* pts;   // the FP32 points (for the L2 prefetch), row stride ldpts
    int64_t ldpts;
    const float* w;     // source side: weights of the n points
    double* mom;        // source side: moment partials [(pair * halves + h) * P + p][q]
    float* absmax;      // source side: max |z| over the points
    unsigned* err;
};

// dynamic shared memory: the stage ring, the barriers and (target side) the q x 512
// coefficients; at most 226 KB (q = 16)
__host__ __device__ constexpr size_t pair_smem_bytes(int beta_terms) {
    return 1024 + static_cast<size_t>(QSTAGES) * QSTAGE_BYTES + ((sizeof(PairSmem) + 15) & ~size_t(15)) +
           static_cast<size_t>(QMAX_P) * beta_terms * sizeof(float);
}
constexpr size_t kPairSmemMax = pair_smem_bytes(16);

// Convert 16 of one stage's 128 FP32 rows (rows 16 wi .. 16 wi + 15; the stage holds two
// unswizzled 32-column boxes of 128 bytes per row) to centred BF16 in place over the first
// box, 128-byte swizzle (16-byte chunk c of row r at c ^ (r % 8)); rows at or beyond n are
// written as zeros.  Lane l takes columns 4j..4j+3 (j = l % 16) of rows 2u + l / 16; m holds
// the centre at those columns (the same arithmetic as the single-CTA converting kernel).
__device__ __forceinline__ void convert_rows16(unsigned char* cv, int lane, int wi, const float (&m)[4], int row0,
                                               int n) {
    constexpr int HALF = QM * 128;
    const int j = lane & 15, rr = lane >> 4;
    const unsigned char* src = cv + (j >> 3) * HALF + (j & 7) * 16;
    const int r0 = wi * 16;
    float4 v[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) v[u] = *reinterpret_cast<const float4*>(src + (r0 + 2 * u + rr) * 128);
    __syncwarp();
#pragma unroll
    for (int u = 0; u < 8; ++u) {
        const int r = r0 + 2 * u + rr;
        union { __nv_bfloat162 h[2]; uint2 u2; } pk;
        pk.h[0] = __floats2bfloat162_rn(v[u].x - m[0], v[u].y - m[1]);
        pk.h[1] = __floats2bfloat162_rn(v[u].z - m[2], v[u].w - m[3]);
        if (row0 + r >= n) pk.u2 = make_uint2(0u, 0u);
        *reinterpret_cast<uint2*>(cv + r * 128 + (((j >> 1) ^ (r & 7)) << 4) + ((j & 1) << 3)) = pk.u2;
    }
}

template <int SIDE>
__global__ void __launch_bounds__(QTHREADS, 1)
    k_pair_cheb(const __grid_constant__ CUtensorMap map_pts, const __grid_constant__ CUtensorMap map_dir, PairArgs a) {
    extern __shared__ unsigned char smem_raw[];
    unsigned char* base = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    PairSmem* sm = reinterpret_cast<PairSmem*>(base + QSTAGES * QSTAGE_BYTES);
    float* sbeta = reinterpret_cast<float*>(base + QSTAGES * QSTAGE_BYTES + ((sizeof(PairSmem) + 15) & ~size_t(15)));
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t rank = cluster_rank();
    const int pair = static_cast<int>(blockIdx.x >> 1), npairs = static_cast<int>(gridDim.x >> 1);
    const int kblocks = (a.d + QK - 1) / QK;
    const int nsub = a.P > QN ? 2 : 1;
    const uint32_t stage_tx = CVT_BYTES + nsub * DIR_BYTES;

    if (threadIdx.x == 0) {
        for (int s = 0; s < QSTAGES; ++s) {
            mbar_init(&sm->raw[s], 1);
            mbar_init(&sm->full[s], 2 * WORKER_WARPS);  // one arrival per worker warp of each CTA
            mbar_init(&sm->empty[s], 1);
        }
        mbar_init(&sm->acc_full, 1);
        mbar_init(&sm->acc_empty, 2 * WORKER_WARPS);
        mbar_init(&sm->drain, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (SIDE == SIDE_TARGET)
        for (int e = threadIdx.x; e < QMAX_P * a.q; e += blockDim.x) {
            const int l = e / QMAX_P, p = e - l * QMAX_P;
            sbeta[e] = p < a.P ? a.beta[static_cast<int64_t>(p) * a.q + l] : 0.0f;
        }
    if (warp == 2) tmem_alloc_pair(&sm->tmem_base, QTMEM_COLS);
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    // both CTAs' barriers initialised and tensor memory allocated before any remote arrival
    cluster_barrier();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = sm->tmem_base;

    int ntile = 0;
    for (int t = pair; t < a.tiles; t += npairs) ++ntile;
    const int total = ntile * kblocks;

    if (warp == 0) {
        // ---------------- producer: TMA loads of this CTA's stages, L2 prefetch of its next tile
        if (lane == 0) {
            int issued = 0;
            // rows of the next tile brought into L2 a chunk per stage (contiguous bytes of
            // the row-major points), so that the TMA loads of a tile find it there
            const int chunk = (QM + kblocks - 1) / kblocks;
            auto prefetch_rows = [&](int tile, int kb) {
                const int rbase = tile * (2 * QM) + static_cast<int>(rank) * QM;
                const int r0 = rbase + kb * chunk;
                int r1 = r0 + chunk;
                if (r1 > rbase + QM) r1 = rbase + QM;
                if (r1 > a.n) r1 = a.n;
                if (tile >= a.tiles || r0 >= r1) return;
                // from the first element of row r0 to the last element of row r1 - 1, rounded
                // down to 16 bytes (never past the caller's rows)
                const int64_t bytes = ((static_cast<int64_t>(r1 - r0 - 1) * a.ldpts + a.d) * 4) & ~int64_t(15);
                if (bytes > 0)
                    bulk_prefetch_l2(a.pts + static_cast<int64_t>(r0) * a.ldpts, static_cast<uint32_t>(bytes));
            };
            for (int gg = 0; gg < total; ++gg) {
                const int tile = pair + (gg / kblocks) * npairs, kb = gg % kblocks, s = gg % QSTAGES;
                if (gg >= QSTAGES) {
                    // released by the pair's MMAs: on the even CTA by their commit, on the odd
                    // CTA by the even CTA's producer forwarding that release
                    const bool ok = rank == 0 ? mbar_wait(&sm->empty[s], ((gg / QSTAGES) - 1) & 1)
                                              : mbar_wait_cluster(&sm->empty[s], ((gg / QSTAGES) - 1) & 1);
                    if (!ok) {
                        atomicOr(a.err, 8u);
                        break;
                    }
                    if (rank == 0) mbar_arrive_cluster(cluster_addr(&sm->empty[s], 1));
                }
                const int prow = tile * (2 * QM) + static_cast<int>(rank) * QM;
                unsigned char* st = base + s * QSTAGE_BYTES;
                mbar_expect_tx(&sm->raw[s], stage_tx);
                tma_load_2d(st, &map_pts, &sm->raw[s], kb * QK, prow);
                tma_load_2d(st + QM * 128, &map_pts, &sm->raw[s], kb * QK + 32, prow);
                for (int j = 0; j < nsub; ++j)
                    tma_load_2d(st + CVT_BYTES + j * DIR_BYTES, &map_dir, &sm->raw[s], kb * QK,
                                j * QN + static_cast<int>(rank) * QM);
                ++issued;
                prefetch_rows(tile + npairs, kb);
            }
            drain_fills(sm->raw, QSTAGES, issued);
        }
    } else if (warp == 1) {
        // ---------------- MMA issuer (even CTA): M = 256 over the pair, one or two sub-tiles
        if (rank == 0 && lane == 0) {
            const uint32_t idesc = instr_desc(1u, 2 * QM, QN);
            for (int g = 0; g < total; ++g) {
                const int kb = g % kblocks, t = g / kblocks, s = g % QSTAGES;
                if (kb == 0 && t >= 1 && !mbar_wait_cluster(&sm->acc_empty, (t - 1) & 1)) {
                    atomicOr(a.err, 16u);
                    break;
                }
                if (!mbar_wait_cluster(&sm->full[s], (g / QSTAGES) & 1)) {
                    atomicOr(a.err, 16u);
                    break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                unsigned char* st = base + s * QSTAGE_BYTES;
#pragma unroll
                for (int k = 0; k < QK / 16; ++k)
                    for (int j = 0; j < nsub; ++j) {
                        const uint64_t dp = smem_desc(st + k * 32);
                        const uint64_t dd = smem_desc(st + CVT_BYTES + j * DIR_BYTES + k * 32);
                        if (SIDE == SIDE_TARGET)
                            umma_f16_pair(tmem + j * QN, dp, dd, idesc, (kb > 0 || k > 0) ? 1u : 0u);
                        else
                            umma_f16_pair(tmem + j * QN, dd, dp, idesc, (kb > 0 || k > 0) ? 1u : 0u);
                    }
                umma_commit_pair(&sm->empty[s]);
                if (kb == kblocks - 1) umma_commit_pair(&sm->acc_full);
            }
            drain_mma_pair(&sm->drain, a.err, 16u);
        }
    } else if (warp >= WORKER0) {
        // ---------------- workers (warps 4-11; warps 2-3 have no role): for each tile, convert this warp's 16 rows of
        // every stage as it lands, then read the finished accumulators back (TMEM lane
        // quarter warp % 4, column group (warp - 2) / 4)
        const int wi = warp - WORKER0, q4 = warp & 3, grp = wi >> 2;
        const uint32_t lane_off = static_cast<uint32_t>(q4 * 32) << 16;
        const uint32_t full0 = cluster_addr(&sm->full[0], 0);
        const uint32_t acc_empty0 = cluster_addr(&sm->acc_empty, 0);
        const uint32_t peer_full = cluster_addr(&sm->acc_full, 1);
        const bool forwarder = rank == 0 && wi == 0 && lane == 0;
        // the centre's four columns of this lane for the next stage, loaded a stage ahead
        float mnext[4];
        auto load_mu = [&](int kb) {
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const int k = kb * QK + 4 * (lane & 15) + e;
                mnext[e] = k < a.d ? __ldg(a.mu + k) : 0.0f;
            }
        };
        load_mu(0);
        bool ok = true;
        // convert the stages of local tile t; false on a timeout
        auto convert_tile = [&](int t) {
            const int tile = pair + t * npairs;
            for (int kb = 0; kb < kblocks; ++kb) {
                const int g = t * kblocks + kb, s = g % QSTAGES;
                float m[4] = {mnext[0], mnext[1], mnext[2], mnext[3]};
                load_mu(kb + 1 < kblocks ? kb + 1 : 0);
                const bool got = mbar_wait(&sm->raw[s], (g / QSTAGES) & 1);
                if (!__all_sync(0xffffffffu, got)) {
                    if (lane == 0) atomicOr(a.err, 8u);
                    return false;
                }
                convert_rows16(base + s * QSTAGE_BYTES, lane, wi, m, tile * (2 * QM) + static_cast<int>(rank) * QM,
                               a.n);
                // generic-proxy writes, read next by the tensor core (async proxy)
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                __syncwarp();
                if (lane == 0) mbar_arrive_cluster(full0 + static_cast<uint32_t>(s * sizeof(uint64_t)));
            }
            return true;
        };
        auto wait_acc = [&](int t) {
            if (!mbar_wait_cluster(&sm->acc_full, t & 1)) {
                atomicOr(a.err, 32u);
                return false;
            }
            if (forwarder) mbar_arrive_cluster(peer_full);
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            return true;
        };
        auto release_acc = [&]() {
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            __syncwarp();
            if (lane == 0) mbar_arrive_cluster(acc_empty0);
        };
        if (SIDE == SIDE_TARGET) {
            // row sums of t_p(z) over the slices of this warp's column group
            const uint32_t col0 = nsub == 2 ? grp * QN : grp * (QN / 2);
            const int ncols = nsub == 2 ? QN : QN / 2;
            bool bad = false;
            auto run = [&](auto qp_tag, auto horner_tag) {
                constexpr int QP = decltype(qp_tag)::value;
                constexpr bool HORNER = decltype(horner_tag)::value;
                for (int t = 0; t < ntile && ok; ++t) {
                    if (!convert_tile(t) || !wait_acc(t)) {
                        ok = false;
                        break;
                    }
                    const int tile = pair + t * npairs;
                    const int row = tile * (2 * QM) + static_cast<int>(rank) * QM + q4 * 32 + lane;
                    float sum = 0.0f, comp = 0.0f;  // Kahan
                    uint32_t ra[32], rb[32];
                    const uint32_t tbase = tmem + lane_off + col0;
                    tmem_ld32_issue(tbase, ra);
                    tmem_wait32(ra);
                    for (int cc = 0; cc < ncols; cc += 64) {
                        tmem_ld32_issue(tbase + cc + 32, rb);
                        cheb_chunk32<QP, HORNER>(ra, sbeta + col0 + cc, QMAX_P, a.R, a.inv_R, sum, comp, bad);
                        tmem_wait32(rb);
                        if (cc + 64 < ncols) tmem_ld32_issue(tbase + cc + 64, ra);
                        cheb_chunk32<QP, HORNER>(rb, sbeta + col0 + cc + 32, QMAX_P, a.R, a.inv_R, sum, comp, bad);
                        if (cc + 64 < ncols) tmem_wait32(ra);
                    }
                    release_acc();
                    if (row < a.n)
                        a.part[static_cast<int64_t>(grp) * a.ldp + row] =
                            static_cast<double>(sum) - static_cast<double>(comp);
                }
            };
            using T_ = std::true_type;
            using F_ = std::false_type;
            if (a.q == 10) a.horner ? run(std::integral_constant<int, 10>{}, T_{}) : run(std::integral_constant<int, 10>{}, F_{});
            else if (a.q == 12) a.horner ? run(std::integral_constant<int, 12>{}, T_{}) : run(std::integral_constant<int, 12>{}, F_{});
            else if (a.q == 8) a.horner ? run(std::integral_constant<int, 8>{}, T_{}) : run(std::integral_constant<int, 8>{}, F_{});
            else a.horner ? run(std::integral_constant<int, 16>{}, T_{}) : run(std::integral_constant<int, 16>{}, F_{});
            if (bad) atomicOr(a.err, 4u);
        } else {
            // one slice's moments per thread over all tiles: two sub-tiles, group j owns the
            // slices of accumulator j (all 256 points); one sub-tile, both groups own the same
            // slices, each over half of the points
            const uint32_t col0 = nsub == 2 ? grp * QN : 0;
            const int pt_off = nsub == 2 ? 0 : grp * (QN / 2);
            const int ncols = nsub == 2 ? QN : QN / 2;
            const int slice = (nsub == 2 ? grp * QN : 0) + static_cast<int>(rank) * QM + q4 * 32 + lane;
            float mx = 0.0f;
            auto run = [&](auto qp_tag) {
                constexpr int QP = decltype(qp_tag)::value;
                float hi[QP], lo[QP];
#pragma unroll
                for (int k = 0; k < QP; ++k) hi[k] = lo[k] = 0.0f;
                auto chunk = [&](const uint32_t (&r)[32], int tile, int cc, float (&tt)[QP]) {
                    // accumulator column c holds point tile * 256 + c (columns 0-127 from the
                    // even CTA's rows of B, 128-255 from the odd CTA's)
                    const int pt0 = tile * (2 * QM) + pt_off + cc;
                    const float wl = pt0 + lane < a.n ? __ldg(a.w + pt0 + lane) : 0.0f;
                    float v[32];
#pragma unroll
                    for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
                    mom_chunk<QP>(v, wl, a.inv_R, a.n - pt0, tt, mx);
                };
                for (int t = 0; t < ntile && ok; ++t) {
                    if (!convert_tile(t) || !wait_acc(t)) {
                        ok = false;
                        break;
                    }
                    const int tile = pair + t * npairs;
                    float tt[QP];
#pragma unroll
                    for (int k = 0; k < QP; ++k) tt[k] = 0.0f;
                    uint32_t ra[32], rb[32];
                    const uint32_t tbase = tmem + lane_off + col0 + pt_off;
                    tmem_ld32_issue(tbase, ra);
                    tmem_wait32(ra);
                    for (int cc = 0; cc < ncols; cc += 64) {
                        tmem_ld32_issue(tbase + cc + 32, rb);
                        chunk(ra, tile, cc, tt);
                        tmem_wait32(rb);
                        if (cc + 64 < ncols) tmem_ld32_issue(tbase + cc + 64, ra);
                        chunk(rb, tile, cc + 32, tt);
                        if (cc + 64 < ncols) tmem_wait32(ra);
                    }
                    release_acc();
#pragma unroll
                    for (int k = 0; k < QP; ++k) two_sum_into(hi[k], lo[k], tt[k]);
                }
                if (slice < a.P) {
                    const int halves = nsub == 2 ? 1 : 2;
                    const int h = nsub == 2 ? 0 : grp;
                    double* out = a.mom + (static_cast<int64_t>(pair * halves + h) * a.P + slice) * QP;
#pragma unroll
                    for (int k = 0; k < QP; ++k) out[k] = static_cast<double>(hi[k]) + static_cast<double>(lo[k]);
                }
            };
            if (a.q == 10) run(std::integral_constant<int, 10>{});
            else if (a.q == 12) run(std::integral_constant<int, 12>{});
            else if (a.q == 8) run(std::integral_constant<int, 8>{});
            else run(std::integral_constant<int, 16>{});
            if (slice >= a.P) mx = 0.0f;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
            if (lane == 0 && a.absmax) atomicMax(reinterpret_cast<unsigned int*>(a.absmax), __float_as_uint(mx));
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    // neither CTA frees its tensor memory or leaves while the pair's MMAs or arrivals
    // may still reach it
    cluster_barrier();
    if (warp == 2) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        tmem_dealloc_pair(tmem, QTMEM_COLS);
    }
}

}  // namespace

bool pair_cheb_fits(int P, int q) { return P >= 1 && P <= QMAX_P && (q == 8 || q == 10 || q == 12 || q == 16); }

namespace {

// Co-resident CTA pairs of the kernel on the current device; sets its shared-memory limit.
template <int SIDE>
int pair_units() {
    static int units[128] = {};
    int dev = 0;
    SLK_CHECK_CUDA(cudaGetDevice(&dev));
    SLK_REQUIRE(dev >= 0 && dev < 128, "device index out of range");
    if (!units[dev]) {
        SLK_CHECK_CUDA(cudaFuncSetAttribute(k_pair_cheb<SIDE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                            static_cast<int>(kPairSmemMax)));
        int sms = 0;
        SLK_CHECK_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
        cudaLaunchConfig_t cfg = {};
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = 2;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.gridDim = dim3(static_cast<unsigned>(sms / 2 * 2));
        cfg.blockDim = dim3(QTHREADS);
        cfg.dynamicSmemBytes = kPairSmemMax;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        int clusters = 0;
        SLK_CHECK_CUDA(cudaOccupancyMaxActiveClusters(&clusters, k_pair_cheb<SIDE>, &cfg));
        SLK_REQUIRE(clusters > 0, "no CTA pair of the fused Chebyshev kernel fits on this device");
        units[dev] = clusters;
    }
    return units[dev];
}

template <int SIDE>
void launch_pairs(const CUtensorMap& mp, const CUtensorMap& md, const PairArgs& a, int npairs, cudaStream_t st) {
    static_assert(kPairSmemMax <= 227 * 1024, "shared memory of the pair kernel");
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = 2;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.gridDim = dim3(static_cast<unsigned>(2 * npairs));
    cfg.blockDim = dim3(QTHREADS);
    cfg.dynamicSmemBytes = pair_smem_bytes(SIDE == SIDE_TARGET ? a.q : 0);
    cfg.stream = st;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    SLK_CHECK_CUDA(cudaLaunchKernelEx(&cfg, k_pair_cheb<SIDE>, mp, md, a));
}

PairArgs pair_args(int64_t n, int P, int d, int q, double R, const float* mu, unsigned* err) {
    PairArgs a{};
    a.n = static_cast<int>(n);
    a.P = P;
    a.d = d;
    a.tiles = static_cast<int>(ceil_div(n, 2 * QM));
    a.q = q;
    a.R = static_cast<float>(R);
    a.inv_R = static_cast<float>(1.0 / R);
    a.mu = mu;
    a.err = err;
    return a;
}

}  // namespace

void launch_pair_cheb_target(const float* y, int64_t ldy, const float* mu, int64_t n, const void* xib, int P, int d,
                             const float* coef, int q, int horner, double R, double* part, int64_t ldp, unsigned* err,
                             cudaStream_t st) {
    if (n <= 0) return;
    SLK_REQUIRE(pair_cheb_fits(P, q), "slice or term count unsupported by the CTA-pair Chebyshev kernel");
    SLK_REQUIRE(umma_f32_operand_ok(y, ldy), "FP32 targets need 16-byte aligned rows");
    SLK_REQUIRE(n < (int64_t(1) << 31) - 2 * QM, "too many targets for one launch");
    const CUtensorMap mp = tmap_f32_rows(y, n, d, ldy, QM);
    const CUtensorMap md = tmap_bf16_sw128(xib, P, d, umma_operand_ld(d), QM);
    PairArgs a = pair_args(n, P, d, q, R, mu, err);
    a.pts = y;
    a.ldpts = ldy;
    a.horner = horner;
    a.beta = coef;
    a.part = part;
    a.ldp = ldp;
    const int units = pair_units<SIDE_TARGET>();
    const int npairs = a.tiles < units ? a.tiles : units;
    SLK_TIMED("pair_cheb_target", st);
    launch_pairs<SIDE_TARGET>(mp, md, a, npairs, st);
}

int64_t pair_moments_chunks(int P) {
    const int halves = P > QN ? 1 : 2;
    return static_cast<int64_t>(pair_units<SIDE_SOURCE>()) * halves;
}

void launch_pair_moments(const float* x, int64_t ldx, const float* mu, int64_t n, const void* xib, int P, int d,
                         const float* w, int q, double R, double* mom, float* absmax, unsigned* err, cudaStream_t st) {
    SLK_REQUIRE(pair_cheb_fits(P, q), "slice or term count unsupported by the CTA-pair Chebyshev kernel");
    SLK_REQUIRE(umma_f32_operand_ok(x, ldx), "FP32 sources need 16-byte aligned rows");
    SLK_REQUIRE(n >= 1 && n < (int64_t(1) << 31) - 2 * QM, "source count out of range for one launch");
    const CUtensorMap mp = tmap_f32_rows(x, n, d, ldx, QM);
    const CUtensorMap md = tmap_bf16_sw128(xib, P, d, umma_operand_ld(d), QM);
    PairArgs a = pair_args(n, P, d, q, R, mu, err);
    a.pts = x;
    a.ldpts = ldx;
    a.w = w;
    a.mom = mom;
    a.absmax = absmax;
    SLK_TIMED("pair_cheb_moments", st);
    // every pair writes its partial moments (zeros when it has no tile)
    launch_pairs<SIDE_SOURCE>(mp, md, a, pair_units<SIDE_SOURCE>(), st);
}

}  // namespace slk
