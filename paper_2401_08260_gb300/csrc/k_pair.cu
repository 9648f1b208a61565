// Fused Chebyshev kernels on CTA pairs (tcgen05 cta_group::2, sm_103a).
//
// Both sides of the Chebyshev evaluation of the truncated Fourier sum (Section 3.1,
// with the projection of Algorithm 1 fused in) read the caller's FP32 points directly:
//   target side  t(y) = sum_p sum_l beta[p][l] T_l(<xi_p, y - mu> / R)   (row sums per point)
//   source side  mom[p][j] = sum_n w_n T_j(<xi_p, x_n - mu> / R)          (moments per slice)
//
// Work item: one 256-point tile against one 256-slice half of the P <= 512 directions,
// computed by the two CTAs of a cluster of two.  Each CTA brings in, per 64-wide K stage,
// its own 128 FP32 point rows (two 32-column TMA boxes, converted in place to centred BF16
// in the tensor core's 128-byte-swizzled layout by three converter warps) and its own 128
// rows of the half's directions; the even CTA issues M = 256, N = 256 MMAs (kind::f16,
// FP32 accumulate) into one of two 256-column accumulators of each CTA's tensor memory,
// so that the epilogue of one item overlaps the MMAs of the next:
//   target side: A = points (rows = TMEM lanes), B = directions, D[point][slice];
//   source side: A = directions (rows = slices), B = points, D[slice][point].
// Items go round the pairs in order, so with an even number of pairs the two pairs that
// take the two halves of a tile work on it at the same time and the second read of its
// points is served by L2; while a CTA works on an item, its poller streams the rows of
// its next item's tile into L2, one contiguous chunk per stage.
//
// One thread of each CTA (warp 0) polls its barriers without blocking and issues
// whatever is ready: TMA loads of free stages and, on the even CTA, the MMAs of converted
// stages.  Signals between the CTAs are remote mbarrier arrivals at cluster scope:
//   odd CTA's converter warps    -> full[s] of the even CTA (release: their writes)
//   even CTA's poller            -> empty[s] of the odd CTA when the pair's MMAs released it
//                                   (relaxed: a pure signal)
//   one even-CTA epilogue thread -> acc_full[b] of the odd CTA
//   epilogue warps of both       -> acc_empty[b] of the even CTA (16 arrivals)
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
constexpr int QSTAGES = 4;
constexpr int QTHREADS = 384;                // warp 0 poller, 1-3 converters, 4-11 epilogue
constexpr int CVT_WARPS = 3;
constexpr int EPI0 = 4;                      // first epilogue warp (TMEM lane quarter = warp % 4)
constexpr int CVT_BYTES = QM * QK * 4;       // 128 FP32 rows x 64 (two 32-column boxes)
constexpr int DIR_BYTES = QM * QK * 2;       // 128 BF16 direction rows x 64
constexpr int QSTAGE_BYTES = CVT_BYTES + DIR_BYTES;
constexpr int QMAX_P = 2 * QN;               // two halves of 256 slices
constexpr uint32_t QTMEM_COLS = 512;         // two 256-column accumulators

enum { SIDE_TARGET = 0, SIDE_SOURCE = 1 };

struct PairSmem {
    uint64_t raw[QSTAGES];    // this CTA's TMA bytes of a stage have landed
    uint64_t cvt[QSTAGES];    // even CTA: its converters finished a stage (3 arrivals)
    uint64_t full[QSTAGES];   // even CTA: the odd CTA's converters finished a stage (3 arrivals)
    uint64_t empty[QSTAGES];  // the stage may be refilled
    uint64_t acc_full[2];     // an accumulator holds a finished item
    uint64_t acc_empty[2];    // even CTA: both CTAs' epilogues have read it
    uint64_t drain;           // even CTA: its last MMAs completed
    uint32_t tmem_base;
};

struct PairArgs {
    int n;          // points
    int P;          // slices (<= 512)
    int d;
    int tiles;      // 256-point tiles
    int halves;     // 256-slice halves (1 or 2)
    int q;          // Chebyshev terms
    int horner;     // target side: monomial coefficients
    float R, inv_R;
    const float* mu;    // centre (d values)
    const float* beta;  // target side: P x q coefficients
    double* part;       // target side: 2 * halves rows of ldp FP64 row sums
    int64_t ldp;
    const float* pts;   // the FP32 points (for the L2 prefetch), row stride ldpts
    int64_t ldpts;
    const float* w;     // source side: weights of the n points
    double* mom;        // source side: moment partials [chunk * P + p][q]
    float* absmax;      // source side: max |z| over the points
    unsigned* err;
};

// dynamic shared memory: the stage ring, the barriers, (target side) the q x 512
// coefficients and the d values of the centre (read by the converters from shared memory,
// so that no global load is outstanding when they signal the other CTA)
__host__ __device__ constexpr size_t pair_beta_offset() {
    return static_cast<size_t>(QSTAGES) * QSTAGE_BYTES + ((sizeof(PairSmem) + 15) & ~size_t(15));
}
__host__ __device__ constexpr size_t pair_smem_bytes(int beta_terms, int d) {
    return 1024 + pair_beta_offset() + static_cast<size_t>(QMAX_P) * beta_terms * sizeof(float) +
           ((static_cast<size_t>(d) * sizeof(float) + 15) & ~size_t(15));
}
constexpr size_t kPairSmemMax = 227 * 1024;

// Convert one converter warp's share of a stage's 128 FP32 rows (the stage holds two
// unswizzled 32-column boxes of 128 bytes per row) to centred BF16 in place over the first
// box, 128-byte swizzle (16-byte chunk c of row r at c ^ (r % 8)); rows at or beyond n are
// written as zeros.  The warp takes the 16-row batches cw, cw + CVT_WARPS, ... and reads all
// of them before it writes any (one round trip to shared memory instead of one per batch; a
// batch's rows are read and written only by its warp).  Lane l takes columns 4j..4j+3
// (j = l % 16) of rows 2u + l / 16 of each batch; m holds the centre at those columns (the
// same arithmetic as the single-CTA converting kernel).
__device__ __forceinline__ void convert_share(unsigned char* cv, int lane, int cw, const float (&m)[4], int row0,
                                              int n) {
    constexpr int HALF = QM * 128;
    constexpr int NBATCH = QM / 16;
    constexpr int PER_WARP = (NBATCH + CVT_WARPS - 1) / CVT_WARPS;
    const int j = lane & 15, rr = lane >> 4;
    const unsigned char* src = cv + (j >> 3) * HALF + (j & 7) * 16;
    float4 v[PER_WARP][8];
#pragma unroll
    for (int b = 0; b < PER_WARP; ++b) {
        const int bi = cw + b * CVT_WARPS;
        if (bi < NBATCH) {
#pragma unroll
            for (int u = 0; u < 8; ++u)
                v[b][u] = *reinterpret_cast<const float4*>(src + (bi * 16 + 2 * u + rr) * 128);
        }
    }
    __syncwarp();
    // x - m as x + (-m), two columns per packed add (the same bits as the scalar subtraction)
    const float2 nm01 = make_float2(-m[0], -m[1]), nm23 = make_float2(-m[2], -m[3]);
#pragma unroll
    for (int b = 0; b < PER_WARP; ++b) {
        const int bi = cw + b * CVT_WARPS;
        if (bi >= NBATCH) continue;
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int r = bi * 16 + 2 * u + rr;
            union { __nv_bfloat162 h[2]; uint2 u2; } pk;
            const float2 c01 = __fadd2_rn(make_float2(v[b][u].x, v[b][u].y), nm01);
            const float2 c23 = __fadd2_rn(make_float2(v[b][u].z, v[b][u].w), nm23);
            pk.h[0] = __floats2bfloat162_rn(c01.x, c01.y);
            pk.h[1] = __floats2bfloat162_rn(c23.x, c23.y);
            if (row0 + r >= n) pk.u2 = make_uint2(0u, 0u);
            *reinterpret_cast<uint2*>(cv + r * 128 + (((j >> 1) ^ (r & 7)) << 4) + ((j & 1) << 3)) = pk.u2;
        }
    }
}

template <int SIDE>
__global__ void __launch_bounds__(QTHREADS, 1)
    k_pair_cheb(const __grid_constant__ CUtensorMap map_pts, const __grid_constant__ CUtensorMap map_dir, PairArgs a) {
    extern __shared__ unsigned char smem_raw[];
    // 1024-byte aligned start, derived from the shared array itself so that every access
    // through it compiles to a shared-memory instruction
    unsigned char* base = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
    PairSmem* sm = reinterpret_cast<PairSmem*>(base + QSTAGES * QSTAGE_BYTES);
    float* sbeta = reinterpret_cast<float*>(base + pair_beta_offset());
    float* smu = sbeta + (SIDE == SIDE_TARGET ? QMAX_P * a.q : 0);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t rank = cluster_rank();
    const int pair = static_cast<int>(blockIdx.x >> 1), npairs = static_cast<int>(gridDim.x >> 1);
    const int kblocks = (a.d + QK - 1) / QK;
    const int items = a.tiles * a.halves;

    if (threadIdx.x == 0) {
        for (int s = 0; s < QSTAGES; ++s) {
            mbar_init(&sm->raw[s], 1);
            mbar_init(&sm->cvt[s], CVT_WARPS);
            mbar_init(&sm->full[s], CVT_WARPS);  // even CTA: one arrival per converter warp of the odd CTA
            mbar_init(&sm->empty[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&sm->acc_full[b], 1);
            mbar_init(&sm->acc_empty[b], 2 * 8);
        }
        mbar_init(&sm->drain, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (SIDE == SIDE_TARGET)
        for (int e = threadIdx.x; e < QMAX_P * a.q; e += blockDim.x) {
            const int l = e / QMAX_P, p = e - l * QMAX_P;
            sbeta[e] = p < a.P ? a.beta[static_cast<int64_t>(p) * a.q + l] : 0.0f;
        }
    for (int k = threadIdx.x; k < a.d; k += blockDim.x) smu[k] = a.mu[k];
    if (warp == 2) tmem_alloc_pair(&sm->tmem_base, QTMEM_COLS);
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    // both CTAs' barriers initialised and tensor memory allocated before any remote arrival
    cluster_barrier();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = sm->tmem_base;

    // this pair's items: pair, pair + npairs, ...; item -> (tile, half)
    int nloc = 0;
    for (int it = pair; it < items; it += npairs) ++nloc;
    const int total = nloc * kblocks;
    auto item_of = [&](int li) { return pair + li * npairs; };
    auto prow_of = [&](int li) { return (item_of(li) / a.halves) * (2 * QM) + static_cast<int>(rank) * QM; };

    if (warp == 0) {
        // ---------------- poller (one thread): TMA loads, the even CTA's MMAs, the odd CTA's forwards
        if (lane == 0) {
            // rows of the next item's tile brought into L2 a chunk per stage (contiguous bytes
            // of the row-major points), so that its TMA loads find them there
            const int chunk = (QM + kblocks - 1) / kblocks;
            auto prefetch_rows = [&](int li, int kb) {
                if (li >= nloc) return;
                const int rbase = prow_of(li);
                const int r0 = rbase + kb * chunk;
                int r1 = r0 + chunk;
                if (r1 > rbase + QM) r1 = rbase + QM;
                if (r1 > a.n) r1 = a.n;
                if (r0 >= r1) return;
                // from the first element of row r0 to the last element of row r1 - 1, rounded
                // down to 16 bytes (never past the caller's rows)
                const int64_t bytes = ((static_cast<int64_t>(r1 - r0 - 1) * a.ldpts + a.d) * 4) & ~int64_t(15);
                if (bytes > 0)
                    bulk_prefetch_l2(a.pts + static_cast<int64_t>(r0) * a.ldpts, static_cast<uint32_t>(bytes));
            };
            auto issue = [&](int g) {
                const int li = g / kblocks, kb = g % kblocks, s = g % QSTAGES;
                const int half = item_of(li) % a.halves;
                unsigned char* st = base + s * QSTAGE_BYTES;
                mbar_expect_tx(&sm->raw[s], CVT_BYTES + DIR_BYTES);
                tma_load_2d(st, &map_pts, &sm->raw[s], kb * QK, prow_of(li));
                tma_load_2d(st + QM * 128, &map_pts, &sm->raw[s], kb * QK + 32, prow_of(li));
                tma_load_2d(st + CVT_BYTES, &map_dir, &sm->raw[s], kb * QK, half * QN + static_cast<int>(rank) * QM);
                prefetch_rows(li + 1, kb);
            };
            const uint32_t idesc = instr_desc(1u, 2 * QM, QN);
            const uint32_t peer_empty0 = cluster_addr(&sm->empty[0], 1);
            int gf = 0, gm = 0;  // next fill, next MMA stage (even CTA)
            unsigned idle = 0;
            while (gf < total || (rank == 0 && gm < total)) {
                bool progress = false;
                if (gf < total) {
                    const int s = gf % QSTAGES;
                    const uint32_t ph = ((gf / QSTAGES) - 1) & 1;
                    if (gf < QSTAGES || mbar_test_cta(&sm->empty[s], ph)) {
                        // the even CTA passes the release of the stage on to the odd CTA (a pure
                        // signal: the MMAs that read the stage have completed)
                        if (rank == 0 && gf >= QSTAGES)
                            mbar_arrive_cluster_relaxed(peer_empty0 + static_cast<uint32_t>(s * sizeof(uint64_t)));
                        issue(gf);
                        ++gf;
                        progress = true;
                    }
                }
                if (rank == 0 && gm < gf) {
                    const int s = gm % QSTAGES, kb = gm % kblocks, li = gm / kblocks, b = li & 1;
                    const uint32_t ph = (gm / QSTAGES) & 1;
                    const bool acc_free = kb != 0 || li < 2 || mbar_test(&sm->acc_empty[b], ((li >> 1) - 1) & 1);
                    if (acc_free && mbar_test_cta(&sm->cvt[s], ph) && mbar_test(&sm->full[s], ph)) {
                        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                        unsigned char* st = base + s * QSTAGE_BYTES;
#pragma unroll
                        for (int k = 0; k < QK / 16; ++k) {
                            const uint64_t dp = smem_desc(st + k * 32);
                            const uint64_t dd = smem_desc(st + CVT_BYTES + k * 32);
                            if (SIDE == SIDE_TARGET)
                                umma_f16_pair(tmem + b * QN, dp, dd, idesc, (kb > 0 || k > 0) ? 1u : 0u);
                            else
                                umma_f16_pair(tmem + b * QN, dd, dp, idesc, (kb > 0 || k > 0) ? 1u : 0u);
                        }
                        umma_commit_pair(&sm->empty[s]);
                        if (kb == kblocks - 1) umma_commit_pair(&sm->acc_full[b]);
                        ++gm;
                        progress = true;
                    }
                }
                if (progress) {
                    idle = 0;
                } else if (++idle > WAIT_LIMIT) {
                    atomicOr(a.err, rank == 0 ? 16u : 8u);
                    break;
                }
            }
            drain_fills(sm->raw, QSTAGES, gf);
            if (rank == 0) drain_mma_pair(&sm->drain, a.err, 16u);
        }
    } else if (warp < EPI0) {
        // ---------------- converters (warps 1-3) of this CTA's points: 16-row batches
        // cw, cw + 3, ... of every stage
        const int cw = warp - 1;
        const uint32_t lead_full0 = cluster_addr(&sm->full[0], 0);
        for (int g = 0; g < total; ++g) {
            const int s = g % QSTAGES, kb = g % kblocks;
            float m[4];
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const int k = kb * QK + 4 * (lane & 15) + e;
                m[e] = k < a.d ? smu[k] : 0.0f;
            }
            const bool got = mbar_wait(&sm->raw[s], (g / QSTAGES) & 1);
            if (!__all_sync(0xffffffffu, got)) {
                if (lane == 0) atomicOr(a.err, 8u);
                break;
            }
            const int row0 = prow_of(g / kblocks);
            convert_share(base + s * QSTAGE_BYTES, lane, cw, m, row0, a.n);
            // generic-proxy writes, read next by the tensor core (async proxy)
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            __syncwarp();
            // even CTA: its own converters' barrier; odd CTA: straight to the even CTA's full[s]
            if (lane == 0) {
                if (rank == 0) mbar_arrive(&sm->cvt[s]);
                else mbar_arrive_cluster(lead_full0 + static_cast<uint32_t>(s * sizeof(uint64_t)));
            }
        }
    } else {
        // ---------------- epilogue (warps 4-11): TMEM lane quarter warp % 4, column half
        // grp = (warp - 4) / 4 of the item's accumulator
        const int q4 = warp & 3, grp = (warp - EPI0) >> 2;
        const uint32_t lane_off = static_cast<uint32_t>(q4 * 32) << 16;
        const uint32_t acc_empty0 = cluster_addr(&sm->acc_empty[0], 0);
        const uint32_t peer_full0 = cluster_addr(&sm->acc_full[0], 1);
        const bool forwarder = rank == 0 && warp == EPI0 && lane == 0;
        auto wait_acc = [&](int li) {
            const int b = li & 1;
            if (!mbar_wait_cluster(&sm->acc_full[b], (li >> 1) & 1)) {
                atomicOr(a.err, 32u);
                return false;
            }
            if (forwarder) mbar_arrive_cluster(peer_full0 + static_cast<uint32_t>(b * sizeof(uint64_t)));
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            return true;
        };
        auto release_acc = [&](int li) {
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            __syncwarp();
            if (lane == 0) mbar_arrive_cluster(acc_empty0 + static_cast<uint32_t>((li & 1) * sizeof(uint64_t)));
        };
        constexpr int NC = QN / 2;  // columns per thread
        if (SIDE == SIDE_TARGET) {
            // row sums of t_p(z) over this warp's 128 slices of the item's half
            bool bad = false;
            float mabs = 0.0f;  // max |z| of the Horner chunks, checked against R at the end
            auto run = [&](auto qp_tag, auto horner_tag) {
                constexpr int QP = decltype(qp_tag)::value;
                constexpr bool HORNER = decltype(horner_tag)::value;
                auto chunk = [&](const uint32_t (&r)[32], const float* bt0, float& s_, float& c_) {
                    if constexpr (HORNER) horner_chunk32<QP>(r, bt0, QMAX_P, a.inv_R, s_, c_, mabs);
                    else cheb_chunk32<QP, false>(r, bt0, QMAX_P, a.R, a.inv_R, s_, c_, bad);
                };
                for (int li = 0; li < nloc; ++li) {
                    if (!wait_acc(li)) break;
                    const int item = item_of(li), half = item % a.halves;
                    const int row = (item / a.halves) * (2 * QM) + static_cast<int>(rank) * QM + q4 * 32 + lane;
                    const float* bt = sbeta + half * QN + grp * NC;
                    float sum = 0.0f, comp = 0.0f;  // Kahan
                    uint32_t ra[32], rb[32];
                    const uint32_t tbase = tmem + lane_off + (li & 1) * QN + grp * NC;
                    tmem_ld32_issue(tbase, ra);
                    tmem_wait32(ra);
#pragma unroll 1
                    for (int cc = 0; cc < NC; cc += 64) {
                        tmem_ld32_issue(tbase + cc + 32, rb);
                        chunk(ra, bt + cc, sum, comp);
                        tmem_wait32(rb);
                        if (cc + 64 < NC) tmem_ld32_issue(tbase + cc + 64, ra);
                        chunk(rb, bt + cc + 32, sum, comp);
                        if (cc + 64 < NC) tmem_wait32(ra);
                    }
                    release_acc(li);
                    if (!(sum == sum)) bad = true;  // a NaN projection
                    if (row < a.n)
                        a.part[static_cast<int64_t>(half * 2 + grp) * a.ldp + row] =
                            static_cast<double>(sum) - static_cast<double>(comp);
                }
            };
            using T_ = std::true_type;
            using F_ = std::false_type;
            if (a.q == 10) a.horner ? run(std::integral_constant<int, 10>{}, T_{}) : run(std::integral_constant<int, 10>{}, F_{});
            else if (a.q == 12) a.horner ? run(std::integral_constant<int, 12>{}, T_{}) : run(std::integral_constant<int, 12>{}, F_{});
            else if (a.q == 8) a.horner ? run(std::integral_constant<int, 8>{}, T_{}) : run(std::integral_constant<int, 8>{}, F_{});
            else a.horner ? run(std::integral_constant<int, 16>{}, T_{}) : run(std::integral_constant<int, 16>{}, F_{});
            if (!(mabs <= a.R)) bad = true;
            if (bad) atomicOr(a.err, 4u);
        } else {
            // one slice's moments per thread over this warp's 128 points of every item; a pair
            // keeps one half of the slices throughout (the host launches an even number of
            // pairs when there are two halves)
            const int half = pair % a.halves;
            const int slice = half * QN + static_cast<int>(rank) * QM + q4 * 32 + lane;
            float mx = 0.0f;
            auto run = [&](auto qp_tag) {
                constexpr int QP = decltype(qp_tag)::value;
                float hi[QP], lo[QP];
#pragma unroll
                for (int k = 0; k < QP; ++k) hi[k] = lo[k] = 0.0f;
                for (int li = 0; li < nloc; ++li) {
                    if (!wait_acc(li)) break;
                    const int tile = item_of(li) / a.halves;
                    float2 tt[QP];  // this item's sums over its even and odd points
#pragma unroll
                    for (int k = 0; k < QP; ++k) tt[k] = make_float2(0.0f, 0.0f);
                    auto chunk = [&](const uint32_t (&r)[32], int cc) {
                        // accumulator column c holds point tile * 256 + c (columns 0-127 from the
                        // even CTA's rows of B, 128-255 from the odd CTA's)
                        const int pt0 = tile * (2 * QM) + grp * NC + cc;
                        const float wl = pt0 + lane < a.n ? __ldg(a.w + pt0 + lane) : 0.0f;
                        float v[32];
#pragma unroll
                        for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
                        mom_chunk2<QP>(v, wl, a.inv_R, a.n - pt0, tt, mx);
                    };
                    uint32_t ra[32], rb[32];
                    const uint32_t tbase = tmem + lane_off + (li & 1) * QN + grp * NC;
                    tmem_ld32_issue(tbase, ra);
                    tmem_wait32(ra);
#pragma unroll 1
                    for (int cc = 0; cc < NC; cc += 64) {
                        tmem_ld32_issue(tbase + cc + 32, rb);
                        chunk(ra, cc);
                        tmem_wait32(rb);
                        if (cc + 64 < NC) tmem_ld32_issue(tbase + cc + 64, ra);
                        chunk(rb, cc + 32);
                        if (cc + 64 < NC) tmem_wait32(ra);
                    }
                    release_acc(li);
#pragma unroll
                    for (int k = 0; k < QP; ++k) two_sum_into(hi[k], lo[k], tt[k].x + tt[k].y);
                }
                if (slice < a.P) {
                    // chunk: the pair (of a pair of pairs with two halves) and the column half
                    const int c = (a.halves == 2 ? pair >> 1 : pair) * 2 + grp;
                    double* out = a.mom + (static_cast<int64_t>(c) * a.P + slice) * QP;
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

// ---------------------------------------------------------------- FP16 hi/lo projection
// Z = Xi (X - mu)^T to FP32 accuracy on CTA pairs: the split of the single-CTA kernel
// k_umma_project_x3 (a = a_hi + 2^-11 a_lo' for both operands; per 16-wide K step the
// correction products a_hi b_lo' + a_lo' b_hi, then a_hi b_hi with the accumulator scaled by
// 2^-11 on input, into a fresh accumulator that the epilogue adds into FP32 registers with
// round-to-nearest), with a pair computing a 256-point x 256-slice tile by M = 256, N = 256
// MMAs: each CTA loads its own 128 point rows and its own 128 direction rows (hi and lo) per
// 64-wide K stage, so every byte brought into shared memory feeds twice the MMA work of the
// single CTA's 128 x 128 tile.
//   warp 0:     poller: TMA loads; even CTA: the MMAs and the release of a stage to the odd
//               CTA; odd CTA: a remote arrival on the even CTA's peer_full when its bytes landed
//   warp 1:     tensor memory (two 256-column accumulators per CTA); even CTA: passes each
//               finished K step on to the odd CTA's epilogue
//   warps 2-17: epilogue, TMEM lane quarter warp % 4 and 64 columns (warp - 2) / 4 each
constexpr int X3P_STAGES = 3;
constexpr int X3P_THREADS = 576;
constexpr int X3P_EPI0 = 2;
constexpr int X3P_EPI_WARPS = 16;
constexpr int X3P_TILE_BYTES = QM * QK * 2;  // 128 rows x 64 16-bit values
constexpr int X3P_STAGE_BYTES = 4 * X3P_TILE_BYTES;
constexpr uint32_t X3P_TMEM_COLS = 512;

struct X3PairSmem {
    uint64_t full[X3P_STAGES];       // this CTA's TMA bytes of a stage have landed
    uint64_t peer_full[X3P_STAGES];  // even CTA: the odd CTA's bytes of a stage have landed
    uint64_t empty[X3P_STAGES];      // the stage may be refilled
    uint64_t d_full[2];              // an accumulator holds a finished K step
    uint64_t d_empty[2];             // even CTA: both CTAs' epilogue warps have read it
    uint64_t drain;                  // even CTA: its last MMAs completed
    uint32_t tmem_base;
};

struct X3PairArgs {
    int n, P, d, col_tiles;
    float* Z;
    int64_t ldz;
    float* absmax;
    unsigned* err;
};

__host__ __device__ constexpr size_t x3_pair_smem_bytes() {
    return 1024 + static_cast<size_t>(X3P_STAGES) * X3P_STAGE_BYTES + sizeof(X3PairSmem);
}

__global__ void __launch_bounds__(X3P_THREADS, 1)
    k_pair_project_x3(const __grid_constant__ CUtensorMap map_a, const __grid_constant__ CUtensorMap map_b,
                      const __grid_constant__ CUtensorMap map_a2, const __grid_constant__ CUtensorMap map_b2,
                      X3PairArgs a) {
    extern __shared__ unsigned char smem_raw[];
    unsigned char* base = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
    X3PairSmem* sm = reinterpret_cast<X3PairSmem*>(base + X3P_STAGES * X3P_STAGE_BYTES);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t rank = cluster_rank();
    const int pair = static_cast<int>(blockIdx.x >> 1);
    const int row0 = (pair / a.col_tiles) * (2 * QM) + static_cast<int>(rank) * QM;  // this CTA's points
    const int col0 = (pair % a.col_tiles) * QN;                                     // the pair's slices
    const int brow0 = col0 + static_cast<int>(rank) * QM;                           // this CTA's directions
    const int kblocks = (a.d + QK - 1) / QK;
    const int ksteps = kblocks * (QK / 16);

    if (threadIdx.x == 0) {
        for (int s = 0; s < X3P_STAGES; ++s) {
            mbar_init(&sm->full[s], 1);
            mbar_init(&sm->peer_full[s], 1);
            mbar_init(&sm->empty[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&sm->d_full[b], 1);
            mbar_init(&sm->d_empty[b], 2 * X3P_EPI_WARPS);
        }
        mbar_init(&sm->drain, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) tmem_alloc_pair(&sm->tmem_base, X3P_TMEM_COLS);
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    // both CTAs' barriers initialised and tensor memory allocated before any remote arrival
    cluster_barrier();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = sm->tmem_base;

    if (warp == 0) {
        if (lane == 0) {
            const uint32_t idesc = instr_desc(0u, 2 * QM, QN);
            const uint32_t peer_empty0 = cluster_addr(&sm->empty[0], 1);
            const uint32_t lead_pfull0 = cluster_addr(&sm->peer_full[0], 0);
            int gf = 0, gp = 0, gk = 0;  // next fill, next forward (odd), next K step (even)
            unsigned idle = 0;
            while (gf < kblocks || (rank == 1 && gp < kblocks) || (rank == 0 && gk < ksteps)) {
                bool progress = false;
                if (gf < kblocks) {
                    const int s = gf % X3P_STAGES;
                    if (gf < X3P_STAGES || mbar_test_cta(&sm->empty[s], ((gf / X3P_STAGES) - 1) & 1)) {
                        // the even CTA passes the release of the stage on to the odd CTA
                        if (rank == 0 && gf >= X3P_STAGES)
                            mbar_arrive_cluster_relaxed(peer_empty0 + static_cast<uint32_t>(s * sizeof(uint64_t)));
                        unsigned char* st = base + s * X3P_STAGE_BYTES;
                        mbar_expect_tx(&sm->full[s], X3P_STAGE_BYTES);
                        tma_load_2d(st, &map_a, &sm->full[s], gf * QK, row0);
                        tma_load_2d(st + X3P_TILE_BYTES, &map_b, &sm->full[s], gf * QK, brow0);
                        tma_load_2d(st + 2 * X3P_TILE_BYTES, &map_a2, &sm->full[s], gf * QK, row0);
                        tma_load_2d(st + 3 * X3P_TILE_BYTES, &map_b2, &sm->full[s], gf * QK, brow0);
                        ++gf;
                        progress = true;
                    }
                }
                if (rank == 1 && gp < gf) {
                    const int s = gp % X3P_STAGES;
                    if (mbar_test_cta(&sm->full[s], (gp / X3P_STAGES) & 1)) {
                        mbar_arrive_cluster(lead_pfull0 + static_cast<uint32_t>(s * sizeof(uint64_t)));
                        ++gp;
                        progress = true;
                    }
                }
                if (rank == 0 && gk < ksteps) {
                    const int g = gk >> 2, k = gk & 3, s = g % X3P_STAGES, b = gk & 1;
                    bool ready = g < gf;
                    if (ready && k == 0)
                        ready = mbar_test_cta(&sm->full[s], (g / X3P_STAGES) & 1) &&
                                mbar_test(&sm->peer_full[s], (g / X3P_STAGES) & 1);
                    if (ready && gk >= 2) ready = mbar_test(&sm->d_empty[b], ((gk >> 1) - 1) & 1);
                    if (ready) {
                        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                        unsigned char* st = base + s * X3P_STAGE_BYTES;
                        const uint64_t ah = smem_desc(st + k * 32);
                        const uint64_t bh = smem_desc(st + X3P_TILE_BYTES + k * 32);
                        const uint64_t al = smem_desc(st + 2 * X3P_TILE_BYTES + k * 32);
                        const uint64_t bl = smem_desc(st + 3 * X3P_TILE_BYTES + k * 32);
                        const uint32_t dt = tmem + static_cast<uint32_t>(b * QN);
                        umma_f16_pair(dt, ah, bl, idesc, 0u);
                        umma_f16_pair(dt, al, bh, idesc, 1u);
                        umma_f16_pair_scale_d<11>(dt, ah, bh, idesc);
                        umma_commit_pair(&sm->d_full[b]);
                        if (k == QK / 16 - 1) umma_commit_pair(&sm->empty[s]);
                        ++gk;
                        progress = true;
                    }
                }
                if (progress) {
                    idle = 0;
                } else if (++idle > WAIT_LIMIT) {
                    atomicOr(a.err, rank == 0 ? 16u : 8u);
                    break;
                }
            }
            drain_fills(sm->full, X3P_STAGES, gf);
            if (rank == 0) drain_mma_pair(&sm->drain, a.err, 16u);
        }
    } else if (warp == 1) {
        // even CTA: pass every finished K step on to the odd CTA's epilogue as soon as it lands
        if (rank == 0 && lane == 0) {
            const uint32_t peer_dfull0 = cluster_addr(&sm->d_full[0], 1);
            for (int t = 0; t < ksteps; ++t) {
                const int b = t & 1;
                if (!mbar_wait_cluster(&sm->d_full[b], (t >> 1) & 1)) {
                    atomicOr(a.err, 32u);
                    break;
                }
                mbar_arrive_cluster(peer_dfull0 + static_cast<uint32_t>(b * sizeof(uint64_t)));
            }
        }
    } else if (warp >= X3P_EPI0) {
        const int q4 = warp & 3, cg = (warp - X3P_EPI0) >> 2;
        const uint32_t lane_off = static_cast<uint32_t>(q4 * 32) << 16;
        const uint32_t d_empty0 = cluster_addr(&sm->d_empty[0], 0);
        float acc[64];
#pragma unroll
        for (int j = 0; j < 64; ++j) acc[j] = 0.0f;
        bool ok = true;
        for (int t = 0; t < ksteps; ++t) {
            const int b = t & 1;
            if (!mbar_wait_cluster(&sm->d_full[b], (t >> 1) & 1)) {
                atomicOr(a.err, 32u);
                ok = false;
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            // 16 columns at a time (the 64 running sums leave room for one load in flight)
            const uint32_t ta = tmem + lane_off + static_cast<uint32_t>(b * QN + cg * 64);
            uint32_t v[16];
#pragma unroll
            for (int c = 0; c < 48; c += 16) {
                tmem_ld16_issue(ta + c, v);
                tmem_wait16(v);
#pragma unroll
                for (int j = 0; j < 16; ++j) acc[c + j] = __fadd_rn(acc[c + j], __uint_as_float(v[j]));
            }
            tmem_ld16_issue(ta + 48, v);
            tmem_wait16(v);
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            __syncwarp();
            if (lane == 0) mbar_arrive_cluster(d_empty0 + static_cast<uint32_t>(b * sizeof(uint64_t)));
#pragma unroll
            for (int j = 0; j < 16; ++j) acc[48 + j] = __fadd_rn(acc[48 + j], __uint_as_float(v[j]));
        }
        float mx = 0.0f;
        const int row = row0 + q4 * 32 + lane;
        if (ok && row < a.n) {
#pragma unroll
            for (int j = 0; j < 64; ++j) {
                const int p = col0 + cg * 64 + j;
                if (p < a.P) {
                    a.Z[static_cast<int64_t>(p) * a.ldz + row] = acc[j];
                    mx = fmaxf(mx, fabsf(acc[j]));
                }
            }
        }
        if (a.absmax) {
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
            if (lane == 0) atomicMax(reinterpret_cast<unsigned int*>(a.absmax), __float_as_uint(mx));
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    // neither CTA frees its tensor memory or leaves while the pair's MMAs or arrivals may
    // still reach it
    cluster_barrier();
    if (warp == 1) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        tmem_dealloc_pair(tmem, X3P_TMEM_COLS);
    }
}

}  // namespace
bool pair_cheb_fits(int P, int q, int d) {
    return P >= 1 && P <= QMAX_P && (q == 8 || q == 10 || q == 12 || q == 16) && d >= 1 &&
           pair_smem_bytes(q, d) <= kPairSmemMax;
}

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
    cfg.dynamicSmemBytes = pair_smem_bytes(SIDE == SIDE_TARGET ? a.q : 0, a.d);
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
    a.halves = P > QN ? 2 : 1;
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
    SLK_REQUIRE(pair_cheb_fits(P, q, d), "slice count, term count or dimension unsupported by the CTA-pair Chebyshev kernel");
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
    const int items = a.tiles * a.halves;
    // an even number of pairs (when there are more items) keeps the two halves of a tile together
    const int npairs = items < units ? items : (units & ~1);
    SLK_TIMED("pair_cheb_target", st);
    launch_pairs<SIDE_TARGET>(mp, md, a, npairs, st);
}

int64_t pair_cheb_parts(int P) { return P > QN ? 4 : 2; }

// Source-side launches use every co-resident pair (an even number of them with two halves,
// each pair keeping one half of the slices in its registers).
static int source_pairs(int P) {
    const int units = pair_units<SIDE_SOURCE>();
    const int pairs = P > QN ? (units & ~1) : units;
    SLK_REQUIRE(pairs >= 1, "too few co-resident CTA pairs for the fused moments kernel");
    return pairs;
}

int64_t pair_moments_chunks(int P) { return 2 * static_cast<int64_t>(P > QN ? source_pairs(P) / 2 : source_pairs(P)); }

void launch_pair_moments(const float* x, int64_t ldx, const float* mu, int64_t n, const void* xib, int P, int d,
                         const float* w, int q, double R, double* mom, float* absmax, unsigned* err, cudaStream_t st) {
    SLK_REQUIRE(pair_cheb_fits(P, q, d), "slice count, term count or dimension unsupported by the CTA-pair Chebyshev kernel");
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
    launch_pairs<SIDE_SOURCE>(mp, md, a, source_pairs(P), st);
}

void launch_pair_project_x3(const void* xa, const void* xa_lo, int64_t n, const void* xib, const void* xib_lo, int P,
                            int d, float* Z, int64_t ldz, float* absmax, unsigned* err, cudaStream_t st) {
    if (n <= 0) return;
    SLK_REQUIRE(n < (int64_t(1) << 31) - 2 * QM, "too many points for one projection");
    const int64_t ld = umma_operand_ld(d);
    // the FP16 operands move through the 16-bit, 128-byte-swizzled maps of the BF16 path
    const CUtensorMap ma = tmap_bf16_sw128(xa, n, d, ld, QM);
    const CUtensorMap mb = tmap_bf16_sw128(xib, P, d, ld, QM);
    const CUtensorMap ma2 = tmap_bf16_sw128(xa_lo, n, d, ld, QM);
    const CUtensorMap mb2 = tmap_bf16_sw128(xib_lo, P, d, ld, QM);
    X3PairArgs a{};
    a.n = static_cast<int>(n);
    a.P = P;
    a.d = d;
    a.col_tiles = static_cast<int>(ceil_div(P, QN));
    a.Z = Z;
    a.ldz = ldz;
    a.absmax = absmax;
    a.err = err;
    const int64_t pairs = ceil_div(n, 2 * QM) * a.col_tiles;
    SLK_REQUIRE(2 * pairs < (int64_t(1) << 31), "too many points for one projection");
    static bool attr = false;
    if (!attr) {
        SLK_CHECK_CUDA(cudaFuncSetAttribute(k_pair_project_x3, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                            static_cast<int>(x3_pair_smem_bytes())));
        attr = true;
    }
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attrs[1];
    attrs[0].id = cudaLaunchAttributeClusterDimension;
    attrs[0].val.clusterDim.x = 2;
    attrs[0].val.clusterDim.y = 1;
    attrs[0].val.clusterDim.z = 1;
    cfg.gridDim = dim3(static_cast<unsigned>(2 * pairs));
    cfg.blockDim = dim3(X3P_THREADS);
    cfg.dynamicSmemBytes = x3_pair_smem_bytes();
    cfg.stream = st;
    cfg.attrs = attrs;
    cfg.numAttrs = 1;
    SLK_TIMED("pair_project_x3", st);
    SLK_CHECK_CUDA(cudaLaunchKernelEx(&cfg, k_pair_project_x3, ma, mb, ma2, mb2, a));
}

}  // namespace slk
