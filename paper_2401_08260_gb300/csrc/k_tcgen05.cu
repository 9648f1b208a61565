// Tensor-core projection Z = Xi (X - mu)^T on sm_103a (tcgen05 + TMA).
//
// The projection of Algorithm 1 is the one dense contraction of the path:
// Z[p][i] = sum_k xi[p][k] (x[i][k] - mu[k]) for P directions and n points.
// Per CTA: a 128-point x 256-slice output tile.  A (points, K-major) and B
// (directions, K-major) tiles of 64 K-elements are brought in by TMA with the
// 128-byte swizzle into a 4-stage shared-memory ring; one thread issues
// tcgen05.mma (kind::f16, BF16 or FP16 inputs, FP32 accumulate) into a
// 128 x 256 FP32 accumulator in tensor memory; four epilogue warps read it back
// with tcgen05.ld and store Z slice-major (coalesced along points), keeping
// the largest |z| on the way.
//
// The fused Chebyshev target kernel also comes in a variant that reads the
// targets as FP32 rows straight from the caller's array: TMA brings each
// 64-column stage in as two 32-column halves, three converter warps centre and
// round them to BF16 in shared memory, in place, in the swizzled layout the
// tensor core reads, and only then release the stage to the MMA issuer.  This
// removes the separate centring pass over the targets (an FP32 read and a BF16
// write and re-read of every target) and leaves bit-identical operands.
//
// The FP16 "x3" variant (k_umma_project_x3) splits both operands into a high
// and a scaled low FP16 part (a = a_hi + 2^-11 a_lo') and forms
// a_hi b_hi + 2^-11 (a_hi b_lo' + a_lo' b_hi) (error ~ 2^-22 relative per
// product, about FP32), promoting each 16-wide K step's three products, folded
// into one accumulator, to FP32 registers (see the kernel's comment).
//
// Every mbarrier wait is bounded: on timeout the kernel records an error bit,
// skips the remaining work, still frees its tensor memory and returns.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <type_traits>

#include "kernels.cuh"
#include "cheb_epi.cuh"
#include "umma.cuh"

namespace slk {

namespace {

using namespace umma;

constexpr int BM = 128;       // points per tile (TMEM lanes)
constexpr int BN = 256;       // slices per tile (TMEM columns per accumulator)
constexpr int BK = 64;        // K elements per stage (128 bytes of 16-bit data)
constexpr int STAGES_1 = 4;  // one 16-bit product: 48 KB per stage
constexpr int THREADS = 256;  // warp 0: TMA, warp 1: MMA, warp 2: TMEM alloc, warps 4-7: epilogue

template <class Half>
__device__ __forceinline__ Half to_half(float v);
template <>
__device__ __forceinline__ __nv_bfloat16 to_half<__nv_bfloat16>(float v) { return __float2bfloat16_rn(v); }
template <>
__device__ __forceinline__ __half to_half<__half>(float v) { return __float2half_rn(v); }

struct Smem {
    // follows the stage buffers (each stage: A tile then B tile, 1024-byte aligned)
    uint64_t full[STAGES_1];
    uint64_t empty[STAGES_1];
    uint64_t raw_full[STAGES_1];  // FP32-input variant: the TMA bytes of a stage have landed
    uint64_t acc_full[2];
    uint64_t acc_empty[2];
    uint64_t drain;  // the MMA issuer's last commit (all its MMAs complete)
    uint32_t tmem_base;
};

// Stage geometry of the persistent projection.  CVT (target side only): the targets
// arrive as FP32 rows (two 32-column halves of 128 bytes per row, unswizzled) and are
// centred and rounded to BF16 in shared memory, in place over the first half, by the
// converter warps; three stages of 64 KB.
template <bool CVT>
struct Geo {
    static constexpr int A_BYTES = CVT ? BM * BK * 4 : BM * BK * 2;
    static constexpr int B_BYTES = BN * BK * 2;
    static constexpr int STAGE_BYTES = A_BYTES + B_BYTES;
    static constexpr int STAGES = CVT ? 3 : STAGES_1;
};

// BF16 projection, persistent: each CTA walks tiles blockIdx.x, blockIdx.x + gridDim.x, ...
// (column tile fastest, so the CTAs that share a block of points run together and the
// second read of A hits L2).  Two 256-column TMEM accumulators alternate between tiles:
// the epilogue of one tile overlaps the MMAs of the next.
// Epilogues:
//   EPI_Z:    Z[col * ldz + row] (slice-major projections), largest |z| into *absmax;
//   EPI_ROW:  Z[row * ldz + col] * rowscale(row), rowscale = scale * (rs ? rs[row] : 1)
//             (the backward product, rows = targets, columns = coordinates);
//   EPI_CHEB: the target side of the Chebyshev evaluation fused in: for every row
//             (target) and column (slice p) t_p = sum_l beta[p][l] T_l(z / R) by Clenshaw,
//             summed over the tile's columns; Z receives the FP64 partial row sums
//             Z_part[(col_tile * 2 + half) * n + row] (no projection is stored).
//   EPI_MOM:  the source side of the Chebyshev evaluation fused in, with the roles turned
//             round: A = directions (rows = slices), B = points (columns); every thread
//             keeps one slice's moments mu_j = sum_n w_n T_j(z / R) in registers over all the
//             point tiles of its CTA and writes them once (no projection is stored).
enum { EPI_Z = 0, EPI_ROW = 1, EPI_CHEB = 2, EPI_MOM = 3 };

struct ChebEpi {
    const float* beta;  // P x q: Chebyshev coefficients, or monomial ones when horner
    int q;
    int horner;
    float inv_R, R;
    double* part;  // (2 * col_tiles) x ldp
    int64_t ldp;
    // EPI_MOM: weights of the npts points, moment partials mom[(chunk * P + slice) * q + j]
    const float* w;
    int npts;
    double* mom;
    // FP32-target variant: the centre subtracted from the targets (d values)
    const float* mu;
};

//
// Work items: item -> slice tile (item % col_tiles), point block (item / col_tiles).
// Each CTA loads its own A and B tiles into its own shared memory (no loads are shared
// between CTAs).
template <int EPI, bool CVT>
__global__ void __launch_bounds__(EPI == EPI_CHEB || EPI == EPI_MOM ? 384 : 256, 1)
    k_umma_project(const __grid_constant__ CUtensorMap map_a, const __grid_constant__ CUtensorMap map_b, int n, int P,
                   int d, int col_tiles, int tiles, float* __restrict__ Z, int64_t ldz, float* __restrict__ absmax,
                   unsigned* __restrict__ err, const float* __restrict__ rs, float scale, ChebEpi ce) {
    static_assert(!CVT || EPI == EPI_CHEB, "FP32 targets: fused target epilogue only");
    using G = Geo<CVT>;
    constexpr bool ROWMAJOR = EPI == EPI_ROW;
    int unit = static_cast<int>(blockIdx.x), nunits = static_cast<int>(gridDim.x);
    // EPI_MOM: a CTA keeps one slice block for all its point tiles, so its threads can
    // accumulate their slices' moments across tiles
    int mom_group = 0, mom_chunk_id = -1;
    if (EPI == EPI_MOM) {
        const int groups = static_cast<int>((n + BM - 1) / BM);
        const int per_group = nunits / groups;
        mom_group = unit % groups;
        mom_chunk_id = unit / groups < per_group ? unit / groups : -1;
        unit = mom_chunk_id >= 0 ? mom_chunk_id : tiles;  // idle units take no tile
        nunits = per_group > 0 ? per_group : 1;
    }
    auto row_of = [&](int item) {
        return EPI == EPI_MOM ? mom_group * BM : (item / col_tiles) * BM;
    };
    auto col_of = [&](int item) { return EPI == EPI_MOM ? item * BN : (item % col_tiles) * BN; };
    constexpr int EPI_WARPS = EPI == EPI_CHEB || EPI == EPI_MOM ? 8 : 4;
    constexpr int STAGES = G::STAGES;
    extern __shared__ unsigned char smem_raw[];
    // 1024-byte aligned start, derived from the shared array itself so that every access
    // through it compiles to a shared-memory instruction
    unsigned char* base = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
    constexpr int A_BYTES = G::A_BYTES, B_BYTES = G::B_BYTES;
    constexpr int STAGE_BYTES = G::STAGE_BYTES;
    Smem* sm = reinterpret_cast<Smem*>(base + STAGES * STAGE_BYTES);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int kblocks = (d + BK - 1) / BK;
    constexpr uint32_t TMEM_COLS = 512;

    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(&sm->full[s], CVT ? 96 : 1);  // CVT: one arrival per converter thread
            mbar_init(&sm->empty[s], 1);  // one MMA commit
            mbar_init(&sm->raw_full[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&sm->acc_full[b], 1);
            mbar_init(&sm->acc_empty[b], EPI_WARPS);  // one arrival per epilogue warp
        }
        mbar_init(&sm->drain, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    // Chebyshev coefficients in shared memory (after the Smem struct), degree-major
    // sbeta[l * ppad + p], zero for the padding slices p >= P (whose projections are 0)
    const int ppad = col_tiles * BN;
    float* sbeta = reinterpret_cast<float*>(base + STAGES * STAGE_BYTES + ((sizeof(Smem) + 15) & ~size_t(15)));
    if (EPI == EPI_CHEB)
        for (int e = threadIdx.x; e < ppad * ce.q; e += blockDim.x) {
            const int l = e / ppad, p = e - l * ppad;
            sbeta[e] = p < P ? ce.beta[static_cast<int64_t>(p) * ce.q + l] : 0.0f;
        }
    if (warp == 2) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&sm->tmem_base)),
                     "r"(TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = sm->tmem_base;

    if (!CVT && warp == 0 && lane == 0) {
        // ---------------- TMA producer: one ring across all tiles of this CTA
        int g = 0;
        bool ok = true;
        for (int tile = unit; tile < tiles && ok; tile += nunits) {
            const int row0 = row_of(tile), col0 = col_of(tile);
            for (int kb = 0; kb < kblocks; ++kb, ++g) {
                const int s = g % STAGES;
                if (g >= STAGES && !mbar_wait(&sm->empty[s], ((g / STAGES) - 1) & 1)) {
                    atomicOr(err, 8u);
                    ok = false;
                    break;
                }
                unsigned char* st = base + s * STAGE_BYTES;
                mbar_expect_tx(&sm->full[s], STAGE_BYTES);
                tma_load_2d(st, &map_a, &sm->full[s], kb * BK, row0);
                tma_load_2d(st + A_BYTES, &map_b, &sm->full[s], kb * BK, col0);
            }
        }
        // Before the CTA may exit, the bytes of every stage it filled have landed: the
        // last fill of each stage completed its full barrier (at once on the normal path,
        // where the MMA issuer waited on them; bounded after an error on either side).
        drain_fills(sm->full, STAGES, g);
    } else if (!CVT && warp == 1 && lane == 0) {
        // ---------------- MMA issuer
        const uint32_t idesc = instr_desc(1u, BM, BN);
        int g = 0, local = 0;
        bool ok = true;
        for (int tile = unit; tile < tiles && ok; tile += nunits, ++local) {
            const int b = local & 1;
            if (local >= 2 && !mbar_wait(&sm->acc_empty[b], ((local >> 1) - 1) & 1)) {
                atomicOr(err, 16u);
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t acc_t = tmem + b * BN;
            for (int kb = 0; kb < kblocks; ++kb, ++g) {
                const int s = g % STAGES;
                if (!mbar_wait(&sm->full[s], (g / STAGES) & 1)) {
                    atomicOr(err, 16u);
                    ok = false;
                    break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                unsigned char* st = base + s * STAGE_BYTES;
#pragma unroll
                for (int k = 0; k < BK / 16; ++k) {
                    // advancing 16 elements (32 bytes) inside the 128-byte swizzled row
                    umma_f16(acc_t, smem_desc(st + k * 32), smem_desc(st + A_BYTES + k * 32), idesc,
                             (kb > 0 || k > 0) ? 1u : 0u);
                }
                umma_commit(&sm->empty[s]);
            }
            umma_commit(&sm->acc_full[b]);
        }
        // no MMA of this CTA may still write tensor memory when it is freed
        drain_mma(&sm->drain, err);
    } else if (CVT && warp == 0) {
        // ---------------- control of the FP32-target variant (one thread): TMA loads, L2
        // prefetches and MMA issue in one loop over this CTA's stages g = (tile, k block).
        // Stage g + STAGES - 1 is loaded right after the MMAs of stage g are issued (its
        // buffer is the one stage g - 1 used, released once those MMAs, issued one step
        // earlier, complete); the points of stage g + PF are prefetched into L2 so that the
        // loads find them there.
        if (lane == 0) {
            constexpr int PF = 8;
            int ntile = 0;
            for (int t = unit; t < tiles; t += nunits) ++ntile;
            const int total = ntile * kblocks;
            int issued = 0;
            auto issue = [&](int gg) {
                ++issued;
                const int tile = unit + (gg / kblocks) * nunits, kb = gg % kblocks, s = gg % STAGES;
                const int r0 = row_of(tile), c0 = col_of(tile);
                unsigned char* st = base + s * STAGE_BYTES;
                uint64_t* tb = &sm->raw_full[s];
                mbar_expect_tx(tb, STAGE_BYTES);
                // the two 32-column halves of the FP32 targets, and the directions
                tma_load_2d(st, &map_a, tb, kb * BK, r0);
                tma_load_2d(st + BM * 128, &map_a, tb, kb * BK + 32, r0);
                tma_load_2d(st + A_BYTES, &map_b, tb, kb * BK, c0);
            };
            auto prefetch = [&](int gg) {
                const int tile = unit + (gg / kblocks) * nunits, kb = gg % kblocks;
                tma_prefetch_2d(&map_a, kb * BK, row_of(tile));
                tma_prefetch_2d(&map_a, kb * BK + 32, row_of(tile));
            };
            const uint32_t idesc = instr_desc(1u, BM, BN);
            for (int gg = 0; gg < total && gg < PF; ++gg) prefetch(gg);
            for (int gg = 0; gg < total && gg < STAGES - 1; ++gg) issue(gg);
            bool ok = true;
            for (int g = 0; g < total; ++g) {
                const int kb = g % kblocks, local = g / kblocks, b = local & 1, s = g % STAGES;
                if (kb == 0 && local >= 2 && !mbar_wait(&sm->acc_empty[b], ((local >> 1) - 1) & 1)) {
                    atomicOr(err, 16u);
                    ok = false;
                    break;
                }
                if (!mbar_wait(&sm->full[s], (g / STAGES) & 1)) {
                    atomicOr(err, 16u);
                    ok = false;
                    break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                unsigned char* st = base + s * STAGE_BYTES;
#pragma unroll
                for (int k = 0; k < BK / 16; ++k)
                    umma_f16(tmem + b * BN, smem_desc(st + k * 32), smem_desc(st + A_BYTES + k * 32), idesc,
                             (kb > 0 || k > 0) ? 1u : 0u);
                umma_commit(&sm->empty[s]);
                if (kb == kblocks - 1) umma_commit(&sm->acc_full[b]);
                const int gn = g + STAGES - 1;
                if (gn < total) {
                    if (gn >= STAGES && !mbar_wait(&sm->empty[gn % STAGES], ((gn / STAGES) - 1) & 1)) {
                        atomicOr(err, 8u);
                        ok = false;
                        break;
                    }
                    issue(gn);
                }
                if (g + PF < total) prefetch(g + PF);
            }
            (void)ok;
            // before exit: the TMA bytes of every issued stage have landed and no MMA still
            // writes tensor memory (immediate on the normal path, bounded after an error)
            drain_fills(sm->raw_full, STAGES, issued);
            drain_mma(&sm->drain, err);
        }
    } else if (CVT && warp <= 3) {
        // ---------------- converters (warps 1-3): FP32 targets -> centred BF16 operand, in place
        // Lane l takes columns 4j..4j+3 (j = l % 16) of one row of a pair (l / 16): it reads
        // them from the first (j < 8) or second 32-column half and writes their BF16 values,
        // x - mu rounded to nearest (the same arithmetic as the separate centring cast), to
        // the row's 128-byte line with the 128-byte swizzle (16-byte chunk c at c ^ (row % 8)).
        // A row's BF16 line is its own line of the first half, so each row is converted by
        // one warp: all of a batch's loads precede its stores (__syncwarp), and rows beyond
        // the targets are written as zeros.  Batches of 16 rows go round the three warps.
        constexpr int HALF = BM * 128, NB = BM / 16;
        const int j = lane & 15, rr = lane >> 4, cw = warp - 1;
        const int npts = n;
        int g = 0;
        bool ok = true;
        for (int tile = unit; tile < tiles && ok; tile += nunits) {
            const int p0 = row_of(tile);
            for (int kb = 0; kb < kblocks; ++kb, ++g) {
                const int s = g % STAGES;
                // every lane waits (and so observes the TMA bytes); the vote keeps the warp together
                const bool got = mbar_wait(&sm->raw_full[s], (g / STAGES) & 1);
                if (!__all_sync(0xffffffffu, got)) {
                    if (lane == 0) atomicOr(err, 8u);
                    ok = false;
                    break;
                }
                unsigned char* cv = base + s * STAGE_BYTES;
                const unsigned char* src = cv + (j >> 3) * HALF + (j & 7) * 16;
                float m[4];
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    const int k = kb * BK + 4 * j + e;
                    m[e] = k < d ? __ldg(ce.mu + k) : 0.0f;
                }
                for (int bi = cw; bi < NB; bi += 3) {
                    const int r0 = bi * 16;
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
                        if (p0 + r >= npts) pk.u2 = make_uint2(0u, 0u);
                        *reinterpret_cast<uint2*>(cv + r * 128 + (((j >> 1) ^ (r & 7)) << 4) + ((j & 1) << 3)) = pk.u2;
                    }
                }
                // generic-proxy writes, read next by the tensor core (async proxy)
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                mbar_arrive(&sm->full[s]);
            }
        }
    } else if (warp >= 4 && EPI == EPI_MOM) {
        // ---------------- fused source side: moments of one slice per thread
        const int q4 = warp & 3, half = (warp - 4) >> 2;  // TMEM lane quarter (slices), column half (points)
        const uint32_t lane_off = static_cast<uint32_t>(q4 * 32) << 16;
        const int slice = row_of(0) + q4 * 32 + lane;
        float mx = 0.0f;
        bool ok = true;
        auto run = [&](auto qp_tag) {
            constexpr int QP = decltype(qp_tag)::value;
            float hi[QP], lo[QP];
#pragma unroll
            for (int k = 0; k < QP; ++k) hi[k] = lo[k] = 0.0f;
            int local = 0;
            for (int tile = unit; tile < tiles; tile += nunits, ++local) {
                const int b = local & 1;
                if (!mbar_wait(&sm->acc_full[b], (local >> 1) & 1)) {
                    atomicOr(err, 32u);
                    ok = false;
                    break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                float t[QP];
#pragma unroll
                for (int k = 0; k < QP; ++k) t[k] = 0.0f;
                for (int cc = 0; cc < BN / 2; cc += 32) {
                    float v[32];
                    tmem_ld32(tmem + lane_off + b * BN + half * (BN / 2) + cc, v);
                    const int pt0 = col_of(tile) + half * (BN / 2) + cc;
                    const float wl = pt0 + lane < ce.npts ? __ldg(ce.w + pt0 + lane) : 0.0f;
                    mom_chunk<QP>(v, wl, ce.inv_R, ce.npts - pt0, t, mx);
                }
                asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
                __syncwarp();
                if (lane == 0) mbar_arrive(&sm->acc_empty[b]);
                // a tile's FP32 sums (128 points) into the running double-float moments
#pragma unroll
                for (int k = 0; k < QP; ++k) two_sum_into(hi[k], lo[k], t[k]);
            }
            if (mom_chunk_id >= 0 && slice < n) {
                double* out = ce.mom + (static_cast<int64_t>(mom_chunk_id * 2 + half) * n + slice) * QP;
#pragma unroll
                for (int k = 0; k < QP; ++k) out[k] = static_cast<double>(hi[k]) + static_cast<double>(lo[k]);
            }
        };
        if (ce.q == 8) run(std::integral_constant<int, 8>{});
        else if (ce.q == 10) run(std::integral_constant<int, 10>{});
        else if (ce.q == 12) run(std::integral_constant<int, 12>{});
        else run(std::integral_constant<int, 16>{});
        if (slice >= n) mx = 0.0f;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        if (lane == 0 && absmax) atomicMax(reinterpret_cast<unsigned int*>(absmax), __float_as_uint(mx));
        (void)ok;
    } else if (warp >= 4 && EPI == EPI_CHEB) {
        // ---------------- fused target side: t_p(z) per (row, slice), row sums per tile
        const int q4 = warp & 3, half = (warp - 4) >> 2;  // TMEM lane quarter, column half
        const uint32_t lane_off = static_cast<uint32_t>(q4 * 32) << 16;
        const int qn = ce.q;
        bool bad = false;
        int local = 0;
        for (int tile = unit; tile < tiles; tile += nunits, ++local) {
            const int b = local & 1;
            const int ct = tile % col_tiles;
            const int row = row_of(tile) + q4 * 32 + lane, col0 = ct * BN + half * (BN / 2);
            if (!mbar_wait(&sm->acc_full[b], (local >> 1) & 1)) {
                atomicOr(err, 32u);
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            float s = 0.0f, c = 0.0f;  // Kahan
            for (int cc = 0; cc < BN / 2; cc += 8) {
                float v[8];
                tmem_ld8(tmem + lane_off + b * BN + half * (BN / 2) + cc, v);
                const float* bt = sbeta + col0 + cc;
                if (qn == 12) {
                    if (ce.horner) cheb_chunk<12, true>(v, bt, ppad, ce.R, ce.inv_R, s, c, bad);
                    else cheb_chunk<12, false>(v, bt, ppad, ce.R, ce.inv_R, s, c, bad);
                } else if (qn == 10) {
                    if (ce.horner) cheb_chunk<10, true>(v, bt, ppad, ce.R, ce.inv_R, s, c, bad);
                    else cheb_chunk<10, false>(v, bt, ppad, ce.R, ce.inv_R, s, c, bad);
                } else if (qn == 8) {
                    if (ce.horner) cheb_chunk<8, true>(v, bt, ppad, ce.R, ce.inv_R, s, c, bad);
                    else cheb_chunk<8, false>(v, bt, ppad, ce.R, ce.inv_R, s, c, bad);
                } else {
                    if (ce.horner) cheb_chunk<16, true>(v, bt, ppad, ce.R, ce.inv_R, s, c, bad);
                    else cheb_chunk<16, false>(v, bt, ppad, ce.R, ce.inv_R, s, c, bad);
                }
            }
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            __syncwarp();
            if (lane == 0) mbar_arrive(&sm->acc_empty[b]);
            if (row < n) ce.part[static_cast<int64_t>(ct * 2 + half) * ce.ldp + row] = static_cast<double>(s) - static_cast<double>(c);
        }
        if (bad) atomicOr(err, 4u);
    } else if (warp >= 4 && warp < 8) {
        // ---------------- epilogue: TMEM -> registers -> Z (slice-major)
        const int q = warp - 4;  // TMEM lane quarter
        const uint32_t lane_off = static_cast<uint32_t>(q * 32) << 16;
        float mx = 0.0f;
        int local = 0;
        for (int tile = unit; tile < tiles; tile += nunits, ++local) {
            const int b = local & 1;
            const int row = row_of(tile) + q * 32 + lane, col0 = col_of(tile);
            if (!mbar_wait(&sm->acc_full[b], (local >> 1) & 1)) {
                atomicOr(err, 32u);
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const float rsc = ROWMAJOR && row < n ? scale * (rs ? rs[row] : 1.0f) : 1.0f;
            for (int c = 0; c < BN; c += 32) {
                float v[32];
                tmem_ld32(tmem + lane_off + b * BN + c, v);
                if (row < n) {
                    if constexpr (ROWMAJOR) {
                        float* out = Z + static_cast<int64_t>(row) * ldz + col0 + c;
                        if (col0 + c + 32 <= P && (ldz % 4) == 0) {
#pragma unroll
                            for (int j = 0; j < 32; j += 4)
                                *reinterpret_cast<float4*>(out + j) =
                                    make_float4(v[j] * rsc, v[j + 1] * rsc, v[j + 2] * rsc, v[j + 3] * rsc);
                        } else {
#pragma unroll
                            for (int j = 0; j < 32; ++j)
                                if (col0 + c + j < P) out[j] = v[j] * rsc;
                        }
                    } else {
#pragma unroll
                        for (int j = 0; j < 32; ++j) {
                            const int p = col0 + c + j;
                            if (p < P) {
                                Z[static_cast<int64_t>(p) * ldz + row] = v[j];
                                mx = fmaxf(mx, fabsf(v[j]));
                            }
                        }
                    }
                }
            }
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            __syncwarp();
            if (lane == 0) mbar_arrive(&sm->acc_empty[b]);
        }
        if (absmax) {
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
            if (lane == 0) atomicMax(reinterpret_cast<unsigned int*>(absmax), __float_as_uint(mx));
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 2) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS) : "memory");
    }
}

// FP16 hi/lo split with promotion.  The tensor core's FP32 accumulation
// rounds toward zero inside each MMA, so every partial sum it forms is biased
// towards zero by about 2^-24 of itself; summed over K these biases add up to
// a systematic relative error (about the number of chained MMA steps x 2^-24)
// that slicing does not average out.  Here every 16-wide K step goes to a fresh
// accumulator (four TMEM buffers in rotation): the two correction products
// a_hi b_lo' + a_lo' b_hi first (2^11-scaled low parts), then the dominant
// product a_hi b_hi with the accumulator scaled by 2^-11 on input (the MMA's
// input-D scale), so the buffer holds the whole step's contribution after one
// rounding of a 16-term group.  The epilogue warps add each buffer into FP32
// registers with round-to-nearest.
// Tile: 128 points x 128 slices; TMEM columns: D[0..3] at 0, 128, 256, 384.
// Warps: 0 TMA, 1 MMA, 2 TMEM allocation, 4-11 epilogue (warp 4 + q + 4 h owns
// TMEM lanes 32q..32q+31 and columns 64h..64h+63).
constexpr int X3_BN = 128;
constexpr int X3_STAGES = 3;
constexpr int X3_BUF = 4;
constexpr int X3_THREADS = 384;

struct SmemX3 {
    uint64_t full[X3_STAGES];
    uint64_t empty[X3_STAGES];
    uint64_t d1_full[X3_BUF];
    uint64_t d1_empty[X3_BUF];
    uint64_t drain;
    uint32_t tmem_base;
};

__global__ void __launch_bounds__(X3_THREADS, 1)
    k_umma_project_x3(const __grid_constant__ CUtensorMap map_a, const __grid_constant__ CUtensorMap map_b,
                      const __grid_constant__ CUtensorMap map_a2, const __grid_constant__ CUtensorMap map_b2, int n,
                      int P, int d, int col_tiles, int tiles, float* __restrict__ Z, int64_t ldz,
                      float* __restrict__ absmax, unsigned* __restrict__ err) {
    extern __shared__ unsigned char smem_raw[];
    // 1024-byte aligned start, derived from the shared array itself so that every access
    // through it compiles to a shared-memory instruction
    unsigned char* base = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
    constexpr int A_BYTES = BM * BK * 2, B_BYTES = X3_BN * BK * 2;
    constexpr int STAGE_BYTES = 2 * (A_BYTES + B_BYTES);
    SmemX3* sm = reinterpret_cast<SmemX3*>(base + X3_STAGES * STAGE_BYTES);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int kblocks = (d + BK - 1) / BK;
    const int ksteps = kblocks * (BK / 16);
    // persistent: this CTA's tiles are blockIdx.x, blockIdx.x + gridDim.x, ...; tile ->
    // (row tile, column tile) with the column tiles of a row tile adjacent
    int ntile = 0;
    for (int tl = static_cast<int>(blockIdx.x); tl < tiles; tl += static_cast<int>(gridDim.x)) ++ntile;
    const int total = ntile * kblocks;
    auto tile_of = [&](int li) { return static_cast<int>(blockIdx.x) + li * static_cast<int>(gridDim.x); };
    constexpr uint32_t TMEM_COLS = 512;
    static_assert(X3_BUF * X3_BN <= static_cast<int>(TMEM_COLS), "accumulators exceed tensor memory");

    if (threadIdx.x == 0) {
        for (int s = 0; s < X3_STAGES; ++s) {
            mbar_init(&sm->full[s], 1);
            mbar_init(&sm->empty[s], 1);
        }
        for (int b = 0; b < X3_BUF; ++b) {
            mbar_init(&sm->d1_full[b], 1);
            mbar_init(&sm->d1_empty[b], 8);  // one arrival per epilogue warp
        }
        mbar_init(&sm->drain, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 2) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&sm->tmem_base)),
                     "r"(TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = sm->tmem_base;

    if (warp == 0 && lane == 0) {
        int fills = 0;
        for (int g = 0; g < total; ++g, ++fills) {
            const int s = g % X3_STAGES, kb = g % kblocks, tile = tile_of(g / kblocks);
            const int row0 = (tile / col_tiles) * BM, col0 = (tile % col_tiles) * X3_BN;
            if (g >= X3_STAGES && !mbar_wait(&sm->empty[s], ((g / X3_STAGES) - 1) & 1)) {
                atomicOr(err, 8u);
                break;
            }
            unsigned char* st = base + s * STAGE_BYTES;
            mbar_expect_tx(&sm->full[s], STAGE_BYTES);
            tma_load_2d(st, &map_a, &sm->full[s], kb * BK, row0);
            tma_load_2d(st + A_BYTES, &map_b, &sm->full[s], kb * BK, col0);
            tma_load_2d(st + A_BYTES + B_BYTES, &map_a2, &sm->full[s], kb * BK, row0);
            tma_load_2d(st + 2 * A_BYTES + B_BYTES, &map_b2, &sm->full[s], kb * BK, col0);
        }
        drain_fills(sm->full, X3_STAGES, fills);
    } else if (warp == 1 && lane == 0) {
        const uint32_t idesc = instr_desc(0u, BM, X3_BN);
        bool ok = true;
        for (int g = 0; g < total && ok; ++g) {
            const int s = g % X3_STAGES;
            if (!mbar_wait(&sm->full[s], (g / X3_STAGES) & 1)) {
                atomicOr(err, 16u);
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            unsigned char* st = base + s * STAGE_BYTES;
            for (int k = 0; k < BK / 16; ++k) {
                const int t = g * (BK / 16) + k;  // K step, counted over this CTA's tiles
                const int b = t % X3_BUF;
                if (t >= X3_BUF && !mbar_wait(&sm->d1_empty[b], ((t / X3_BUF) - 1) & 1)) {
                    atomicOr(err, 16u);
                    ok = false;
                    break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const uint64_t ah = smem_desc(st + k * 32), bh = smem_desc(st + A_BYTES + k * 32);
                const uint64_t al = smem_desc(st + A_BYTES + B_BYTES + k * 32);
                const uint64_t bl = smem_desc(st + 2 * A_BYTES + B_BYTES + k * 32);
                const uint32_t dt = tmem + b * X3_BN;
                umma_f16(dt, ah, bl, idesc, 0u);
                umma_f16(dt, al, bh, idesc, 1u);
                umma_f16_scale_d<11>(dt, ah, bh, idesc);
                umma_commit(&sm->d1_full[b]);
            }
            umma_commit(&sm->empty[s]);
        }
        drain_mma(&sm->drain, err);
    } else if (warp >= 4) {
        const int q = warp & 3, h = (warp - 4) >> 2;
        const uint32_t lane_off = static_cast<uint32_t>(q * 32) << 16;
        const int cbase = h * 64;
        float mx = 0.0f;
        bool ok = true;
        int t = 0;  // K step, counted over this CTA's tiles
        for (int li = 0; li < ntile && ok; ++li) {
            const int tile = tile_of(li);
            const int row = (tile / col_tiles) * BM + q * 32 + lane, col0 = (tile % col_tiles) * X3_BN;
            float acc[64];
#pragma unroll
            for (int j = 0; j < 64; ++j) acc[j] = 0.0f;
            for (int k = 0; k < ksteps; ++k, ++t) {
                const int b = t % X3_BUF;
                if (!mbar_wait(&sm->d1_full[b], (t / X3_BUF) & 1)) {
                    atomicOr(err, 32u);
                    ok = false;
                    break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                uint32_t v0[32], v1[32];
                tmem_ld32_issue(tmem + lane_off + b * X3_BN + cbase, v0);
                tmem_ld32_issue(tmem + lane_off + b * X3_BN + cbase + 32, v1);
                tmem_wait32(v0);
                tmem_wait32(v1);
                asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
                __syncwarp();
                if (lane == 0) mbar_arrive(&sm->d1_empty[b]);
#pragma unroll
                for (int j = 0; j < 32; ++j) {
                    acc[j] = __fadd_rn(acc[j], __uint_as_float(v0[j]));
                    acc[32 + j] = __fadd_rn(acc[32 + j], __uint_as_float(v1[j]));
                }
            }
            if (ok && row < n) {
#pragma unroll
                for (int j = 0; j < 64; ++j) {
                    const int p = col0 + cbase + j;
                    if (p < P) {
                        Z[static_cast<int64_t>(p) * ldz + row] = acc[j];
                        mx = fmaxf(mx, fabsf(acc[j]));
                    }
                }
            }
        }
        if (absmax) {
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
            if (lane == 0) atomicMax(reinterpret_cast<unsigned int*>(absmax), __float_as_uint(mx));
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 2) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS) : "memory");
    }
}

size_t x3_smem_bytes() {
    constexpr int A_BYTES = BM * BK * 2, B_BYTES = X3_BN * BK * 2;
    return 1024 + X3_STAGES * 2 * (A_BYTES + B_BYTES) + sizeof(SmemX3);
}

// centre and convert: out[i][k] = (16-bit)(x[i][k] - mu[k]) for k < d, 0 for d <= k < ldo;
// SPLIT also writes the scaled low part 2^11 (x - mu - hi) into out_lo.  One thread
// converts 8 consecutive elements of a row (one 16-byte store per output), four such
// groups per step with their loads issued together, so that a small grid (one sharing
// the SMs with the projection) still keeps enough reads in flight.

template <class Half, int SPLIT>
__global__ void __launch_bounds__(256) k_center_cast(const float* __restrict__ x, int64_t n, int d, int64_t ldx,
                                                     const float* __restrict__ mu, Half* __restrict__ out,
                                                     Half* __restrict__ out_lo, int ldo, int vec_ok) {
    constexpr int U = 4;
    const int chunks = ldo / 8;
    const int64_t total = n * static_cast<int64_t>(chunks);
    const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
    for (int64_t e0 = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; e0 < total; e0 += U * stride) {
        float v[U][8];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int64_t e = e0 + u * stride;
            const int64_t i = e / chunks;
            const int k0 = static_cast<int>(e - i * chunks) * 8;
            const float* row = x + i * ldx + k0;
            if (e < total && vec_ok && k0 + 8 <= d) {
                const float4 a = __ldg(reinterpret_cast<const float4*>(row));
                const float4 b = __ldg(reinterpret_cast<const float4*>(row + 4));
                v[u][0] = a.x; v[u][1] = a.y; v[u][2] = a.z; v[u][3] = a.w;
                v[u][4] = b.x; v[u][5] = b.y; v[u][6] = b.z; v[u][7] = b.w;
            } else {
#pragma unroll
                for (int j = 0; j < 8; ++j) v[u][j] = e < total && k0 + j < d ? row[j] : 0.0f;
            }
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int64_t e = e0 + u * stride;
            if (e >= total) break;
            const int64_t i = e / chunks;
            const int k0 = static_cast<int>(e - i * chunks) * 8;
            union { Half h[8]; uint4 u4; } hi, lo;
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const float c = k0 + j < d ? v[u][j] - (mu ? __ldg(mu + k0 + j) : 0.0f) : 0.0f;
                hi.h[j] = to_half<Half>(c);
                if constexpr (SPLIT != 0) lo.h[j] = __float2half_rn((c - static_cast<float>(hi.h[j])) * 2048.0f);
            }
            *reinterpret_cast<uint4*>(out + i * ldo + k0) = hi.u4;
            if constexpr (SPLIT != 0) *reinterpret_cast<uint4*>(out_lo + i * ldo + k0) = lo.u4;
        }
    }
}

PFN_cuTensorMapEncodeTiled_v12000 get_encode() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        SLK_CHECK_CUDA(cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q));
        if (q != cudaDriverEntryPointSuccess || !p) fail(SLK_ERR_CUDA, "cuTensorMapEncodeTiled is unavailable");
        fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    }
    return fn;
}

// 2-D tensor map over a row-major [rows][ld] 16-bit matrix, box = 64 x box_rows, 128B swizzle
CUtensorMap make_map(const void* ptr, CUtensorMapDataType dt, int64_t rows, int cols, int64_t ld, int box_rows) {
    CUtensorMap m;
    cuuint64_t gdim[2] = {static_cast<cuuint64_t>(cols), static_cast<cuuint64_t>(rows)};
    cuuint64_t gstride[1] = {static_cast<cuuint64_t>(ld * 2)};
    cuuint32_t box[2] = {static_cast<cuuint32_t>(BK), static_cast<cuuint32_t>(box_rows)};
    cuuint32_t estride[2] = {1, 1};
    CUresult r = get_encode()(&m, dt, 2, const_cast<void*>(ptr), gdim, gstride, box, estride,
                              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                              CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) fail(SLK_ERR_CUDA, "cuTensorMapEncodeTiled failed (%d)", static_cast<int>(r));
    return m;
}

// 2-D tensor map over row-major [rows][ld] FP32 points, box = 32 columns (128 bytes) x
// box_rows, no swizzle: the FP32 input of the converting projection (two boxes per
// 64-column stage); columns >= cols and rows >= rows read as zeros.
CUtensorMap make_map_f32(const float* ptr, int64_t rows, int cols, int64_t ld, int box_rows) {
    CUtensorMap m;
    cuuint64_t gdim[2] = {static_cast<cuuint64_t>(cols), static_cast<cuuint64_t>(rows)};
    cuuint64_t gstride[1] = {static_cast<cuuint64_t>(ld * 4)};
    cuuint32_t box[2] = {32u, static_cast<cuuint32_t>(box_rows)};
    cuuint32_t estride[2] = {1, 1};
    CUresult r = get_encode()(&m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float*>(ptr), gdim, gstride, box,
                              estride, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                              CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) fail(SLK_ERR_CUDA, "cuTensorMapEncodeTiled (FP32) failed (%d)", static_cast<int>(r));
    return m;
}

template <bool CVT>
size_t umma_smem_bytes(size_t extra = 0) {
    using G = Geo<CVT>;
    return 1024 + static_cast<size_t>(G::STAGES) * G::STAGE_BYTES + ((sizeof(Smem) + 15) & ~size_t(15)) + extra;
}
// room for beta (padded P x q floats) in the fused kernel; kept a few KB under the SM's
// capacity so that small kernels of another stream can share the SM
constexpr size_t kChebSmem = 28 * 1024;

template <int EPI, bool CVT>
size_t epi_smem() {
    return umma_smem_bytes<CVT>(EPI == EPI_CHEB ? kChebSmem : 0);
}
template <int EPI>
constexpr int epi_threads() {
    return EPI == EPI_CHEB || EPI == EPI_MOM ? 384 : THREADS;
}

// Co-resident CTAs of the persistent kernel on the current device (one per SM); sets the
// kernel's shared-memory limit once.
template <int EPI, bool CVT = false>
int persistent_units() {
    static int units[128] = {};
    int dev = 0;
    SLK_CHECK_CUDA(cudaGetDevice(&dev));
    SLK_REQUIRE(dev >= 0 && dev < 128, "device index out of range");
    if (!units[dev]) {
        SLK_CHECK_CUDA(cudaFuncSetAttribute(k_umma_project<EPI, CVT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                            static_cast<int>(epi_smem<EPI, CVT>())));
        int sms = 0;
        SLK_CHECK_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
        units[dev] = sms;
    }
    return units[dev];
}

// Launch the persistent projection over n rows (A) and col_tiles 256-wide column tiles (B).
template <int EPI, bool CVT = false>
void launch_persistent(const CUtensorMap& ma, const CUtensorMap& mb, int64_t n, int P, int d, int col_tiles, float* Z,
                       int64_t ldz, float* absmax, unsigned* err, const float* rs, float scale, const ChebEpi& ce,
                       cudaStream_t st) {
    const int64_t items = ceil_div(n, BM) * col_tiles;
    SLK_REQUIRE(items < (int64_t(1) << 31) && n < (int64_t(1) << 31), "too many points for one projection");
    const int64_t units = persistent_units<EPI, CVT>();
    const int64_t grid = items < units ? items : units;
    k_umma_project<EPI, CVT><<<static_cast<unsigned>(grid), epi_threads<EPI>(), epi_smem<EPI, CVT>(), st>>>(
        ma, mb, static_cast<int>(n), P, d, col_tiles, static_cast<int>(items), Z, ldz, absmax, err, rs, scale, ce);
    SLK_CHECK_LAUNCH();
}

int sm_count_dev() {
    static int sms[128] = {};
    int dev = 0;
    SLK_CHECK_CUDA(cudaGetDevice(&dev));
    SLK_REQUIRE(dev >= 0 && dev < 128, "device index out of range");
    if (!sms[dev]) SLK_CHECK_CUDA(cudaDeviceGetAttribute(&sms[dev], cudaDevAttrMultiProcessorCount, dev));
    return sms[dev];
}

template <class Half>
__global__ void k_transpose_cast(const float* __restrict__ src, int rows, int cols, Half* __restrict__ dst, int ldd) {
    // dst[c][r] = src[r][c] for r < rows, 0 for rows <= r < ldd
    for (int64_t e = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; e < static_cast<int64_t>(cols) * ldd;
         e += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const int c = static_cast<int>(e / ldd), r = static_cast<int>(e % ldd);
        dst[e] = to_half<Half>(r < rows ? src[static_cast<int64_t>(r) * cols + c] : 0.0f);
    }
}

// g16[m][p] = BF16(G[p * ldG + m]) through a 32 x 32 shared tile (reads coalesced along m,
// writes along p), zero for P <= p < ldo
__global__ void __launch_bounds__(256) k_derivs_bf16(const float* __restrict__ G, int P, int64_t M, int64_t ldG,
                                                     __nv_bfloat16* __restrict__ g16, int ldo) {
    __shared__ float tile[32][33];
    const int64_t m0 = static_cast<int64_t>(blockIdx.x) * 32;
    const int p0 = static_cast<int>(blockIdx.y) * 32;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
#pragma unroll
    for (int j = 0; j < 32; j += 8) {
        const int p = p0 + ty + j;
        const int64_t m = m0 + tx;
        tile[ty + j][tx] = (p < P && m < M) ? G[static_cast<int64_t>(p) * ldG + m] : 0.0f;
    }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < 32; j += 8) {
        const int64_t m = m0 + ty + j;
        const int p = p0 + tx;
        if (m < M && p < ldo) g16[m * ldo + p] = __float2bfloat16_rn(tile[tx][ty + j]);
    }
}

}  // namespace

int64_t umma_operand_ld(int d) { return (d + 7) / 8 * 8; }

CUtensorMap tmap_bf16_sw128(const void* ptr, int64_t rows, int cols, int64_t ld, int box_rows) {
    return make_map(ptr, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, rows, cols, ld, box_rows);
}

CUtensorMap tmap_f32_rows(const float* ptr, int64_t rows, int cols, int64_t ld, int box_rows) {
    return make_map_f32(ptr, rows, cols, ld, box_rows);
}

void launch_transpose_bf16(const float* src, int rows, int cols, void* dst, cudaStream_t st) {
    const int ldd = static_cast<int>(umma_operand_ld(rows));
    const int64_t total = static_cast<int64_t>(cols) * ldd;
    SLK_TIMED("transpose_cast", st);
    k_transpose_cast<__nv_bfloat16><<<static_cast<unsigned>(ceil_div(total, 256) < 4096 ? ceil_div(total, 256) : 4096),
                                      256, 0, st>>>(src, rows, cols, static_cast<__nv_bfloat16*>(dst), ldd);
    SLK_CHECK_LAUNCH();
}

void launch_derivs_bf16(const float* G, int P, int64_t M, int64_t ldG, void* g16, cudaStream_t st) {
    if (M <= 0) return;
    const int ldo = static_cast<int>(umma_operand_ld(P));
    dim3 grid(static_cast<unsigned>(ceil_div(M, 32)), static_cast<unsigned>(ceil_div(ldo, 32)));
    SLK_REQUIRE(grid.y <= 65535 && ceil_div(M, 32) <= 2147483647, "derivative matrix too large for one cast");
    {
        SLK_TIMED("derivs_bf16", st);
        k_derivs_bf16<<<grid, 256, 0, st>>>(G, P, M, ldG, static_cast<__nv_bfloat16*>(g16), ldo);
    }
    SLK_CHECK_LAUNCH();
}

int64_t umma_cheb_parts(int P) { return 2 * ceil_div(P, BN); }

bool umma_cheb_fits(int P, int q) {
    return (q == 8 || q == 10 || q == 12 || q == 16) &&
           static_cast<size_t>(ceil_div(P, BN) * BN) * q * sizeof(float) <= kChebSmem;
}

void launch_umma_cheb_target(const void* xa, int64_t n, const void* xib, int P, int d, const float* coef, int q,
                             int horner, double R, double* part, int64_t ldp, unsigned* err, cudaStream_t st) {
    if (n <= 0) return;
    SLK_REQUIRE(umma_cheb_fits(P, q), "Chebyshev coefficients do not fit the fused kernel");
    const int64_t ld = umma_operand_ld(d);
    CUtensorMap ma = make_map(xa, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, n, d, ld, BM);
    CUtensorMap mb = make_map(xib, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, P, d, ld, BN);
    const int col_tiles = static_cast<int>(ceil_div(P, BN));
    ChebEpi ce{coef, q, horner, static_cast<float>(1.0 / R), static_cast<float>(R), part, ldp};
    SLK_TIMED("umma_cheb_target", st);
    launch_persistent<EPI_CHEB>(ma, mb, n, P, d, col_tiles, nullptr, 0, nullptr, err, nullptr, 1.0f, ce,
                                              st);
}

bool umma_f32_operand_ok(const float* x, int64_t ld) {
    return reinterpret_cast<uintptr_t>(x) % 16 == 0 && ld % 4 == 0;
}

void launch_umma_cheb_target_f32(const float* y, int64_t ldy, const float* mu, int64_t n, const void* xib, int P, int d,
                                 const float* coef, int q, int horner, double R, double* part, int64_t ldp,
                                 unsigned* err, cudaStream_t st) {
    if (n <= 0) return;
    SLK_REQUIRE(umma_cheb_fits(P, q), "Chebyshev coefficients do not fit the fused kernel");
    SLK_REQUIRE(umma_f32_operand_ok(y, ldy), "FP32 targets need 16-byte aligned rows");
    const int64_t ld = umma_operand_ld(d);
    CUtensorMap ma = make_map_f32(y, n, d, ldy, BM);
    CUtensorMap mb = make_map(xib, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, P, d, ld, BN);
    const int col_tiles = static_cast<int>(ceil_div(P, BN));
    ChebEpi ce{coef, q, horner, static_cast<float>(1.0 / R), static_cast<float>(R), part, ldp};
    ce.mu = mu;
    SLK_TIMED("umma_cheb_target", st);
    launch_persistent<EPI_CHEB, true>(ma, mb, n, P, d, col_tiles, nullptr, 0, nullptr, err, nullptr,
                                                    1.0f, ce, st);
}

bool umma_moments_fit(int q) { return q == 8 || q == 10 || q == 12 || q == 16; }

int64_t umma_moments_chunks(int P) {
    const int groups = static_cast<int>(ceil_div(P, BM));
    const int units = persistent_units<EPI_MOM>();
    SLK_REQUIRE(units >= groups, "too many slices for the fused moments kernel");
    return 2 * static_cast<int64_t>(units / groups);
}

void launch_umma_moments(const void* xa, int64_t n, const void* xib, int P, int d, const float* w, int q, double R,
                         double* mom, float* absmax, unsigned* err, cudaStream_t st) {
    SLK_REQUIRE(umma_moments_fit(q), "Chebyshev term count unsupported by the fused moments kernel");
    SLK_REQUIRE(n < (int64_t(1) << 31), "too many points for one projection");
    const int64_t ld = umma_operand_ld(d);
    // A = directions (slices as rows), B = points (256-point tiles)
    CUtensorMap ma = make_map(xib, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, P, d, ld, BM);
    CUtensorMap mb = make_map(xa, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, n, d, ld, BN);
    const int groups = static_cast<int>(ceil_div(P, BM));
    const int units = persistent_units<EPI_MOM>();
    const int per_group = units / groups;
    const int point_tiles = static_cast<int>(ceil_div(n, BN));
    ChebEpi ce{};
    ce.q = q;
    ce.inv_R = static_cast<float>(1.0 / R);
    ce.R = static_cast<float>(R);
    ce.w = w;
    ce.npts = static_cast<int>(n);
    ce.mom = mom;
    SLK_TIMED("umma_cheb_moments", st);
    // "n" of the kernel is the row count (slices), "P" the column count (points)
    k_umma_project<EPI_MOM, false><<<static_cast<unsigned>(per_group * groups), epi_threads<EPI_MOM>(),
                                     epi_smem<EPI_MOM, false>(), st>>>(
        ma, mb, P, static_cast<int>(n), d, point_tiles, point_tiles, static_cast<float*>(nullptr), int64_t(0), absmax,
        err, static_cast<const float*>(nullptr), 1.0f, ce);
    SLK_CHECK_LAUNCH();
}

void launch_grad_umma(const void* g16, int64_t M, int P, const void* xit16, int d, const float* gs, double scale,
                      float* gy, int64_t ldg, unsigned* err, cudaStream_t st) {
    if (M <= 0) return;
    SLK_REQUIRE(M < (int64_t(1) << 31), "too many targets for one backward product");
    const int64_t ld = umma_operand_ld(P);
    CUtensorMap ma = make_map(g16, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, M, P, ld, BM);
    CUtensorMap mb = make_map(xit16, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, d, P, ld, BN);
    const int col_tiles = static_cast<int>(ceil_div(d, BN));
    SLK_TIMED("umma_grad_bf16", st);
    launch_persistent<EPI_ROW>(ma, mb, M, d, P, col_tiles, gy, ldg, nullptr, err, gs, static_cast<float>(scale),
                                  ChebEpi{}, st);
}

int device_sm_count() { return sm_count_dev(); }

void launch_center_cast(const float* x, int64_t n, int d, int64_t ldx, const float* mu, void* out, void* out_lo,
                        int split, cudaStream_t st, const char* label, int max_blocks) {
    if (n <= 0) return;
    const int ldo = static_cast<int>(umma_operand_ld(d));
    const int64_t total = n * (ldo / 8);
    const int64_t cap = max_blocks > 0 ? max_blocks : 8 * sm_count_dev();
    const unsigned blocks = static_cast<unsigned>(ceil_div(total, 256) < cap ? ceil_div(total, 256) : cap);
    const int vec_ok = (ldx % 4 == 0) && (reinterpret_cast<uintptr_t>(x) % 16 == 0);
    SLK_TIMED(label, st);
    if (split)
        k_center_cast<__half, 1><<<blocks, 256, 0, st>>>(x, n, d, ldx, mu, static_cast<__half*>(out),
                                                        static_cast<__half*>(out_lo), ldo, vec_ok);
    else
        k_center_cast<__nv_bfloat16, 0><<<blocks, 256, 0, st>>>(x, n, d, ldx, mu, static_cast<__nv_bfloat16*>(out),
                                                               nullptr, ldo, vec_ok);
    SLK_CHECK_LAUNCH();
}

void launch_project_umma(const void* xa, const void* xa_lo, int64_t n, const void* xib, const void* xib_lo, int P,
                         int d, int split, float* Z, int64_t ldz, float* absmax, unsigned* err, cudaStream_t st) {
    if (n <= 0) return;
    SLK_REQUIRE(n < (int64_t(1) << 31), "too many points for one projection");
    const int64_t ld = umma_operand_ld(d);
    const CUtensorMapDataType dt = split ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
    const int bn = split ? X3_BN : BN;
    CUtensorMap ma = make_map(xa, dt, n, d, ld, BM);
    CUtensorMap mb = make_map(xib, dt, P, d, ld, bn);
    CUtensorMap ma2 = split ? make_map(xa_lo, dt, n, d, ld, BM) : ma;
    CUtensorMap mb2 = split ? make_map(xib_lo, dt, P, d, ld, bn) : mb;
    const int col_tiles = static_cast<int>(ceil_div(P, bn));
    const int64_t blocks = ceil_div(n, BM) * col_tiles;
    SLK_REQUIRE(blocks < (int64_t(1) << 31), "too many points");
    dim3 grid(static_cast<unsigned>(blocks));
    if (split && P > X3_BN) {
        // more slices than one 128-column tile: CTA pairs with 256 x 256 tiles (twice the MMA
        // work per byte of operands brought into shared memory)
        launch_pair_project_x3(xa, xa_lo, n, xib, xib_lo, P, d, Z, ldz, absmax, err, st);
        return;
    }
    if (split) {
        static bool attr = false;
        if (!attr) {
            SLK_CHECK_CUDA(cudaFuncSetAttribute(k_umma_project_x3, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                static_cast<int>(x3_smem_bytes())));
            attr = true;
        }
        // persistent: one CTA per SM (shared memory and tensor memory admit one), tiles in turn
        const int sms = sm_count_dev();
        const unsigned cta = static_cast<unsigned>(blocks < sms ? blocks : sms);
        SLK_TIMED("umma_project_x3", st);
        k_umma_project_x3<<<cta, X3_THREADS, x3_smem_bytes(), st>>>(ma, mb, ma2, mb2, static_cast<int>(n), P, d,
                                                                    col_tiles, static_cast<int>(blocks), Z, ldz,
                                                                    absmax, err);
    } else {
        SLK_TIMED("umma_project_bf16", st);
        launch_persistent<EPI_Z>(ma, mb, n, P, d, col_tiles, Z, ldz, absmax, err, nullptr, 1.0f,
                                               ChebEpi{}, st);
    }
    SLK_CHECK_LAUNCH();
}

}  // namespace slk
