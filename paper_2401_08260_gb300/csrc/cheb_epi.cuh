// Epilogue arithmetic of the fused Chebyshev kernels (target-side evaluation of the
// Chebyshev or monomial form per slice, source-side moments per slice), shared by the
// single-CTA and the CTA-pair tensor-core kernels.
#pragma once

#include <cstdint>

namespace slk {
namespace umma {

// Target-side evaluation of one 8-column accumulator chunk (one row per thread): four
// slices at a time, the QP coefficients of the group loaded up front (one broadcast
// LDS.128 per degree from the degree-major table), then Horner's rule on monomial
// coefficients or Clenshaw's recurrence on Chebyshev ones; the 32 values are added to
// (s, c) with Kahan compensation.  Projections outside [-R, R] (or NaN) set bad.
// Chunks of 8 keep the unrolled evaluation within the register budget of 384 threads.
template <int QP, bool HORNER>
__device__ __forceinline__ void cheb_chunk(const float (&v)[8], const float* __restrict__ bt0, int ppad, float R,
                                           float inv_R, float& s, float& c, bool& bad) {
#pragma unroll
    for (int j = 0; j < 8; j += 4) {
        float u[4], b1[4], b2[4];
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            const float z = v[j + r];
            if (!(z <= R && z >= -R)) bad = true;
            u[r] = z * inv_R;
            b1[r] = 0.0f;
            b2[r] = 0.0f;
        }
        // fully unrolled over the degrees: the coefficient loads carry no loop dependence
#pragma unroll
        for (int k = QP - 1; k >= 0; --k) {
            const float4 c4 = *reinterpret_cast<const float4*>(bt0 + j + k * ppad);
            const float cv[4] = {c4.x, c4.y, c4.z, c4.w};
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                if (HORNER) {
                    b1[r] = fmaf(b1[r], u[r], cv[r]);
                } else if (k >= 1) {
                    const float bk = fmaf(u[r] + u[r], b1[r], cv[r] - b2[r]);
                    b2[r] = b1[r];
                    b1[r] = bk;
                } else {
                    b1[r] = fmaf(u[r], b1[r], cv[r] - b2[r]);
                }
            }
        }
        // the group's four values added plainly, the group sum with Kahan compensation
        const float y = ((b1[0] + b1[1]) + (b1[2] + b1[3])) - c;
        const float tt = s + y;
        c = (tt - s) - y;
        s = tt;
    }
}


// Target-side evaluation of one 32-column accumulator chunk (one row per thread, raw
// TMEM words in r): twice 16 independent Horner (monomial coefficients) or Clenshaw
// (Chebyshev coefficients) chains over the degrees, the coefficients of 16 slices read as
// four broadcast LDS.128 per degree from the degree-major table bt0[k * ppad + p]; the
// values are added to (s, c) four at a time, each group sum with Kahan compensation.
// Projections outside [-R, R] (or NaN) set bad.
template <int QP, bool HORNER>
__device__ __forceinline__ void cheb_chunk32(const uint32_t (&r)[32], const float* __restrict__ bt0, int ppad,
                                             float R, float inv_R, float& s, float& c, bool& bad) {
    // two halves of 16 independent chains (the register budget of 384 threads)
    constexpr int W = 16;
#pragma unroll
    for (int h = 0; h < 32; h += W) {
        float u[W], b1[W], b2[HORNER ? 1 : W];
#pragma unroll
        for (int i = 0; i < W; ++i) {
            const float z = __uint_as_float(r[h + i]);
            if (!(z <= R && z >= -R)) bad = true;
            u[i] = z * inv_R;
            b1[i] = 0.0f;
            if (!HORNER) b2[i] = 0.0f;
        }
#pragma unroll
        for (int k = QP - 1; k >= 0; --k) {
#pragma unroll
            for (int g = 0; g < W / 4; ++g) {
                const float4 c4 = *reinterpret_cast<const float4*>(bt0 + h + 4 * g + k * ppad);
                const float cv[4] = {c4.x, c4.y, c4.z, c4.w};
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    const int i = 4 * g + e;
                    if (HORNER) {
                        b1[i] = fmaf(b1[i], u[i], cv[e]);
                    } else if (k >= 1) {
                        const float bk = fmaf(u[i] + u[i], b1[i], cv[e] - b2[i]);
                        b2[i] = b1[i];
                        b1[i] = bk;
                    } else {
                        b1[i] = fmaf(u[i], b1[i], cv[e] - b2[i]);
                    }
                }
            }
        }
#pragma unroll
        for (int g = 0; g < W / 4; ++g) {
            const float y = ((b1[4 * g] + b1[4 * g + 1]) + (b1[4 * g + 2] + b1[4 * g + 3])) - c;
            const float tt = s + y;
            c = (tt - s) - y;
            s = tt;
        }
    }
}

// Moments of one slice over a 32-point accumulator chunk: z[j] for the chunk's points,
// the lane-th point's weight in wl (zero beyond the points); t holds this tile's FP32 sums.
template <int QP>
__device__ __forceinline__ void mom_chunk(const float (&v)[32], float wl, float inv_R, int valid_pts, float (&t)[QP],
                                          float& mx) {
#pragma unroll
    for (int j = 0; j < 32; ++j) {
        const float wj = __shfl_sync(0xffffffffu, wl, j);
        const float z = v[j];
        if (j < valid_pts) mx = fmaxf(mx, fabsf(z));
        const float u = z * inv_R, u2 = u + u;
        float tm1 = 1.0f, tc = u;  // T_0, T_1
        t[0] += wj;
#pragma unroll
        for (int k = 1; k < QP; ++k) {
            t[k] = fmaf(wj, tc, t[k]);
            const float tn = fmaf(u2, tc, -tm1);
            tm1 = tc;
            tc = tn;
        }
    }
}

// Add a float into an unevaluated pair hi + lo without rounding loss (TwoSum).
__device__ __forceinline__ void two_sum_into(float& hi, float& lo, float x) {
    const float s = hi + x, bp = s - hi;
    lo += (hi - (s - bp)) + (x - bp);
    hi = s;
}

}  // namespace umma
}  // namespace slk
