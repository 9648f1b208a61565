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

// Moments of one slice over a 32-point accumulator chunk, two points at a time with packed
// FP32 arithmetic (FFMA2: each half rounds exactly as a scalar fmaf): the even points of
// the chunk go to t[k].x, the odd ones to t[k].y.  Otherwise as mom_chunk.
template <int QP>
__device__ __forceinline__ void mom_chunk2(const float (&v)[32], float wl, float inv_R, int valid_pts,
                                           float2 (&t)[QP], float& mx) {
    if (valid_pts >= 32) {
#pragma unroll
        for (int j = 0; j < 32; ++j) mx = fmaxf(mx, fabsf(v[j]));
    } else {
#pragma unroll
        for (int j = 0; j < 32; ++j)
            if (j < valid_pts) mx = fmaxf(mx, fabsf(v[j]));
    }
    const float2 ir = make_float2(inv_R, inv_R);
#pragma unroll
    for (int j = 0; j < 32; j += 2) {
        const float2 w2 = make_float2(__shfl_sync(0xffffffffu, wl, j), __shfl_sync(0xffffffffu, wl, j + 1));
        const float2 u = __fmul2_rn(make_float2(v[j], v[j + 1]), ir);
        const float2 u2 = __fadd2_rn(u, u);
        float2 tm1 = make_float2(1.0f, 1.0f), tc = u;  // T_0, T_1
        t[0] = __fadd2_rn(t[0], w2);
#pragma unroll
        for (int k = 1; k < QP; ++k) {
            t[k] = __ffma2_rn(w2, tc, t[k]);
            if (k + 1 < QP) {
                const float2 tn = __ffma2_rn(u2, tc, make_float2(-tm1.x, -tm1.y));
                tm1 = tc;
                tc = tn;
            }
        }
    }
}

// Target-side Horner evaluation (monomial coefficients) of one 32-column accumulator chunk,
// two slices at a time with packed FP32 FMAs (each half rounds exactly as the scalar
// fmaf of cheb_chunk32, so for finite projections the values and their Kahan sum are
// the same bits): the coefficients of four slices come as one broadcast LDS.128 per
// degree from the degree-major table bt0[k * ppad + p].  |z| is folded into mabs (the
// caller checks it against R); a NaN projection makes the sum NaN.
template <int QP>
__device__ __forceinline__ void horner_chunk32(const uint32_t (&r)[32], const float* __restrict__ bt0, int ppad,
                                               float inv_R, float& s, float& c, float& mabs) {
    constexpr int W = 16;
    const float2 ir = make_float2(inv_R, inv_R);
#pragma unroll
    for (int h = 0; h < 32; h += W) {
        float2 u[W / 2], b[W / 2];
#pragma unroll
        for (int g = 0; g < W / 4; ++g) {
            const float4 c4 = *reinterpret_cast<const float4*>(bt0 + h + 4 * g + (QP - 1) * ppad);
            b[2 * g] = make_float2(c4.x, c4.y);
            b[2 * g + 1] = make_float2(c4.z, c4.w);
        }
#pragma unroll
        for (int i = 0; i < W / 2; ++i) {
            const float z0 = __uint_as_float(r[h + 2 * i]), z1 = __uint_as_float(r[h + 2 * i + 1]);
            mabs = fmaxf(mabs, fmaxf(fabsf(z0), fabsf(z1)));
            u[i] = __fmul2_rn(make_float2(z0, z1), ir);
        }
#pragma unroll
        for (int k = QP - 2; k >= 0; --k) {
#pragma unroll
            for (int g = 0; g < W / 4; ++g) {
                const float4 c4 = *reinterpret_cast<const float4*>(bt0 + h + 4 * g + k * ppad);
                b[2 * g] = __ffma2_rn(b[2 * g], u[2 * g], make_float2(c4.x, c4.y));
                b[2 * g + 1] = __ffma2_rn(b[2 * g + 1], u[2 * g + 1], make_float2(c4.z, c4.w));
            }
        }
#pragma unroll
        for (int g = 0; g < W / 4; ++g) {
            const float y = ((b[2 * g].x + b[2 * g].y) + (b[2 * g + 1].x + b[2 * g + 1].y)) - c;
            const float tt = s + y;
            c = (tt - s) - y;
            s = tt;
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
