// SIMT projection  Z = Xi (X - mu)^T  and the backward product  gy = diag(s) G Xi.
//
// Tiled shared-memory GEMM: a 64 x 64 output tile per 256-thread block, each
// thread owns a 4 x 4 register tile, K staged 16 at a time.  Used for the FP64
// path, the FP32 path and the backward product; the tensor-core projection for
// BF16 / FP16x3 precisions lives in k_tcgen05.cu.
#include "kernels.cuh"

namespace slk {

namespace {

constexpr int BM = 64, BN = 64, BK = 16;

// C(r, c) = sum_q A(r, q) B(c, q)
//   A(r, q) = A[r * sAr + q * sAq],  B(c, q) = B[c * sBc + q * sBq] (- mu[q] if mu)
//   C[r * sCr + c] = acc * scale * (rowscale ? rowscale[r] : 1)
template <class TA, class TB, class TC, class ACC>
__global__ void __launch_bounds__(256) k_gemm_tile(int64_t R, int64_t C, int Q, const TA* __restrict__ A, int64_t sAr,
                                                   int64_t sAq, const TB* __restrict__ B, int64_t sBc, int64_t sBq,
                                                   const TB* __restrict__ mu, TC* __restrict__ Cout, int64_t sCr,
                                                   double scale, const TC* __restrict__ rowscale, int rows_on_x) {
    __shared__ ACC As[BK][BM + 4];
    __shared__ ACC Bs[BK][BN + 4];
    const int tid = threadIdx.x;
    const int tx = tid % 16, ty = tid / 16;
    const int64_t r0 = static_cast<int64_t>(rows_on_x ? blockIdx.x : blockIdx.y) * BM;
    const int64_t c0 = static_cast<int64_t>(rows_on_x ? blockIdx.y : blockIdx.x) * BN;
    ACC acc[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = ACC(0);

    for (int q0 = 0; q0 < Q; q0 += BK) {
        // 1024 elements per tile, 4 per thread.  The fast-varying index follows
        // the unit stride of each operand so that a warp reads contiguous memory.
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            int idx = tid + e * 256;
            int rr, qq;
            if (sAq == 1) { qq = idx % BK; rr = idx / BK; } else { rr = idx % BM; qq = idx / BM; }
            int64_t r = r0 + rr;
            int q = q0 + qq;
            As[qq][rr] = (r < R && q < Q) ? static_cast<ACC>(A[r * sAr + q * sAq]) : ACC(0);
            int cc;
            if (sBq == 1) { qq = idx % BK; cc = idx / BK; } else { cc = idx % BN; qq = idx / BN; }
            int64_t c = c0 + cc;
            q = q0 + qq;
            ACC v = ACC(0);
            if (c < C && q < Q) {
                v = static_cast<ACC>(B[c * sBc + q * sBq]);
                if (mu) v -= static_cast<ACC>(mu[q]);
            }
            Bs[qq][cc] = v;
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < BK; ++k) {
            ACC a[4], b[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                a[i] = As[k][ty * 4 + i];
                b[i] = Bs[k][tx * 4 + i];
            }
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        int64_t r = r0 + ty * 4 + i;
        if (r >= R) continue;
        double rs = scale * (rowscale ? static_cast<double>(rowscale[r]) : 1.0);
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            int64_t c = c0 + tx * 4 + j;
            if (c < C) Cout[r * sCr + c] = static_cast<TC>(static_cast<double>(acc[i][j]) * rs);
        }
    }
}

}  // namespace

template <class T>
void launch_project_simt(const T* xi, int P, const T* x, int64_t n, int d, int64_t ldx, const T* mu, T* Z, int64_t ldz,
                         cudaStream_t st) {
    if (n <= 0) return;
    dim3 grid(static_cast<unsigned>(ceil_div(n, BN)), static_cast<unsigned>(ceil_div(P, BM)));
    SLK_REQUIRE(grid.y <= 65535, "too many slices for one projection launch");
    {
        SLK_TIMED("gemm_tile", st);
        k_gemm_tile<T, T, T, T><<<grid, 256, 0, st>>>(P, n, d, xi, d, 1, x, ldx, 1, mu, Z, ldz, 1.0, nullptr, 0);
    }
    SLK_CHECK_LAUNCH();
}

template <class T>
void launch_grad_gemm(const T* G, int64_t ldG, int64_t M, int P, const T* xi, int d, const T* gs, double scale, T* gy,
                      int64_t ldg, cudaStream_t st) {
    if (M <= 0) return;
    // rows r = targets (A(m, p) = G[p * ldG + m], slice-major), columns c = coordinates
    // (B(c, p) = xi[p][c])
    dim3 grid(static_cast<unsigned>(ceil_div(M, BM)), static_cast<unsigned>(ceil_div(d, BN)));
    SLK_REQUIRE(grid.y <= 65535, "dimension too large for one backward launch");
    {
        SLK_TIMED("gemm_tile", st);
        k_gemm_tile<T, T, T, T><<<grid, 256, 0, st>>>(M, d, P, G, 1, ldG, xi, 1, d, nullptr, gy, ldg, scale, gs, 1);
    }
    SLK_CHECK_LAUNCH();
}

template void launch_project_simt<float>(const float*, int, const float*, int64_t, int, int64_t, const float*, float*,
                                         int64_t, cudaStream_t);
template void launch_project_simt<double>(const double*, int, const double*, int64_t, int, int64_t, const double*,
                                          double*, int64_t, cudaStream_t);
template void launch_grad_gemm<float>(const float*, int64_t, int64_t, int, const float*, int, const float*, double,
                                      float*, int64_t, cudaStream_t);
template void launch_grad_gemm<double>(const double*, int64_t, int64_t, int, const double*, int, const double*, double,
                                       double*, int64_t, cudaStream_t);

}  // namespace slk
