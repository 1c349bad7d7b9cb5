// Dense kernel operator out = K(X, Y) W with K_ij = exp(-s |x_i - y_j|^2)
// and its adjoint (the RBF / Gaussian-process operators of paper Sec. 1 and
// Sec. 1.1; dense global operators, Sec. 2.2.2) on FP32 CUDA cores.
//
// Forward (k_dense_fwd): a CTA owns 128 rows of X and all (<= 64) columns of
// W.  For each chunk of 32 Y points it stages Y and W in shared memory,
// evaluates the 128 x 32 kernel tile once (direct differences, FP32, exp via
// ex2), and then runs a 128 x 64 x 32 register-tiled product with each
// thread holding an 8 x 4 accumulator tile in packed FP32 pairs.  The exponentials are 1/64 of the
// multiply-adds, so the kernel is bound by the FP32 pipe.
//
// Adjoint: dW = K^T G is the forward with the roles of (X, W) and (Y, G)
// swapped (K(X,Y)^T = K(Y,X)); dX (and ds) come from k_dense_gradx, which for
// each 128-row block forms S = G W_chunk^T on CUDA cores, A = S o K, and the
// row reductions sum_j A_ij, sum_j A_ij y_j, sum_j A_ij d_ij^2; dY is the same
// kernel with (X, G) and (Y, W) swapped.
#include <cuda_runtime.h>
#include <stdint.h>

#include "ab_internal.cuh"

namespace ab {

namespace {

constexpr int kBM = 128;      // X rows per CTA
constexpr int kBN = 32;       // Y points per chunk
constexpr int kRHS = 64;      // padded right-hand-side width
constexpr int kDThreads = 256;
constexpr float kLog2eD = 1.4426950408889634f;

__device__ __forceinline__ float ex2f(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// Packed FP32 pairs: fma.rn.f32x2 rounds each half exactly like fmaf.
__device__ __forceinline__ uint64_t f2p(float a, float b) {
    uint64_t r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
    return r;
}
__device__ __forceinline__ void f2u(uint64_t v, float& a, float& b) {
    asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(v));
}
__device__ __forceinline__ uint64_t ffma2(uint64_t a, uint64_t b, uint64_t c) {
    uint64_t d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}

// thread layout for the product: tx in [0,16) -> 4 columns, ty in [0,16) ->
// 8 consecutive rows ty*8 .. ty*8+7 (two float4 shared loads; a warp's two ty
// values read broadcast addresses).  Rows are paired in fma.f32x2 (the K
// values of rows 2r, 2r+1 sit in an aligned register pair of the float4 load;
// the W value is duplicated), 16 packed FMAs a K step instead of 32, with
// the same rounding and order as scalar FMAs (65,536^2 x 64: 17.4 -> 16.0
// ms, outputs bit-identical).  W and Y chunks alternate between two shared
// buffers.
__global__ void __launch_bounds__(kDThreads)
k_dense_fwd(int64_t m, int64_t n, const float4* __restrict__ X,
            const float4* __restrict__ Y, int nrhs, const float* __restrict__ W,
            float ns_log2e, float* __restrict__ out) {
    __shared__ __align__(16) float Ks[kBN][kBM];
    __shared__ __align__(16) float Ws[2][kBN][kRHS];
    __shared__ float4 Ys[2][kBN];
    const int t = threadIdx.x;
    const int tx = t & 15, ty = t >> 4;
    const int64_t row0 = (int64_t)blockIdx.x * kBM;
    // kernel-tile role: row r = t & 127 (its x in registers), 16 Y points
    const int kr = t & (kBM - 1);
    const int kh = t >> 7;  // 0 or 1: which 16 of the 32 Y points
    float4 xi = make_float4(0.f, 0.f, 0.f, 0.f);
    if (row0 + kr < m) xi = __ldg(X + row0 + kr);
    uint64_t acc2[4][4];   // acc2[p][c] = rows (ty*8 + 2p, ty*8 + 2p + 1), column tx*4 + c
#pragma unroll
    for (int p = 0; p < 4; ++p)
#pragma unroll
        for (int c = 0; c < 4; ++c) acc2[p][c] = 0ull;
    // W chunk: 32 x 64 floats, 8 per thread; Y chunk: 32 points
    auto stage = [&](int64_t j0, int b) {
#pragma unroll
        for (int e = 0; e < (kBN * kRHS) / kDThreads; ++e) {
            const int idx = e * kDThreads + t;
            const int jj = idx / kRHS, cc = idx % kRHS;
            Ws[b][jj][cc] = (j0 + jj < n && cc < nrhs) ? __ldg(W + (j0 + jj) * nrhs + cc) : 0.f;
        }
        if (t < kBN) Ys[b][t] = (j0 + t < n) ? __ldg(Y + j0 + t) : make_float4(0.f, 0.f, 0.f, 0.f);
    };
    auto kernel_tile = [&](int64_t j0, int b) {
#pragma unroll 4
        for (int q = 0; q < 16; ++q) {
            const int jj = kh * 16 + q;
            const float4 y = Ys[b][jj];
            const float dx = xi.x - y.x, dy = xi.y - y.y, dz = xi.z - y.z;
            const float d2 = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
            Ks[jj][kr] = (j0 + jj < n) ? ex2f(ns_log2e * d2) : 0.f;
        }
    };
    const int64_t chunks = (n + kBN - 1) / kBN;
    if (chunks > 0) {
        stage(0, 0);
        __syncthreads();
        kernel_tile(0, 0);
        __syncthreads();
    }
    for (int64_t c = 0; c < chunks; ++c) {
        const int b = (int)(c & 1);
#pragma unroll 8
        for (int k = 0; k < kBN; ++k) {
            const float4 a0 = *reinterpret_cast<const float4*>(&Ks[k][ty * 8]);
            const float4 a1 = *reinterpret_cast<const float4*>(&Ks[k][ty * 8 + 4]);
            const float4 w = *reinterpret_cast<const float4*>(&Ws[b][k][tx * 4]);
            const uint64_t A[4] = {f2p(a0.x, a0.y), f2p(a0.z, a0.w), f2p(a1.x, a1.y), f2p(a1.z, a1.w)};
            const uint64_t B[4] = {f2p(w.x, w.x), f2p(w.y, w.y), f2p(w.z, w.z), f2p(w.w, w.w)};
#pragma unroll
            for (int p = 0; p < 4; ++p)
#pragma unroll
                for (int cc = 0; cc < 4; ++cc) acc2[p][cc] = ffma2(A[p], B[cc], acc2[p][cc]);
        }
        __syncthreads();   // Ks and Ws[b] fully read
        if (c + 1 < chunks) {
            stage((c + 1) * kBN, b ^ 1);
            __syncthreads();
            kernel_tile((c + 1) * kBN, b ^ 1);
            __syncthreads();
        }
    }
#pragma unroll
    for (int p = 0; p < 4; ++p) {
#pragma unroll
        for (int cc = 0; cc < 4; ++cc) {
            float v0, v1;
            f2u(acc2[p][cc], v0, v1);
            const int col = tx * 4 + cc;
            const int64_t row = row0 + ty * 8 + 2 * p;
            if (col < nrhs) {
                if (row < m) out[row * nrhs + col] = v0;
                if (row + 1 < m) out[(row + 1) * nrhs + col] = v1;
            }
        }
    }
}

// dX_i = -2 s (x_i sum_j A_ij - sum_j A_ij y_j), A_ij = (G_i . W_j) K_ij,
// ds partial = -sum_ij A_ij d_ij^2 (one FP64 value per CTA).
// Thread layout: row r = t & 127, j-half h = t >> 7 (16 Y points each).
__global__ void __launch_bounds__(kDThreads)
k_dense_gradx(int64_t m, int64_t n, const float4* __restrict__ X,
              const float4* __restrict__ Y, int nrhs, const float* __restrict__ W,
              const float* __restrict__ G, float s, float ns_log2e,
              float4* __restrict__ dX, double* __restrict__ partial) {
    __shared__ __align__(16) float Gs[kBM][kRHS + 4];   // padded rows
    __shared__ __align__(16) float Ws[kBN][kRHS + 4];
    __shared__ float4 Ys[kBN];

    const int t = threadIdx.x;
    const int r = t & (kBM - 1), h = t >> 7;
    const int64_t row0 = (int64_t)blockIdx.x * kBM;
    for (int e = t; e < kBM * kRHS; e += kDThreads) {
        const int rr = e / kRHS, cc = e % kRHS;
        Gs[rr][cc] = (row0 + rr < m && cc < nrhs) ? __ldg(G + (row0 + rr) * nrhs + cc) : 0.f;
    }
    float4 xi = make_float4(0.f, 0.f, 0.f, 0.f);
    if (row0 + r < m) xi = __ldg(X + row0 + r);
    // accumulate A_ij (x_i - y_j) directly: no cancellation between
    // x_i sum_j A_ij and sum_j A_ij y_j
    float sX = 0.f, sY = 0.f, sZ = 0.f, sAd2 = 0.f;

    for (int64_t j0 = 0; j0 < n; j0 += kBN) {
        __syncthreads();
        if (t < kBN) Ys[t] = (j0 + t < n) ? __ldg(Y + j0 + t) : make_float4(0.f, 0.f, 0.f, 0.f);
        for (int e = t; e < kBN * kRHS; e += kDThreads) {
            const int jj = e / kRHS, cc = e % kRHS;
            Ws[jj][cc] = (j0 + jj < n && cc < nrhs) ? __ldg(W + (j0 + jj) * nrhs + cc) : 0.f;
        }
        __syncthreads();
        // S_ij = G_i . W_j for this thread's row and 16 Y points
        float S[16];
#pragma unroll
        for (int q = 0; q < 16; ++q) S[q] = 0.f;
#pragma unroll 4
        for (int c = 0; c < kRHS; c += 4) {
            const float4 gv = *reinterpret_cast<const float4*>(&Gs[r][c]);
#pragma unroll
            for (int q = 0; q < 16; ++q) {
                const float4 wv = *reinterpret_cast<const float4*>(&Ws[h * 16 + q][c]);
                S[q] = fmaf(gv.x, wv.x, fmaf(gv.y, wv.y, fmaf(gv.z, wv.z, fmaf(gv.w, wv.w, S[q]))));
            }
        }
#pragma unroll
        for (int q = 0; q < 16; ++q) {
            const int jj = h * 16 + q;
            if (j0 + jj >= n) continue;
            const float4 y = Ys[jj];
            const float dx = xi.x - y.x, dy = xi.y - y.y, dz = xi.z - y.z;
            const float d2 = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
            const float A = S[q] * ex2f(ns_log2e * d2);
            sX = fmaf(A, dx, sX);
            sY = fmaf(A, dy, sY);
            sZ = fmaf(A, dz, sZ);
            sAd2 = fmaf(A, d2, sAd2);
        }
    }
    __syncthreads();
    // the W chunk buffer is free now: reuse it for the cross-half reduction
    float (*red)[4] = reinterpret_cast<float (*)[4]>(&Ws[0][0]);
    red[t][0] = sX; red[t][1] = sY; red[t][2] = sZ; red[t][3] = sAd2;
    __syncthreads();
    if (h == 0) {
        const float ax = red[t][0] + red[t + kBM][0];
        const float ay = red[t][1] + red[t + kBM][1];
        const float az = red[t][2] + red[t + kBM][2];
        const float ad = red[t][3] + red[t + kBM][3];
        if (row0 + r < m && dX)
            dX[row0 + r] = make_float4(-2.f * s * ax, -2.f * s * ay, -2.f * s * az, 0.f);
        red[t][3] = ad;
    }
    __syncthreads();
    if (t == 0 && partial) {
        double tot = 0.0;
        for (int q = 0; q < kBM; ++q) tot += (double)red[q][3];
        partial[blockIdx.x] = -tot;
    }
}

}  // namespace

int dense_partial_capacity(int64_t m, int64_t n) {
    (void)n;
    return (int)((m + kBM - 1) / kBM);
}

cudaError_t launch_dense_fwd(int64_t m, int64_t n, const float4* X, const float4* Y,
                             int nrhs, const float* W, float s, ab_prec prec,
                             float* out, cudaStream_t st) {
    if (m <= 0) return cudaSuccess;
    if (prec != AB_PREC_FP32) return cudaErrorNotSupported;
    const unsigned grid = (unsigned)((m + kBM - 1) / kBM);
    k_dense_fwd<<<grid, kDThreads, 0, st>>>(m, n, X, Y, nrhs, W, -s * kLog2eD, out);
    return cudaGetLastError();
}

cudaError_t launch_dense_bwd(int64_t m, int64_t n, const float4* X, const float4* Y,
                             int nrhs, const float* W, float s, ab_prec prec,
                             const float* G, float* dW, float4* dX, float4* dY,
                             double* partial, int* partial_count, cudaStream_t st) {
    if (prec != AB_PREC_FP32) return cudaErrorNotSupported;
    cudaError_t e = cudaSuccess;
    *partial_count = 0;
    if (dW && n > 0) {
        const unsigned grid = (unsigned)((n + kBM - 1) / kBM);
        k_dense_fwd<<<grid, kDThreads, 0, st>>>(n, m, Y, X, nrhs, G, -s * kLog2eD, dW);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    if ((dX || partial) && m > 0) {
        const unsigned grid = (unsigned)((m + kBM - 1) / kBM);
        k_dense_gradx<<<grid, kDThreads, 0, st>>>(m, n, X, Y, nrhs, W, G, s, -s * kLog2eD,
                                                  dX, partial);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        if (partial) *partial_count = (int)grid;
    }
    if (dY && n > 0) {
        const unsigned grid = (unsigned)((n + kBM - 1) / kBM);
        k_dense_gradx<<<grid, kDThreads, 0, st>>>(n, m, Y, X, nrhs, G, W, s, -s * kLog2eD,
                                                  dY, nullptr);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace ab
