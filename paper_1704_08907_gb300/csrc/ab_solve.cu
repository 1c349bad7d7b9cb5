// Kernel kernels of the conjugate-gradient solve of (K(X, X) + sigma^2 I) W = B
// (the linear system of RBF interpolation with a nugget and of the
// Gaussian-process posterior mean, paper Sec. 1.1; Hestenes and Stiefel's
// method, one independent CG per right-hand side).
//
// Vectors are float32 [n][nrhs] row-major.  Every inner product is a per-
// column FP64 sum: a block of 4 x 64 threads covers 64 columns and a range of
// rows, reduces its rows in shared memory, and writes one partial per
// (block, column); a second kernel adds the partials of each column in a
// fixed order, so the result is the same on every run.  The step lengths
// alpha = (r.r) / (p.Ap) and beta = (r'.r') / (r.r) are formed on the device
// in FP64; a column whose residual has reached tol ||b|| is frozen (alpha =
// beta = 0, p = 0).  A p = K p + sigma^2 p is never stored: the kernels that
// need it take K p and p.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <vector>

#include "ab_internal.cuh"

namespace ab {

namespace {

constexpr int kCols = 64;       // columns per block (threadIdx.x)
constexpr int kRowLanes = 4;    // row lanes per block (threadIdx.y)

// Per-column scalars of the iteration (device, FP64).
struct Col {
    double bb;      // b.b
    double rs;      // r.r of the current residual
    double pap;     // p.(K p + sigma^2 p)
    double rs_new;  // r.r after the update
    double beta;    // rs_new / rs
    int active;     // 1 while ||r|| > tol ||b||
    int pad;
};

__device__ __forceinline__ void row_range(int64_t n, int64_t& r0, int64_t& r1) {
    const int64_t per = (n + gridDim.x - 1) / gridDim.x;
    r0 = per * blockIdx.x;
    r1 = r0 + per < n ? r0 + per : n;
}

// Reduce v over threadIdx.y and store partial[blockIdx.x][c].
__device__ __forceinline__ void col_partial(double v, int c, int nrhs, double* partial) {
    __shared__ double s[kRowLanes][kCols];
    s[threadIdx.y][threadIdx.x] = v;
    __syncthreads();
    if (threadIdx.y == 0 && c < nrhs) {
        double t = 0.0;
#pragma unroll
        for (int q = 0; q < kRowLanes; ++q) t += s[q][threadIdx.x];
        partial[(int64_t)blockIdx.x * nrhs + c] = t;
    }
}

// R = B, P = B, W = 0; partial of b.b
__global__ void __launch_bounds__(kCols * kRowLanes)
k_solve_init(int64_t n, int nrhs, const float* __restrict__ B, float* __restrict__ R,
             float* __restrict__ P, float* __restrict__ W, double* __restrict__ partial) {
    const int c = blockIdx.y * kCols + threadIdx.x;
    int64_t r0, r1;
    row_range(n, r0, r1);
    double acc = 0.0;
    if (c < nrhs) {
        for (int64_t i = r0 + threadIdx.y; i < r1; i += kRowLanes) {
            const int64_t e = i * nrhs + c;
            const float b = __ldg(B + e);
            R[e] = b;
            P[e] = b;
            W[e] = 0.0f;
            acc += (double)b * b;
        }
    }
    col_partial(acc, c, nrhs, partial);
}

// partial of p.(q + sigma^2 p), q = K p
__global__ void __launch_bounds__(kCols * kRowLanes)
k_solve_pap(int64_t n, int nrhs, const float* __restrict__ P, const float* __restrict__ Q,
            float sigma2, double* __restrict__ partial) {
    const int c = blockIdx.y * kCols + threadIdx.x;
    int64_t r0, r1;
    row_range(n, r0, r1);
    double acc = 0.0;
    if (c < nrhs) {
        for (int64_t i = r0 + threadIdx.y; i < r1; i += kRowLanes) {
            const int64_t e = i * nrhs + c;
            const double p = __ldg(P + e);
            acc += p * ((double)__ldg(Q + e) + (double)sigma2 * p);
        }
    }
    col_partial(acc, c, nrhs, partial);
}

// W += alpha p, R -= alpha (q + sigma^2 p); partial of the new r.r
__global__ void __launch_bounds__(kCols * kRowLanes)
k_solve_update(int64_t n, int nrhs, const float* __restrict__ P, const float* __restrict__ Q,
               float sigma2, const Col* __restrict__ col, float* __restrict__ R,
               float* __restrict__ W, double* __restrict__ partial) {
    const int c = blockIdx.y * kCols + threadIdx.x;
    int64_t r0, r1;
    row_range(n, r0, r1);
    double acc = 0.0;
    if (c < nrhs) {
        const Col k = col[c];
        const float alpha = (k.active && k.pap > 0.0) ? (float)(k.rs / k.pap) : 0.0f;
        for (int64_t i = r0 + threadIdx.y; i < r1; i += kRowLanes) {
            const int64_t e = i * nrhs + c;
            const float p = __ldg(P + e);
            const float ap = fmaf(sigma2, p, __ldg(Q + e));
            W[e] = fmaf(alpha, p, W[e]);
            const float r = fmaf(-alpha, ap, R[e]);
            R[e] = r;
            acc += (double)r * r;
        }
    }
    col_partial(acc, c, nrhs, partial);
}

// P = R + beta P (frozen columns: P = 0)
__global__ void __launch_bounds__(kCols * kRowLanes)
k_solve_dir(int64_t n, int nrhs, const float* __restrict__ R, const Col* __restrict__ col,
            float* __restrict__ P) {
    const int c = blockIdx.y * kCols + threadIdx.x;
    int64_t r0, r1;
    row_range(n, r0, r1);
    if (c >= nrhs) return;
    const Col k = col[c];
    const float beta = (float)k.beta;
    for (int64_t i = r0 + threadIdx.y; i < r1; i += kRowLanes) {
        const int64_t e = i * nrhs + c;
        P[e] = k.active ? fmaf(beta, P[e], __ldg(R + e)) : 0.0f;
    }
}

// Column sums of the partials in a fixed order, then the scalar step for
// what = 0: b.b (initialise), 1: p.Ap, 2: r'.r' (beta, activity, counts).
__global__ void k_solve_finish(const double* __restrict__ partial, int blocks, int nrhs, int what,
                               double tol2, Col* __restrict__ col, int* __restrict__ n_active) {
    for (int c = threadIdx.x; c < nrhs; c += blockDim.x) {
        double t = 0.0;
        for (int b = 0; b < blocks; ++b) t += partial[(int64_t)b * nrhs + c];
        Col k = col[c];
        if (what == 0) {
            k.bb = t;
            k.rs = t;
            k.pap = 0.0;
            k.rs_new = t;
            k.beta = 0.0;
            k.active = t > 0.0;
        } else if (what == 1) {
            k.pap = t;
        } else {
            k.rs_new = t;
            if (k.active) {
                k.beta = k.rs > 0.0 ? t / k.rs : 0.0;
                k.rs = t;
                k.active = t > tol2 * k.bb;
            } else {
                k.beta = 0.0;
            }
        }
        col[c] = k;
        if (what != 1 && k.active) atomicAdd(n_active, 1);
    }
}

int solve_blocks(int64_t n) {
    const int64_t b = (n + 255) / 256;
    return (int)(b < 1024 ? (b > 0 ? b : 1) : 1024);
}

}  // namespace

size_t solve_workspace_bytes(int64_t n, int nrhs) {
    const size_t v = (size_t)n * nrhs * sizeof(float);
    return 3 * v + (size_t)solve_blocks(n) * nrhs * sizeof(double) + (size_t)nrhs * sizeof(Col) +
           256 * 4;
}

// Conjugate gradients; the matvec Q = K(X, X) P is supplied by the caller.
cudaError_t run_solve(int64_t n, int nrhs, const float* B, float sigma2, float tol, int max_iter,
                      float* W, void* ws, const SolveMatvec& mv, int* iters, float* relres,
                      cudaStream_t st) {
    const size_t v = (size_t)n * nrhs;
    float* R = (float*)ws;
    float* P = R + v;
    float* Q = P + v;
    double* partial = (double*)(Q + v);
    const int blocks = solve_blocks(n);
    Col* col = (Col*)(partial + (size_t)blocks * nrhs);
    int* n_active_dev = (int*)(col + nrhs);
    const dim3 grid((unsigned)blocks, (unsigned)((nrhs + kCols - 1) / kCols)), block(kCols, kRowLanes);
    const double tol2 = (double)tol * tol;
    int n_active = 0;
    cudaError_t e;
    auto finish = [&](int what) -> cudaError_t {
        cudaError_t r = cudaMemsetAsync(n_active_dev, 0, sizeof(int), st);
        if (r != cudaSuccess) return r;
        k_solve_finish<<<1, 256, 0, st>>>(partial, blocks, nrhs, what, tol2, col, n_active_dev);
        return cudaGetLastError();
    };
    k_solve_init<<<grid, block, 0, st>>>(n, nrhs, B, R, P, W, partial);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if ((e = finish(0)) != cudaSuccess) return e;
    if ((e = cudaMemcpyAsync(&n_active, n_active_dev, sizeof(int), cudaMemcpyDeviceToHost, st)) != cudaSuccess)
        return e;
    if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return e;
    int it = 0;
    while (n_active > 0 && it < max_iter) {
        if ((e = mv(P, Q)) != cudaSuccess) return e;
        k_solve_pap<<<grid, block, 0, st>>>(n, nrhs, P, Q, sigma2, partial);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        if ((e = finish(1)) != cudaSuccess) return e;
        k_solve_update<<<grid, block, 0, st>>>(n, nrhs, P, Q, sigma2, col, R, W, partial);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        if ((e = finish(2)) != cudaSuccess) return e;
        k_solve_dir<<<grid, block, 0, st>>>(n, nrhs, R, col, P);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        ++it;
        if ((e = cudaMemcpyAsync(&n_active, n_active_dev, sizeof(int), cudaMemcpyDeviceToHost, st)) !=
            cudaSuccess)
            return e;
        if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return e;
    }
    // largest relative residual (the recurrence's r.r over b.b)
    std::vector<Col> hc((size_t)nrhs);
    if ((e = cudaMemcpyAsync(hc.data(), col, (size_t)nrhs * sizeof(Col), cudaMemcpyDeviceToHost, st)) !=
            cudaSuccess ||
        (e = cudaStreamSynchronize(st)) != cudaSuccess)
        return e;
    double worst = 0.0;
    for (const Col& k : hc) {
        const double q = k.bb > 0.0 ? k.rs / k.bb : 0.0;
        if (q > worst) worst = q;
    }
    if (iters) *iters = it;
    if (relres) *relres = (float)sqrt(worst);
    return cudaSuccess;
}

}  // namespace ab
