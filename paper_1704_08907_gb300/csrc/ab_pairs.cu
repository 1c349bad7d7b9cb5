// Fixed-radius pair sums over the cell list (paper Sec. 2.2.2 box search:
// a particle's cell and its adjacent cells; Sec. 3, Eq. 1 and the velocity-
// update listing: the radius-filtered sum over the shortest separation).
//
// One thread per sorted particle i.  Sorted order puts the particles of one
// cell in consecutive threads, so a warp walks the same few neighbour cells
// and the float4 neighbour loads hit L1.  Along x the three stencil cells of
// a row are contiguous in sorted order, so a 3-D stencil is 9 row segments
// (plus one extra segment where a row wraps through a periodic face).
//
// Exact neighbour predicate.  The canonical rule (also the oracle's) is
//   dx = fl(x_j - x_i); periodic axis: dx > L/2 -> fl(dx - L),
//                                      dx < -L/2 -> fl(dx + L);
//   d2 = fl(fl(fl(dx0*dx0) + fl(dx1*dx1)) + fl(dx2*dx2)); pair iff d2 < r2.
// The __fsub_rn/__fmul_rn/__fadd_rn intrinsics are never contracted into FMA.
// Fast path: when every periodic axis has >= 5 cells the wrap decision is
// fixed per stencil cell -- a neighbour cell reached through the face is at
// least 3 cells (> L/2) away the other way, and one reached directly is at
// most 2 cells (< L/2) away -- so dx = fl(fl(x_j - x_i) + shift) with a
// per-segment shift in {-L, 0, +L} is bit-identical to the canonical rule
// (adding 0 is exact).  Otherwise the kernel applies the canonical rule per
// candidate (GENERAL).
#include <cuda_runtime.h>
#include <stdint.h>

#include "ab_internal.cuh"

namespace ab {

namespace {

constexpr int kPairThreads = 128;
constexpr float kLog2e = 1.4426950408889634f;

struct PairParams {
    const float4* __restrict__ spos;
    const uint32_t* __restrict__ cell_start;
    const uint32_t* __restrict__ perm;
    const float2* __restrict__ sv;
    int64_t n;
    Geom g;
    float s, s_log2e, eps, sig2, c, k, r;
};

__device__ __forceinline__ float ex2_approx(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float rcp_approx(float x) {
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float rsqrt_approx(float x) {
    float y;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// Canonical FP32 minimum image along one periodic axis.
__device__ __forceinline__ float min_image(float d, float L, float halfL) {
    if (d > halfL) return __fsub_rn(d, L);
    if (d < -halfL) return __fadd_rn(d, L);
    return d;
}

// Stencil along axis y or z: up to 3 distinct neighbour cell coordinates and
// the fast-path shift of each.
__device__ __forceinline__ int axis_stencil(const Geom& g, int k, int c, bool general,
                                            int (&cell)[3], float (&shift)[3]) {
    const int n = g.n[k];
    int m = 0;
    if (!g.periodic[k]) {
#pragma unroll
        for (int o = -1; o <= 1; ++o) {
            int t = c + o;
            if (t >= 0 && t < n) { cell[m] = t; shift[m] = 0.0f; ++m; }
        }
        return m;
    }
    if (general) {
        // distinct cells of {c-1, c, c+1} mod n (n may be 1 or 2)
        if (n == 1) { cell[0] = 0; shift[0] = 0.0f; return 1; }
        if (n == 2) { cell[0] = 0; cell[1] = 1; shift[0] = shift[1] = 0.0f; return 2; }
        cell[0] = (c + n - 1) % n; cell[1] = c; cell[2] = (c + 1) % n;
        shift[0] = shift[1] = shift[2] = 0.0f;
        return 3;
    }
    cell[0] = c - 1; shift[0] = 0.0f;
    if (c == 0) { cell[0] = n - 1; shift[0] = -g.L[k]; }
    cell[1] = c; shift[1] = 0.0f;
    cell[2] = c + 1; shift[2] = 0.0f;
    if (c == n - 1) { cell[2] = 0; shift[2] = g.L[k]; }
    return 3;
}

// Row segments along x: inclusive cell ranges [a, b] and their shifts.
__device__ __forceinline__ int x_segments(const Geom& g, int c, bool general,
                                          int (&a)[3], int (&b)[3], float (&shift)[3]) {
    const int n = g.n[0];
    if (!g.periodic[0]) {
        a[0] = c > 0 ? c - 1 : 0;
        b[0] = c < n - 1 ? c + 1 : n - 1;
        shift[0] = 0.0f;
        return 1;
    }
    if (general) {
        if (n <= 3) { a[0] = 0; b[0] = n - 1; shift[0] = 0.0f; return 1; }
        // n == 4 (n >= 5 periodic never selects the general path on its own,
        // but the general path is also used for n >= 5 when another axis
        // needs it): the three distinct cells as contiguous pieces
        if (c == 0) {
            a[0] = 0; b[0] = 1; a[1] = n - 1; b[1] = n - 1;
            shift[0] = shift[1] = 0.0f;
            return 2;
        }
        if (c == n - 1) {
            a[0] = n - 2; b[0] = n - 1; a[1] = 0; b[1] = 0;
            shift[0] = shift[1] = 0.0f;
            return 2;
        }
        a[0] = c - 1; b[0] = c + 1; shift[0] = 0.0f;
        return 1;
    }
    if (c == 0) {
        a[0] = 0; b[0] = 1; shift[0] = 0.0f;
        a[1] = n - 1; b[1] = n - 1; shift[1] = -g.L[0];
        return 2;
    }
    if (c == n - 1) {
        a[0] = n - 2; b[0] = n - 1; shift[0] = 0.0f;
        a[1] = 0; b[1] = 0; shift[1] = g.L[0];
        return 2;
    }
    a[0] = c - 1; b[0] = c + 1; shift[0] = 0.0f;
    return 1;
}

// Visit every neighbour j of sorted particle s (position pi):
// f(j, pj, dx, dy, dz, d2) is called for each accepted pair.
template <int DIM, bool GENERAL, class F>
__device__ __forceinline__ void visit_pairs(const PairParams& P, uint32_t s,
                                            const float4& pi, F&& f) {
    const Geom& g = P.g;
    const int cx = cell_coord(pi.x, g.lo[0], g.inv_w[0], g.n[0]);
    const int cy = cell_coord(pi.y, g.lo[1], g.inv_w[1], g.n[1]);
    const int cz = DIM == 3 ? cell_coord(pi.z, g.lo[2], g.inv_w[2], g.n[2]) : 0;
    int ycell[3], zcell[3];
    float yshift[3], zshift[3];
    const int ny = axis_stencil(g, 1, cy, GENERAL, ycell, yshift);
    int nz = 1;
    zcell[0] = 0;
    zshift[0] = 0.0f;
    if (DIM == 3) nz = axis_stencil(g, 2, cz, GENERAL, zcell, zshift);
    int xa[3], xb[3];
    float xshift[3];
    const int nseg = x_segments(g, cx, GENERAL, xa, xb, xshift);
    const float r2 = g.r2;

#pragma unroll 1
    for (int iz = 0; iz < nz; ++iz) {
#pragma unroll 1
        for (int iy = 0; iy < ny; ++iy) {
            const int64_t row = ((int64_t)zcell[iz] * g.n[1] + ycell[iy]) * g.n[0];
            const float sy = yshift[iy], sz = zshift[iz];
#pragma unroll 1
            for (int sg = 0; sg < nseg; ++sg) {
                const uint32_t a = __ldg(P.cell_start + row + xa[sg]);
                const uint32_t b = __ldg(P.cell_start + row + xb[sg] + 1);
                const float sx = xshift[sg];
#pragma unroll 2
                for (uint32_t j = a; j < b; ++j) {
                    const float4 pj = __ldg(P.spos + j);
                    float dx = __fsub_rn(pj.x, pi.x);
                    float dy = __fsub_rn(pj.y, pi.y);
                    float dz = DIM == 3 ? __fsub_rn(pj.z, pi.z) : 0.0f;
                    if (GENERAL) {
                        if (g.periodic[0]) dx = min_image(dx, g.L[0], g.halfL[0]);
                        if (g.periodic[1]) dy = min_image(dy, g.L[1], g.halfL[1]);
                        if (DIM == 3 && g.periodic[2]) dz = min_image(dz, g.L[2], g.halfL[2]);
                    } else {
                        dx = __fadd_rn(dx, sx);
                        dy = __fadd_rn(dy, sy);
                        if (DIM == 3) dz = __fadd_rn(dz, sz);
                    }
                    float d2 = __fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy));
                    if (DIM == 3) d2 = __fadd_rn(d2, __fmul_rn(dz, dz));
                    if (d2 < r2 && j != s) f(j, pj, dx, dy, dz, d2);
                }
            }
        }
    }
}

// FP64 block sum of one value per thread into partial[blockIdx.x].
__device__ __forceinline__ void block_partial(double v, double* partial) {
    __shared__ double s_red[kPairThreads / 32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) s_red[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
#pragma unroll
        for (int w = 0; w < kPairThreads / 32; ++w) t += s_red[w];
        partial[blockIdx.x] = t;
    }
}

template <int DIM, bool GENERAL, int OP>
__global__ void __launch_bounds__(kPairThreads)
k_pair_fwd(PairParams P, PairOut o) {
    const uint32_t s = blockIdx.x * kPairThreads + threadIdx.x;
    const bool live = s < P.n;
    float a0 = 0.0f, a1 = 0.0f, a2 = 0.0f;
    if (live) {
        const float4 pi = __ldg(P.spos + s);
        visit_pairs<DIM, GENERAL>(P, s, pi,
            [&](uint32_t j, const float4& pj, float dx, float dy, float dz, float d2) {
                if (OP == AB_OP_COUNT) {
                    a0 += 1.0f;
                } else if (OP == AB_OP_GAUSS) {
                    a0 += __ldg(&P.sv[j].x) * ex2_approx(-P.s_log2e * d2);
                } else if (OP == AB_OP_LJ) {
                    float sr2 = P.sig2 * rcp_approx(d2);
                    float sr6 = sr2 * sr2 * sr2;
                    a0 += sr6 * (sr6 - 1.0f);
                } else {  // EXPF, SOFT: vector forces, skip coincident points
                    if (d2 > 0.0f) {
                        float inv_d = rsqrt_approx(d2);
                        float d = d2 * inv_d;
                        float mag = (OP == AB_OP_EXPF)
                                        ? -P.c * ex2_approx(-kLog2e * d) * inv_d
                                        : -P.k * (P.r - d) * inv_d;
                        a0 += mag * dx;
                        a1 += mag * dy;
                        a2 += mag * dz;
                    }
                }
            });
        const uint32_t p = __ldg(P.perm + s);
        if (OP == AB_OP_COUNT || OP == AB_OP_GAUSS) {
            o.out[p] = a0;
        } else if (OP == AB_OP_LJ) {
            a0 *= 0.5f * P.eps;
            o.out[p] = a0;
        } else {
            o.out4[p] = make_float4(a0, a1, DIM == 3 ? a2 : 0.0f, 0.0f);
        }
    }
    if (OP == AB_OP_LJ && o.partial) block_partial(live ? (double)a0 : 0.0, o.partial);
}

template <int DIM, bool GENERAL, int OP>
__global__ void __launch_bounds__(kPairThreads)
k_pair_bwd(PairParams P, PairOut o) {
    const uint32_t s = blockIdx.x * kPairThreads + threadIdx.x;
    const bool live = s < P.n;
    float gx = 0.0f, gy = 0.0f, gz = 0.0f, dw = 0.0f, ds = 0.0f;
    float2 vi = make_float2(0.0f, 0.0f);
    if (live) {
        const float4 pi = __ldg(P.spos + s);
        vi = __ldg(P.sv + s);
        visit_pairs<DIM, GENERAL>(P, s, pi,
            [&](uint32_t j, const float4& pj, float dx, float dy, float dz, float d2) {
                const float2 vj = __ldg(P.sv + j);
                if (OP == AB_OP_GAUSS) {
                    float k = ex2_approx(-P.s_log2e * d2);
                    float coef = (vi.y * vj.x + vj.y * vi.x) * k;
                    gx += coef * dx;
                    gy += coef * dy;
                    gz += coef * dz;
                    dw += vj.y * k;
                    ds += vj.x * k * d2;
                } else {  // LJ: 1/2 (g_i + g_j) eps (12 sr12 - 6 sr6) / d2
                    float inv = rcp_approx(d2);
                    float sr2 = P.sig2 * inv;
                    float sr6 = sr2 * sr2 * sr2;
                    float coef = (vi.y + vj.y) * (sr6 * (6.0f * sr6 - 3.0f)) * inv;
                    gx += coef * dx;
                    gy += coef * dy;
                    gz += coef * dz;
                }
            });
        const uint32_t p = __ldg(P.perm + s);
        if (OP == AB_OP_GAUSS) {
            const float two_s = 2.0f * P.s;
            if (o.grad_pos)
                o.grad_pos[p] = make_float4(two_s * gx, two_s * gy,
                                            DIM == 3 ? two_s * gz : 0.0f, 0.0f);
            if (o.grad_w) o.grad_w[p] = dw;
        } else {
            if (o.grad_pos)
                o.grad_pos[p] = make_float4(P.eps * gx, P.eps * gy,
                                            DIM == 3 ? P.eps * gz : 0.0f, 0.0f);
        }
    }
    if (OP == AB_OP_GAUSS && o.partial)
        block_partial(live ? -(double)vi.y * (double)ds : 0.0, o.partial);
}

template <int DIM, bool GENERAL>
__global__ void __launch_bounds__(kPairThreads)
k_pair_count(PairParams P, uint32_t* __restrict__ counts) {
    const uint32_t s = blockIdx.x * kPairThreads + threadIdx.x;
    if (s >= P.n) return;
    const float4 pi = __ldg(P.spos + s);
    uint32_t c = 0;
    visit_pairs<DIM, GENERAL>(P, s, pi,
        [&](uint32_t, const float4&, float, float, float, float) { ++c; });
    counts[__ldg(P.perm + s)] = c;
}

template <int DIM, bool GENERAL>
__global__ void __launch_bounds__(kPairThreads)
k_pair_emit(PairParams P, const int64_t* __restrict__ offsets, int32_t* __restrict__ idx) {
    const uint32_t s = blockIdx.x * kPairThreads + threadIdx.x;
    if (s >= P.n) return;
    const float4 pi = __ldg(P.spos + s);
    int64_t at = offsets[__ldg(P.perm + s)];
    visit_pairs<DIM, GENERAL>(P, s, pi,
        [&](uint32_t j, const float4&, float, float, float, float) {
            idx[at++] = (int32_t)__ldg(P.perm + j);
        });
}

PairParams make_params(const CellList& cl, const ab_op_params& prm, const float2* sv) {
    PairParams P;
    P.spos = cl.spos;
    P.cell_start = cl.cell_start;
    P.perm = cl.perm;
    P.sv = sv;
    P.n = cl.n;
    P.g = cl.g;
    P.s = prm.s;
    P.s_log2e = prm.s * kLog2e;
    P.eps = prm.eps;
    P.sig2 = prm.sigma * prm.sigma;
    P.c = prm.c;
    P.k = prm.k;
    P.r = cl.g.r;
    return P;
}

}  // namespace

int pair_grid(int64_t n) { return (int)((n + kPairThreads - 1) / kPairThreads); }

#define COMMA_OP(x) , x

#define AB_DISPATCH_DG(KERNEL, OPARGS, ...)                                          \
    do {                                                                             \
        const int grid = pair_grid(cl.n);                                            \
        if (cl.g.dim == 3) {                                                         \
            if (cl.g.general) KERNEL<3, true OPARGS><<<grid, kPairThreads, 0, st>>>(__VA_ARGS__); \
            else KERNEL<3, false OPARGS><<<grid, kPairThreads, 0, st>>>(__VA_ARGS__);  \
        } else {                                                                     \
            if (cl.g.general) KERNEL<2, true OPARGS><<<grid, kPairThreads, 0, st>>>(__VA_ARGS__); \
            else KERNEL<2, false OPARGS><<<grid, kPairThreads, 0, st>>>(__VA_ARGS__);  \
        }                                                                            \
    } while (0)

cudaError_t launch_pair_fwd(const CellList& cl, ab_op op, const ab_op_params& prm,
                            const float2* sv, PairOut& o, cudaStream_t st) {
    if (cl.n <= 0) return cudaSuccess;
    PairParams P = make_params(cl, prm, sv);
    switch (op) {
        case AB_OP_COUNT: AB_DISPATCH_DG(k_pair_fwd, COMMA_OP(AB_OP_COUNT), P, o); break;
        case AB_OP_GAUSS: AB_DISPATCH_DG(k_pair_fwd, COMMA_OP(AB_OP_GAUSS), P, o); break;
        case AB_OP_LJ: AB_DISPATCH_DG(k_pair_fwd, COMMA_OP(AB_OP_LJ), P, o); break;
        case AB_OP_EXPF: AB_DISPATCH_DG(k_pair_fwd, COMMA_OP(AB_OP_EXPF), P, o); break;
        case AB_OP_SOFT: AB_DISPATCH_DG(k_pair_fwd, COMMA_OP(AB_OP_SOFT), P, o); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_pair_bwd(const CellList& cl, ab_op op, const ab_op_params& prm,
                            const float2* sv, PairOut& o, cudaStream_t st) {
    if (cl.n <= 0) return cudaSuccess;
    PairParams P = make_params(cl, prm, sv);
    switch (op) {
        case AB_OP_GAUSS: AB_DISPATCH_DG(k_pair_bwd, COMMA_OP(AB_OP_GAUSS), P, o); break;
        case AB_OP_LJ: AB_DISPATCH_DG(k_pair_bwd, COMMA_OP(AB_OP_LJ), P, o); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_pair_count(const CellList& cl, uint32_t* counts, cudaStream_t st) {
    if (cl.n <= 0) return cudaSuccess;
    ab_op_params prm{};
    PairParams P = make_params(cl, prm, nullptr);
    AB_DISPATCH_DG(k_pair_count, , P, counts);
    return cudaGetLastError();
}

cudaError_t launch_pair_emit(const CellList& cl, const int64_t* offsets, int32_t* idx,
                             cudaStream_t st) {
    if (cl.n <= 0) return cudaSuccess;
    ab_op_params prm{};
    PairParams P = make_params(cl, prm, nullptr);
    AB_DISPATCH_DG(k_pair_emit, , P, offsets, idx);
    return cudaGetLastError();
}

}  // namespace ab
