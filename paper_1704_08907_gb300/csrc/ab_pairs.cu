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
    const uint32_t* __restrict__ cell_start;   // dense: per cell; compact: per occupied cell
    const uint4* __restrict__ occ;             // compact: occupancy words (see cell_bound)
    const uint32_t* __restrict__ perm;
    const float2* __restrict__ sv;
    int64_t n;
    Geom g;
    float s, s_log2e, eps, sig2, c, k, r;
    float zero;   // 0.0f, passed at run time (see sq2)
    float wend_a;         // Wendland C2 normalisation a (SPH)
    float inv_r;          // 1 / r
    float wend_grad;      // -20 a / r^2: W'(d)/d = wend_grad (1 - d/r)^3
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
// Wendland C2 with support r: t = 1 - d/r (and q = d/r) for a pair at d^2.
__device__ __forceinline__ float wend_t(float d2, float inv_r, float& q) {
    const float d = d2 > 0.0f ? d2 * rsqrt_approx(d2) : 0.0f;
    q = d * inv_r;
    return fmaxf(1.0f - q, 0.0f);
}

// Canonical FP32 minimum image along one periodic axis.
__device__ __forceinline__ float min_image(float d, float L, float halfL) {
    if (d > halfL) return __fsub_rn(d, L);
    if (d < -halfL) return __fadd_rn(d, L);
    return d;
}

// One neighbour coordinate along axis k for offset o (|o| <= reach): returns
// false if the offset leaves a non-periodic box or repeats a cell already
// visited (periodic axes with fewer than 3 cells, general path only);
// *shift receives the fast-path shift (-L when reaching through the lower
// face, +L through the upper face; meaningful when every periodic axis has
// at least 2 reach + 3 cells).
__device__ __forceinline__ bool stencil_coord(const Geom& g, int k, int c, int o, int& t,
                                              float& shift) {
    const int n = g.n[k];
    t = c + o;
    shift = 0.0f;
    if (!g.periodic[k]) return t >= 0 && t < n;
    if (n == 1) return o == 0;
    if (n == 2) {                 // cells {0, 1}: offsets 0 and +1 cover both
        if (o == -1) return false;
        t = (c + o) & 1;
        return true;
    }
    if (t < 0) { t += n; shift = -g.L[k]; }
    else if (t >= n) { t -= n; shift = g.L[k]; }
    return true;
}

// Value separation along one axis, accurate to one rounding: the canonical
// minimum image of x_j - x_i, where a wrapped difference is corrected by the
// rounding error of fl(x_j - x_i) (Knuth's TwoSum).  fl(x_j - x_i) has
// magnitude above L/2 when it wraps, so fl(. -+ L) is exact (Sterbenz) and
// only the final addition of the error term rounds.  Without the correction
// a pair straddling a periodic face would carry an absolute error of
// ulp(L)/2 in a separation of size ~r.  The neighbour predicate never uses
// this value; it uses the canonical FP32 rule only.
__device__ __forceinline__ float two_sum_err(float a, float b, float s) {
    const float bp = __fsub_rn(s, a);
    const float ap = __fsub_rn(s, bp);
    return __fadd_rn(__fsub_rn(a, ap), __fsub_rn(b, bp));
}

__device__ __forceinline__ float value_sep(float xi, float xj, bool periodic, float L,
                                           float halfL) {
    const float s = __fsub_rn(xj, xi);
    if (periodic && (s > halfL || s < -halfL)) {
        const float e = two_sum_err(xj, -xi, s);
        const float w = (s > halfL) ? __fsub_rn(s, L) : __fadd_rn(s, L);
        return __fadd_rn(w, e);
    }
    return s;
}

// Kernel modes: the fast path over a dense cell table, the general path
// (canonical wrap per candidate, dense table), and the fast path over the
// compacted table of occupied cells.
constexpr int kModeFast = 0, kModeGeneral = 1, kModeCompact = 2;

// First sorted slot of cell c (c = n_cells gives n).  Dense table: one load.
// Compacted table: occ[c / 64] packs the occupancy bits of cells 64w ..
// 64w + 63 (x, y) and the number of occupied cells before them (z); the
// occupied cells before c index the compact offsets (an empty cell starts
// where the next occupied one does).
template <int MODE>
__device__ __forceinline__ uint32_t cell_bound(const PairParams& P, int64_t c) {
    if (MODE != kModeCompact) return __ldg(P.cell_start + c);
    const uint4 q = __ldg(P.occ + (c >> 6));
    const uint64_t bits = ((uint64_t)q.y << 32) | q.x;
    const uint32_t rank = q.z + (uint32_t)__popcll(bits & ((1ull << (c & 63)) - 1ull));
    return __ldg(P.cell_start + rank);
}

// Walk the stencil of the particle at pi: seg(a, b, sx, sy, sz) is called for
// each contiguous range [a, b) of sorted particles with its fast-path shift.
// Rows along x are contiguous in sorted order; a row that wraps through the
// periodic x face splits into two segments.
template <int DIM, int MODE, class S>
__device__ __forceinline__ void for_each_segment(const PairParams& P, const float4& pi,
                                                 S&& seg) {
    constexpr bool GENERAL = MODE == kModeGeneral;
    const Geom& g = P.g;
    const int cx = cell_coord(pi.x, g.lo[0], g.inv_w[0], g.n[0]);
    const int cy = cell_coord(pi.y, g.lo[1], g.inv_w[1], g.n[1]);
    const int cz = DIM == 3 ? cell_coord(pi.z, g.lo[2], g.inv_w[2], g.n[2]) : 0;
    const int nx = g.n[0];
    // x segments: [xa0, xb0] with shift xs0, optional [xa1, xb1] with xs1;
    // the stencil reaches kx cells each way along x (kx = 1 on the general
    // path)
    const int kx = GENERAL ? 1 : g.kx;
    int xa0, xb0, xa1 = 0, xb1 = -1;
    float xs0 = 0.0f, xs1 = 0.0f;
    if (!g.periodic[0]) {
        xa0 = cx > kx - 1 ? cx - kx : 0;
        xb0 = cx < nx - kx ? cx + kx : nx - 1;
    } else if (nx <= 3) {
        xa0 = 0;
        xb0 = nx - 1;
    } else if (cx - kx < 0) {
        xa0 = 0; xb0 = cx + kx; xa1 = nx - (kx - cx); xb1 = nx - 1; xs1 = GENERAL ? 0.0f : -g.L[0];
    } else if (cx + kx >= nx) {
        xa0 = cx - kx; xb0 = nx - 1; xa1 = 0; xb1 = cx + kx - nx; xs1 = GENERAL ? 0.0f : g.L[0];
    } else {
        xa0 = cx - kx; xb0 = cx + kx;
    }
    const int ky = GENERAL ? 1 : g.ky, kz = GENERAL ? 1 : g.kz;
#pragma unroll 1
    for (int oz = (DIM == 3 ? -kz : 0); oz <= (DIM == 3 ? kz : 0); ++oz) {
        int z = 0;
        float sz = 0.0f;
        if (DIM == 3 && !stencil_coord(g, 2, cz, oz, z, sz)) continue;
#pragma unroll 1
        for (int oy = -ky; oy <= ky; ++oy) {
            int y;
            float sy;
            if (!stencil_coord(g, 1, cy, oy, y, sy)) continue;
            if (GENERAL) sy = sz = 0.0f;
            const int64_t row = ((int64_t)z * g.n[1] + y) * nx;
            seg(cell_bound<MODE>(P, row + xa0), cell_bound<MODE>(P, row + xb0 + 1), xs0, sy, sz);
            if (xb1 >= xa1)
                seg(cell_bound<MODE>(P, row + xa1), cell_bound<MODE>(P, row + xb1 + 1), xs1, sy, sz);
        }
    }
}

// Packed FP32 pairs (sm_100+ f32x2 arithmetic; each half rounds exactly like
// the scalar FP32 instruction).  The x and y components of one float4 sit in
// an aligned register pair, so the predicate forms (dx, dy) and their squares
// with one instruction each.  Squares are fma(d, d, z) with z a zero known
// only at run time: rounded once, exactly like fl(d * d), and never
// contracted further with the following addition.
__device__ __forceinline__ uint64_t f2pack(float a, float b) {
    uint64_t r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
    return r;
}
__device__ __forceinline__ void f2unpack(uint64_t v, float& a, float& b) {
    asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(v));
}
__device__ __forceinline__ uint64_t sub2(uint64_t a, uint64_t b) {
    uint64_t d;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ uint64_t add2(uint64_t a, uint64_t b) {
    uint64_t d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ uint64_t sq2(uint64_t a, uint64_t z) {
    uint64_t d;
    asm("fma.rn.f32x2 %0, %1, %1, %2;" : "=l"(d) : "l"(a), "l"(z));
    return d;
}

// Predicate separation (canonical FP32 rule) for candidate pj.
template <int DIM, bool GENERAL, bool SHIFTED>
__device__ __forceinline__ float pred_d2(const Geom& g, const float4& pi, const float4& pj,
                                         float sx, float sy, float sz, float& dx, float& dy,
                                         float& dz, float zero) {
    if (GENERAL) {
        dx = __fsub_rn(pj.x, pi.x);
        dy = __fsub_rn(pj.y, pi.y);
        dz = DIM == 3 ? __fsub_rn(pj.z, pi.z) : 0.0f;
        if (g.periodic[0]) dx = min_image(dx, g.L[0], g.halfL[0]);
        if (g.periodic[1]) dy = min_image(dy, g.L[1], g.halfL[1]);
        if (DIM == 3 && g.periodic[2]) dz = min_image(dz, g.L[2], g.halfL[2]);
        float d2 = __fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy));
        if (DIM == 3) d2 = __fadd_rn(d2, __fmul_rn(dz, dz));
        return d2;
    }
    uint64_t dxy = sub2(f2pack(pj.x, pj.y), f2pack(pi.x, pi.y));
    dz = DIM == 3 ? __fsub_rn(pj.z, pi.z) : 0.0f;
    if (SHIFTED) {
        dxy = add2(dxy, f2pack(sx, sy));
        if (DIM == 3) dz = __fadd_rn(dz, sz);
    }
    float qx, qy;
    f2unpack(sq2(dxy, f2pack(zero, zero)), qx, qy);
    f2unpack(dxy, dx, dy);
    float d2 = __fadd_rn(qx, qy);
    if (DIM == 3) d2 = __fadd_rn(d2, __fmul_rn(dz, dz));
    return d2;
}

// Direct visit: f(j, pj, dx, dy, dz, d2) for every accepted pair, with value
// separations accurate to one rounding (see value_sep).  Used by every pair
// kernel.  UNROLL is the unroll factor of the candidate loop, measured per
// kernel: 2 where the body is short or rarely taken (forwards, COUNT, the
// fused LJ kernel), 4 for the adjoints and the EXPF / SOFT forces.
template <int DIM, int MODE, int UNROLL = 4, class F>
__device__ __forceinline__ void visit_pairs(const PairParams& P, uint32_t s,
                                            const float4& pi, F&& f) {
    constexpr bool GENERAL = MODE == kModeGeneral;
    const Geom& g = P.g;
    const float r2 = g.r2;
    for_each_segment<DIM, MODE>(P, pi, [&](uint32_t a0, uint32_t b0, float sx, float sy,
                                              float sz) {
      // the segment holding the particle itself is walked as [a0, s), (s, b0)
      uint32_t a = a0, b = (a0 <= s && s < b0) ? s : b0;
      for (;;) {
        if (GENERAL || sx != 0.0f || sy != 0.0f || sz != 0.0f) {
#pragma unroll 1
            for (uint32_t j = a; j < b; ++j) {
                const float4 pj = __ldg(P.spos + j);
                float dx, dy, dz;
                const float d2 = pred_d2<DIM, GENERAL, true>(g, pi, pj, sx, sy, sz, dx, dy, dz, P.zero);
                if (d2 < r2) {
                    dx = value_sep(pi.x, pj.x, g.periodic[0], g.L[0], g.halfL[0]);
                    dy = value_sep(pi.y, pj.y, g.periodic[1], g.L[1], g.halfL[1]);
                    if (DIM == 3) dz = value_sep(pi.z, pj.z, g.periodic[2], g.L[2], g.halfL[2]);
                    f(j, pj, dx, dy, dz, fmaf(dz, dz, fmaf(dy, dy, dx * dx)));
                }
            }
        } else {
#pragma unroll UNROLL
            for (uint32_t j = a; j < b; ++j) {
                const float4 pj = __ldg(P.spos + j);
                float dx, dy, dz;
                const float d2 = pred_d2<DIM, false, false>(g, pi, pj, 0.f, 0.f, 0.f, dx, dy, dz, P.zero);
                if (d2 < r2) f(j, pj, dx, dy, dz, d2);
            }
        }
        if (b >= b0) break;
        a = b + 1;
        b = b0;
      }
    });
}

// Lets a programmatic dependent launch of the partials' reduction begin
// (its blocks then wait for this grid to finish): called at the start of
// every kernel that writes block partials.
__device__ __forceinline__ void allow_dependents() {
    asm volatile("griddepcontrol.launch_dependents;");
}

// Every pair kernel is a programmatic dependent launch of the kernel before
// it on the stream (normally the build): it may be scheduled while that
// kernel finishes, and waits here, before its first global read, until that
// grid has completed and its writes are visible.  Without a prerequisite
// grid the wait returns at once.
__device__ __forceinline__ void wait_prerequisite() {
    asm volatile("griddepcontrol.wait;" ::: "memory");
}

// FP64 block sum of one value per thread into partial[blockIdx.x].
template <int THREADS>
__device__ __forceinline__ void block_partial(double v, double* partial) {
    __shared__ double s_red[THREADS / 32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) s_red[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
#pragma unroll
        for (int w = 0; w < THREADS / 32; ++w) t += s_red[w];
        partial[blockIdx.x] = t;
    }
}

// Forward for the cheap operators (COUNT, GAUSS, SPH density): direct visit.
// The weight w_j (GAUSS) or mass m_j (SPH) comes in the pad component of the
// sorted position, loaded with the candidate.
template <int DIM, int MODE, int OP>
__global__ void __launch_bounds__(kPairThreads, 8)
k_pair_fwd(PairParams P, PairOut o) {
    wait_prerequisite();
    const uint32_t s = blockIdx.x * kPairThreads + threadIdx.x;
    if (s >= P.n) return;
    const float4 pi = __ldg(P.spos + s);
    float a0 = 0.0f;
    visit_pairs<DIM, MODE, 2>(P, s, pi,
        [&](uint32_t, const float4& pj, float, float, float, float d2) {
            if (OP == AB_OP_COUNT) {
                a0 += 1.0f;
            } else if (OP == AB_OP_GAUSS) {
                a0 = fmaf(pj.w, ex2_approx(-P.s_log2e * d2), a0);
            } else {   // SPH_DENSITY: m_j W(d)
                float q;
                const float t = wend_t(d2, P.inv_r, q);
                const float t2 = t * t;
                a0 = fmaf(pj.w * P.wend_a, t2 * t2 * fmaf(4.0f, q, 1.0f), a0);
            }
        });
    if (OP == AB_OP_SPH_DENSITY) a0 = fmaf(pi.w, P.wend_a, a0);   // the particle itself
    o.out[__ldg(P.perm + s)] = a0;
}

// Forward for LJ / EXPF / SOFT: direct visit.
template <int DIM, int MODE, int OP>
__global__ void __launch_bounds__(kPairThreads, 8)
k_pair_fwd_q(PairParams P, PairOut o) {
    allow_dependents();
    wait_prerequisite();
    const uint32_t s = blockIdx.x * kPairThreads + threadIdx.x;
    const bool live = s < P.n;
    const float4 pi = live ? __ldg(P.spos + s) : make_float4(0.f, 0.f, 0.f, 0.f);
    float a0 = 0.0f, a1 = 0.0f, a2 = 0.0f;
    const float ai = (OP == AB_OP_SPH_FORCE && live) ? __ldg(&P.sv[s].y) : 0.0f;
    if (live) visit_pairs<DIM, MODE, (OP == AB_OP_EXPF || OP == AB_OP_SOFT) ? 4 : 2>(P, s, pi,
        [&](uint32_t j, const float4&, float dx, float dy, float dz, float d2) {
            if (OP == AB_OP_SPH_FORCE) {
                // m_j (A_i + A_j) W'(d)/d dx, W'(d)/d = wend_grad t^3
                const float2 vj = __ldg(P.sv + j);
                float q;
                const float t = wend_t(d2, P.inv_r, q);
                const float coef = vj.x * (ai + vj.y) * (P.wend_grad * (t * t * t));
                a0 = fmaf(coef, dx, a0);
                a1 = fmaf(coef, dy, a1);
                a2 = fmaf(coef, dz, a2);
            } else if (OP == AB_OP_LJ) {
                const float sr2 = P.sig2 * rcp_approx(d2);
                const float sr6 = sr2 * sr2 * sr2;
                a0 = fmaf(sr6, sr6 - 1.0f, a0);
            } else if (d2 > 0.0f) {   // EXPF, SOFT: coincident points contribute 0
                float mag;
                if (OP == AB_OP_EXPF) {
                    const float inv_d = rsqrt_approx(d2);
                    mag = -P.c * ex2_approx(-kLog2e * (d2 * inv_d)) * inv_d;
                } else {
                    // -k (r - d) / d with r - d = (r^2 - d^2) / (r + d): the
                    // fma rounds r^2 - d^2 once, so the term keeps its relative
                    // accuracy up to the cut-off, where r - d cancels, and d
                    // enters only through 1/d and r + d (approximate
                    // reciprocals, a few ulp)
                    const float inv_d = rsqrt_approx(d2);
                    const float d = d2 * inv_d;
                    mag = (-P.k * fmaf(P.r, P.r, -d2)) * (inv_d * rcp_approx(P.r + d));
                }
                a0 = fmaf(mag, dx, a0);
                a1 = fmaf(mag, dy, a1);
                a2 = fmaf(mag, dz, a2);
            }
        });
    if (live) {
        const uint32_t p = __ldg(P.perm + s);
        if (OP == AB_OP_LJ) {
            a0 *= 0.5f * P.eps;
            o.out[p] = a0;
        } else {
            o.out4[p] = make_float4(a0, a1, DIM == 3 ? a2 : 0.0f, 0.0f);
        }
    }
    if (OP == AB_OP_LJ && o.partial) block_partial<kPairThreads>(live ? (double)a0 : 0.0, o.partial);
}

// Adjoints (GAUSS, LJ): direct visit.  (A batched variant that collected
// acceptances in a per-lane bit mask and evaluated the bodies when draining
// it measured 6-15% slower once the predicate was packed.)
// VALUE: the forward value of the same operator in the same walk (the
// upstream gradient is known when the forward runs); each forward term is
// the forward kernel's expression, accumulated in the same visit order, so
// both outputs equal the separate kernels' bit for bit.  With VALUE the
// partials carry the LJ energy (GAUSS: still ds).
template <int DIM, int MODE, int OP, bool VALUE>
__global__ void __launch_bounds__(kPairThreads, 8)
k_pair_bwd(PairParams P, PairOut o) {
    allow_dependents();
    wait_prerequisite();
    const uint32_t s = blockIdx.x * kPairThreads + threadIdx.x;
    const bool live = s < P.n;
    const float4 pi = live ? __ldg(P.spos + s) : make_float4(0.f, 0.f, 0.f, 0.f);
    // the upstream gradient g rides in the pad component of the sorted
    // positions; GAUSS also needs w, a float per particle (sv as float[n])
    const float* __restrict__ wv = reinterpret_cast<const float*>(P.sv);
    const float wi = (live && OP == AB_OP_GAUSS) ? __ldg(wv + s) : 0.0f;
    float gx = 0.0f, gy = 0.0f, gz = 0.0f, dw = 0.0f, ds = 0.0f, y = 0.0f;
    if (live) visit_pairs<DIM, MODE>(P, s, pi,
        [&](uint32_t j, const float4& pj, float dx, float dy, float dz, float d2) {
            if (OP == AB_OP_GAUSS) {
                const float wj = __ldg(wv + j);
                const float k = ex2_approx(-P.s_log2e * d2);
                if (VALUE) y = fmaf(wj, k, y);
                const float coef = fmaf(pi.w, wj, pj.w * wi) * k;
                gx = fmaf(coef, dx, gx);
                gy = fmaf(coef, dy, gy);
                gz = fmaf(coef, dz, gz);
                dw = fmaf(pj.w, k, dw);
                ds = fmaf(wj * k, d2, ds);
            } else {  // LJ: 1/2 (g_i + g_j) eps (12 sr12 - 6 sr6) / d2
                const float inv = rcp_approx(d2);
                const float sr2 = P.sig2 * inv;
                const float sr6 = sr2 * sr2 * sr2;
                if (VALUE) y = fmaf(sr6, sr6 - 1.0f, y);
                const float coef = (pi.w + pj.w) * (sr6 * fmaf(6.0f, sr6, -3.0f)) * inv;
                gx = fmaf(coef, dx, gx);
                gy = fmaf(coef, dy, gy);
                gz = fmaf(coef, dz, gz);
            }
        });
    if (VALUE && OP == AB_OP_LJ) y *= 0.5f * P.eps;
    if (live) {
        const uint32_t p = __ldg(P.perm + s);
        if (VALUE && o.out) o.out[p] = y;
        if (OP == AB_OP_GAUSS) {
            const float two_s = 2.0f * P.s;
            if (o.grad_pos)
                o.grad_pos[p] = make_float4(two_s * gx, two_s * gy,
                                            DIM == 3 ? two_s * gz : 0.0f, 0.0f);
            if (o.grad_w) o.grad_w[p] = dw;
        } else if (o.grad_pos) {
            o.grad_pos[p] = make_float4(P.eps * gx, P.eps * gy, DIM == 3 ? P.eps * gz : 0.0f, 0.0f);
        }
    }
    if (OP == AB_OP_GAUSS && o.partial)
        block_partial<kPairThreads>(live ? -(double)pi.w * (double)ds : 0.0, o.partial);
    if (VALUE && OP == AB_OP_LJ && o.partial)
        block_partial<kPairThreads>(live ? (double)y : 0.0, o.partial);
}

// LJ energy and its gradient in one walk, for a loss equal to the total
// energy (every per-particle energy has upstream gradient 1): the forward's
// E_i = 1/2 eps sum_j ((sig/d)^12 - (sig/d)^6) and the adjoint's
// dE/dx_i = eps sum_j (g_i + g_j) C_ij dx_ij with g = 1, sharing the
// predicate and the powers of sig/d.  Bit for bit the results of k_pair_fwd_q
// (LJ) and of k_pair_bwd (LJ) with g = 1: the same visit order, the same
// expressions, and (g_i + g_j) = 2 exactly.
template <int DIM, int MODE>
__global__ void __launch_bounds__(kPairThreads, 8)
k_pair_lj_eg(PairParams P, PairOut o) {
    allow_dependents();
    wait_prerequisite();
    const uint32_t s = blockIdx.x * kPairThreads + threadIdx.x;
    const bool live = s < P.n;
    const float4 pi = live ? __ldg(P.spos + s) : make_float4(0.f, 0.f, 0.f, 0.f);
    float e = 0.0f, gx = 0.0f, gy = 0.0f, gz = 0.0f;
    if (live) visit_pairs<DIM, MODE, 2>(P, s, pi,
        [&](uint32_t, const float4&, float dx, float dy, float dz, float d2) {
            const float inv = rcp_approx(d2);
            const float sr2 = P.sig2 * inv;
            const float sr6 = sr2 * sr2 * sr2;
            e = fmaf(sr6, sr6 - 1.0f, e);
            // (g_i + g_j) (sr6 (6 sr6 - 3)) / d2 with g = 1: the factor 2 is
            // folded into the fma, exactly (scaling by 2 commutes with
            // rounding; 6 sr6 - 3 is 0 or far from the subnormal range)
            const float coef = (sr6 * fmaf(12.0f, sr6, -6.0f)) * inv;
            gx = fmaf(coef, dx, gx);
            gy = fmaf(coef, dy, gy);
            gz = fmaf(coef, dz, gz);
        });
    if (live) {
        const uint32_t p = __ldg(P.perm + s);
        e *= 0.5f * P.eps;
        if (o.out) o.out[p] = e;
        if (o.grad_pos)
            o.grad_pos[p] = make_float4(P.eps * gx, P.eps * gy, DIM == 3 ? P.eps * gz : 0.0f, 0.0f);
        if (o.grad_packed) {   // DIM floats per particle
            float* q = o.grad_packed + (int64_t)p * DIM;
            q[0] = P.eps * gx;
            q[1] = P.eps * gy;
            if (DIM == 3) q[2] = P.eps * gz;
        }
    }
    if (o.partial) block_partial<kPairThreads>(live ? (double)e : 0.0, o.partial);
}

template <int DIM, int MODE>
__global__ void __launch_bounds__(kPairThreads, 8)
k_pair_count(PairParams P, uint32_t* __restrict__ counts) {
    wait_prerequisite();
    const uint32_t s = blockIdx.x * kPairThreads + threadIdx.x;
    if (s >= P.n) return;
    const float4 pi = __ldg(P.spos + s);
    uint32_t c = 0;
    visit_pairs<DIM, MODE, 2>(P, s, pi,
        [&](uint32_t, const float4&, float, float, float, float) { ++c; });
    counts[__ldg(P.perm + s)] = c;
}

template <int DIM, int MODE>
__global__ void __launch_bounds__(kPairThreads, 8)
k_pair_emit(PairParams P, const int64_t* __restrict__ offsets, int32_t* __restrict__ idx) {
    wait_prerequisite();
    const uint32_t s = blockIdx.x * kPairThreads + threadIdx.x;
    if (s >= P.n) return;
    const float4 pi = __ldg(P.spos + s);
    int64_t at = offsets[__ldg(P.perm + s)];
    visit_pairs<DIM, MODE, 2>(P, s, pi,
        [&](uint32_t j, const float4&, float, float, float, float) {
            idx[at++] = (int32_t)__ldg(P.perm + j);
        });
}

PairParams make_params(const CellList& cl, const ab_op_params& prm, const float2* sv) {
    PairParams P;
    P.spos = cl.spos;
    P.cell_start = cl.cell_start;
    P.occ = cl.occ;
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
    P.zero = 0.0f;
    const double r = (double)cl.g.r, pi = 3.14159265358979323846;
    const double a = cl.g.dim == 3 ? 21.0 / (2.0 * pi * r * r * r) : 7.0 / (pi * r * r);
    P.wend_a = (float)a;
    P.inv_r = (float)(1.0 / r);
    P.wend_grad = (float)(-20.0 * a / (r * r));
    return P;
}

}  // namespace

int pair_grid(int64_t n) { return (int)((n + kPairThreads - 1) / kPairThreads); }

// Launch as a programmatic dependent of the previous kernel on the stream
// (see wait_prerequisite).
template <class... KArgs, class... Args>
static cudaError_t pdl_launch(void (*kern)(KArgs...), int grid, int threads, cudaStream_t st,
                              Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3((unsigned)threads);
    cfg.stream = st;
    cudaLaunchAttribute attr;
    attr.id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr.val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = &attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, args...);
}

#define COMMA_OP(x) , x

#define AB_DISPATCH_DG(KERNEL, THREADS, OPARGS, ...)                                  \
    do {                                                                              \
        const int grid = (int)((cl.n + THREADS - 1) / THREADS);                       \
        cudaError_t le_;                                                              \
        if (cl.g.dim == 3) {                                                          \
            if (cl.g.general) le_ = pdl_launch(KERNEL<3, kModeGeneral OPARGS>, grid, THREADS, st, __VA_ARGS__); \
            else if (cl.g.compact) le_ = pdl_launch(KERNEL<3, kModeCompact OPARGS>, grid, THREADS, st, __VA_ARGS__); \
            else le_ = pdl_launch(KERNEL<3, kModeFast OPARGS>, grid, THREADS, st, __VA_ARGS__); \
        } else {                                                                      \
            if (cl.g.general) le_ = pdl_launch(KERNEL<2, kModeGeneral OPARGS>, grid, THREADS, st, __VA_ARGS__); \
            else if (cl.g.compact) le_ = pdl_launch(KERNEL<2, kModeCompact OPARGS>, grid, THREADS, st, __VA_ARGS__); \
            else le_ = pdl_launch(KERNEL<2, kModeFast OPARGS>, grid, THREADS, st, __VA_ARGS__); \
        }                                                                             \
        if (le_ != cudaSuccess) return le_;                                           \
    } while (0)

cudaError_t launch_pair_fwd(const CellList& cl, ab_op op, const ab_op_params& prm,
                            const float2* sv, PairOut& o, cudaStream_t st) {
    if (cl.n <= 0) return cudaSuccess;
    PairParams P = make_params(cl, prm, sv);
    switch (op) {
        case AB_OP_COUNT: AB_DISPATCH_DG(k_pair_fwd, kPairThreads, COMMA_OP(AB_OP_COUNT), P, o); break;
        case AB_OP_GAUSS: AB_DISPATCH_DG(k_pair_fwd, kPairThreads, COMMA_OP(AB_OP_GAUSS), P, o); break;
        case AB_OP_LJ: AB_DISPATCH_DG(k_pair_fwd_q, kPairThreads, COMMA_OP(AB_OP_LJ), P, o); break;
        case AB_OP_EXPF: AB_DISPATCH_DG(k_pair_fwd_q, kPairThreads, COMMA_OP(AB_OP_EXPF), P, o); break;
        case AB_OP_SOFT: AB_DISPATCH_DG(k_pair_fwd_q, kPairThreads, COMMA_OP(AB_OP_SOFT), P, o); break;
        case AB_OP_SPH_DENSITY:
            AB_DISPATCH_DG(k_pair_fwd, kPairThreads, COMMA_OP(AB_OP_SPH_DENSITY), P, o);
            break;
        case AB_OP_SPH_FORCE:
            AB_DISPATCH_DG(k_pair_fwd_q, kPairThreads, COMMA_OP(AB_OP_SPH_FORCE), P, o);
            break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_pair_bwd(const CellList& cl, ab_op op, const ab_op_params& prm,
                            const float2* sv, PairOut& o, cudaStream_t st, bool value) {
    if (cl.n <= 0) return cudaSuccess;
    PairParams P = make_params(cl, prm, sv);
    switch (op) {
        case AB_OP_GAUSS:
            if (value) AB_DISPATCH_DG(k_pair_bwd, kPairThreads, COMMA_OP(AB_OP_GAUSS) COMMA_OP(true), P, o);
            else AB_DISPATCH_DG(k_pair_bwd, kPairThreads, COMMA_OP(AB_OP_GAUSS) COMMA_OP(false), P, o);
            break;
        case AB_OP_LJ:
            if (value) AB_DISPATCH_DG(k_pair_bwd, kPairThreads, COMMA_OP(AB_OP_LJ) COMMA_OP(true), P, o);
            else AB_DISPATCH_DG(k_pair_bwd, kPairThreads, COMMA_OP(AB_OP_LJ) COMMA_OP(false), P, o);
            break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_pair_energy_grad(const CellList& cl, ab_op op, const ab_op_params& prm,
                                   PairOut& o, cudaStream_t st) {
    if (cl.n <= 0) return cudaSuccess;
    if (op != AB_OP_LJ) return cudaErrorNotSupported;
    PairParams P = make_params(cl, prm, nullptr);
    AB_DISPATCH_DG(k_pair_lj_eg, kPairThreads, , P, o);
    return cudaGetLastError();
}

cudaError_t launch_pair_count(const CellList& cl, uint32_t* counts, cudaStream_t st) {
    if (cl.n <= 0) return cudaSuccess;
    ab_op_params prm{};
    PairParams P = make_params(cl, prm, nullptr);
    AB_DISPATCH_DG(k_pair_count, kPairThreads, , P, counts);
    return cudaGetLastError();
}

cudaError_t launch_pair_emit(const CellList& cl, const int64_t* offsets, int32_t* idx,
                             cudaStream_t st) {
    if (cl.n <= 0) return cudaSuccess;
    ab_op_params prm{};
    PairParams P = make_params(cl, prm, nullptr);
    AB_DISPATCH_DG(k_pair_emit, kPairThreads, , P, offsets, idx);
    return cudaGetLastError();
}

}  // namespace ab
