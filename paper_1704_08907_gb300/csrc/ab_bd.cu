// One Euler-Maruyama Brownian-dynamics step (Brownian dynamics is one of the
// paper's particle methods, Sec. 1; Sec. 2.2.1 names rapidly moving Brownian
// particles as the case that rebuilds the search structure every step).
//
//   x_k += dt F_k + sqrt(2 D dt) z_k
//
// Noise: Philox4x64-10 (Salmon, Moraes, Dror, Shaw, SC'11) keyed by
// (seed, 0) on the counter (i, step, 0, 0); each 64-bit word w gives the
// uniform u = ((w >> 40) + 1) 2^-24 in (0, 1] (exact in FP32), and the
// Box-Muller transform maps (u0, u1) -> (z0, z1) and (u2, u3) -> z2.
// Periodic axes wrap into [lo, hi); non-periodic axes reflect once.
// Element-wise and HBM-bound: one float4 read, one float4 force read, one
// float4 write per particle.
//
// Also here: the semi-implicit (symplectic) Euler step of the paper's worked
// molecular-dynamics example (Sec. 3, Eqs. 2-3), generalised to a step dt:
//   v_i <- v_i + dt a_i,   x_i <- x_i + dt v_i  (the new velocity),
// with a_i the summed pair force (the EXPF pair sum of Eq. 1, or any other).
// Periodic axes wrap as above; at a wall of a non-periodic axis the position
// is reflected once and that velocity component reversed.
#include <cuda_runtime.h>
#include <stdint.h>

#include "ab_internal.cuh"

namespace ab {


namespace {

constexpr uint64_t kPhiloxM0 = 0xD2E7470EE14C6C93ull;
constexpr uint64_t kPhiloxM1 = 0xCA5A826395121157ull;
constexpr uint64_t kPhiloxW0 = 0x9E3779B97F4A7C15ull;
constexpr uint64_t kPhiloxW1 = 0xBB67AE8584CAA73Bull;

struct U64x4 {
    uint64_t v[4];
};

__device__ __forceinline__ U64x4 philox4x64_10(U64x4 c, uint64_t k0, uint64_t k1) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r > 0) {
            k0 += kPhiloxW0;
            k1 += kPhiloxW1;
        }
        const uint64_t hi0 = __umul64hi(kPhiloxM0, c.v[0]);
        const uint64_t lo0 = kPhiloxM0 * c.v[0];
        const uint64_t hi1 = __umul64hi(kPhiloxM1, c.v[2]);
        const uint64_t lo1 = kPhiloxM1 * c.v[2];
        U64x4 n;
        n.v[0] = hi1 ^ c.v[1] ^ k0;
        n.v[1] = lo1;
        n.v[2] = hi0 ^ c.v[3] ^ k1;
        n.v[3] = lo0;
        c = n;
    }
    return c;
}

__device__ __forceinline__ float uniform24(uint64_t w) {
    return (float)((uint32_t)(w >> 40) + 1u) * 5.9604644775390625e-8f;  // 2^-24
}

struct StepGeom {
    int dim;
    int periodic[3];
    float lo[3], hi[3], L[3];
};

__device__ __forceinline__ float advance(float x, float drift, float kick, int k,
                                         const StepGeom& g) {
    float y = x + drift + kick;
    if (g.periodic[k]) {
        const float t = floorf(__fdiv_rn(y - g.lo[k], g.L[k]));
        y = y - t * g.L[k];
        if (y >= g.hi[k] || y < g.lo[k]) y = g.lo[k];
    } else {
        if (y < g.lo[k]) y = 2.0f * g.lo[k] - y;
        if (y > g.hi[k]) y = 2.0f * g.hi[k] - y;
    }
    return y;
}

__global__ void __launch_bounds__(256)
k_bd_step(int64_t n, float4* __restrict__ pos, const float4* __restrict__ force,
          StepGeom g, float dt, float amp, uint64_t seed, uint64_t step) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        U64x4 c;
        c.v[0] = (uint64_t)i;
        c.v[1] = step;
        c.v[2] = 0;
        c.v[3] = 0;
        const U64x4 w = philox4x64_10(c, seed, 0);
        const float u0 = uniform24(w.v[0]), u1 = uniform24(w.v[1]);
        const float rad01 = sqrtf(-2.0f * logf(u0));
        float s01, c01;
        sincospif(2.0f * u1, &s01, &c01);
        float z[3] = {rad01 * c01, rad01 * s01, 0.0f};
        if (g.dim == 3) {
            const float u2 = uniform24(w.v[2]), u3 = uniform24(w.v[3]);
            float s23, c23;
            sincospif(2.0f * u3, &s23, &c23);
            z[2] = sqrtf(-2.0f * logf(u2)) * c23;
        }
        float4 p = pos[i];
        const float4 f = force ? __ldg(force + i) : make_float4(0.f, 0.f, 0.f, 0.f);
        p.x = advance(p.x, dt * f.x, amp * z[0], 0, g);
        p.y = advance(p.y, dt * f.y, amp * z[1], 1, g);
        if (g.dim == 3) p.z = advance(p.z, dt * f.z, amp * z[2], 2, g);
        pos[i] = p;
    }
}

__global__ void __launch_bounds__(256)
k_md_step(int64_t n, float4* __restrict__ pos, float4* __restrict__ vel,
          const float4* __restrict__ acc, StepGeom g, float dt) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        float4 p = pos[i], v = vel[i];
        const float4 a = __ldg(acc + i);
        float pp[3] = {p.x, p.y, p.z}, vv[3] = {v.x, v.y, v.z};
        const float aa[3] = {a.x, a.y, a.z};
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            if (k >= g.dim) break;
            float vk = __fadd_rn(vv[k], __fmul_rn(dt, aa[k]));   // Eq. 2
            float y = __fadd_rn(pp[k], __fmul_rn(dt, vk));        // Eq. 3
            if (g.periodic[k]) {
                const float t = floorf(__fdiv_rn(y - g.lo[k], g.L[k]));
                y = y - t * g.L[k];
                if (y >= g.hi[k] || y < g.lo[k]) y = g.lo[k];
            } else {
                if (y < g.lo[k]) {
                    y = 2.0f * g.lo[k] - y;
                    vk = -vk;
                }
                if (y > g.hi[k]) {
                    y = 2.0f * g.hi[k] - y;
                    vk = -vk;
                }
            }
            pp[k] = y;
            vv[k] = vk;
        }
        pos[i] = make_float4(pp[0], pp[1], pp[2], p.w);
        vel[i] = make_float4(vv[0], vv[1], vv[2], v.w);
    }
}

StepGeom step_geom(const Geom& geo) {
    StepGeom g;
    g.dim = geo.dim;
    for (int k = 0; k < 3; ++k) {
        g.periodic[k] = geo.periodic[k];
        g.lo[k] = geo.lo[k];
        g.L[k] = geo.L[k];
        g.hi[k] = geo.lo[k] + geo.L[k];
    }
    return g;
}

}  // namespace

cudaError_t launch_md_step(const Geom& geo, int64_t n, float4* pos, float4* vel,
                           const float4* acc, float dt, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    int64_t blocks = (n + 255) / 256;
    const int64_t cap = (int64_t)num_sms() * 8;
    if (blocks > cap) blocks = cap;
    k_md_step<<<(unsigned)blocks, 256, 0, st>>>(n, pos, vel, acc, step_geom(geo), dt);
    return cudaGetLastError();
}

cudaError_t launch_bd_step(const Geom& geo, int64_t n, float4* pos, const float4* force,
                           float dt, float D, uint64_t seed, uint64_t step,
                           cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    const StepGeom g = step_geom(geo);
    const float amp = (float)sqrt(2.0 * (double)D * (double)dt);
    int64_t blocks = (n + 255) / 256;
    const int64_t cap = (int64_t)num_sms() * 8;
    if (blocks > cap) blocks = cap;
    k_bd_step<<<(unsigned)blocks, 256, 0, st>>>(n, pos, force, g, dt, amp, seed, step);
    return cudaGetLastError();
}

}  // namespace ab
