// Dense kernel operator out = K(X, Y) W on the tcgen05 tensor cores
// (RBF / Gaussian-process operators, paper Sec. 1 and Sec. 1.1; dense global
// operators, Sec. 2.2.2).
//
// One CTA per 128 rows of X, looping over tiles of 128 Y points:
//   epilogue warps 0-15 warp w serves rows 32 (w % 4) .. +31 (its TMEM lane
//                       quadrant) and columns 32 (w / 4) .. +31 of each tile,
//                       so four warps per scheduler hide MUFU/FMA latency;
//                       thread = row i: the base-2 exponent -s log2(e) d2 in
//                       the centred expanded form (see k_prep_y: 3 FMA + 1 add
//                       per element), p = ex2 of it, p split into
//                       bf16 p_hi + p_lo, both written to TMEM with
//                       tcgen05.st (the A operand of the next MMA);
//   warp 16 (one elected lane) tcgen05.mma kind::f16 / kind::tf32, A = P from TMEM,
//                       B = W tile from shared memory, FP32 accumulator in
//                       TMEM: split paths D[128 x 128] += P_hi [W_hi | W_lo]
//                       (N = 128) and D[:, :64] += P_lo W_hi (N = 64) per K
//                       step; the result is D[:, :64] + D[:, 64:]; plain
//                       paths D[128 x 64] += P_hi W_hi;
//   warp 17 (one elected lane) cp.async.bulk of the next W tiles into a 3-stage ring.
// W is prepared once per call (k_prep_w): split into bf16 hi/lo and laid out
// tile by tile in exactly the shared-memory image the MMA reads (K-major,
// 128-byte swizzle), so each tile arrives by one contiguous bulk copy.
// Three P buffers let the epilogue run up to two tiles ahead of the MMAs.
// The bound is the epilogue's instruction stream (exponent, ex2 and the
// hi/lo split: about 5.5 warp instructions per element), with the MMAs
// overlapped behind it; on the split paths the power cap sets the clock.
//
// Every wait is bounded: a role that waits longer than kWaitLimitNs raises
// the CTA's abort flag and the device error word, every role leaves its loop,
// the MMA warp waits (bounded) for its issued MMAs, the producer for its
// copies, and the TMEM is freed before the CTA exits.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

#include "ab_internal.cuh"

namespace ab {


namespace {

constexpr int kTM = 128;            // rows of X per CTA (= TMEM lanes)
constexpr int kRhs = 64;            // MMA N
constexpr int kStages = 3;          // G/W ring depth of the adjoint
constexpr int kFwdStages = 3;       // W ring depth of the forward
// A W tile is 64 rows x 256 bytes of K in either precision: 128 bf16 points
// or 64 tf32 points.  Its P block is 64 TMEM columns either way.
constexpr int kTileBytes = kRhs * 256;              // one hi or lo image: 16 KB
constexpr int kImgBytes = 2 * kTileBytes;           // hi + lo images of one W tile
constexpr int kEpiWarps = 16;       // four warps per TMEM lane quadrant (column quarters)
template <bool TF32>
struct Tile {
    static constexpr int TN = TF32 ? 64 : 128;              // Y points per tile
    static constexpr int YBytes = TN * 16;                   // yhat of one tile
    static constexpr int StageBytes = kImgBytes + YBytes;    // 33 or 34 KB
    static constexpr int ColsPerWarp = TN / (kEpiWarps / 4); // 16 or 32
};
constexpr int kStageBytesMax = Tile<false>::StageBytes;
static_assert(Tile<false>::StageBytes % 1024 == 0 && Tile<true>::StageBytes % 1024 == 0,
              "stages keep the 1024-byte swizzle alignment");
constexpr int kThreadsTC = 32 * (kEpiWarps + 2);   // + MMA warp + producer warp
constexpr uint32_t kTmemCols = 512;
constexpr uint32_t kColD = 0;       // D: columns [0, 128) (split: [P W_hi | P W_lo])
constexpr uint32_t kColP = 128;     // P buffer b: hi at 128 + 128 b, lo at +64
constexpr int kPBufs = 3;           // TMEM: 128 + 3 * 128 = 512 columns
constexpr long long kWaitLimitNs = 2000000000ll;
constexpr float kLog2eTC = 1.4426950408889634f;

struct SmemLayout {
    // W ring first: each stage must be 1024-byte aligned for the swizzle atoms
    static constexpr int w = 0;
    static constexpr int bars = kFwdStages * kStageBytesMax;    // 102 KB at 3 stages
    static constexpr int full = bars;                           // [kFwdStages]
    static constexpr int empty = full + 8 * kFwdStages;            // [kFwdStages]
    static constexpr int pfull = empty + 8 * kFwdStages;           // [kPBufs]
    static constexpr int pempty = pfull + 8 * kPBufs;           // [kPBufs]
    static constexpr int accfull = pempty + 8 * kPBufs;
    static constexpr int tmem_slot = accfull + 8;
    static constexpr int abort_flag = tmem_slot + 4;
    static constexpr int fold_max = abort_flag + 4;   // bits of max over the rows of -c_i
    static constexpr int bytes = fold_max + 4;
};
// + alignment slack; rounded up past half of the SM's 228 KB so that only
// one CTA is resident per SM (each CTA allocates all 512 TMEM columns)
constexpr int kSmemBytes = SmemLayout::bytes + 1024 > 120 * 1024
                               ? (SmemLayout::bytes + 1024 + 1023) / 1024 * 1024
                               : 120 * 1024;
static_assert(kSmemBytes <= 227 * 1024, "shared memory per CTA");
static_assert(SmemLayout::bytes + 1024 <= kSmemBytes, "shared memory layout");

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ long long gtimer() {
    long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}
// One lane of a converged warp (elect.sync).  The MMA and producer roles run
// their loops on the whole warp and issue tcgen05.mma, tcgen05.commit and the
// bulk copies from the elected lane: issued from inside a one-lane branch
// instead, each of these warp-uniform instructions is wrapped by the compiler
// in a loop over the active lanes (about ten extra instructions per MMA on the
// scheduler that also runs epilogue warps).
__device__ __forceinline__ bool elect_one_sync() {
    uint32_t pred = 0;
    asm volatile(
        "{\n\t.reg .pred P;\n\t"
        "elect.sync _|P, 0xffffffff;\n\t"
        "selp.u32 %0, 1, 0, P;\n\t}"
        : "=r"(pred));
    return pred != 0;
}
// The same test with a suspend-time hint: a thread whose phase is not yet
// complete sleeps in the barrier (until the phase completes, or for up to
// 1 ms) instead of spinning.
__device__ __forceinline__ bool mbar_try_wait_sleep(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity), "r"(1000000u)
        : "memory");
    return ok != 0;
}
// Bounded wait on a phase parity.  Returns false if this CTA aborted (here or
// in another role); raises the abort flag and the device error on timeout.
// SLEEP selects the suspend-time hint (each try then returns within 1 ms, so
// the bound still holds).
template <bool SLEEP = false>
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, volatile int* abort_flag,
                                          uint32_t* err) {
    if (SLEEP ? mbar_try_wait_sleep(bar, parity) : mbar_try_wait(bar, parity)) return true;
    const long long t0 = gtimer();
    for (;;) {
        if (SLEEP ? mbar_try_wait_sleep(bar, parity) : mbar_try_wait(bar, parity)) return true;
        if (*abort_flag) return false;
        if (gtimer() - t0 > kWaitLimitNs) {
            *abort_flag = 1;
            atomicOr(err, DEVERR_TC_TIMEOUT);
            return false;
        }
    }
}
__device__ __forceinline__ void bulk_copy(uint32_t dst, const void* src, uint32_t bytes,
                                          uint32_t bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
        "l"(src), "r"(bytes), "r"(bar)
        : "memory");
}
__device__ __forceinline__ float4 lds128(uint32_t addr) {
    float4 v;
    asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];"
                 : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
                 : "r"(addr));
    return v;
}
__device__ __forceinline__ void tc_fence_before() {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_commit(uint32_t bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
                 : "memory");
}
// D[tmem] (+)= A[tmem] * B[smem desc], kind::f16 (bf16 inputs, fp32 accumulate)
__device__ __forceinline__ void mma_ts(uint32_t d_tmem, uint32_t a_tmem, uint64_t b_desc,
                                       uint32_t idesc, uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n\t}" ::"r"(d_tmem),
        "r"(a_tmem), "l"(b_desc), "r"(idesc), "r"(accumulate)
        : "memory");
}
__device__ __forceinline__ void mma_ts_tf32(uint32_t d_tmem, uint32_t a_tmem, uint64_t b_desc,
                                            uint32_t idesc, uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], [%1], %2, %3, p;\n\t}" ::"r"(d_tmem),
        "r"(a_tmem), "l"(b_desc), "r"(idesc), "r"(accumulate)
        : "memory");
}
__device__ __forceinline__ void tmem_st16(uint32_t taddr, const uint32_t (&v)[16]) {
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], "
        "{%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, %16};" ::"r"(taddr),
        "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]), "r"(v[7]),
        "r"(v[8]), "r"(v[9]), "r"(v[10]), "r"(v[11]), "r"(v[12]), "r"(v[13]), "r"(v[14]),
        "r"(v[15])
        : "memory");
}
// 16 lanes x 16 columns: thread t holds, per 8-column repetition r,
// v[4r + 0, 1] = lane t/4, columns 8r + 2 (t%4) + {0, 1} and
// v[4r + 2, 3] = lane t/4 + 8, the same columns.
__device__ __forceinline__ void tmem_st_16x256b_x2(uint32_t taddr, const uint32_t (&v)[8]) {
    asm volatile(
        "tcgen05.st.sync.aligned.16x256b.x2.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};" ::"r"(
            taddr),
        "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]), "r"(v[7])
        : "memory");
}
// 16 lanes x 32 columns, the load counterpart of tmem_st_16x256b_x2 (four
// 8-column repetitions of four registers each).
__device__ __forceinline__ void tmem_ld_16x256b_x4(uint32_t taddr, uint32_t (&v)[16]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.16x256b.x4.b32 "
        "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
          "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]),
          "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
        : "r"(taddr)
        : "memory");
}
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&v)[16]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
        "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
          "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]),
          "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
        : "r"(taddr)
        : "memory");
}
__device__ __forceinline__ void tmem_wait_st() {
    asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_wait_ld() {
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// Shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row groups
// 1024 bytes apart (stride byte offset), descriptor version 1.
__device__ __forceinline__ uint64_t sw128_desc(uint32_t smem_addr) {
    uint64_t d = 0;
    d |= (uint64_t)((smem_addr & 0x3FFFFu) >> 4);
    d |= (uint64_t)1 << 16;                  // leading byte offset (unused here): 16 B
    d |= (uint64_t)(1024 >> 4) << 32;        // stride byte offset
    d |= (uint64_t)1 << 46;                  // version
    d |= (uint64_t)2 << 61;                  // 128-byte swizzle
    return d;
}

// Instruction descriptor, kind::f16: D fp32, A and B bf16, both K-major,
// N = 64, M = 128.
constexpr uint32_t kIdescBf16 = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(kRhs >> 3) << 17) |
                                ((uint32_t)(kTM >> 4) << 24);
// kind::tf32: D fp32, A and B tf32 (format 2), both K-major, N = 64, M = 128.
constexpr uint32_t kIdescTf32 = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(kRhs >> 3) << 17) |
                                ((uint32_t)(kTM >> 4) << 24);
// The same with N = 128: B = [W_hi | W_lo] stacked along N.
constexpr uint32_t kIdescBf16N128 = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(128 >> 3) << 17) |
                                    ((uint32_t)(kTM >> 4) << 24);
constexpr uint32_t kIdescTf32N128 = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(128 >> 3) << 17) |
                                    ((uint32_t)(kTM >> 4) << 24);

__device__ __forceinline__ float ex2f_tc(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
// Packed FP32 pairs (sm_100+ f32x2 arithmetic: each half rounds exactly like
// the scalar FP32 instruction) for the epilogue, which evaluates two columns
// per instruction.
__device__ __forceinline__ uint64_t f2pack(float a, float b) {
    uint64_t r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
    return r;
}
__device__ __forceinline__ void f2unpack(uint64_t v, float& a, float& b) {
    asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(v));
}
__device__ __forceinline__ uint64_t fma2(uint64_t a, uint64_t b, uint64_t c) {
    uint64_t d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}
__device__ __forceinline__ uint64_t mul2(uint64_t a, uint64_t b) {
    uint64_t d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ uint64_t add2(uint64_t a, uint64_t b) {
    uint64_t d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ uint64_t sub2(uint64_t a, uint64_t b) {
    uint64_t d;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
// Two floats -> packed bf16x2 (lo element in the low half), round to nearest.
__device__ __forceinline__ uint32_t pack_bf16x2(float lo, float hi) {
    uint32_t r;
    asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(r) : "f"(hi), "f"(lo));
    return r;
}
__device__ __forceinline__ float bf16lo_to_f(uint32_t v) { return __uint_as_float(v << 16); }
// fp32 -> tf32 (round to nearest, ties away), as an fp32 bit pattern
__device__ __forceinline__ uint32_t to_tf32(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ float bf16hi_to_f(uint32_t v) { return __uint_as_float(v & 0xFFFF0000u); }

// ---------------------------------------------------------------------------
// W -> tile-native hi/lo images.  Tile t covers TN points (128 bf16 or 64
// tf32) and occupies 32 KB: two 16 KB K-blocks of 128 bytes of K each; a
// K-block holds 128 rows, rows 0-63 the hi parts of the 64 right-hand sides
// and rows 64-127 the lo parts, so B = [W_hi | W_lo] is one N = 128 operand.
// Row n of a K-block sits at (n / 8) * 1024 + (n % 8) * 128 with its 16-byte
// chunk c stored at chunk c ^ (n % 8) (the 128-byte swizzle).  One thread
// writes one 16-byte chunk of one hi row and of its lo row.  bf16: hi is
// W rounded to nearest, lo the rounded remainder; tf32 likewise with
// cvt.rna.tf32.
// ---------------------------------------------------------------------------
template <bool TF32>
__global__ void __launch_bounds__(256)
k_prep_w(int64_t n, int nrhs, const float* __restrict__ W, int64_t tiles,
         uint8_t* __restrict__ img, uint32_t* __restrict__ wmax) {
    constexpr int TN = Tile<TF32>::TN;
    constexpr int PTS = TF32 ? 4 : 8;                    // points per 16-byte chunk
    const int64_t total = tiles * kRhs * 16;
    uint32_t amax = 0;   // bits of max |W| seen by this thread (NaN bits order above inf)
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int chunk = (int)(e % 16);                 // 16-byte chunk along K
        const int row = (int)((e / 16) % kRhs);          // right-hand side
        const int64_t t = e / (16 * kRhs);
        const int kb = chunk / 8, c = chunk % 8;
        uint32_t hi[4], lo[4];
        if (TF32) {
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int64_t j = t * TN + chunk * PTS + q;
                const float v = (j < n && row < nrhs) ? __ldg(W + j * nrhs + row) : 0.0f;
                amax = max(amax, __float_as_uint(v) & 0x7FFFFFFFu);
                hi[q] = to_tf32(v);
                lo[q] = to_tf32(v - __uint_as_float(hi[q]));
            }
        } else {
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                float v[2];
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int64_t j = t * TN + chunk * PTS + 2 * q + h;
                    v[h] = (j < n && row < nrhs) ? __ldg(W + j * nrhs + row) : 0.0f;
                    amax = max(amax, __float_as_uint(v[h]) & 0x7FFFFFFFu);
                }
                hi[q] = pack_bf16x2(v[0], v[1]);
                lo[q] = pack_bf16x2(v[0] - bf16lo_to_f(hi[q]), v[1] - bf16hi_to_f(hi[q]));
            }
        }
        const int64_t off = kb * 16384 + (row / 8) * 1024 + (row % 8) * 128 + ((c ^ (row % 8)) * 16);
        uint8_t* base = img + t * (int64_t)kImgBytes;
        *reinterpret_cast<uint4*>(base + off) = make_uint4(hi[0], hi[1], hi[2], hi[3]);
        // the lo row 64 + row: same (row % 8), 8 row groups (8 KB) further
        *reinterpret_cast<uint4*>(base + off + 8192) = make_uint4(lo[0], lo[1], lo[2], lo[3]);
    }
    amax = __reduce_max_sync(0xffffffffu, amax);
    if ((threadIdx.x & 31) == 0 && amax) atomicMax(wmax, amax);
}

// Order-independent float min/max through their sortable integer images.
__device__ __forceinline__ uint32_t f2ord(float f) {
    const uint32_t u = __float_as_uint(f);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__device__ __forceinline__ float ord2f(uint32_t u) {
    return __uint_as_float((u & 0x80000000u) ? (u & 0x7FFFFFFFu) : ~u);
}

// Bounding box of Y (bbox[0..2] = min, bbox[4..6] = max, as ordered ints;
// initialised by the caller to (0xFFFFFFFF, 0)).
__global__ void __launch_bounds__(256)
k_bbox(int64_t n, const float4* __restrict__ Y, uint32_t* __restrict__ bbox) {
    uint32_t mn[3] = {0xFFFFFFFFu, 0xFFFFFFFFu, 0xFFFFFFFFu}, mx[3] = {0u, 0u, 0u};
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n;
         j += (int64_t)gridDim.x * blockDim.x) {
        const float4 y = __ldg(Y + j);
        const float v[3] = {y.x, y.y, y.z};
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            mn[k] = min(mn[k], f2ord(v[k]));
            mx[k] = max(mx[k], f2ord(v[k]));
        }
    }
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        for (int o = 16; o > 0; o >>= 1) {
            mn[k] = min(mn[k], __shfl_xor_sync(0xffffffffu, mn[k], o));
            mx[k] = max(mx[k], __shfl_xor_sync(0xffffffffu, mx[k], o));
        }
        if ((threadIdx.x & 31) == 0) {
            atomicMin(bbox + k, mn[k]);
            atomicMax(bbox + 4 + k, mx[k]);
        }
    }
}

// Per Y point, centred on c = bounding-box midpoint:
//   yhat = (2 s' (y - c), -s' |y - c|^2),  s' = s log2(e)
// so that for a row x the exponent of K in base 2 is
//   x~ . yhat.xyz + yhat.w - s' |x~|^2 = -s' |x - y|^2,   x~ = x - c.
// Centring keeps every term below s' * (half-diagonal^2) in magnitude, so the
// FP32 rounding of the expanded form stays ~1e-5 in the exponent.  Padding
// points get yhat = (0, 0, 0, -inf): their kernel values are exactly 0.
// Layout: points in pairs (2p, 2p+1), each pair as two float4
//   A = (x0, x1, y0, y1), B = (z0, z1, w0, w1)
// so the epilogue loads a column pair's components as packed FP32 pairs.
// BLOCKED (bf16 tiles): within each block of 16 points (pairs 2c + e,
// c = 0..3, e = 0..1) the float4 at 16 * block + 4 * (2 e + {A: 0, B: 1}) + c,
// so that the four column quads c of one 16-point block, read by the four
// threads of a TMEM lane group at once, are 64 contiguous bytes (no bank
// conflict).  Otherwise pair p at float4 2p (A) and 2p + 1 (B).
template <bool BLOCKED>
__global__ void __launch_bounds__(256)
k_prep_y(int64_t n, const float4* __restrict__ Y, int64_t npad, const uint32_t* __restrict__ bbox,
         float sl2e, float4* __restrict__ Yhat, float4* __restrict__ centre) {
    const float c0 = 0.5f * (ord2f(bbox[0]) + ord2f(bbox[4]));
    const float c1 = 0.5f * (ord2f(bbox[1]) + ord2f(bbox[5]));
    const float c2 = 0.5f * (ord2f(bbox[2]) + ord2f(bbox[6]));
    if (blockIdx.x == 0 && threadIdx.x == 0) *centre = make_float4(c0, c1, c2, 0.0f);
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; 2 * p < npad;
         p += (int64_t)gridDim.x * blockDim.x) {
        float4 h[2];
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            const int64_t j = 2 * p + u;
            if (j < n) {
                const float4 y = __ldg(Y + j);
                const float a = y.x - c0, b = y.y - c1, c = y.z - c2;
                const float nrm = fmaf(c, c, fmaf(b, b, a * a));
                h[u] = make_float4(2.0f * sl2e * a, 2.0f * sl2e * b, 2.0f * sl2e * c, -sl2e * nrm);
            } else {
                h[u] = make_float4(0.0f, 0.0f, 0.0f, -__int_as_float(0x7f800000));
            }
        }
        int64_t ia = 2 * p, ib = 2 * p + 1;
        if (BLOCKED) {
            const int64_t blk = p >> 3;
            const int c = (int)(p >> 1) & 3, e = (int)p & 1;
            ia = 16 * blk + 4 * (2 * e) + c;
            ib = 16 * blk + 4 * (2 * e + 1) + c;
        }
        Yhat[ia] = make_float4(h[0].x, h[1].x, h[0].y, h[1].y);
        Yhat[ib] = make_float4(h[0].z, h[1].z, h[0].w, h[1].w);
    }
}

template <bool TF32, bool SPLIT>
__global__ void __launch_bounds__(kThreadsTC, 1)
k_dense_tc_fwd(int64_t m, int64_t total_tiles, const float4* __restrict__ X,
               const float4* __restrict__ Yhat, const float4* __restrict__ centre,
               const uint8_t* __restrict__ wimg, const uint32_t* __restrict__ wmax, float sl2e,
               float* __restrict__ out, uint32_t* __restrict__ err) {
    // blockIdx.y selects a contiguous range of Y tiles; with gridDim.y == 2
    // the two partial sums are added into a zeroed output (0 + a + b is the
    // same in either order, so the result stays deterministic)
    constexpr int kTN = Tile<TF32>::TN;
    constexpr int kYBytes = Tile<TF32>::YBytes;
    constexpr int kStageBytes = Tile<TF32>::StageBytes;
    constexpr int kColsPerWarp = Tile<TF32>::ColsPerWarp;
    // plain paths: the producer and MMA warps sleep in their barrier waits
    // instead of spinning on the schedulers the epilogue warps use (BF16
    // 1.18 -> 1.04 ms, TF32 1.73 -> 1.70 ms); the split paths measured no
    // better (BF16X3) or worse (TF32X3 2.11 -> 2.20 ms) with it
    constexpr bool kSleep = !SPLIT;
    const int64_t t_begin = total_tiles * blockIdx.y / gridDim.y;
    const int64_t tiles = total_tiles * (blockIdx.y + 1) / gridDim.y - t_begin;
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    const uint32_t sbase = smem_u32(smem);
    const uint32_t bar_full = sbase + SmemLayout::full;
    const uint32_t bar_empty = sbase + SmemLayout::empty;
    const uint32_t bar_pfull = sbase + SmemLayout::pfull;
    const uint32_t bar_pempty = sbase + SmemLayout::pempty;
    const uint32_t bar_acc = sbase + SmemLayout::accfull;
    uint32_t* tmem_slot = (uint32_t*)(smem + SmemLayout::tmem_slot);
    volatile int* abort_flag = (volatile int*)(smem + SmemLayout::abort_flag);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int s = 0; s < kFwdStages; ++s) {
            mbar_init(bar_full + 8 * s, 1);
            mbar_init(bar_empty + 8 * s, 1 + kEpiWarps);   // MMA commit + one per epilogue warp
        }
        for (int b = 0; b < kPBufs; ++b) {
            mbar_init(bar_pfull + 8 * b, 32 * kEpiWarps);
            mbar_init(bar_pempty + 8 * b, 1);
        }
        mbar_init(bar_acc, 1);
        *abort_flag = 0;
        *(uint32_t*)(smem + SmemLayout::fold_max) = 0u;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == kEpiWarps) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         sbase + SmemLayout::tmem_slot),
                     "r"(kTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    const int64_t row0 = (int64_t)blockIdx.x * kTM;

    if (warp == kEpiWarps + 1) {
        // ---------------- producer: W tiles into the ring ----------------
        int64_t issued = 0;
        int s = 0;
        uint32_t ph = 0;   // (t / kFwdStages) & 1
        for (int64_t t = 0; t < tiles; ++t) {
            if (t >= kFwdStages) {
                const bool ok = mbar_wait<kSleep>(bar_empty + 8 * s, ph ^ 1u, abort_flag, err);
                if (!__all_sync(0xffffffffu, ok)) break;
            }
            const int64_t gt = t_begin + t;
            if (elect_one_sync()) {
                mbar_arrive_expect_tx(bar_full + 8 * s, kStageBytes);
                bulk_copy(sbase + SmemLayout::w + s * kStageBytes, wimg + gt * (int64_t)kImgBytes,
                          kImgBytes, bar_full + 8 * s);
                bulk_copy(sbase + SmemLayout::w + s * kStageBytes + kImgBytes, Yhat + gt * kTN, kYBytes,
                          bar_full + 8 * s);
            }
            __syncwarp();
            issued = t + 1;
            if (++s == kFwdStages) { s = 0; ph ^= 1u; }
        }
        // copies still in flight must land before the CTA may exit
        if (lane == 0) {
            for (int64_t t = issued > kFwdStages ? issued - kFwdStages : 0; t < issued; ++t) {
                const int q = (int)(t % kFwdStages);
                const long long t0 = gtimer();
                while (!mbar_try_wait(bar_full + 8 * q, (uint32_t)(t / kFwdStages) & 1)) {
                    if (gtimer() - t0 > kWaitLimitNs) {
                        atomicOr(err, DEVERR_TC_TIMEOUT);
                        break;
                    }
                }
            }
        }
    } else if (warp == kEpiWarps) {
        // ---------------- MMA issuer: the warp waits, one lane issues ----------------
        int s = 0, b = 0;
        uint32_t sph = 0, bph = 0;   // (t / kFwdStages) & 1, (t / kPBufs) & 1
        for (int64_t t = 0; t < tiles; ++t) {
            bool ok = mbar_wait<kSleep>(bar_full + 8 * s, sph, abort_flag, err);
            ok = ok && mbar_wait<kSleep>(bar_pfull + 8 * b, bph, abort_flag, err);
            if (!__all_sync(0xffffffffu, ok)) break;
            tc_fence_after();
            const uint32_t a_hi = tmem + kColP + 128 * b;
            const uint32_t a_lo = a_hi + 64;
            // descriptor of the stage; K step ks starts (ks / 4) 16 KB + (ks % 4)
            // 32 bytes further (the address field counts 16-byte units)
            const uint64_t d0 = sw128_desc(sbase + SmemLayout::w + s * kStageBytes);
            if (elect_one_sync()) {
                // 8 K steps of 32 bytes (16 bf16 or 8 tf32 points = 8 TMEM columns);
                // split: D[:, 0:128] += P_hi [W_hi | W_lo] (N = 128) and
                // D[:, 0:64] += P_lo W_hi (N = 64): the three products.  A fourth,
                // P_lo W_lo (2^-16 of the result), would cost a quarter more
                // tensor work and, under the power cap, measurably lower clocks.
#pragma unroll
                for (int ks = 0; ks < 8; ++ks) {
                    const uint64_t bdesc = d0 + (uint64_t)(((ks / 4) * 16384 + (ks % 4) * 32) >> 4);
                    const uint32_t acol = ks * 8;
                    const uint32_t acc0 = (t > 0 || ks > 0) ? 1u : 0u;
                    if (TF32) {
                        if (SPLIT) {
                            mma_ts_tf32(tmem + kColD, a_hi + acol, bdesc, kIdescTf32N128, acc0);
                            mma_ts_tf32(tmem + kColD, a_lo + acol, bdesc, kIdescTf32, 1u);
                        } else {
                            mma_ts_tf32(tmem + kColD, a_hi + acol, bdesc, kIdescTf32, acc0);
                        }
                    } else {
                        if (SPLIT) {
                            mma_ts(tmem + kColD, a_hi + acol, bdesc, kIdescBf16N128, acc0);
                            mma_ts(tmem + kColD, a_lo + acol, bdesc, kIdescBf16, 1u);
                        } else {
                            mma_ts(tmem + kColD, a_hi + acol, bdesc, kIdescBf16, acc0);
                        }
                    }
                }
                tc_commit(bar_empty + 8 * s);
                tc_commit(bar_pempty + 8 * b);
            }
            __syncwarp();
            if (++s == kFwdStages) { s = 0; sph ^= 1u; }
            if (++b == kPBufs) { b = 0; bph ^= 1u; }
        }
        // always signal the epilogue; after an abort it only waits for the
        // MMAs already issued before freeing TMEM
        if (elect_one_sync()) tc_commit(bar_acc);
        __syncwarp();
    } else {
        // ---------------- epilogue warps: row i, one column half ----------------
        const int quad = warp & 3, part = warp >> 2;   // lane quadrant, column slice
        const int i = quad * 32 + lane;   // TMEM lane = row of this thread
        const uint32_t lane_base = tmem + ((uint32_t)(quad * 32) << 16);
        // row in centred coordinates; a padding row gets -inf: K = 0
        float xa = 0.f, xb = 0.f, xc = 0.f, ci = -__int_as_float(0x7f800000);
        if (row0 + i < m) {
            const float4 x = __ldg(X + row0 + i), c = __ldg(centre);
            xa = x.x - c.x;
            xb = x.y - c.y;
            xc = x.z - c.z;
            ci = -sl2e * fmaf(xc, xc, fmaf(xb, xb, xa * xa));
        }
        const uint64_t xa2 = f2pack(xa, xa), xb2 = f2pack(xb, xb), xc2 = f2pack(xc, xc);
        const uint64_t ci2 = f2pack(ci, ci);
        // Fold the row term c_i out of the per-element exponent when the
        // range allows.  P' = 2^(e - c_i) <= 2^(-c_i) (e <= 0), so
        // sum_j P' |W_j| <= n max|W| 2^M with M the CTA's largest -c_i; the
        // rows are scaled by 2^c_i after the MMAs.  The fold is taken only if
        // that bound stays below 2^120 (and nothing is NaN), so the FP32
        // accumulator cannot overflow where the unfolded form would not.
        bool fold;
        {
            uint32_t* fm = (uint32_t*)(smem + SmemLayout::fold_max);
            atomicMax(fm, __float_as_uint(row0 + i < m ? -ci : 0.0f));   // -ci >= 0 (or NaN)
            asm volatile("bar.sync 1, %0;" ::"r"(32 * kEpiWarps) : "memory");   // epilogue warps
            const float M = __uint_as_float(*(volatile uint32_t*)fm);
            const float wm = __uint_as_float(__ldg(wmax));
            fold = M + log2f(wm) + log2f((float)total_tiles * Tile<TF32>::TN) < 120.0f;
        }
        // bf16 paths: thread (g4, c4) = (lane / 4, lane % 4) evaluates rows
        // 8 r + g4 (r = 0..3) of its quadrant at column quads c4, so one
        // yhat load serves four rows (the 16x256b TMEM store layout)
        const int g4 = lane >> 2, c4 = lane & 3;
        uint64_t xq[4][4];   // row r: xa, xb, xc, ci as duplicated pairs
        if (!TF32) {
            const float4 c = __ldg(centre);
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                const int64_t row = row0 + quad * 32 + 8 * r + g4;
                float a = 0.f, bb = 0.f, cc = 0.f, ck = -__int_as_float(0x7f800000);
                if (row < m) {
                    const float4 x = __ldg(X + row);
                    a = x.x - c.x;
                    bb = x.y - c.y;
                    cc = x.z - c.z;
                    ck = -sl2e * fmaf(cc, cc, fmaf(bb, bb, a * a));
                }
                xq[r][0] = f2pack(a, a);
                xq[r][1] = f2pack(bb, bb);
                xq[r][2] = f2pack(cc, cc);
                xq[r][3] = f2pack(ck, ck);
            }
        }
        // the tile loop, compiled with and without the fold
        auto tile_loop = [&](auto fold_c) {
        constexpr bool FOLD = decltype(fold_c)::value;
        // ring positions and phase parities kept incrementally: a 64-bit
        // division per tile costs ~10% of the epilogue's issue slots
        int b = 0, st = 0;
        uint32_t pround = 0, sround = 0;   // (t / kPBufs) & 1, (t / kFwdStages) & 1
        const int ntiles = (int)tiles;
        for (int t = 0; t < ntiles; ++t) {
            bool ok = true;
            if (t >= kPBufs) ok = mbar_wait(bar_pempty + 8 * b, pround ^ 1u, abort_flag, err);
            ok = ok && mbar_wait(bar_full + 8 * st, sround, abort_flag, err);
            if (!__all_sync(0xffffffffu, ok)) break;   // tcgen05.st needs the whole warp
            tc_fence_after();
            // yhat of this tile, read with explicit shared loads (a generic
            // pointer here would send every read down the global-load path)
            const uint32_t yt = sbase + SmemLayout::w + st * kStageBytes + kImgBytes +
                                part * kColsPerWarp * 16;
            // exponent of a column pair with packed FP32 pairs:
            //   e = xa yx + (xb yy + (xc yz + (yw + ci)))  (+ ci dropped when folded)
            auto exponent2 = [&](int pair, float& e0, float& e1) {
                const float4 A = lds128(yt + 32 * pair), B = lds128(yt + 32 * pair + 16);
                uint64_t e = FOLD ? f2pack(B.z, B.w) : add2(f2pack(B.z, B.w), ci2);
                e = fma2(xc2, f2pack(B.x, B.y), e);
                e = fma2(xb2, f2pack(A.z, A.w), e);
                e = fma2(xa2, f2pack(A.x, A.y), e);
                f2unpack(e, e0, e1);
            };
            if (TF32) {
                // 16 columns: one tf32 value per TMEM column; hi keeps the top
                // 19 bits of p (truncation), lo = p - hi exactly (the MMA then
                // reads lo's top 19 bits: relative error <= 2^-20 of p)
                uint32_t hi[16], lo[16];
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    float e0, e1;
                    exponent2(q, e0, e1);
                    const float p0 = ex2f_tc(e0), p1 = ex2f_tc(e1);
                    hi[2 * q] = __float_as_uint(p0) & 0xFFFFE000u;
                    hi[2 * q + 1] = __float_as_uint(p1) & 0xFFFFE000u;
                    if (SPLIT) {
                        float r0, r1;
                        f2unpack(sub2(f2pack(p0, p1), f2pack(__uint_as_float(hi[2 * q]),
                                                             __uint_as_float(hi[2 * q + 1]))),
                                 r0, r1);
                        lo[2 * q] = __float_as_uint(r0);
                        lo[2 * q + 1] = __float_as_uint(r1);
                    }
                }
                const uint32_t col = kColP + 128 * b + part * kColsPerWarp;
                tmem_st16(lane_base + col, hi);
                if (SPLIT) tmem_st16(lane_base + col + 64, lo);
            } else {
                // two 16-column blocks; per block four 16-byte yhat loads
                // (column pairs 2 c4 and 2 c4 + 1, parts A and B) serve
                // 4 rows x 4 columns
                uint32_t hi[2][8], lo[2][8];   // [lane half][16x256b register]
#pragma unroll
                for (int k = 0; k < 2; ++k) {
                    const uint32_t yb = yt + 256 * k + 16 * c4;
                    const float4 Ae = lds128(yb), Be = lds128(yb + 64);
                    const float4 Ao = lds128(yb + 128), Bo = lds128(yb + 192);
#pragma unroll
                    for (int r = 0; r < 4; ++r) {
#pragma unroll
                        for (int jp = 0; jp < 2; ++jp) {
                            const float4 A = jp ? Ao : Ae, B = jp ? Bo : Be;
                            uint64_t e = FOLD ? f2pack(B.z, B.w) : add2(f2pack(B.z, B.w), xq[r][3]);
                            e = fma2(xq[r][2], f2pack(B.x, B.y), e);
                            e = fma2(xq[r][1], f2pack(A.z, A.w), e);
                            e = fma2(xq[r][0], f2pack(A.x, A.y), e);
                            float e0, e1;
                            f2unpack(e, e0, e1);
                            const float p0 = ex2f_tc(e0), p1 = ex2f_tc(e1);
                            const int q = 4 * k + 2 * (r & 1) + jp;
                            if (SPLIT) {
                                // hi = top 16 bits of p (truncation, integer ops only:
                                // the conversion unit is already busy with ex2), lo =
                                // p - hi exactly, then its top 16 bits: relative
                                // error <= 2^-16 of p
                                const uint32_t b0 = __float_as_uint(p0), b1 = __float_as_uint(p1);
                                const float r0 = p0 - __uint_as_float(b0 & 0xFFFF0000u);
                                const float r1 = p1 - __uint_as_float(b1 & 0xFFFF0000u);
                                hi[r >> 1][q] = __byte_perm(b0, b1, 0x7632);
                                lo[r >> 1][q] = __byte_perm(__float_as_uint(r0), __float_as_uint(r1), 0x7632);
                            } else {
                                hi[r >> 1][q] = pack_bf16x2(p0, p1);
                            }
                        }
                    }
                }
                const uint32_t col = kColP + 128 * b + part * (kColsPerWarp / 2);
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const uint32_t ta = lane_base + ((uint32_t)(16 * h) << 16) + col;
                    tmem_st_16x256b_x2(ta, hi[h]);
                    if (SPLIT) tmem_st_16x256b_x2(ta + 64, lo[h]);
                }
            }
            tmem_wait_st();
            tc_fence_before();
            mbar_arrive(bar_pfull + 8 * b);
            __syncwarp();
            if (lane == 0) mbar_arrive(bar_empty + 8 * st);   // this warp is done with yhat
            if (++b == kPBufs) { b = 0; pround ^= 1u; }
            if (++st == kFwdStages) { st = 0; sround ^= 1u; }
        }
        };
        if (fold) tile_loop(std::true_type{});
        else tile_loop(std::false_type{});
        // accumulator ready (or aborted: the wait is still bounded)
        bool ok = mbar_wait(bar_acc, 0, abort_flag, err);
        ok = __all_sync(0xffffffffu, ok && !*abort_flag);   // tcgen05.ld needs the whole warp
        tc_fence_after();
        if (ok) {
            float* orow = out + (row0 + i) * kRhs;
#pragma unroll 1
            for (int c0 = part * (kRhs / 4); c0 < (part + 1) * (kRhs / 4); c0 += 16) {
                uint32_t v[16];
                tmem_ld16(lane_base + kColD + c0, v);
                tmem_wait_ld();
                if (SPLIT) {
                    uint32_t u[16];
                    tmem_ld16(lane_base + kColD + 64 + c0, u);
                    tmem_wait_ld();
#pragma unroll
                    for (int q = 0; q < 16; ++q)
                        v[q] = __float_as_uint(__uint_as_float(v[q]) + __uint_as_float(u[q]));
                }
                if (fold) {   // the row term folded out of the exponent
                    const float sc = ex2f_tc(ci);
#pragma unroll
                    for (int q = 0; q < 16; ++q) v[q] = __float_as_uint(__uint_as_float(v[q]) * sc);
                }
                if (row0 + i < m) {
#pragma unroll
                    for (int q = 0; q < 16; q += 4) {
                        const float4 r = make_float4(__uint_as_float(v[q]), __uint_as_float(v[q + 1]),
                                                     __uint_as_float(v[q + 2]), __uint_as_float(v[q + 3]));
                        if (gridDim.y == 1) *reinterpret_cast<float4*>(orow + c0 + q) = r;
                        else atomicAdd(reinterpret_cast<float4*>(orow + c0 + q), r);
                    }
                }
            }
        }
    }
    // The MMA thread's final commit arrives on bar_acc once its MMAs are done;
    // make sure that has happened (bounded) before TMEM is released.
    if (warp == kEpiWarps && lane == 0) {
        const long long t0 = gtimer();
        while (!mbar_try_wait(bar_acc, 0)) {
            if (gtimer() - t0 > kWaitLimitNs) {
                atomicOr(err, DEVERR_TC_TIMEOUT);
                break;
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == kEpiWarps)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                     "r"(kTmemCols)
                     : "memory");
}


// ===========================================================================
// Adjoint for the rows: dX_i = -2 s sum_j A_ij (x_i - y_j) and
// ds = -sum_ij A_ij d_ij^2, A_ij = (G_i . W_j) K_ij.
//
// S = G W^T on the tensor cores (kind::f16, both operands from shared
// memory): G and W are split into bf16 hi + lo and S = G_hi W_hi + G_hi W_lo
// + G_lo W_hi (three products, AB_PREC_*X3) or G_hi W_hi; the accumulator is
// a 128 x 128 fp32 tile in TMEM, double-buffered.  The epilogue warps read S
// with tcgen05.ld, recompute K_ij from the centred expanded exponent, and
// accumulate A (x~_i - y~_j) and A * exponent in registers, so the row sums
// never cancel.  One CTA per 128 rows; warps 0-15 epilogue (lane quadrant
// w % 4, 32 of the 128 points of a tile), 16 MMA, 17 producer.  Both the G
// image of the CTA's rows (once) and the W image + y tile of each Y tile
// (3-stage ring) arrive by bulk copies.  The same kernel with X <-> Y and
// G <-> W gives dY.
// ===========================================================================
constexpr int kGImg = 2 * 128 * 128;                 // hi + lo blocks, 128 rows x 128 B: 32 KB
constexpr int kGStage = kGImg + 128 * 16;            // W image + y~ tile: 34 KB
struct GradSmem {
    static constexpr int a = 0;                                  // G image (32 KB)
    static constexpr int ring = kGImg;                            // 3 stages
    static constexpr int red = ring + kStages * kGStage;          // 4 x 128 x 4 floats
    static constexpr int bars = red + 4 * 128 * 4 * 4;
    static constexpr int afull = bars;
    static constexpr int full = afull + 8;
    static constexpr int empty = full + 8 * kStages;
    static constexpr int sfull = empty + 8 * kStages;             // [2]
    static constexpr int sempty = sfull + 16;                     // [2]
    static constexpr int done = sempty + 16;
    static constexpr int tmem_slot = done + 8;
    static constexpr int abort_flag = tmem_slot + 4;
    static constexpr int bytes = abort_flag + 4;
};
constexpr int kGradSmemBytes = GradSmem::bytes + 1024;
static_assert(kGImg % 1024 == 0 && kGStage % 1024 == 0, "swizzle alignment");

__device__ __forceinline__ void mma_ss(uint32_t d_tmem, uint64_t a_desc, uint64_t b_desc,
                                       uint32_t idesc, uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(a_desc), "l"(b_desc), "r"(idesc), "r"(accumulate)
        : "memory");
}

// [rows x 64] fp32 -> per block of 128 rows: bf16 hi image then lo image,
// each 128 rows x 128 B, K-major with the 128-byte swizzle.  Rows past
// `rows` are zero.  One thread per (row, 16-byte chunk).
__global__ void __launch_bounds__(256)
k_prep_rows64(int64_t rows, int ncols, const float* __restrict__ src, int64_t blocks,
              uint8_t* __restrict__ img) {
    const int64_t total = blocks * 128 * 8;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int c = (int)(e % 8);
        const int64_t r = e / 8;
        const int rb = (int)(r % 128);
        const int64_t blk = r / 128;
        uint32_t hi[4], lo[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            float v[2];
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int col = c * 8 + 2 * q + h;
                v[h] = (r < rows && col < ncols) ? __ldg(src + r * ncols + col) : 0.0f;
            }
            hi[q] = pack_bf16x2(v[0], v[1]);
            lo[q] = pack_bf16x2(v[0] - bf16lo_to_f(hi[q]), v[1] - bf16hi_to_f(hi[q]));
        }
        const int64_t off = blk * (int64_t)kGImg + (rb / 8) * 1024 + (rb % 8) * 128 + ((c ^ (rb % 8)) * 16);
        *reinterpret_cast<uint4*>(img + off) = make_uint4(hi[0], hi[1], hi[2], hi[3]);
        *reinterpret_cast<uint4*>(img + off + 16384) = make_uint4(lo[0], lo[1], lo[2], lo[3]);
    }
}

// Centred, scaled points for the gradient, y~ = q (y - c) with q = sqrt(s'),
// s' = s log2(e), so that |x~ - y~|^2 is the base-2 exponent's magnitude
// directly; in pairs (2p, 2p + 1) as two float4 (x0, x1, y0, y1),
// (z0, z1, 0, 0), so the epilogue reads a column pair's components as
// packed FP32 pairs.  Padding points are 0; their column of S = G W^T is
// exactly 0 (zero rows of W), so they add nothing.
__global__ void __launch_bounds__(256)
k_prep_ytil(int64_t n, const float4* __restrict__ Y, int64_t npad, const uint32_t* __restrict__ bbox,
            float q, float4* __restrict__ Yt, float4* __restrict__ centre) {
    const float c0 = 0.5f * (ord2f(bbox[0]) + ord2f(bbox[4]));
    const float c1 = 0.5f * (ord2f(bbox[1]) + ord2f(bbox[5]));
    const float c2 = 0.5f * (ord2f(bbox[2]) + ord2f(bbox[6]));
    if (blockIdx.x == 0 && threadIdx.x == 0) *centre = make_float4(c0, c1, c2, 0.0f);
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; 2 * p < npad;
         p += (int64_t)gridDim.x * blockDim.x) {
        float3 h[2];
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            const int64_t j = 2 * p + u;
            h[u] = make_float3(0.0f, 0.0f, 0.0f);
            if (j < n) {
                const float4 y = __ldg(Y + j);
                h[u] = make_float3(q * (y.x - c0), q * (y.y - c1), q * (y.z - c2));
            }
        }
        Yt[2 * p] = make_float4(h[0].x, h[1].x, h[0].y, h[1].y);
        Yt[2 * p + 1] = make_float4(h[0].z, h[1].z, 0.0f, 0.0f);
    }
}

template <bool SPLIT>
__global__ void __launch_bounds__(kThreadsTC, 1)
k_dense_tc_gradx(int64_t m, int64_t total_tiles, const float4* __restrict__ X,
                 const float4* __restrict__ Yt, const float4* __restrict__ centre,
                 const uint8_t* __restrict__ gimg, const uint8_t* __restrict__ wimg, float sl2e,
                 float s, float4* __restrict__ dX, double* __restrict__ partial,
                 uint32_t* __restrict__ err) {
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    const uint32_t sbase = smem_u32(smem);
    const uint32_t bar_afull = sbase + GradSmem::afull;
    const uint32_t bar_full = sbase + GradSmem::full;
    const uint32_t bar_empty = sbase + GradSmem::empty;
    const uint32_t bar_sfull = sbase + GradSmem::sfull;
    const uint32_t bar_sempty = sbase + GradSmem::sempty;
    const uint32_t bar_done = sbase + GradSmem::done;
    uint32_t* tmem_slot = (uint32_t*)(smem + GradSmem::tmem_slot);
    volatile int* abort_flag = (volatile int*)(smem + GradSmem::abort_flag);
    const int64_t t_begin = total_tiles * blockIdx.y / gridDim.y;
    const int64_t tiles = total_tiles * (blockIdx.y + 1) / gridDim.y - t_begin;
    constexpr uint32_t kCols = 256;   // two S buffers of 128 columns

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        mbar_init(bar_afull, 1);
        for (int q = 0; q < kStages; ++q) {
            mbar_init(bar_full + 8 * q, 1);
            mbar_init(bar_empty + 8 * q, 1 + kEpiWarps);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(bar_sfull + 8 * b, 1);
            mbar_init(bar_sempty + 8 * b, kEpiWarps);
        }
        mbar_init(bar_done, 1);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == kEpiWarps) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         sbase + GradSmem::tmem_slot),
                     "r"(kCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    const int64_t row0 = (int64_t)blockIdx.x * kTM;

    if (warp == kEpiWarps + 1) {
        // producer: the warp waits, one elected lane copies
        if (elect_one_sync()) {
            mbar_arrive_expect_tx(bar_afull, kGImg);
            bulk_copy(sbase + GradSmem::a, gimg + blockIdx.x * (int64_t)kGImg, kGImg, bar_afull);
        }
        __syncwarp();
        int64_t issued = 0;
        int q = 0;
        uint32_t ph = 0;   // (t / kStages) & 1
        for (int64_t t = 0; t < tiles; ++t) {
            if (t >= kStages) {
                const bool ok = mbar_wait(bar_empty + 8 * q, ph ^ 1u, abort_flag, err);
                if (!__all_sync(0xffffffffu, ok)) break;
            }
            const int64_t gt = t_begin + t;
            if (elect_one_sync()) {
                mbar_arrive_expect_tx(bar_full + 8 * q, kGStage);
                bulk_copy(sbase + GradSmem::ring + q * kGStage, wimg + gt * (int64_t)kGImg, kGImg,
                          bar_full + 8 * q);
                bulk_copy(sbase + GradSmem::ring + q * kGStage + kGImg, Yt + gt * 128, 128 * 16,
                          bar_full + 8 * q);
            }
            __syncwarp();
            issued = t + 1;
            if (++q == kStages) { q = 0; ph ^= 1u; }
        }
        if (lane == 0) {
            for (int64_t t = issued > kStages ? issued - kStages : 0; t < issued; ++t) {
                const int qq = (int)(t % kStages);
                const long long t0 = gtimer();
                while (!mbar_try_wait(bar_full + 8 * qq, (uint32_t)(t / kStages) & 1)) {
                    if (gtimer() - t0 > kWaitLimitNs) {
                        atomicOr(err, DEVERR_TC_TIMEOUT);
                        break;
                    }
                }
            }
            const long long t0 = gtimer();
            while (!mbar_try_wait(bar_afull, 0)) {
                if (gtimer() - t0 > kWaitLimitNs) {
                    atomicOr(err, DEVERR_TC_TIMEOUT);
                    break;
                }
            }
        }
    } else if (warp == kEpiWarps) {
        // MMA issuer: the warp waits, one elected lane issues
        const bool aok = __all_sync(0xffffffffu, mbar_wait(bar_afull, 0, abort_flag, err));
        int q = 0;
        uint32_t qph = 0;   // (t / kStages) & 1
        // descriptors of the G image (hi at 0, lo 16 KB further); K step ks
        // starts ks 32 bytes further (the address field counts 16-byte units)
        const uint64_t ga0 = sw128_desc(sbase + GradSmem::a);
        for (int64_t t = 0; aok && t < tiles; ++t) {
            const int b = (int)(t & 1);
            bool ok = mbar_wait(bar_full + 8 * q, qph, abort_flag, err);
            if (t >= 2) ok = ok && mbar_wait(bar_sempty + 8 * b, (uint32_t)((t - 2) >> 1) & 1, abort_flag, err);
            if (!__all_sync(0xffffffffu, ok)) break;
            tc_fence_after();
            const uint64_t wb0 = sw128_desc(sbase + GradSmem::ring + q * kGStage);
            const uint32_t dcol = tmem + 128 * b;
            if (elect_one_sync()) {
#pragma unroll
                for (int ks = 0; ks < 4; ++ks) {
                    const uint64_t ahi = ga0 + (uint64_t)(ks * 2), bhi = wb0 + (uint64_t)(ks * 2);
                    mma_ss(dcol, ahi, bhi, kIdescBf16N128, ks > 0 ? 1u : 0u);
                    if (SPLIT) {
                        const uint64_t alo = ahi + (uint64_t)(16384 >> 4);
                        const uint64_t blo = bhi + (uint64_t)(16384 >> 4);
                        mma_ss(dcol, ahi, blo, kIdescBf16N128, 1u);
                        mma_ss(dcol, alo, bhi, kIdescBf16N128, 1u);
                    }
                }
                tc_commit(bar_sfull + 8 * b);
                tc_commit(bar_empty + 8 * q);
            }
            __syncwarp();
            if (++q == kStages) { q = 0; qph ^= 1u; }
        }
        // completes once every MMA issued above has finished (also after
        // an abort); waited for before TMEM is released
        if (elect_one_sync()) tc_commit(bar_done);
        __syncwarp();
    } else {
        // Warp w serves TMEM lane quadrant w % 4, lane half (w / 4) % 2 and
        // columns 64 (w / 8) .. +63 of each S tile.  Thread (g4, c4) =
        // (lane / 4, lane % 4) holds rows 16 h + 8 u + g4 (u = 0, 1) of the
        // quadrant at column pairs 8 k + 2 c4 (the 16x256b TMEM load layout):
        // one y~ load serves two rows, and every step works on column pairs
        // with packed FP32 arithmetic.  Coordinates are scaled by sqrt(s'),
        // so the exponent comes from the differences d = x~ - y~ that the
        // sums need anyway: K = 2^-|d|^2.
        const int quad = warp & 3, half = (warp >> 2) & 1, cpart = warp >> 3;
        const int g4 = lane >> 2, c4 = lane & 3;
        const uint32_t lane_base = tmem + ((uint32_t)(quad * 32 + 16 * half) << 16);
        uint64_t xt[2][3];   // row u: x~ components as duplicated pairs (padding rows: S = 0)
        const float qs = sqrtf(sl2e);   // the scale of the y~ image
        {
            const float4 c = __ldg(centre);
#pragma unroll
            for (int u = 0; u < 2; ++u) {
                const int64_t row = row0 + quad * 32 + 16 * half + 8 * u + g4;
                float a = 0.f, bb = 0.f, cc = 0.f;
                if (row < m) {
                    const float4 x = __ldg(X + row);
                    a = qs * (x.x - c.x);
                    bb = qs * (x.y - c.y);
                    cc = qs * (x.z - c.z);
                }
                xt[u][0] = f2pack(a, a);
                xt[u][1] = f2pack(bb, bb);
                xt[u][2] = f2pack(cc, cc);
            }
        }
        // per row: sums of A dx, A dy, A dz and A * exponent, even and odd
        // columns in the two halves of each packed pair
        uint64_t acc[2][4];
#pragma unroll
        for (int u = 0; u < 2; ++u)
#pragma unroll
            for (int k = 0; k < 4; ++k) acc[u][k] = 0ull;
        int q = 0;
        uint32_t qround = 0;   // ring position t % kStages and parity (t / kStages) & 1
        for (int64_t t = 0; t < tiles; ++t) {
            const int b = (int)(t & 1);
            bool ok = mbar_wait(bar_sfull + 8 * b, (uint32_t)(t >> 1) & 1, abort_flag, err);
            ok = ok && mbar_wait(bar_full + 8 * q, qround, abort_flag, err);
            if (!__all_sync(0xffffffffu, ok)) break;
            tc_fence_after();
            // pair record (64 cpart + 8 k + c0) / 2 + c4 of this tile's y~
            const uint32_t yt = sbase + GradSmem::ring + q * kGStage + kGImg + cpart * 64 * 16 + 32 * c4;
#pragma unroll 1
            for (int c0 = 0; c0 < 64; c0 += 32) {
                uint32_t v[16];
                tmem_ld_16x256b_x4(lane_base + 128 * b + cpart * 64 + c0, v);
                tmem_wait_ld();
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    const float4 P = lds128(yt + 16 * (c0 + 8 * k)), Q = lds128(yt + 16 * (c0 + 8 * k) + 16);
                    const uint64_t yx = f2pack(P.x, P.y), yy = f2pack(P.z, P.w), yz = f2pack(Q.x, Q.y);
#pragma unroll
                    for (int u = 0; u < 2; ++u) {
                        const uint64_t d0 = sub2(xt[u][0], yx), d1 = sub2(xt[u][1], yy);
                        const uint64_t d2 = sub2(xt[u][2], yz);
                        uint64_t e = mul2(d0, d0);   // s' |x - y|^2: K = 2^-e
                        e = fma2(d1, d1, e);
                        e = fma2(d2, d2, e);
                        float e0, e1;
                        f2unpack(e, e0, e1);
                        const uint64_t A = mul2(f2pack(__uint_as_float(v[4 * k + 2 * u]),
                                                       __uint_as_float(v[4 * k + 2 * u + 1])),
                                                f2pack(ex2f_tc(-e0), ex2f_tc(-e1)));
                        acc[u][0] = fma2(A, d0, acc[u][0]);
                        acc[u][1] = fma2(A, d1, acc[u][1]);
                        acc[u][2] = fma2(A, d2, acc[u][2]);
                        acc[u][3] = fma2(A, e, acc[u][3]);
                    }
                }
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) {
                mbar_arrive(bar_sempty + 8 * b);
                mbar_arrive(bar_empty + 8 * q);
            }
            if (++q == kStages) { q = 0; qround ^= 1u; }
        }
        // fold each row's column pairs and its four column-quad lanes, then
        // combine the two column halves of the tile through shared memory
        float* red = (float*)(smem + GradSmem::red);
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            const int i = quad * 32 + 16 * half + 8 * u + g4;
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                float lo, hi;
                f2unpack(acc[u][k], lo, hi);
                float v = lo + hi;
                v += __shfl_xor_sync(0xffffffffu, v, 1);
                v += __shfl_xor_sync(0xffffffffu, v, 2);
                if (c4 == 0) red[(cpart * 128 + i) * 4 + k] = v;
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (threadIdx.x < 128) {
        const float* red = (const float*)(smem + GradSmem::red);
        const int i = threadIdx.x;
        float sx = 0.f, sy = 0.f, sz = 0.f, se = 0.f;
#pragma unroll
        for (int pp = 0; pp < 2; ++pp) {
            sx += red[(pp * 128 + i) * 4 + 0];
            sy += red[(pp * 128 + i) * 4 + 1];
            sz += red[(pp * 128 + i) * 4 + 2];
            se += red[(pp * 128 + i) * 4 + 3];
        }
        if (row0 + i < m && dX && !*abort_flag) {
            // the sums carry the scale q of the differences
            const float f = -2.0f * s / sqrtf(sl2e);
            const float4 g = make_float4(f * sx, f * sy, f * sz, 0.0f);
            if (gridDim.y == 1) dX[row0 + i] = g;
            else atomicAdd(dX + row0 + i, g);
        }
        // ds = -sum A d2 = -(1/s') sum A e, e = s' d2
        double v = (row0 + i < m) ? -(double)se / (double)sl2e : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        __shared__ double wsum[4];
        if ((i & 31) == 0) wsum[i >> 5] = v;
        asm volatile("bar.sync 1, 128;" ::: "memory");   // warps 0-3 only
        if (i == 0 && partial)
            partial[(int64_t)blockIdx.y * gridDim.x + blockIdx.x] = wsum[0] + wsum[1] + wsum[2] + wsum[3];
    }
    if (warp == kEpiWarps && lane == 0) {
        const long long t0 = gtimer();
        while (!mbar_try_wait(bar_done, 0)) {
            if (gtimer() - t0 > kWaitLimitNs) {
                atomicOr(err, DEVERR_TC_TIMEOUT);
                break;
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == kEpiWarps)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kCols)
                     : "memory");
}

}  // namespace

size_t dense_tc_workspace_bytes(int64_t n) {
    // sized for the tf32 tiling (64 points per 32 KB image), the larger one
    const int64_t tiles = (n + 63) / 64;
    return (size_t)tiles * kImgBytes + (size_t)tiles * 64 * 16 + 16 + 32 + 256;
}

template <bool TF32, bool SPLIT>
static cudaError_t launch_tc(int64_t m, int64_t n, const float4* X, const float4* Y, int nrhs,
                             const float* W, float s, float* out, void* ws, uint32_t* err,
                             cudaStream_t st) {
    constexpr int TN = Tile<TF32>::TN;
    const int64_t tiles = (n + TN - 1) / TN;
    if (tiles == 0) return cudaMemsetAsync(out, 0, (size_t)m * nrhs * sizeof(float), st);
    uint8_t* wimg = (uint8_t*)ws;                                    // 1024-aligned (cudaMalloc)
    float4* Yhat = (float4*)(wimg + (size_t)tiles * kImgBytes);
    float4* centre = Yhat + tiles * TN;
    uint32_t* bbox = (uint32_t*)(centre + 1);
    uint32_t* wmax = bbox + 8;   // max |W| (float bits), in the workspace's slack
    const int64_t prep_items = tiles * kRhs * 16;
    cudaError_t e = cudaMemsetAsync(wmax, 0, sizeof(uint32_t), st);
    if (e != cudaSuccess) return e;
    k_prep_w<TF32><<<(unsigned)((prep_items + 255) / 256 < 4096 ? (prep_items + 255) / 256 : 4096), 256,
                     0, st>>>(n, nrhs, W, tiles, wimg, wmax);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(bbox, 0xFF, 4 * sizeof(uint32_t), st)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(bbox + 4, 0x00, 4 * sizeof(uint32_t), st)) != cudaSuccess) return e;
    k_bbox<<<(unsigned)((n + 255) / 256 < 1024 ? (n + 255) / 256 : 1024), 256, 0, st>>>(n, Y, bbox);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    const float sl2e = s * kLog2eTC;
    k_prep_y<!TF32><<<(unsigned)((tiles * TN / 2 + 255) / 256), 256, 0, st>>>(n, Y, tiles * TN, bbox, sl2e,
                                                                          Yhat, centre);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    const int64_t mblocks = (m + kTM - 1) / kTM;
    // split the Y range in two when the row blocks alone leave a ragged last
    // wave (fewer than four waves of one CTA per SM)
    const int split = (mblocks < 4 * (int64_t)num_sms() && tiles >= 2) ? 2 : 1;
    if (split == 2 && (e = cudaMemsetAsync(out, 0, (size_t)m * nrhs * sizeof(float), st)) != cudaSuccess)
        return e;
    // set on every launch: the attribute belongs to the current device, and
    // contexts on several devices may share this process (a microsecond
    // against a kernel of milliseconds)
    e = cudaFuncSetAttribute(k_dense_tc_fwd<TF32, SPLIT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             kSmemBytes);
    if (e != cudaSuccess) return e;
    const dim3 grid((unsigned)mblocks, (unsigned)split);
    k_dense_tc_fwd<TF32, SPLIT><<<grid, kThreadsTC, kSmemBytes, st>>>(m, tiles, X, Yhat, centre, wimg,
                                                                      wmax, sl2e, out, err);
    return cudaGetLastError();
}

size_t dense_tc_grad_workspace_bytes(int64_t m, int64_t n) {
    const int64_t mb = (m + 127) / 128, nb = (n + 127) / 128;
    return (size_t)(mb + nb) * kGImg + (size_t)nb * 128 * 16 + 16 + 32 + 256;
}

// dX (and ds partials) for rows X against points Y with row weights G and
// point weights W (both [.][64]); see k_dense_tc_gradx.
cudaError_t launch_dense_tc_gradx(int64_t m, int64_t n, const float4* X, const float4* Y,
                                  const float* G, const float* W, float s, ab_prec prec,
                                  float4* dX, double* partial, int* partial_count, void* ws,
                                  uint32_t* err, cudaStream_t st) {
    *partial_count = 0;
    if (m <= 0) return cudaSuccess;
    const int64_t mb = (m + 127) / 128, nb = (n + 127) / 128;
    cudaError_t e;
    if (nb == 0) {
        if (dX) e = cudaMemsetAsync(dX, 0, (size_t)m * sizeof(float4), st);
        else e = cudaSuccess;
        return e;
    }
    uint8_t* gimg = (uint8_t*)ws;
    uint8_t* wimg = gimg + (size_t)mb * kGImg;
    float4* Yt = (float4*)(wimg + (size_t)nb * kGImg);
    float4* centre = Yt + nb * 128;
    uint32_t* bbox = (uint32_t*)(centre + 1);
    k_prep_rows64<<<(unsigned)((mb * 1024 + 255) / 256 < 4096 ? (mb * 1024 + 255) / 256 : 4096), 256, 0,
                    st>>>(m, kRhs, G, mb, gimg);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    k_prep_rows64<<<(unsigned)((nb * 1024 + 255) / 256 < 4096 ? (nb * 1024 + 255) / 256 : 4096), 256, 0,
                    st>>>(n, kRhs, W, nb, wimg);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(bbox, 0xFF, 4 * sizeof(uint32_t), st)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(bbox + 4, 0x00, 4 * sizeof(uint32_t), st)) != cudaSuccess) return e;
    k_bbox<<<(unsigned)((n + 255) / 256 < 1024 ? (n + 255) / 256 : 1024), 256, 0, st>>>(n, Y, bbox);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    const float sl2e = s * kLog2eTC;
    k_prep_ytil<<<(unsigned)((nb * 64 + 255) / 256), 256, 0, st>>>(n, Y, nb * 128, bbox, sqrtf(sl2e), Yt,
                                                                   centre);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    const int split = (mb < 4 * (int64_t)num_sms() && nb >= 2) ? 2 : 1;
    if (split == 2 && dX && (e = cudaMemsetAsync(dX, 0, (size_t)m * sizeof(float4), st)) != cudaSuccess)
        return e;
    const dim3 grid((unsigned)mb, (unsigned)split);
    if (prec == AB_PREC_BF16 || prec == AB_PREC_TF32) {
        if ((e = cudaFuncSetAttribute(k_dense_tc_gradx<false>,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      kGradSmemBytes)) != cudaSuccess)
            return e;   // per device: set on every launch
        k_dense_tc_gradx<false><<<grid, kThreadsTC, kGradSmemBytes, st>>>(m, nb, X, Yt, centre, gimg,
                                                                          wimg, sl2e, s, dX, partial, err);
    } else {
        if ((e = cudaFuncSetAttribute(k_dense_tc_gradx<true>,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      kGradSmemBytes)) != cudaSuccess)
            return e;   // per device: set on every launch
        k_dense_tc_gradx<true><<<grid, kThreadsTC, kGradSmemBytes, st>>>(m, nb, X, Yt, centre, gimg,
                                                                         wimg, sl2e, s, dX, partial, err);
    }
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    *partial_count = (int)(mb * split);
    return cudaSuccess;
}

cudaError_t launch_dense_tc_fwd(int64_t m, int64_t n, const float4* X, const float4* Y, int nrhs,
                                const float* W, float s, ab_prec prec, float* out, void* ws,
                                uint32_t* err, cudaStream_t st) {
    if (m <= 0) return cudaSuccess;
    if (nrhs != kRhs) return cudaErrorNotSupported;
    switch (prec) {
        case AB_PREC_BF16X3: return launch_tc<false, true>(m, n, X, Y, nrhs, W, s, out, ws, err, st);
        case AB_PREC_BF16: return launch_tc<false, false>(m, n, X, Y, nrhs, W, s, out, ws, err, st);
        case AB_PREC_TF32X3: return launch_tc<true, true>(m, n, X, Y, nrhs, W, s, out, ws, err, st);
        case AB_PREC_TF32: return launch_tc<true, false>(m, n, X, Y, nrhs, W, s, out, ws, err, st);
        default: return cudaErrorNotSupported;
    }
}

}  // namespace ab
