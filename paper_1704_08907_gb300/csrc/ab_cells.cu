// Cell-list build: cell hash + histogram, exclusive scan of the counts,
// stable counting-sort scatter (paper Sec. 2.2.1: a lattice of hypercube
// cells, filled in parallel by reordering the particles; Sec. 3: cell width
// r_cut).  Everything is HBM-bound element-wise work: float4 coalesced loads,
// grid-stride loops sized to the SM count, a single-pass decoupled look-back
// scan with bounded waits.
#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>

#include "ab_internal.cuh"

namespace ab {


namespace {

constexpr int kThreads = 256;

inline int ew_grid(int64_t n) {
    // one thread per element up to 64 blocks per SM: the build kernels are
    // latency-bound (dependent loads and atomics), so they want many loads in
    // flight rather than long grid-stride loops
    int64_t b = (n + kThreads - 1) / kThreads;
    int64_t cap = (int64_t)num_sms() * 64;
    if (b > cap) b = cap;
    return b < 1 ? 1 : (int)b;
}

// Position i of the caller's array: float4 (x, y, z, pad) records, or
// PACKED records of DIM floats (x, y[, z]).
template <int DIM, bool PACKED>
__device__ __forceinline__ float4 load_pos(const float* __restrict__ pos, int64_t i) {
    if (!PACKED) return __ldg(reinterpret_cast<const float4*>(pos) + i);
    const float* q = pos + i * DIM;
    return make_float4(__ldg(q), __ldg(q + 1), DIM == 3 ? __ldg(q + 2) : 0.0f, 0.0f);
}

// ---------------------------------------------------------------------------
// (a1) cell hash + histogram.  The atomic's return value is the particle's
// arrival rank inside its cell (order not deterministic; fixed up below).
// ---------------------------------------------------------------------------
template <int DIM, bool PACKED>
__global__ void __launch_bounds__(kThreads)
k_hash(const float* __restrict__ pos, int64_t n, Geom g, uint2* __restrict__ cell_rank,
       uint32_t* __restrict__ count) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        float4 p = load_pos<DIM, PACKED>(pos, i);
        uint32_t c = (uint32_t)cell_coord(p.x, g.lo[0], g.inv_w[0], g.n[0]);
        uint32_t cy = (uint32_t)cell_coord(p.y, g.lo[1], g.inv_w[1], g.n[1]);
        c += (uint32_t)g.n[0] * cy;
        if (DIM == 3) {
            uint32_t cz = (uint32_t)cell_coord(p.z, g.lo[2], g.inv_w[2], g.n[2]);
            c += (uint32_t)g.n[0] * (uint32_t)g.n[1] * cz;
        }
        cell_rank[i] = make_uint2(c, atomicAdd(count + c, 1u));
    }
}

// (a3) scatter (original index, cell) into the particle's (unordered) slot.
__global__ void __launch_bounds__(kThreads)
k_scatter(int64_t n, const uint2* __restrict__ cell_rank,
          const uint32_t* __restrict__ cell_start, uint2* __restrict__ tmp) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const uint2 cr = cell_rank[i];
        tmp[cell_start[cr.x] + cr.y] = make_uint2((uint32_t)i, cr.x);
    }
}

// (a3) make the sort stable: the final slot of particle p inside its cell is
// the number of cell members with a smaller original index.  Then gather the
// position into sorted order.
template <int DIM, bool PACKED>
__global__ void __launch_bounds__(kThreads)
k_finalize(int64_t n, const float* __restrict__ pos,
           const uint32_t* __restrict__ cell_start,
           const uint2* __restrict__ tmp, uint32_t* __restrict__ perm,
           float4* __restrict__ spos) {
    for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < n;
         s += (int64_t)gridDim.x * blockDim.x) {
        // the slot carries its cell, so the cell range and the position are
        // fetched side by side
        const uint2 pc = tmp[s];
        const uint32_t p = pc.x, c = pc.y;
        uint32_t a = cell_start[c], b = cell_start[c + 1];
        uint32_t r = 0;
        for (uint32_t t = a; t < b; ++t) r += (__ldg(&tmp[t].x) < p) ? 1u : 0u;
        uint32_t d = a + r;
        perm[d] = p;
        float4 q = load_pos<DIM, PACKED>(pos, p);
        spos[d] = make_float4(q.x, q.y, DIM == 3 ? q.z : 0.0f, 0.0f);
    }
}

// The per-particle weight w, in sorted order, into the pad component of the
// sorted positions: a forward that needs only w (Gaussian sum, SPH density)
// then reads it with the candidate's position, no separate load.
__global__ void __launch_bounds__(kThreads)
k_gather_w_pos(int64_t n, const uint32_t* __restrict__ perm, const float* __restrict__ w,
               float4* __restrict__ spos) {
    for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < n;
         s += (int64_t)gridDim.x * blockDim.x)
        spos[s].w = __ldg(w + perm[s]);
}

__global__ void __launch_bounds__(kThreads)
k_gather_pairs(int64_t n, const uint32_t* __restrict__ perm, const float2* __restrict__ wv,
               float2* __restrict__ sv) {
    for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < n;
         s += (int64_t)gridDim.x * blockDim.x)
        sv[s] = __ldg(wv + perm[s]);
}

// ---------------------------------------------------------------------------
// (a2) single-pass exclusive scan with decoupled look-back
// (Merrill & Garland, "Single-pass parallel prefix scan with decoupled
// look-back", 2016).  Tiles take increasing ids from a ticket counter, so a
// tile only ever waits on tiles that are already running; every wait is still
// bounded by a wall-clock limit after which the tile records
// DEVERR_SCAN_TIMEOUT and carries on (results are then garbage, but the
// kernel always terminates).
// ---------------------------------------------------------------------------
constexpr int kScanItems = 16;
constexpr int kScanTile = kThreads * kScanItems;
constexpr uint64_t kFlagAgg = 1ull << 62;
constexpr uint64_t kFlagPre = 2ull << 62;
constexpr uint64_t kValMask = (1ull << 62) - 1;

__device__ __forceinline__ void st_release(uint64_t* p, uint64_t v) {
    asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ uint64_t ld_acquire(const uint64_t* p) {
    uint64_t v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ long long global_ns() {
    long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

template <typename TOut>
__global__ void __launch_bounds__(kThreads)
k_scan(const uint32_t* in, TOut* out, int64_t n, uint64_t* status,
       uint32_t* ticket, uint32_t* err, int skip_tile, long long limit_ns) {
    __shared__ uint32_t s_tile;
    __shared__ uint64_t s_warp[kThreads / 32];
    __shared__ uint64_t s_prefix;
    if (threadIdx.x == 0) s_tile = atomicAdd(ticket, 1u);
    __syncthreads();
    const int64_t tile = s_tile;
    const int64_t base = tile * kScanTile + (int64_t)threadIdx.x * kScanItems;
    // 16-byte vector accesses when the arrays allow them (in and out may be
    // the same array: every thread reads its items before writing them)
    const bool whole = base + kScanItems <= n;
    const bool vec_in = whole && (((uintptr_t)in & 15u) == 0);
    const bool vec_out = whole && sizeof(TOut) == 4 && (((uintptr_t)out & 15u) == 0);

    uint32_t v[kScanItems];
    if (vec_in) {
#pragma unroll
        for (int q = 0; q < kScanItems / 4; ++q) {
            const uint4 t = reinterpret_cast<const uint4*>(in + base)[q];
            v[4 * q] = t.x;
            v[4 * q + 1] = t.y;
            v[4 * q + 2] = t.z;
            v[4 * q + 3] = t.w;
        }
    } else {
#pragma unroll
        for (int k = 0; k < kScanItems; ++k) v[k] = (base + k < n) ? in[base + k] : 0u;
    }
    uint64_t tsum = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) tsum += v[k];

    // warp inclusive scan of thread sums
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint64_t incl = tsum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint64_t t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += t;
    }
    if (lane == 31) s_warp[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        uint64_t x = (lane < kThreads / 32) ? s_warp[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint64_t t = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += t;
        }
        if (lane < kThreads / 32) s_warp[lane] = x;  // inclusive warp totals
    }
    __syncthreads();
    const uint64_t block_total = s_warp[kThreads / 32 - 1];
    const uint64_t warp_excl = warp ? s_warp[warp - 1] : 0;

    // decoupled look-back by warp 0: lane l reads the status word of tile
    // j - l, so 32 predecessors are examined per poll; the exclusive prefix is
    // the sum of the values from tile - 1 down to the nearest tile that has
    // published its inclusive prefix (a tile before tile 0 counts as prefix 0)
    if (warp == 0) {
        uint64_t excl = 0;
        if (tile == 0) {
            if (lane == 0 && tile != skip_tile) st_release(status, kFlagPre | (block_total & kValMask));
        } else {
            if (lane == 0 && tile != skip_tile)
                st_release(status + tile, kFlagAgg | (block_total & kValMask));
            const long long t0 = global_ns();
            int64_t j = tile - 1;
            for (;;) {
                const int64_t idx = j - lane;
                const uint64_t w = idx >= 0 ? ld_acquire(status + idx) : kFlagPre;
                const uint64_t f = w & ~kValMask;
                const unsigned pre = __ballot_sync(0xffffffffu, f == kFlagPre);
                const unsigned zero = __ballot_sync(0xffffffffu, f == 0);
                const int first = pre ? __ffs(pre) - 1 : 31;
                const unsigned upto = first == 31 ? 0xffffffffu : ((1u << (first + 1)) - 1u);
                if (zero & upto) {   // a tile in the window has not published yet
                    if (global_ns() - t0 > limit_ns) {
                        if (lane == 0) atomicOr(err, DEVERR_SCAN_TIMEOUT);
                        break;
                    }
                    continue;
                }
                uint64_t part = ((upto >> lane) & 1u) ? (w & kValMask) : 0;
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
                excl += part;
                if (pre) break;
                j -= 32;
            }
            if (lane == 0 && tile != skip_tile)
                st_release(status + tile, kFlagPre | ((excl + block_total) & kValMask));
        }
        if (lane == 0) s_prefix = excl;
    }
    __syncthreads();
    uint64_t run = s_prefix + warp_excl + (incl - tsum);
    if (vec_out) {
        uint32_t o[kScanItems];
#pragma unroll
        for (int k = 0; k < kScanItems; ++k) {
            o[k] = (uint32_t)run;
            run += v[k];
        }
#pragma unroll
        for (int q = 0; q < kScanItems / 4; ++q)
            reinterpret_cast<uint4*>(out + base)[q] = make_uint4(o[4 * q], o[4 * q + 1], o[4 * q + 2], o[4 * q + 3]);
    } else {
#pragma unroll
        for (int k = 0; k < kScanItems; ++k) {
            if (base + k < n) out[base + k] = (TOut)run;
            run += v[k];
        }
    }
}

constexpr int kRedThreads = 1024;
__global__ void __launch_bounds__(kRedThreads)
k_reduce_partials(const double* __restrict__ partial, int count, double* __restrict__ out) {
    // launched as a programmatic dependent of the kernel that writes the
    // partials: wait until that grid has finished and its writes are visible
    // (returns at once without a prerequisite grid)
    asm volatile("griddepcontrol.wait;" ::: "memory");
    // fixed assignment and tree order: deterministic for a given count
    __shared__ double s[kRedThreads];
    double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
    int t = threadIdx.x;
    for (; t + 3 * kRedThreads < count; t += 4 * kRedThreads) {
        a0 += partial[t];
        a1 += partial[t + kRedThreads];
        a2 += partial[t + 2 * kRedThreads];
        a3 += partial[t + 3 * kRedThreads];
    }
    for (; t < count; t += kRedThreads) a0 += partial[t];
    s[threadIdx.x] = (a0 + a1) + (a2 + a3);
    __syncthreads();
    for (int w = kRedThreads / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) s[threadIdx.x] += s[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = s[0];
}


// ---------------------------------------------------------------------------
// The whole build in one cooperative launch: the same counting sort as the
// kernels above (hash + histogram, exclusive scan, scatter, stable finalize),
// phase after phase, separated by grid-wide barriers.  Every block is
// resident (cooperative launch), each thread keeps several particles' loads
// in flight, and no phase pays a launch.  Data written by other blocks during
// the launch is read with ld.global.cg (L2), never through L1.
//
// Compact variant (clustered inputs, many more cells than particles): the
// table holds offsets of the occupied cells only.  The hash marks each
// particle's cell in an occupancy bitmap (64 cells a word, with the number of
// occupied cells before the word beside it); the histogram, scan, scatter and
// finalize then run over the compact index of the cell (its rank among the
// occupied cells), which orders particles exactly as the cell id does, so the
// sorted order is the dense table's bit for bit.
// ---------------------------------------------------------------------------
constexpr int kCoopThreads = 1024;
constexpr int kCoopIlp = 4;             // particles per thread per loop trip
constexpr int kCoopScanItems = 16;      // cells per thread per scan tile (4 x 16-byte loads)

struct CoopArgs {
    const float* pos;
    int64_t n;
    Geom g;
    int64_t nc1;               // n_cells + 1 entries in cell_start (dense)
    uint32_t* cell_start;      // counts, then offsets (in place); compact: per occupied cell
    uint4* occ;                // compact: occupancy words
    int64_t n_words;           // compact: occ_words(n_cells)
    uint2* cell_rank;          // per particle: (cell or compact index, arrival rank)
    uint2* tmp;                // per unordered slot: (original index, cell or compact index)
    uint32_t* perm;
    float4* spos;
    uint32_t* block_sum;       // [gridDim.x]
    uint32_t* bar;             // [2]: arrivals, generation (zero at launch)
    uint32_t* err;
    long long limit_ns;
    int skip_block;            // testing: this block never arrives at the first barrier (-1: none)
};

// Grid barrier: arrivals counted on bar[0], the last arrival resets it and
// advances the generation bar[1].  The wait is bounded by a wall-clock limit;
// a block that gives up latches DEVERR_SCAN_TIMEOUT and carries on (results
// are then garbage, but every block still terminates).
__device__ __forceinline__ void coop_barrier(uint32_t* bar, uint32_t* err, long long limit_ns,
                                             bool absent = false) {
    __syncthreads();
    if (threadIdx.x == 0 && !absent) {
        __threadfence();
        const uint32_t gen = *((volatile uint32_t*)(bar + 1));
        if (atomicAdd(bar, 1u) == gridDim.x - 1) {
            atomicExch(bar, 0u);
            __threadfence();
            atomicAdd(bar + 1, 1u);
        } else {
            const long long t0 = global_ns();
            while (*((volatile uint32_t*)(bar + 1)) == gen) {
                if (global_ns() - t0 > limit_ns) {
                    atomicOr(err, DEVERR_SCAN_TIMEOUT);
                    break;
                }
            }
        }
        __threadfence();
    }
    __syncthreads();
}

__device__ __forceinline__ uint32_t ldcg_u32(const uint32_t* p) { return __ldcg(p); }
__device__ __forceinline__ uint2 ldcg_u2(const uint2* p) { return __ldcg(p); }

// Block-wide exclusive scan of one value per thread; returns the thread's
// exclusive prefix and writes the block total to *total.
__device__ __forceinline__ uint32_t block_excl_scan(uint32_t v, uint32_t* s_warp, uint32_t* total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t incl = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += t;
    }
    if (lane == 31) s_warp[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        uint32_t x = lane < (int)(blockDim.x >> 5) ? s_warp[lane] : 0u;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t t = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += t;
        }
        s_warp[lane] = x;   // inclusive warp totals
    }
    __syncthreads();
    const uint32_t before = warp ? s_warp[warp - 1] : 0u;
    *total = s_warp[(blockDim.x >> 5) - 1];
    __syncthreads();    // s_warp is reused by the next call
    return before + incl - v;
}

// Sum of one value per thread over the block (every thread gets it).
__device__ __forceinline__ uint32_t block_sum_u32(uint32_t v, uint32_t* s_red) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) s_red[threadIdx.x >> 5] = v;
    __syncthreads();
    uint32_t t = 0;
    for (int w = 0; w < kCoopThreads / 32; ++w) t += s_red[w];
    __syncthreads();
    return t;
}

// Exclusive prefix of the sums of the blocks before this one.
__device__ __forceinline__ uint32_t earlier_blocks(const uint32_t* block_sum, uint32_t* s_red) {
    uint32_t pre = 0;
    for (int b = threadIdx.x; b < (int)blockIdx.x; b += kCoopThreads) pre += ldcg_u32(block_sum + b);
    return block_sum_u32(pre, s_red);
}

// In-place exclusive scan of arr[0 .. len) by the whole grid: each block
// sums a contiguous chunk (16-byte aligned), a grid barrier, then each block
// scans its chunk in tiles behind the sums of the earlier blocks.
__device__ void coop_scan_u32(uint32_t* arr, int64_t len, const CoopArgs& a, uint32_t* s_warp,
                              uint32_t* s_red) {
    const int64_t chunk = (((len + gridDim.x - 1) / gridDim.x) + 3) & ~(int64_t)3;
    const int64_t c0 = (int64_t)blockIdx.x * chunk;
    const int64_t c1 = c0 + chunk < len ? c0 + chunk : len;
    {
        uint32_t sum = 0;
        int64_t c = c0 + (int64_t)threadIdx.x * 4;
        for (; c + 4 <= c1; c += (int64_t)kCoopThreads * 4) {
            const uint4 v = __ldcg(reinterpret_cast<const uint4*>(arr + c));
            sum += v.x + v.y + v.z + v.w;
        }
        for (; c < c1; ++c) sum += ldcg_u32(arr + c);   // at most one thread's tail of < 4
        const uint32_t t = block_sum_u32(sum, s_red);
        if (threadIdx.x == 0) a.block_sum[blockIdx.x] = t;
    }
    coop_barrier(a.bar, a.err, a.limit_ns);
    uint32_t run = earlier_blocks(a.block_sum, s_red);
    for (int64_t t0 = c0; t0 < c1; t0 += (int64_t)kCoopThreads * kCoopScanItems) {
        const int64_t base = t0 + (int64_t)threadIdx.x * kCoopScanItems;
        uint32_t v[kCoopScanItems];
        const bool whole = base + kCoopScanItems <= c1;
        if (whole) {
#pragma unroll
            for (int q = 0; q < kCoopScanItems / 4; ++q) {
                const uint4 t = __ldcg(reinterpret_cast<const uint4*>(arr + base) + q);
                v[4 * q] = t.x;
                v[4 * q + 1] = t.y;
                v[4 * q + 2] = t.z;
                v[4 * q + 3] = t.w;
            }
        } else {
#pragma unroll
            for (int k = 0; k < kCoopScanItems; ++k) v[k] = base + k < c1 ? ldcg_u32(arr + base + k) : 0u;
        }
        uint32_t tsum = 0;
#pragma unroll
        for (int k = 0; k < kCoopScanItems; ++k) tsum += v[k];
        uint32_t total;
        uint32_t ex = run + block_excl_scan(tsum, s_warp, &total);
        if (whole) {
#pragma unroll
            for (int q = 0; q < kCoopScanItems / 4; ++q) {
                uint4 t;
                t.x = ex; ex += v[4 * q];
                t.y = ex; ex += v[4 * q + 1];
                t.z = ex; ex += v[4 * q + 2];
                t.w = ex; ex += v[4 * q + 3];
                reinterpret_cast<uint4*>(arr + base)[q] = t;
            }
        } else {
#pragma unroll
            for (int k = 0; k < kCoopScanItems; ++k) {
                if (base + k < c1) arr[base + k] = ex;
                ex += v[k];
            }
        }
        run += total;
    }
}

// The cell index of every particle (dense: the cell id; with occ: its rank
// among the occupied cells) -- the hash of the kernel sequence.
template <int DIM, bool PACKED>
__device__ __forceinline__ uint32_t particle_cell(const CoopArgs& a, const float4& p) {
    uint32_t c = (uint32_t)cell_coord(p.x, a.g.lo[0], a.g.inv_w[0], a.g.n[0]);
    c += (uint32_t)a.g.n[0] * (uint32_t)cell_coord(p.y, a.g.lo[1], a.g.inv_w[1], a.g.n[1]);
    if (DIM == 3)
        c += (uint32_t)a.g.n[0] * (uint32_t)a.g.n[1] *
             (uint32_t)cell_coord(p.z, a.g.lo[2], a.g.inv_w[2], a.g.n[2]);
    return c;
}

// Scatter (original index, cell) into the particle's unordered slot.
__device__ __forceinline__ void coop_scatter(const CoopArgs& a, int64_t tid, int64_t nthreads) {
    const int64_t n = a.n;
    for (int64_t i0 = tid; i0 < n; i0 += nthreads * kCoopIlp) {
        uint2 cr[kCoopIlp];
#pragma unroll
        for (int u = 0; u < kCoopIlp; ++u) {
            const int64_t i = i0 + u * nthreads;
            cr[u] = i < n ? ldcg_u2(a.cell_rank + i) : make_uint2(0u, 0u);
        }
        uint32_t st[kCoopIlp];
#pragma unroll
        for (int u = 0; u < kCoopIlp; ++u)
            st[u] = i0 + u * nthreads < n ? ldcg_u32(a.cell_start + cr[u].x) : 0u;
#pragma unroll
        for (int u = 0; u < kCoopIlp; ++u) {
            const int64_t i = i0 + u * nthreads;
            if (i < n) a.tmp[st[u] + cr[u].y] = make_uint2((uint32_t)i, cr[u].x);
        }
    }
}

// Stable rank inside the cell (number of members with a smaller original
// index), then perm and the sorted positions.
template <int DIM, bool PACKED>
__device__ __forceinline__ void coop_finalize(const CoopArgs& a, int64_t tid, int64_t nthreads) {
    const int64_t n = a.n;
    for (int64_t s0 = tid; s0 < n; s0 += nthreads * kCoopIlp) {
        uint2 pc[kCoopIlp];
#pragma unroll
        for (int u = 0; u < kCoopIlp; ++u) {
            const int64_t s = s0 + u * nthreads;
            pc[u] = s < n ? ldcg_u2(a.tmp + s) : make_uint2(0u, 0u);
        }
        uint32_t lo[kCoopIlp], hi[kCoopIlp];
#pragma unroll
        for (int u = 0; u < kCoopIlp; ++u) {
            const bool live = s0 + u * nthreads < n;
            lo[u] = live ? ldcg_u32(a.cell_start + pc[u].y) : 0u;
            hi[u] = live ? ldcg_u32(a.cell_start + pc[u].y + 1) : 0u;
        }
        float4 q[kCoopIlp];
#pragma unroll
        for (int u = 0; u < kCoopIlp; ++u)
            q[u] = s0 + u * nthreads < n ? load_pos<DIM, PACKED>(a.pos, pc[u].x)
                                          : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
        for (int u = 0; u < kCoopIlp; ++u) {
            if (s0 + u * nthreads >= n) continue;
            uint32_t r = 0;
            for (uint32_t t = lo[u]; t < hi[u]; ++t) r += (__ldcg(&a.tmp[t].x) < pc[u].x) ? 1u : 0u;
            const uint32_t d = lo[u] + r;
            a.perm[d] = pc[u].x;
            a.spos[d] = make_float4(q[u].x, q[u].y, DIM == 3 ? q[u].z : 0.0f, 0.0f);
        }
    }
}

// Compact index of dense cell c: its rank among the occupied cells.
__device__ __forceinline__ uint32_t compact_index(const uint4* occ, uint32_t c) {
    const uint4 q = __ldcg(occ + (c >> 6));
    const uint64_t bits = ((uint64_t)q.y << 32) | q.x;
    return q.z + (uint32_t)__popcll(bits & ((1ull << (c & 63u)) - 1ull));
}

// Compact table: scatter the original index (4 bytes) into the particle's
// unordered slot.  The 4-byte slot array stays in L2 on large inputs where
// the 8-byte (index, cell) records of coop_scatter do not.
__device__ __forceinline__ void coop_scatter_idx(const CoopArgs& a, uint32_t* slot_idx,
                                                 int64_t tid, int64_t nthreads) {
    const int64_t n = a.n;
    for (int64_t i0 = tid; i0 < n; i0 += nthreads * kCoopIlp) {
        uint2 kr[kCoopIlp];
#pragma unroll
        for (int u = 0; u < kCoopIlp; ++u) {
            const int64_t i = i0 + u * nthreads;
            kr[u] = i < n ? ldcg_u2(a.cell_rank + i) : make_uint2(0u, 0u);
        }
        uint32_t st[kCoopIlp];
#pragma unroll
        for (int u = 0; u < kCoopIlp; ++u)
            st[u] = i0 + u * nthreads < n ? ldcg_u32(a.cell_start + kr[u].x) : 0u;
#pragma unroll
        for (int u = 0; u < kCoopIlp; ++u) {
            const int64_t i = i0 + u * nthreads;
            if (i < n) slot_idx[st[u] + kr[u].y] = (uint32_t)i;
        }
    }
}

// Compact table: the stable finalize from 4-byte slots.  The slot's cell is
// recomputed from the gathered position (the hash's expression, then the
// compact index), so the slot needs to carry only the original index.
template <int DIM, bool PACKED>
__device__ __forceinline__ void coop_finalize_idx(const CoopArgs& a, const uint32_t* slot_idx,
                                                  int64_t tid, int64_t nthreads) {
    const int64_t n = a.n;
    for (int64_t s0 = tid; s0 < n; s0 += nthreads * kCoopIlp) {
        uint32_t p[kCoopIlp];
#pragma unroll
        for (int u = 0; u < kCoopIlp; ++u) {
            const int64_t s = s0 + u * nthreads;
            p[u] = s < n ? ldcg_u32(slot_idx + s) : 0u;
        }
        float4 q[kCoopIlp];
#pragma unroll
        for (int u = 0; u < kCoopIlp; ++u)
            q[u] = s0 + u * nthreads < n ? load_pos<DIM, PACKED>(a.pos, p[u])
                                          : make_float4(0.f, 0.f, 0.f, 0.f);
        uint32_t k[kCoopIlp];
#pragma unroll
        for (int u = 0; u < kCoopIlp; ++u) k[u] = compact_index(a.occ, particle_cell<DIM, PACKED>(a, q[u]));
        uint32_t lo[kCoopIlp], hi[kCoopIlp];
#pragma unroll
        for (int u = 0; u < kCoopIlp; ++u) {
            const bool live = s0 + u * nthreads < n;
            lo[u] = live ? ldcg_u32(a.cell_start + k[u]) : 0u;
            hi[u] = live ? ldcg_u32(a.cell_start + k[u] + 1) : 0u;
        }
#pragma unroll
        for (int u = 0; u < kCoopIlp; ++u) {
            if (s0 + u * nthreads >= n) continue;
            uint32_t r = 0;
            for (uint32_t t = lo[u]; t < hi[u]; ++t) r += (ldcg_u32(slot_idx + t) < p[u]) ? 1u : 0u;
            const uint32_t d = lo[u] + r;
            a.perm[d] = p[u];
            a.spos[d] = make_float4(q[u].x, q[u].y, DIM == 3 ? q[u].z : 0.0f, 0.0f);
        }
    }
}

template <int DIM, bool PACKED>
__global__ void __launch_bounds__(kCoopThreads, 1)
k_build_coop(CoopArgs a) {
    // the pair kernel that follows may be scheduled now (it waits for this
    // grid to finish before reading anything)
    asm volatile("griddepcontrol.launch_dependents;");
    __shared__ uint32_t s_warp[32];
    __shared__ uint32_t s_red[32];
    const int64_t n = a.n;
    const int64_t tid = (int64_t)blockIdx.x * kCoopThreads + threadIdx.x;
    const int64_t nthreads = (int64_t)gridDim.x * kCoopThreads;

    // P0: zero the counts
    for (int64_t c = tid; c < a.nc1; c += nthreads) a.cell_start[c] = 0u;
    coop_barrier(a.bar, a.err, a.limit_ns, (int)blockIdx.x == a.skip_block);

    // P1: cell hash + histogram; the atomic's return is the arrival rank
    for (int64_t i0 = tid; i0 < n; i0 += nthreads * kCoopIlp) {
        uint32_t c[kCoopIlp], r[kCoopIlp];
#pragma unroll
        for (int u = 0; u < kCoopIlp; ++u) {
            const int64_t i = i0 + u * nthreads;
            c[u] = particle_cell<DIM, PACKED>(a, i < n ? load_pos<DIM, PACKED>(a.pos, i)
                                                         : make_float4(0.f, 0.f, 0.f, 0.f));
        }
#pragma unroll
        for (int u = 0; u < kCoopIlp; ++u)
            if (i0 + u * nthreads < n) r[u] = atomicAdd(a.cell_start + c[u], 1u);
#pragma unroll
        for (int u = 0; u < kCoopIlp; ++u) {
            const int64_t i = i0 + u * nthreads;
            if (i < n) a.cell_rank[i] = make_uint2(c[u], r[u]);
        }
    }
    coop_barrier(a.bar, a.err, a.limit_ns);

    // P2: counts -> offsets (entry n_cells is 0, so the last offset is n)
    coop_scan_u32(a.cell_start, a.nc1, a, s_warp, s_red);
    coop_barrier(a.bar, a.err, a.limit_ns);

    // P3: scatter; P4: stable finalize
    coop_scatter(a, tid, nthreads);
    coop_barrier(a.bar, a.err, a.limit_ns);
    coop_finalize<DIM, PACKED>(a, tid, nthreads);
}

template <int DIM, bool PACKED>
__global__ void __launch_bounds__(kCoopThreads, 1)
k_build_coop_compact(CoopArgs a) {
    // the pair kernel that follows may be scheduled now (it waits for this
    // grid to finish before reading anything)
    asm volatile("griddepcontrol.launch_dependents;");
    __shared__ uint32_t s_warp[32];
    __shared__ uint32_t s_red[32];
    const int64_t n = a.n;
    const int64_t tid = (int64_t)blockIdx.x * kCoopThreads + threadIdx.x;
    const int64_t nthreads = (int64_t)gridDim.x * kCoopThreads;

    // P0: clear the occupancy words and the per-occupied-cell counts (at
    // most n occupied cells, plus the end entry)
    for (int64_t w = tid; w < a.n_words; w += nthreads) a.occ[w] = make_uint4(0u, 0u, 0u, 0u);
    for (int64_t c = tid; c <= n; c += nthreads) a.cell_start[c] = 0u;
    coop_barrier(a.bar, a.err, a.limit_ns, (int)blockIdx.x == a.skip_block);

    // 4-byte per-particle words in the slot buffer: the cell id (P1 -> P3),
    // then the original index of each unordered slot (P5 -> P6)
    uint32_t* const idx32 = reinterpret_cast<uint32_t*>(a.tmp);

    // P1: cell hash; mark the cell occupied, keep its id
    for (int64_t i0 = tid; i0 < n; i0 += nthreads * kCoopIlp) {
        uint32_t c[kCoopIlp];
#pragma unroll
        for (int u = 0; u < kCoopIlp; ++u) {
            const int64_t i = i0 + u * nthreads;
            c[u] = particle_cell<DIM, PACKED>(a, i < n ? load_pos<DIM, PACKED>(a.pos, i)
                                                         : make_float4(0.f, 0.f, 0.f, 0.f));
        }
#pragma unroll
        for (int u = 0; u < kCoopIlp; ++u) {
            const int64_t i = i0 + u * nthreads;
            if (i >= n) continue;
            atomicOr(reinterpret_cast<unsigned long long*>(a.occ + (c[u] >> 6)), 1ull << (c[u] & 63u));
            idx32[i] = c[u];
        }
    }
    coop_barrier(a.bar, a.err, a.limit_ns);

    // P2: occupied cells before each word (exclusive scan of the words'
    // popcounts, into occ[w].z)
    {
        const int64_t chunk = (a.n_words + gridDim.x - 1) / gridDim.x;
        const int64_t w0 = (int64_t)blockIdx.x * chunk;
        const int64_t w1 = w0 + chunk < a.n_words ? w0 + chunk : a.n_words;
        uint32_t sum = 0;
        for (int64_t w = w0 + threadIdx.x; w < w1; w += kCoopThreads) {
            const uint4 q = __ldcg(a.occ + w);
            sum += (uint32_t)__popc(q.x) + (uint32_t)__popc(q.y);
        }
        const uint32_t t = block_sum_u32(sum, s_red);
        if (threadIdx.x == 0) a.block_sum[blockIdx.x] = t;
        coop_barrier(a.bar, a.err, a.limit_ns);
        uint32_t run = earlier_blocks(a.block_sum, s_red);
        for (int64_t t0 = w0; t0 < w1; t0 += kCoopThreads) {
            const int64_t w = t0 + threadIdx.x;
            uint4 q = make_uint4(0u, 0u, 0u, 0u);
            if (w < w1) q = __ldcg(a.occ + w);
            const uint32_t v = (uint32_t)__popc(q.x) + (uint32_t)__popc(q.y);
            uint32_t total;
            const uint32_t ex = run + block_excl_scan(v, s_warp, &total);
            if (w < w1) a.occ[w].z = ex;
            run += total;
        }
    }
    coop_barrier(a.bar, a.err, a.limit_ns);

    // P3: compact index of each particle's cell; arrival rank in it
    for (int64_t i0 = tid; i0 < n; i0 += nthreads * kCoopIlp) {
        uint32_t c[kCoopIlp], k[kCoopIlp], r[kCoopIlp];
#pragma unroll
        for (int u = 0; u < kCoopIlp; ++u) {
            const int64_t i = i0 + u * nthreads;
            c[u] = i < n ? ldcg_u32(idx32 + i) : 0u;
        }
#pragma unroll
        for (int u = 0; u < kCoopIlp; ++u) k[u] = compact_index(a.occ, c[u]);
#pragma unroll
        for (int u = 0; u < kCoopIlp; ++u)
            if (i0 + u * nthreads < n) r[u] = atomicAdd(a.cell_start + k[u], 1u);
#pragma unroll
        for (int u = 0; u < kCoopIlp; ++u) {
            const int64_t i = i0 + u * nthreads;
            if (i < n) a.cell_rank[i] = make_uint2(k[u], r[u]);
        }
    }
    coop_barrier(a.bar, a.err, a.limit_ns);

    // P4: counts -> offsets of the occupied cells (entries past the last
    // occupied cell are 0, so they all become n)
    coop_scan_u32(a.cell_start, n + 1, a, s_warp, s_red);
    coop_barrier(a.bar, a.err, a.limit_ns);

    // P5: scatter; P6: stable finalize (over compact indices)
    coop_scatter_idx(a, idx32, tid, nthreads);
    coop_barrier(a.bar, a.err, a.limit_ns);
    coop_finalize_idx<DIM, PACKED>(a, idx32, tid, nthreads);
}

// Dense offsets of a compact cell list (inspection and export).
__global__ void __launch_bounds__(kThreads)
k_expand_cells(int64_t nc1, const uint4* __restrict__ occ, const uint32_t* __restrict__ cstart,
               uint32_t* __restrict__ out) {
    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < nc1;
         c += (int64_t)gridDim.x * blockDim.x) {
        const uint4 q = occ[c >> 6];
        const uint64_t bits = ((uint64_t)q.y << 32) | q.x;
        out[c] = cstart[q.z + (uint32_t)__popcll(bits & ((1ull << (c & 63)) - 1ull))];
    }
}

}  // namespace

size_t scan_tiles(int64_t n) { return (size_t)((n + kScanTile - 1) / kScanTile); }

template <typename TOut>
static cudaError_t scan_impl(const uint32_t* in, TOut* out, int64_t n,
                             uint64_t* status, uint32_t* ticket, uint32_t* err,
                             int skip_tile, long long limit_ns, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    size_t tiles = scan_tiles(n);
    cudaError_t e = cudaMemsetAsync(status, 0, tiles * sizeof(uint64_t), st);
    if (e != cudaSuccess) return e;
    e = cudaMemsetAsync(ticket, 0, sizeof(uint32_t), st);
    if (e != cudaSuccess) return e;
    k_scan<TOut><<<(unsigned)tiles, kThreads, 0, st>>>(in, out, n, status, ticket,
                                                       err, skip_tile, limit_ns);
    return cudaGetLastError();
}

// One second: a normal look-back waits microseconds.
static const long long kScanLimitNs = 1000000000ll;

cudaError_t launch_scan_u32(const uint32_t* in, uint32_t* out, int64_t n,
                            uint64_t* status, uint32_t* ticket, uint32_t* err,
                            int skip_tile, long long limit_ns, cudaStream_t st) {
    return scan_impl<uint32_t>(in, out, n, status, ticket, err, skip_tile,
                               limit_ns > 0 ? limit_ns : kScanLimitNs, st);
}

cudaError_t launch_scan_u32_to_i64(const uint32_t* in, int64_t* out, int64_t n,
                                   uint64_t* status, uint32_t* ticket,
                                   uint32_t* err, cudaStream_t st) {
    return scan_impl<int64_t>(in, out, n, status, ticket, err, -1, kScanLimitNs, st);
}

cudaError_t launch_reduce_partials(const double* partial, int count, double* out,
                                   cudaStream_t st) {
    // programmatic dependent launch: the one-block reduction is scheduled
    // while the kernel before it runs its last wave (the pair kernels signal
    // launch_dependents at their start) and waits in griddepcontrol.wait, so
    // its launch latency is hidden
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(1);
    cfg.blockDim = dim3(kRedThreads);
    cfg.stream = st;
    cudaLaunchAttribute attr;
    attr.id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr.val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = &attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k_reduce_partials, partial, count, out);
}

// Grid of the cooperative build: every block resident (one 1024-thread block
// per SM at most), and no more blocks than there is work for.
static int coop_grid(const void* fn, int64_t n, int64_t nc1) {
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kCoopThreads, 0) != cudaSuccess ||
        per_sm < 1) {
        cudaGetLastError();
        return 0;
    }
    const int64_t resident = (int64_t)per_sm * num_sms();
    const int64_t work = n > nc1 ? n : nc1;
    int64_t want = (work + (int64_t)kCoopThreads * kCoopIlp - 1) / ((int64_t)kCoopThreads * kCoopIlp);
    if (want < 1) want = 1;
    return (int)(want < resident ? want : resident);
}

size_t coop_scratch_words() { return 2 + 4096; }   // barrier words + block sums

// The counting sort in one launch where the device allows it (the kernel
// sequence above 2^21 particles with a dense table).  The radix sort of
// ab_sort.cu gives the same cell list and is selected only on request: it
// measured slower on every workload here (1M uniform points 98 vs 54 us,
// 16.7M clustered 857-877 vs 844-857 us, 4M 2-D points 241 vs 168 us).
int auto_build_path(int64_t n, const Geom& g) {
    (void)n;
    (void)g;
    return kPathCoop;
}

cudaError_t launch_build(CellList& cl, const float* pos, bool packed, Scratch& sc,
                         uint32_t* err, cudaStream_t st, const BuildOptions& opt) {
    const int64_t n = cl.n;
    const int64_t nc = cl.g.n_cells;
    const bool compact = cl.g.compact != 0;
    // One cooperative launch when the device allows it: always for the
    // compact table (it has no kernel-sequence form), and for a dense table
    // up to kSingleLaunchMaxN particles.  The cooperative grid holds one
    // 1024-thread block per SM (62 registers a thread); above ~2M particles
    // the kernel sequence's full occupancy keeps more loads in flight than
    // the saved launches are worth (measured: 1M uniform points 53.9 vs
    // 56.4 us; 4M points in 2-D 176.8 vs 167.6 us).
    constexpr int64_t kSingleLaunchMaxN = int64_t(1) << 21;
    const int path = opt.path == kPathAuto ? auto_build_path(n, cl.g) : opt.path;
    if (path == kPathRadix && radix_supported(n, nc))
        return launch_build_radix(cl, pos, packed, sc, err, st, opt);
    if (sc.coop && (compact || (path != kPathSequence && n <= kSingleLaunchMaxN))) {
        const void* fn;
        if (compact) {
            if (cl.g.dim == 3) fn = packed ? (const void*)k_build_coop_compact<3, true> : (const void*)k_build_coop_compact<3, false>;
            else fn = packed ? (const void*)k_build_coop_compact<2, true> : (const void*)k_build_coop_compact<2, false>;
        } else {
            if (cl.g.dim == 3) fn = packed ? (const void*)k_build_coop<3, true> : (const void*)k_build_coop<3, false>;
            else fn = packed ? (const void*)k_build_coop<2, true> : (const void*)k_build_coop<2, false>;
        }
        const int64_t n_words = occ_words(nc);
        const int grid = coop_grid(fn, n, compact ? n_words : nc + 1);
        if (grid >= 1 && grid <= 4096) {
            CoopArgs a;
            a.pos = pos;
            a.n = n;
            a.g = cl.g;
            a.nc1 = nc + 1;
            a.cell_start = cl.cell_start;
            a.occ = cl.occ;
            a.n_words = n_words;
            a.cell_rank = cl.cell_rank;
            a.tmp = reinterpret_cast<uint2*>(cl.tmp);
            a.perm = cl.perm;
            a.spos = cl.spos;
            a.bar = sc.coop;
            a.block_sum = sc.coop + 2;
            a.err = err;
            a.limit_ns = opt.limit_ns > 0 ? opt.limit_ns : kScanLimitNs;
            a.skip_block = opt.skip_block < grid ? opt.skip_block : -1;
            cudaError_t e = cudaMemsetAsync(sc.coop, 0, 2 * sizeof(uint32_t), st);
            if (e != cudaSuccess) return e;
            void* args[] = {&a};
            e = cudaLaunchCooperativeKernel(fn, dim3((unsigned)grid), dim3(kCoopThreads), args, 0, st);
            if (e == cudaSuccess || compact) return e;
            cudaGetLastError();   // not launchable here: fall back to the kernel sequence
        }
        if (compact) return cudaErrorNotSupported;
    }
    if (compact) return cudaErrorNotSupported;
    cudaError_t e = cudaMemsetAsync(cl.cell_start, 0, (size_t)(nc + 1) * sizeof(uint32_t), st);
    if (e != cudaSuccess) return e;
    if (n > 0) {
        const int gr = ew_grid(n);
        if (cl.g.dim == 3) {
            if (packed) k_hash<3, true><<<gr, kThreads, 0, st>>>(pos, n, cl.g, cl.cell_rank, cl.cell_start);
            else k_hash<3, false><<<gr, kThreads, 0, st>>>(pos, n, cl.g, cl.cell_rank, cl.cell_start);
        } else {
            if (packed) k_hash<2, true><<<gr, kThreads, 0, st>>>(pos, n, cl.g, cl.cell_rank, cl.cell_start);
            else k_hash<2, false><<<gr, kThreads, 0, st>>>(pos, n, cl.g, cl.cell_rank, cl.cell_start);
        }
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    // counts -> offsets in place; entry nc is 0 so cell_start[nc] = n.
    e = launch_scan_u32(cl.cell_start, cl.cell_start, nc + 1, sc.scan_status,
                        sc.scan_ticket, err, -1, 0, st);
    if (e != cudaSuccess) return e;
    if (n > 0) {
        uint2* tmp = reinterpret_cast<uint2*>(cl.tmp);   // 8 bytes a particle
        k_scatter<<<ew_grid(n), kThreads, 0, st>>>(n, cl.cell_rank, cl.cell_start, tmp);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        const int gr = ew_grid(n);
        if (cl.g.dim == 3) {
            if (packed) k_finalize<3, true><<<gr, kThreads, 0, st>>>(n, pos, cl.cell_start, tmp, cl.perm, cl.spos);
            else k_finalize<3, false><<<gr, kThreads, 0, st>>>(n, pos, cl.cell_start, tmp, cl.perm, cl.spos);
        } else {
            if (packed) k_finalize<2, true><<<gr, kThreads, 0, st>>>(n, pos, cl.cell_start, tmp, cl.perm, cl.spos);
            else k_finalize<2, false><<<gr, kThreads, 0, st>>>(n, pos, cl.cell_start, tmp, cl.perm, cl.spos);
        }
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    return cudaSuccess;
}

cudaError_t launch_expand_cells(const CellList& cl, uint32_t* out, cudaStream_t st) {
    const int64_t nc1 = cl.g.n_cells + 1;
    k_expand_cells<<<ew_grid(nc1), kThreads, 0, st>>>(nc1, cl.occ, cl.cell_start, out);
    return cudaGetLastError();
}

// A per-particle scalar in sorted order: out[s] = v[perm[s]].
__global__ void __launch_bounds__(kThreads)
k_gather_scalar(int64_t n, const uint32_t* __restrict__ perm, const float* __restrict__ v,
                float* __restrict__ out) {
    for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < n;
         s += (int64_t)gridDim.x * blockDim.x)
        out[s] = __ldg(v + perm[s]);
}

cudaError_t launch_gather_scalar(const CellList& cl, const float* v, float* out, cudaStream_t st) {
    if (cl.n <= 0) return cudaSuccess;
    k_gather_scalar<<<ew_grid(cl.n), kThreads, 0, st>>>(cl.n, cl.perm, v, out);
    return cudaGetLastError();
}

cudaError_t launch_gather_w_pos(CellList& cl, const float* w, cudaStream_t st) {
    if (cl.n <= 0) return cudaSuccess;
    k_gather_w_pos<<<ew_grid(cl.n), kThreads, 0, st>>>(cl.n, cl.perm, w, cl.spos);
    return cudaGetLastError();
}

cudaError_t launch_gather_pairs(const CellList& cl, const float2* wv, float2* sv,
                                cudaStream_t st) {
    if (cl.n <= 0) return cudaSuccess;
    k_gather_pairs<<<ew_grid(cl.n), kThreads, 0, st>>>(cl.n, cl.perm, wv, sv);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Allocation-free variant of the cell-offset scan (ab_exclusive_scan_u32_static
// in include/aboria_gpu.h).  The look-back state lives in a file-scope
// __device__ array instead of context workspace, so the call needs no
// cudaMalloc and no context.  Every GPU that loads the library keeps this
// array (about 32 KB) until the process exits.
// ---------------------------------------------------------------------------
constexpr int64_t kStaticScanMaxTiles = 4096;
constexpr int64_t kStaticScanMaxItems = kStaticScanMaxTiles * kScanTile;  // 2^24

struct StaticScanScratch {
    uint64_t status[kStaticScanMaxTiles];
    uint32_t ticket;
    uint32_t err;
};

static __device__ __align__(256) StaticScanScratch g_static_scan;

// After the scan: a wait that gave up is reported through the output itself
// (out[0] of an exclusive scan is always 0, so 0xFFFFFFFF there is
// unambiguous), and the error word is cleared for the next call.
__global__ void k_static_scan_check(uint32_t* out, uint32_t* err) {
    if (*err) {
        out[0] = 0xFFFFFFFFu;
        *err = 0;
    }
}

namespace {
constexpr int kMaxDevices = 64;
std::mutex g_static_mu;
StaticScanScratch* g_static_ptr[kMaxDevices] = {};
}  // namespace

// Device address of g_static_scan on the current device, looked up once per
// device.  In host code the symbol itself is only a host-side stand-in.
static cudaError_t static_scan_scratch(StaticScanScratch** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lk(g_static_mu);
    if (!g_static_ptr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_static_scan);
        if (e != cudaSuccess) return e;
        g_static_ptr[dev] = (StaticScanScratch*)p;
    }
    *out = g_static_ptr[dev];
    return cudaSuccess;
}

}  // namespace ab

#pragma GCC visibility push(default)
extern "C" ab_status ab_exclusive_scan_u32_static(const uint32_t* in, uint32_t* out,
                                                  int64_t n, void* stream) {
    if (n < 0 || n > ab::kStaticScanMaxItems) return AB_ERR_INVALID_ARG;
    if (n == 0) return AB_OK;
    if (!in || !out || ((uintptr_t)in & 3u) || ((uintptr_t)out & 3u)) return AB_ERR_INVALID_ARG;
    const uintptr_t a0 = (uintptr_t)in, b0 = (uintptr_t)out, nb = (uintptr_t)n * 4u;
    if (a0 != b0 && a0 < b0 + nb && b0 < a0 + nb) return AB_ERR_ALIAS;  // partial overlap
    ab::StaticScanScratch* sc = nullptr;
    cudaError_t e = ab::static_scan_scratch(&sc);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return AB_ERR_CUDA;
    }
    cudaStream_t st = (cudaStream_t)stream;
    const size_t tiles = ab::scan_tiles(n);
    // the array keeps the previous call's contents: reset what must start at 0
    e = cudaMemsetAsync(sc->status, 0, tiles * sizeof(uint64_t), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(&sc->ticket, 0, sizeof(uint32_t), st);
    if (e == cudaSuccess) {
        ab::k_scan<uint32_t><<<(unsigned)tiles, ab::kThreads, 0, st>>>(
            in, out, n, sc->status, &sc->ticket, &sc->err, -1, ab::kScanLimitNs);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) {
        ab::k_static_scan_check<<<1, 1, 0, st>>>(out, &sc->err);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) {
        cudaGetLastError();
        return AB_ERR_CUDA;
    }
    return AB_OK;
}
#pragma GCC visibility pop
