// Cell-list build by a stable least-significant-digit radix sort of the
// particles' cell ids (paper Sec. 2.2.1: the particles are reordered so that
// the particles of each cell are contiguous; Sec. 3: cells of width r_cut).
//
// The counting sort of ab_cells.cu takes one global atomic per particle for
// its histogram (and, for the compacted table, one more for the occupancy
// bits); on large and clustered inputs those atomics are most of the build.
// This build takes no per-particle global atomic:
//   1. keys: each particle's cell id (the counting sort's hash), and each
//      tile's count of the first digit (tile = 4096 keys, shared-memory
//      counts), stored bin-major: counts[d * tiles + t];
//   2. one pass per digit of up to 10 bits, least significant first: the
//      tiles' counts of the digit (from the previous pass's output), one
//      exclusive scan of the bin-major counts -- a single-pass scan with
//      decoupled look-back (Merrill & Garland, 2016) -- which gives every
//      tile the global slot of its first key of each digit, then the pass
//      itself: each warp ranks its 256 keys in order, 32 at a time, equal
//      digits grouped by one ballot per digit bit (stable), the tile stages
//      its keys in digit order in shared memory and writes each digit's run
//      to consecutive global slots.  The last pass writes the permutation
//      and gathers the positions into sorted order.  Every pass is stable
//      and the first starts from original order, so the particles of a cell
//      keep increasing original index: the sorted order, and hence the cell
//      list, is the counting sort's bit for bit;
//   3. cell boundaries: a sorted particle whose key differs from its
//      predecessor's starts an occupied cell; its rank among the boundaries
//      (a look-back scan) indexes the offsets of the occupied cells, and its
//      cell's bit is set in the occupancy words;
//   4. the number of occupied cells before each occupancy word (look-back
//      scan over the words' popcounts);
//   5. dense table only: every cell's offset from the occupied cells'.
// Look-back state words carry a 30-bit epoch, unique to one launch, so the
// status array needs no clearing between launches.  Every wait on another
// tile is bounded by a wall-clock limit after which the tile latches
// DEVERR_SCAN_TIMEOUT and carries on (the results are then garbage, but
// every access is checked to stay in its array and every tile terminates).
// Scan tiles take increasing ids from a ticket counter, so a tile only ever
// waits on tiles that are already running.
#include <cuda_runtime.h>
#include <stdint.h>

#include "ab_internal.cuh"

namespace ab {

namespace {

constexpr int kRsThreads = 512;
constexpr int kRsWarps = kRsThreads / 32;
constexpr int kRsItems = 8;                               // keys per thread
constexpr int kRsTile = kRsThreads * kRsItems;            // 4096 keys a tile
constexpr int kRsWarpItems = kRsTile / kRsWarps;          // 256 keys a warp
constexpr int kRsMaxBits = 10;
constexpr int kRsMaxBins = 1 << kRsMaxBits;
constexpr int kRsBinsPerThread = kRsMaxBins / kRsThreads; // 2 consecutive bins
constexpr int kRsMaxPasses = 4;
constexpr int kRsZItems = 8;                              // occupancy words per thread
constexpr int kRsZTile = kRsThreads * kRsZItems;
// ticket counters of the look-back scans (one per digit pass, the boundary
// scan and the occupancy scan)
constexpr int kRsTickets = 8;
constexpr size_t kRsSmallWords = kRsTickets;
// dynamic shared memory of a pass: per-warp digit counts (u16), staged keys
// and values, per-digit output offsets
constexpr size_t kRsPassSmem = (size_t)kRsWarps * kRsMaxBins * sizeof(uint16_t) +
                               2 * (size_t)kRsTile * sizeof(uint32_t) +
                               (size_t)kRsMaxBins * sizeof(uint32_t);

// look-back state word: [63:34] epoch, [33:32] flag, [31:0] value
constexpr uint64_t kRsAgg = 1ull << 32;   // the tile's own count
constexpr uint64_t kRsPre = 2ull << 32;   // inclusive prefix through the tile
constexpr uint32_t kRsEpochMask = (1u << 30) - 1u;

__device__ __forceinline__ uint64_t rs_word(uint32_t epoch, uint64_t flag, uint32_t v) {
    return ((uint64_t)epoch << 34) | flag | (uint64_t)v;
}
__device__ __forceinline__ void rs_st_release(uint64_t* p, uint64_t v) {
    asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ uint64_t rs_ld_acquire(const uint64_t* p) {
    uint64_t v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ long long rs_now_ns() {
    long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

struct RsPlan {
    int passes;
    int shift[kRsMaxPasses];
    int bits[kRsMaxPasses];
};

// Position i of the caller's array: float4 records or PACKED DIM floats.
template <int DIM, bool PACKED>
__device__ __forceinline__ float4 rs_load_pos(const float* __restrict__ pos, int64_t i) {
    if (!PACKED) return __ldg(reinterpret_cast<const float4*>(pos) + i);
    const float* q = pos + i * DIM;
    return make_float4(__ldg(q), __ldg(q + 1), DIM == 3 ? __ldg(q + 2) : 0.0f, 0.0f);
}

// The particle's cell id: the same expression as the counting sort's hash.
template <int DIM>
__device__ __forceinline__ uint32_t rs_cell(const Geom& g, const float4& p) {
    uint32_t c = (uint32_t)cell_coord(p.x, g.lo[0], g.inv_w[0], g.n[0]);
    c += (uint32_t)g.n[0] * (uint32_t)cell_coord(p.y, g.lo[1], g.inv_w[1], g.n[1]);
    if (DIM == 3)
        c += (uint32_t)g.n[0] * (uint32_t)g.n[1] *
             (uint32_t)cell_coord(p.z, g.lo[2], g.inv_w[2], g.n[2]);
    return c;
}

// Block-wide exclusive scan of one 64-bit value per thread (kRsThreads).
__device__ __forceinline__ uint64_t rs_block_scan(uint64_t v, uint64_t* s_warp, uint64_t* total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint64_t incl = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint64_t t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += t;
    }
    if (lane == 31) s_warp[warp] = incl;
    __syncthreads();
    uint64_t before = 0, all = 0;
#pragma unroll
    for (int w = 0; w < kRsWarps; ++w) {
        const uint64_t t = s_warp[w];
        if (w < warp) before += t;
        all += t;
    }
    *total = all;
    __syncthreads();   // s_warp is reused by the next call
    return before + incl - v;
}

// Decoupled look-back for one value per tile, by warp 0: lane l polls the
// word of tile j - l, so 32 predecessors are examined per poll.  Publishes
// the tile's aggregate first and its inclusive prefix last; returns the
// exclusive prefix (valid in lane 0).
__device__ __forceinline__ uint32_t rs_look_back_warp(uint64_t* status, int64_t tile,
                                                      uint32_t total, uint32_t epoch,
                                                      uint32_t* err, long long limit_ns) {
    const int lane = threadIdx.x & 31;
    uint32_t excl = 0;
    if (tile == 0) {
        if (lane == 0) rs_st_release(status, rs_word(epoch, kRsPre, total));
        return 0;
    }
    if (lane == 0) rs_st_release(status + tile, rs_word(epoch, kRsAgg, total));
    const long long t0 = rs_now_ns();
    int64_t j = tile - 1;
    for (;;) {
        const int64_t idx = j - lane;
        const uint64_t w = idx >= 0 ? rs_ld_acquire(status + idx) : rs_word(epoch, kRsPre, 0u);
        const bool ready = (uint32_t)(w >> 34) == epoch;
        const unsigned pre = __ballot_sync(0xffffffffu, ready && (w & kRsPre));
        const unsigned notready = __ballot_sync(0xffffffffu, !ready);
        const int first = pre ? __ffs(pre) - 1 : 31;
        const unsigned upto = first == 31 ? 0xffffffffu : ((1u << (first + 1)) - 1u);
        if (notready & upto) {   // a tile in the window has not published yet
            // one decision for the whole warp (the lanes' clock reads differ)
            if (__any_sync(0xffffffffu, rs_now_ns() - t0 > limit_ns)) {
                if (lane == 0) atomicOr(err, DEVERR_SCAN_TIMEOUT);
                break;
            }
            continue;
        }
        uint32_t part = ((upto >> lane) & 1u) ? (uint32_t)w : 0u;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
        excl += part;
        if (pre) break;
        j -= 32;
    }
    if (lane == 0) rs_st_release(status + tile, rs_word(epoch, kRsPre, excl + total));
    return excl;
}

// For each of the thread's kRsItems keys (one per round of 32 consecutive
// keys of the warp): the lanes of the warp whose key in that round has the
// same digit (shift, bits), among the lanes with ok set (0 for a lane
// without).  One ballot per digit bit and round, the rounds interleaved so
// that their ballots are independent (one __match_any_sync per round measured
// several times slower).
__device__ __forceinline__ void rs_match(const uint32_t (&key)[kRsItems], const bool (&ok)[kRsItems],
                                         int shift, int bits, uint32_t (&peers)[kRsItems]) {
#pragma unroll
    for (int r = 0; r < kRsItems; ++r) peers[r] = __ballot_sync(0xffffffffu, ok[r]);
    for (int b = 0; b < bits; ++b) {
#pragma unroll
        for (int r = 0; r < kRsItems; ++r) {
            const bool bit = (key[r] >> (shift + b)) & 1u;
            const uint32_t x = __ballot_sync(0xffffffffu, bit);
            peers[r] &= bit ? x : ~x;
        }
    }
#pragma unroll
    for (int r = 0; r < kRsItems; ++r)
        if (!ok[r]) peers[r] = 0u;
}

// Adds the thread's keys (ok set) to the shared histogram h of the digit at
// (shift, bits).  Plain shared-memory atomics: in every pass the keys of one
// round have distinct digits almost always (the first pass takes the low
// bits of unsorted cell ids; later passes take bits above the ones the
// previous pass sorted by), and a ballot match per round measured ~3x slower.
__device__ __forceinline__ void rs_count(uint32_t* h, const uint32_t (&key)[kRsItems],
                                         const bool (&ok)[kRsItems], int shift, int bits) {
    const uint32_t m = (1u << bits) - 1u;
#pragma unroll
    for (int r = 0; r < kRsItems; ++r)
        if (ok[r]) atomicAdd(h + ((key[r] >> shift) & m), 1u);
}

// ---------------------------------------------------------------------------
// 1. keys, and the first digit's count in every tile (tile = block); also
//    clears the occupancy words
// counts are bin-major: counts[d * tiles + tile]
// ---------------------------------------------------------------------------
template <int DIM, bool PACKED>
__global__ void __launch_bounds__(kRsThreads)
k_rs_keys(const float* __restrict__ pos, int64_t n, Geom g, int bits,
          uint32_t* __restrict__ keys, uint32_t* __restrict__ counts, int64_t tiles,
          uint4* __restrict__ occ, int64_t n_words) {
    __shared__ uint32_t h[kRsMaxBins];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint32_t bins = 1u << bits;
    for (uint32_t i = tid; i < bins; i += kRsThreads) h[i] = 0u;
    for (int64_t w = (int64_t)blockIdx.x * kRsThreads + tid; w < n_words;
         w += (int64_t)gridDim.x * kRsThreads)
        occ[w] = make_uint4(0u, 0u, 0u, 0u);
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * kRsTile + warp * kRsWarpItems;
    uint32_t key[kRsItems];
    bool ok[kRsItems];
#pragma unroll
    for (int r = 0; r < kRsItems; ++r) {
        const int64_t i = base + r * 32 + lane;
        ok[r] = i < n;
        key[r] = ok[r] ? rs_cell<DIM>(g, rs_load_pos<DIM, PACKED>(pos, i)) : 0u;
    }
#pragma unroll
    for (int r = 0; r < kRsItems; ++r)
        if (ok[r]) keys[base + r * 32 + lane] = key[r];
    rs_count(h, key, ok, 0, bits);
    __syncthreads();
    for (uint32_t d = tid; d < bins; d += kRsThreads) counts[(int64_t)d * tiles + blockIdx.x] = h[d];
}

// ---------------------------------------------------------------------------
// 2a. a later digit's count in every tile of the previous pass's output
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kRsThreads)
k_rs_up(const uint32_t* __restrict__ keys, int64_t n, int shift, int bits,
        uint32_t* __restrict__ counts, int64_t tiles) {
    __shared__ uint32_t h[kRsMaxBins];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint32_t bins = 1u << bits;
    for (uint32_t i = tid; i < bins; i += kRsThreads) h[i] = 0u;
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * kRsTile + warp * kRsWarpItems;
    uint32_t key[kRsItems];
    bool ok[kRsItems];
#pragma unroll
    for (int r = 0; r < kRsItems; ++r) {
        const int64_t i = base + r * 32 + lane;
        ok[r] = i < n;
        key[r] = ok[r] ? keys[i] : 0u;
    }
    rs_count(h, key, ok, shift, bits);
    __syncthreads();
    for (uint32_t d = tid; d < bins; d += kRsThreads) counts[(int64_t)d * tiles + blockIdx.x] = h[d];
}

// ---------------------------------------------------------------------------
// 2b. exclusive scan of the bin-major counts: counts[d * tiles + t] becomes
//     the global slot of tile t's first key of digit d
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kRsThreads)
k_rs_scan(uint32_t* counts, int64_t len, uint64_t* status, uint32_t* ticket, uint32_t epoch,
          uint32_t* err, long long limit_ns, int64_t skip_tile) {
    __shared__ uint64_t s_scan[kRsWarps];
    __shared__ uint32_t s_tile, s_prefix;
    const int tid = threadIdx.x;
    if (tid == 0) s_tile = atomicAdd(ticket, 1u);
    __syncthreads();
    const int64_t tile = s_tile;
    const int64_t i0 = tile * kRsTile + (int64_t)tid * kRsItems;
    uint32_t v[kRsItems];
    uint32_t sum = 0;
    if (i0 + kRsItems <= len) {
#pragma unroll
        for (int q = 0; q < kRsItems / 4; ++q) {
            const uint4 t = reinterpret_cast<const uint4*>(counts + i0)[q];
            v[4 * q] = t.x;
            v[4 * q + 1] = t.y;
            v[4 * q + 2] = t.z;
            v[4 * q + 3] = t.w;
        }
    } else {
#pragma unroll
        for (int k = 0; k < kRsItems; ++k) v[k] = i0 + k < len ? counts[i0 + k] : 0u;
    }
#pragma unroll
    for (int k = 0; k < kRsItems; ++k) sum += v[k];
    uint64_t total;
    const uint32_t before = (uint32_t)rs_block_scan(sum, s_scan, &total);
    if (tid < 32) {
        uint32_t e = 0;
        if (tile != skip_tile)
            e = rs_look_back_warp(status, tile, (uint32_t)total, epoch, err, limit_ns);
        if (tid == 0) s_prefix = e;
    }
    __syncthreads();
    uint32_t r = s_prefix + before;
    if (i0 + kRsItems <= len) {
#pragma unroll
        for (int q = 0; q < kRsItems / 4; ++q) {
            uint4 t;
            t.x = r; r += v[4 * q];
            t.y = r; r += v[4 * q + 1];
            t.z = r; r += v[4 * q + 2];
            t.w = r; r += v[4 * q + 3];
            reinterpret_cast<uint4*>(counts + i0)[q] = t;
        }
    } else {
#pragma unroll
        for (int k = 0; k < kRsItems; ++k) {
            if (i0 + k < len) counts[i0 + k] = r;
            r += v[k];
        }
    }
}

// ---------------------------------------------------------------------------
// 2c. one digit pass (LAST: write perm, sorted keys and sorted positions)
// ---------------------------------------------------------------------------
struct RsPassArgs {
    const uint32_t* keys_in;
    const uint32_t* vals_in;     // nullptr: the value is the key's index
    uint32_t* keys_out;
    uint32_t* vals_out;          // not on the last pass
    uint32_t* perm;              // last pass
    float4* spos;                // last pass
    const float* pos;            // last pass
    int64_t n;
    int shift, bits;
    const uint32_t* offsets;     // scanned bin-major counts of this digit
    int64_t tiles;
};

template <bool LAST, int DIM, bool PACKED>
__global__ void __launch_bounds__(kRsThreads)
k_rs_pass(RsPassArgs a) {
    extern __shared__ __align__(16) unsigned char rs_smem[];
    // cnt[warp][bin]: the warp's count of the digit, then its first tile slot
    uint16_t* cnt = reinterpret_cast<uint16_t*>(rs_smem);
    uint32_t* s_key = reinterpret_cast<uint32_t*>(rs_smem + kRsWarps * kRsMaxBins * sizeof(uint16_t));
    uint32_t* s_val = s_key + kRsTile;
    uint32_t* s_off = s_val + kRsTile;   // per digit: global slot minus tile slot
    __shared__ uint64_t s_scan[kRsWarps];

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint32_t bins = 1u << a.bits, mask = bins - 1u;
    {
        uint32_t* c32 = reinterpret_cast<uint32_t*>(cnt);
        for (int i = tid; i < kRsWarps * kRsMaxBins / 2; i += kRsThreads) c32[i] = 0u;
    }
    const int64_t tile = blockIdx.x;
    const uint32_t b0 = (uint32_t)tid * kRsBinsPerThread;
    uint32_t goff[kRsBinsPerThread];
#pragma unroll
    for (int q = 0; q < kRsBinsPerThread; ++q)
        goff[q] = b0 + q < bins ? a.offsets[(int64_t)(b0 + q) * a.tiles + tile] : 0u;
    __syncthreads();
    const int64_t base = tile * kRsTile;
    const int64_t rem = a.n - base;
    const int tile_n = rem < kRsTile ? (int)rem : kRsTile;

    // this warp's keys, in order: items wbase + 32 r + lane
    const int wbase = warp * kRsWarpItems;
    uint32_t key[kRsItems], val[kRsItems], rank[kRsItems];
    bool ok[kRsItems];
#pragma unroll
    for (int r = 0; r < kRsItems; ++r) {
        const int idx = wbase + r * 32 + lane;
        ok[r] = idx < tile_n;
        key[r] = ok[r] ? a.keys_in[base + idx] : 0u;
        val[r] = ok[r] ? (a.vals_in ? a.vals_in[base + idx] : (uint32_t)(base + idx)) : 0u;
    }
    // stable rank of each key among the warp's keys of the same digit:
    // rounds in order, lanes in order inside a round
    uint16_t* wc = cnt + warp * kRsMaxBins;
    const uint32_t lt = (1u << lane) - 1u;
    {
        uint32_t peers[kRsItems];
        rs_match(key, ok, a.shift, a.bits, peers);
#pragma unroll
        for (int r = 0; r < kRsItems; ++r) {
            const uint32_t d = (key[r] >> a.shift) & mask;
            const uint32_t below = (uint32_t)__popc(peers[r] & lt);
            const uint32_t c = ok[r] ? (uint32_t)wc[d] : 0u;
            __syncwarp();
            if (ok[r] && below == 0) wc[d] = (uint16_t)(c + (uint32_t)__popc(peers[r]));
            __syncwarp();
            rank[r] = c + below;
        }
    }
    __syncthreads();

    // per digit: the tile's count, and each warp's prefix inside the tile
    uint32_t tc[kRsBinsPerThread];
#pragma unroll
    for (int q = 0; q < kRsBinsPerThread; ++q) {
        uint32_t t = 0;
        if (b0 + q < bins) {
#pragma unroll
            for (int w = 0; w < kRsWarps; ++w) {
                const uint32_t v = cnt[w * kRsMaxBins + b0 + q];
                cnt[w * kRsMaxBins + b0 + q] = (uint16_t)t;
                t += v;
            }
        }
        tc[q] = t;
    }
    // tile-local first slot of each digit
    uint32_t mine = 0;
#pragma unroll
    for (int q = 0; q < kRsBinsPerThread; ++q) mine += tc[q];
    uint64_t all;
    uint32_t t = (uint32_t)rs_block_scan(mine, s_scan, &all);
#pragma unroll
    for (int q = 0; q < kRsBinsPerThread; ++q) {
        if (b0 + q < bins) {
#pragma unroll
            for (int w = 0; w < kRsWarps; ++w) cnt[w * kRsMaxBins + b0 + q] += (uint16_t)t;
            s_off[b0 + q] = goff[q] - t;
        }
        t += tc[q];
    }
    __syncthreads();

    // stage the keys in digit order
#pragma unroll
    for (int r = 0; r < kRsItems; ++r) {
        if (ok[r]) {
            const uint32_t p = (uint32_t)wc[(key[r] >> a.shift) & mask] + rank[r];
            s_key[p] = key[r];
            s_val[p] = val[r];
        }
    }
    __syncthreads();

    // write out in digit order: a digit's keys of this tile go to
    // consecutive global slots.  Slots and indices are checked against n:
    // they are always in range unless a bounded wait of the scan gave up
    // (then the results are garbage, but no access leaves the arrays).
    uint32_t* __restrict__ keys_out = a.keys_out;
    const uint32_t n32 = (uint32_t)a.n;
    if (!LAST) {
        uint32_t* __restrict__ vals_out = a.vals_out;
        for (int p = tid; p < tile_n; p += kRsThreads) {
            const uint32_t k = s_key[p];
            const uint32_t dst = s_off[(k >> a.shift) & mask] + (uint32_t)p;
            if (dst >= n32) continue;
            keys_out[dst] = k;
            vals_out[dst] = s_val[p];
        }
    } else {
        uint32_t* __restrict__ perm = a.perm;
        float4* __restrict__ spos = a.spos;
        constexpr int U = 8;
        for (int p0 = tid; p0 < tile_n; p0 += U * kRsThreads) {
            uint32_t k[U], v[U], dst[U];
            float4 q[U];
            bool ok[U];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int p = p0 + u * kRsThreads;
                k[u] = p < tile_n ? s_key[p] : 0u;
                v[u] = p < tile_n ? s_val[p] : 0u;
                dst[u] = s_off[(k[u] >> a.shift) & mask] + (uint32_t)p;
                ok[u] = p < tile_n && dst[u] < n32 && v[u] < n32;
            }
#pragma unroll
            for (int u = 0; u < U; ++u)
                q[u] = ok[u] ? rs_load_pos<DIM, PACKED>(a.pos, v[u]) : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
            for (int u = 0; u < U; ++u) {
                if (!ok[u]) continue;
                keys_out[dst[u]] = k[u];
                perm[dst[u]] = v[u];
                spos[dst[u]] = make_float4(q[u].x, q[u].y, DIM == 3 ? q[u].z : 0.0f, 0.0f);
            }
        }
    }
}

// ---------------------------------------------------------------------------
// 3. cell boundaries: offsets of the occupied cells and their occupancy bits
// ---------------------------------------------------------------------------
struct RsBoundArgs {
    const uint32_t* keys;    // sorted cell ids
    int64_t n;
    int64_t n_words;
    uint32_t* cstart;        // offsets of the occupied cells [n_occ + 1]
    uint4* occ;              // occupancy words (cleared by k_rs_keys)
    uint64_t* status;
    uint32_t* ticket;
    uint32_t epoch;
    uint32_t* err;
    long long limit_ns;
};

// (the word is in range unless a bounded wait of an earlier launch gave up)
__device__ __forceinline__ void rs_or_bits(uint4* occ, int64_t n_words, uint32_t word,
                                           uint64_t bits) {
    if (word < n_words)
        atomicOr(reinterpret_cast<unsigned long long*>(occ + word), (unsigned long long)bits);
}

__global__ void __launch_bounds__(kRsThreads)
k_rs_bounds(RsBoundArgs a) {
    __shared__ uint64_t s_scan[kRsWarps];
    __shared__ uint32_t s_tile, s_prefix;
    const int tid = threadIdx.x;
    if (tid == 0) s_tile = atomicAdd(a.ticket, 1u);
    __syncthreads();
    const int64_t tile = s_tile;
    const int64_t s0 = tile * kRsTile + (int64_t)tid * kRsItems;
    uint32_t k[kRsItems];
    if (s0 + kRsItems <= a.n) {
#pragma unroll
        for (int q = 0; q < kRsItems / 4; ++q) {
            const uint4 t = reinterpret_cast<const uint4*>(a.keys + s0)[q];
            k[4 * q] = t.x;
            k[4 * q + 1] = t.y;
            k[4 * q + 2] = t.z;
            k[4 * q + 3] = t.w;
        }
    } else {
#pragma unroll
        for (int i = 0; i < kRsItems; ++i) k[i] = s0 + i < a.n ? a.keys[s0 + i] : 0u;
    }
    // keys are below n_cells < 2^32 - 1, so the sentinel marks position 0
    const uint32_t prev = (s0 > 0 && s0 <= a.n) ? a.keys[s0 - 1] : 0xFFFFFFFFu;
    uint32_t flags = 0, count = 0;
#pragma unroll
    for (int i = 0; i < kRsItems; ++i) {
        const bool b = s0 + i < a.n && k[i] != (i ? k[i - 1] : prev);
        flags |= (b ? 1u : 0u) << i;
        count += b ? 1u : 0u;
    }
    uint64_t total;
    const uint32_t before = (uint32_t)rs_block_scan(count, s_scan, &total);
    if (tid < 32) {
        const uint32_t e = rs_look_back_warp(a.status, tile, (uint32_t)total, a.epoch, a.err,
                                             a.limit_ns);
        if (tid == 0) s_prefix = e;
    }
    __syncthreads();
    uint32_t r = s_prefix + before;
    uint32_t word = 0xFFFFFFFFu;
    uint64_t bits = 0;
#pragma unroll
    for (int i = 0; i < kRsItems; ++i) {
        if (!((flags >> i) & 1u)) continue;
        if (r < a.n) a.cstart[r] = (uint32_t)(s0 + i);
        ++r;
        const uint32_t w = k[i] >> 6;
        if (w != word) {
            if (bits) rs_or_bits(a.occ, a.n_words, word, bits);
            word = w;
            bits = 0;
        }
        bits |= 1ull << (k[i] & 63u);
    }
    // the thread's last word: lanes hold consecutive sorted keys, so equal
    // last words sit in consecutive lanes; each run is OR-combined (a
    // segmented tree over the lanes) and flushed once by its first lane
    {
        const int lane = tid & 31;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t w2 = __shfl_down_sync(0xffffffffu, word, o);
            const uint64_t b2 = __shfl_down_sync(0xffffffffu, bits, o);
            if (lane + o < 32 && w2 == word) bits |= b2;
        }
        const uint32_t wp = __shfl_up_sync(0xffffffffu, word, 1);
        if (bits && (lane == 0 || wp != word)) rs_or_bits(a.occ, a.n_words, word, bits);
    }
    // the thread holding the last particle closes the table
    if (s0 < a.n && a.n <= s0 + kRsItems && r <= a.n) a.cstart[r] = (uint32_t)a.n;
}

// ---------------------------------------------------------------------------
// 4. occupied cells before each occupancy word
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kRsThreads)
k_rs_occ_prefix(uint4* occ, int64_t n_words, uint64_t* status, uint32_t* ticket,
                uint32_t epoch, uint32_t* err, long long limit_ns) {
    __shared__ uint64_t s_scan[kRsWarps];
    __shared__ uint32_t s_tile, s_prefix;
    const int tid = threadIdx.x;
    if (tid == 0) s_tile = atomicAdd(ticket, 1u);
    __syncthreads();
    const int64_t tile = s_tile;
    const int64_t w0 = tile * kRsZTile + (int64_t)tid * kRsZItems;
    uint32_t v[kRsZItems];
    uint32_t count = 0;
#pragma unroll
    for (int i = 0; i < kRsZItems; ++i) {
        uint4 q = make_uint4(0u, 0u, 0u, 0u);
        if (w0 + i < n_words) q = occ[w0 + i];
        v[i] = (uint32_t)__popc(q.x) + (uint32_t)__popc(q.y);
        count += v[i];
    }
    uint64_t total;
    const uint32_t before = (uint32_t)rs_block_scan(count, s_scan, &total);
    if (tid < 32) {
        const uint32_t e = rs_look_back_warp(status, tile, (uint32_t)total, epoch, err, limit_ns);
        if (tid == 0) s_prefix = e;
    }
    __syncthreads();
    uint32_t r = s_prefix + before;
#pragma unroll
    for (int i = 0; i < kRsZItems; ++i) {
        if (w0 + i < n_words) occ[w0 + i].z = r;
        r += v[i];
    }
}

// ---------------------------------------------------------------------------
// 5. dense table: every cell's offset from the occupied cells'
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kRsThreads)
k_rs_expand(int64_t nc1, const uint4* __restrict__ occ, const uint32_t* __restrict__ cstart,
            uint32_t* __restrict__ out) {
    for (int64_t c = blockIdx.x * (int64_t)kRsThreads + threadIdx.x; c < nc1;
         c += (int64_t)gridDim.x * kRsThreads) {
        const uint4 q = occ[c >> 6];
        const uint64_t bits = ((uint64_t)q.y << 32) | q.x;
        out[c] = cstart[q.z + (uint32_t)__popcll(bits & ((1ull << (c & 63)) - 1ull))];
    }
}

RsPlan make_plan(int64_t n_cells) {
    RsPlan p{};
    int nbits = 1;
    while (nbits < 32 && (uint64_t)(n_cells - 1) >> nbits) ++nbits;
    p.passes = (nbits + kRsMaxBits - 1) / kRsMaxBits;
    int shift = 0;
    for (int i = 0; i < p.passes; ++i) {
        p.bits[i] = nbits / p.passes + (i < nbits % p.passes ? 1 : 0);
        p.shift[i] = shift;
        shift += p.bits[i];
    }
    return p;
}

// Layout of Scratch::rs_status: the bin-major digit counts of one pass
// (tiles x 2^bits u32, at most tiles x kRsMaxBins), then the epoch-tagged
// look-back words of the scans.
int64_t rs_count_words64(int64_t tiles) { return (tiles * kRsMaxBins + 1) / 2 + 1; }
int64_t rs_status_words64(int64_t tiles, int64_t n_words) {
    const int64_t scan_tiles = (tiles * kRsMaxBins + kRsTile - 1) / kRsTile;
    const int64_t zt = (n_words + kRsZTile - 1) / kRsZTile;
    int64_t w = tiles;
    if (scan_tiles > w) w = scan_tiles;
    if (zt > w) w = zt;
    return w + 1;
}

template <int DIM, bool PACKED>
cudaError_t run_radix(CellList& cl, const float* pos, Scratch& sc, uint32_t* err,
                      cudaStream_t st, const BuildOptions& opt) {
    const int64_t n = cl.n;
    const int64_t nc = cl.g.n_cells;
    const int64_t n_words = occ_words(nc);
    const long long limit = opt.limit_ns > 0 ? opt.limit_ns : 1000000000ll;
    const RsPlan plan = make_plan(nc);
    const int64_t tiles = (n + kRsTile - 1) / kRsTile;
    // the per-particle buffers of the counting sort, as two pairs of key and
    // value arrays of cap_n entries each
    uint32_t* A = reinterpret_cast<uint32_t*>(cl.cell_rank);
    uint32_t* B = cl.tmp;
    uint32_t* keys[2] = {A, B};
    uint32_t* vals[2] = {A + cl.cap_n, B + cl.cap_n};
    uint32_t* counts = reinterpret_cast<uint32_t*>(sc.rs_status);
    uint64_t* status = sc.rs_status + rs_count_words64(tiles);
    uint32_t* tickets = sc.rs_small;
    // epochs: one per look-back launch; the status words are cleared when
    // the 30-bit epoch would wrap (and on fresh memory)
    const uint32_t need = (uint32_t)plan.passes + 2u;
    cudaError_t e;
    if (sc.rs_epoch == 0 || sc.rs_epoch + need > kRsEpochMask) {
        e = cudaMemsetAsync(sc.rs_status, 0, sc.cap_rs_status * sizeof(uint64_t), st);
        if (e != cudaSuccess) return e;
        sc.rs_epoch = 1;
    }
    const uint32_t ep0 = sc.rs_epoch;
    sc.rs_epoch += need;
    if ((e = cudaMemsetAsync(tickets, 0, kRsTickets * sizeof(uint32_t), st)) != cudaSuccess) return e;
    if ((e = cudaFuncSetAttribute((const void*)k_rs_pass<true, DIM, PACKED>,
                                  cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)kRsPassSmem)) != cudaSuccess ||
        (e = cudaFuncSetAttribute((const void*)k_rs_pass<false, DIM, PACKED>,
                                  cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)kRsPassSmem)) != cudaSuccess)
        return e;

    k_rs_keys<DIM, PACKED><<<(unsigned)tiles, kRsThreads, 0, st>>>(
        pos, n, cl.g, plan.bits[0], A, counts, tiles, cl.occ, n_words);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    int cur = 0;   // keys[cur] (and vals[cur] after the first pass) hold the input
    for (int p = 0; p < plan.passes; ++p) {
        const bool last = p == plan.passes - 1;
        if (p > 0) {
            k_rs_up<<<(unsigned)tiles, kRsThreads, 0, st>>>(keys[cur], n, plan.shift[p],
                                                            plan.bits[p], counts, tiles);
            if ((e = cudaGetLastError()) != cudaSuccess) return e;
        }
        const int64_t len = tiles << plan.bits[p];
        const int64_t stiles = (len + kRsTile - 1) / kRsTile;
        const int64_t skip = (p == 0 && opt.skip_block >= 0 && opt.skip_block < stiles)
                                 ? opt.skip_block : -1;
        k_rs_scan<<<(unsigned)stiles, kRsThreads, 0, st>>>(counts, len, status, tickets + p,
                                                           ep0 + (uint32_t)p, err, limit, skip);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        RsPassArgs a;
        a.keys_in = keys[cur];
        a.vals_in = p == 0 ? nullptr : vals[cur];
        a.keys_out = keys[cur ^ 1];
        a.vals_out = last ? nullptr : vals[cur ^ 1];
        a.perm = cl.perm;
        a.spos = cl.spos;
        a.pos = pos;
        a.n = n;
        a.shift = plan.shift[p];
        a.bits = plan.bits[p];
        a.offsets = counts;
        a.tiles = tiles;
        if (last) k_rs_pass<true, DIM, PACKED><<<(unsigned)tiles, kRsThreads, kRsPassSmem, st>>>(a);
        else k_rs_pass<false, DIM, PACKED><<<(unsigned)tiles, kRsThreads, kRsPassSmem, st>>>(a);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        cur ^= 1;
    }
    // sorted keys now in keys[cur]; vals[cur] is free
    uint32_t* cstart = cl.g.compact ? cl.cell_start : vals[cur];
    {
        RsBoundArgs b;
        b.keys = keys[cur];
        b.n = n;
        b.n_words = n_words;
        b.cstart = cstart;
        b.occ = cl.occ;
        b.status = status;
        b.ticket = tickets + plan.passes;
        b.epoch = ep0 + (uint32_t)plan.passes;
        b.err = err;
        b.limit_ns = limit;
        k_rs_bounds<<<(unsigned)tiles, kRsThreads, 0, st>>>(b);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    {
        const int64_t zt = (n_words + kRsZTile - 1) / kRsZTile;
        k_rs_occ_prefix<<<(unsigned)zt, kRsThreads, 0, st>>>(
            cl.occ, n_words, status, tickets + plan.passes + 1,
            ep0 + (uint32_t)plan.passes + 1, err, limit);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    if (!cl.g.compact) {
        const int64_t nc1 = nc + 1;
        int64_t grid = (nc1 + kRsThreads - 1) / kRsThreads;
        const int64_t cap = (int64_t)num_sms() * 16;
        if (grid > cap) grid = cap;
        k_rs_expand<<<(unsigned)grid, kRsThreads, 0, st>>>(nc1, cl.occ, cstart, cl.cell_start);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace

size_t radix_status_words(int64_t n, int64_t n_cells) {
    const int64_t tiles = (n + kRsTile - 1) / kRsTile;
    return (size_t)(rs_count_words64(tiles) + rs_status_words64(tiles, occ_words(n_cells)));
}

size_t radix_small_words() { return kRsSmallWords; }

bool radix_supported(int64_t n, int64_t n_cells) {
    // keys and slots are 32-bit; the boundary scan uses 0xFFFFFFFF as "no
    // predecessor", so every cell id must be below it
    return n > 0 && n < (int64_t(1) << 31) && n_cells >= 1 && n_cells < (int64_t(1) << 32) - 1;
}

cudaError_t launch_build_radix(CellList& cl, const float* pos, bool packed, Scratch& sc,
                               uint32_t* err, cudaStream_t st, const BuildOptions& opt) {
    if (!radix_supported(cl.n, cl.g.n_cells) || !sc.rs_status || !sc.rs_small || !cl.occ)
        return cudaErrorInvalidValue;
    if (cl.g.dim == 3)
        return packed ? run_radix<3, true>(cl, pos, sc, err, st, opt)
                      : run_radix<3, false>(cl, pos, sc, err, st, opt);
    return packed ? run_radix<2, true>(cl, pos, sc, err, st, opt)
                  : run_radix<2, false>(cl, pos, sc, err, st, opt);
}

}  // namespace ab
