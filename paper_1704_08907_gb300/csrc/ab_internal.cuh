// Internal declarations shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <functional>

#include "../../include/aboria_gpu.h"

#define AB_HIDDEN __attribute__((visibility("hidden")))

namespace ab {

// Device-side error bits latched in the context's error word.
enum : uint32_t {
    DEVERR_SCAN_TIMEOUT = 1u,
    DEVERR_TC_TIMEOUT = 2u,   // a tensor-core kernel's pipeline wait gave up
};

// Cell-lattice geometry of one build, passed by value to kernels.
struct Geom {
    int dim;
    int n[3];            // cells per axis (1 for unused axes)
    int periodic[3];
    float lo[3];
    float inv_w[3];      // n_k / L_k rounded to FP32
    float L[3];          // hi - lo in FP32
    float halfL[3];      // 0.5f * L in FP32
    float r2;            // fl(r * r)
    float r;             // radius as given
    int general;         // 1 if a periodic axis has fewer than 5 cells
    int kx;              // x cells per cut-off width: the stencil spans cx - kx .. cx + kx
    int ky, kz;          // the same for y and z (stencil rows: (2 ky + 1) (2 kz + 1))
    int compact;         // 1: offsets of occupied cells only, found through CellList::occ
    int64_t n_cells;
};

// Cell coordinate along one axis: floor((x - lo) * inv_w), clamped.
// Every kernel that needs a particle's cell uses exactly this expression, so
// the hash and the stencil search agree bit for bit.
__device__ __forceinline__ int cell_coord(float x, float lo, float inv_w, int n) {
    float u = __fmul_rn(__fsub_rn(x, lo), inv_w);
    float f = floorf(u);
    int c = (f >= (float)n) ? n - 1 : (f < 0.0f ? 0 : (int)f);
    return c;
}

// Library-owned buffers of one cell list.
struct CellList {
    int64_t n = 0;
    Geom g{};
    const float* user_pos = nullptr;  // caller's positions at build time
    bool valid = false;
    float4* spos = nullptr;           // sorted positions (x, y, z, 0)
    uint32_t* perm = nullptr;         // perm[s] = original index
    uint2* cell_rank = nullptr;       // per original particle: (cell, atomic arrival rank)
    uint32_t* tmp = nullptr;          // unordered slot -> original index
    uint32_t* cell_start = nullptr;   // dense: [n_cells + 1]; compact: [n + 1], per occupied cell
    size_t cap_n = 0, cap_cells = 0;
    // compact table: per 64 cells, the occupancy bits (x: cells 0-31, y:
    // 32-63) and the number of occupied cells before them (z)
    uint4* occ = nullptr;
    size_t cap_occ = 0;
};

// Words of the occupancy table of a compact cell list (cells 0 .. n_cells,
// the last one past the end).
inline int64_t occ_words(int64_t n_cells) { return (n_cells + 1 + 63) / 64; }

struct Scratch {
    float2* sv = nullptr;             // sorted per-particle values: (m, P/rho^2) for the SPH
                                      // force, or w as float[n] for the Gaussian adjoint
    size_t cap_sv = 0;
    uint64_t* scan_status = nullptr;  // decoupled look-back tile words
    uint32_t* scan_ticket = nullptr;
    size_t cap_tiles = 0;
    double* partial = nullptr;        // per-block FP64 partial sums
    size_t cap_partial = 0;
    uint32_t* counts = nullptr;       // pair-list counts (user order)
    size_t cap_counts = 0;
    uint8_t* dense_ws = nullptr;      // tensor-core operand images
    size_t cap_dense_ws = 0;
    uint8_t* solve_ws = nullptr;      // CG vectors and scalars
    size_t cap_solve_ws = 0;
    uint32_t* coop = nullptr;         // cooperative build: barrier words + block sums
    uint64_t* rs_status = nullptr;    // radix build: look-back words (epoch-tagged)
    size_t cap_rs_status = 0;
    uint32_t* rs_small = nullptr;     // radix build: tickets + digit counts
    uint32_t rs_epoch = 0;            // next look-back epoch (0: clear rs_status first)
};

// ---- launchers (defined in the .cu files) ----------------------------------

// ab_cells.cu
// How ab_build runs (see ab_testing_build_path): the counting sort as a
// kernel sequence, the counting sort in one cooperative launch, the radix
// sort of ab_sort.cu, or the automatic choice; the last two fields are
// testing hooks of the bounded waits.
enum BuildPath : int { kPathSequence = 0, kPathCoop = 1, kPathRadix = 2, kPathAuto = 3 };
struct BuildOptions {
    int path = kPathAuto;
    int skip_block = -1;          // a block (tile) that never arrives (publishes)
    long long limit_ns = 0;       // wait limit (0: one second)
};
// The path an automatic build takes for n particles and this geometry.
AB_HIDDEN int auto_build_path(int64_t n, const Geom& g);
AB_HIDDEN cudaError_t launch_build(CellList& cl, const float* pos, bool packed, Scratch& sc,
                                   uint32_t* err, cudaStream_t st, const BuildOptions& opt);
// words of Scratch::coop (allocated once per context)
AB_HIDDEN size_t coop_scratch_words();

// ab_sort.cu: the cell list by a stable radix sort of the cell ids (the same
// cell list as launch_build, bit for bit).  Needs cl.occ for the dense table
// too, Scratch::rs_status of radix_status_words() and Scratch::rs_small of
// radix_small_words().
AB_HIDDEN bool radix_supported(int64_t n, int64_t n_cells);
AB_HIDDEN size_t radix_status_words(int64_t n, int64_t n_cells);
AB_HIDDEN size_t radix_small_words();
AB_HIDDEN cudaError_t launch_build_radix(CellList& cl, const float* pos, bool packed,
                                         Scratch& sc, uint32_t* err, cudaStream_t st,
                                         const BuildOptions& opt);
// The dense offsets of a compact cell list: out[c] = first slot of cell c,
// c = 0 .. n_cells (device uint32[n_cells + 1]).
AB_HIDDEN cudaError_t launch_expand_cells(const CellList& cl, uint32_t* out, cudaStream_t st);
AB_HIDDEN cudaError_t launch_gather_w_pos(CellList& cl, const float* w, cudaStream_t st);
AB_HIDDEN cudaError_t launch_gather_scalar(const CellList& cl, const float* v, float* out,
                                           cudaStream_t st);
// sv[s] = wv[perm[s]]: a per-particle pair of values into sorted order
AB_HIDDEN cudaError_t launch_gather_pairs(const CellList& cl, const float2* wv, float2* sv,
                                          cudaStream_t st);
// Exclusive scan of n u32 counts into out (u32 or u64), out[n] = total.
// status/ticket: scratch of scan_tiles(n) words + 1 ticket (zeroed here).
AB_HIDDEN size_t scan_tiles(int64_t n);
AB_HIDDEN cudaError_t launch_scan_u32(const uint32_t* in, uint32_t* out,
                                      int64_t n, uint64_t* status,
                                      uint32_t* ticket, uint32_t* err,
                                      int skip_tile, long long limit_ns,
                                      cudaStream_t st);
AB_HIDDEN cudaError_t launch_scan_u32_to_i64(const uint32_t* in, int64_t* out,
                                             int64_t n, uint64_t* status,
                                             uint32_t* ticket, uint32_t* err,
                                             cudaStream_t st);
AB_HIDDEN cudaError_t launch_reduce_partials(const double* partial, int count,
                                             double* out, cudaStream_t st);

// ab_pairs.cu
struct PairOut {
    float* out = nullptr;        // scalar output (user order)
    float4* out4 = nullptr;      // vector output (user order)
    float4* grad_pos = nullptr;  // bwd
    float* grad_packed = nullptr;  // bwd, dim floats per particle (energy + gradient only)
    float* grad_w = nullptr;     // bwd
    double* partial = nullptr;   // per-block partials (energy or ds)
    int partial_count = 0;
};
AB_HIDDEN int pair_grid(int64_t n);
AB_HIDDEN int num_sms();   // SM count of the current device
AB_HIDDEN cudaError_t launch_pair_fwd(const CellList& cl, ab_op op,
                                      const ab_op_params& prm, const float2* sv,
                                      PairOut& o, cudaStream_t st);
// value: also the forward values (o.out) in the same walk; LJ energy
// partials then go to o.partial
AB_HIDDEN cudaError_t launch_pair_bwd(const CellList& cl, ab_op op,
                                      const ab_op_params& prm, const float2* sv,
                                      PairOut& o, cudaStream_t st, bool value = false);
// LJ energy + gradient of the total energy in one walk (PairOut out, grad_pos,
// partial)
AB_HIDDEN cudaError_t launch_pair_energy_grad(const CellList& cl, ab_op op,
                                              const ab_op_params& prm, PairOut& o,
                                              cudaStream_t st);
AB_HIDDEN cudaError_t launch_pair_count(const CellList& cl, uint32_t* counts,
                                        cudaStream_t st);
AB_HIDDEN cudaError_t launch_pair_emit(const CellList& cl, const int64_t* offsets,
                                       int32_t* idx, cudaStream_t st);

// ab_dense.cu
AB_HIDDEN cudaError_t launch_dense_fwd(int64_t m, int64_t n, const float4* X,
                                       const float4* Y, int nrhs, const float* W,
                                       float s, ab_prec prec, float* out,
                                       cudaStream_t st);
AB_HIDDEN cudaError_t launch_dense_bwd(int64_t m, int64_t n, const float4* X,
                                       const float4* Y, int nrhs, const float* W,
                                       float s, ab_prec prec, const float* G,
                                       float* dW, float4* dX, float4* dY,
                                       double* partial, int* partial_count,
                                       cudaStream_t st);
AB_HIDDEN int dense_partial_capacity(int64_t m, int64_t n);

// ab_dense_tc.cu (tcgen05 path; nrhs must be 64)
AB_HIDDEN size_t dense_tc_workspace_bytes(int64_t n);
AB_HIDDEN cudaError_t launch_dense_tc_fwd(int64_t m, int64_t n, const float4* X, const float4* Y,
                                          int nrhs, const float* W, float s, ab_prec prec,
                                          float* out, void* ws, uint32_t* err, cudaStream_t st);
AB_HIDDEN size_t dense_tc_grad_workspace_bytes(int64_t m, int64_t n);
AB_HIDDEN cudaError_t launch_dense_tc_gradx(int64_t m, int64_t n, const float4* X, const float4* Y,
                                            const float* G, const float* W, float s, ab_prec prec,
                                            float4* dX, double* partial, int* partial_count,
                                            void* ws, uint32_t* err, cudaStream_t st);

// ab_solve.cu: conjugate gradients for (K(X, X) + sigma^2 I) W = B; the
// matvec Q = K(X, X) P is supplied by the caller
using SolveMatvec = std::function<cudaError_t(const float* P, float* Q)>;
AB_HIDDEN size_t solve_workspace_bytes(int64_t n, int nrhs);
AB_HIDDEN cudaError_t run_solve(int64_t n, int nrhs, const float* B, float sigma2, float tol,
                                int max_iter, float* W, void* ws, const SolveMatvec& mv,
                                int* iters, float* relres, cudaStream_t st);

// ab_bd.cu
AB_HIDDEN cudaError_t launch_bd_step(const Geom& g, int64_t n, float4* pos,
                                     const float4* force, float dt, float D,
                                     uint64_t seed, uint64_t step,
                                     cudaStream_t st);
AB_HIDDEN cudaError_t launch_md_step(const Geom& g, int64_t n, float4* pos, float4* vel,
                                     const float4* acc, float dt, cudaStream_t st);

}  // namespace ab
