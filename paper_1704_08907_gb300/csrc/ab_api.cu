// C ABI entry points: argument validation, workspace management and launch
// sequencing.  Every step of the computation runs in the kernels of
// ab_cells.cu, ab_pairs.cu, ab_dense.cu and ab_bd.cu; this file only checks,
// allocates and orders.
#include <cuda_runtime.h>
#include <math.h>
#include <stdarg.h>
#include <stdint.h>
#include <stdio.h>
#include <string.h>

#include <atomic>
#include <string>

#include "ab_internal.cuh"
#include "../../include/aboria_gpu_testing.h"

namespace ab {
// SM count of the current device, looked up once per device.  The cache
// entries are atomics: concurrent first calls store the same value.
int num_sms() {
    static std::atomic<int> cache[64];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 152;
    int v = cache[dev].load(std::memory_order_relaxed);
    if (v <= 0) {
        if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
            v <= 0)
            return 152;
        cache[dev].store(v, std::memory_order_relaxed);
    }
    return v;
}

// Makes the context's device current for one entry point and restores the
// caller's current device on every return path.
struct DeviceGuard {
    int prev = -1;
    bool ok = false, switched = false;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess) {
            cudaGetLastError();
            prev = -1;
        }
        if (prev == dev) {
            ok = true;
            return;
        }
        ok = switched = cudaSetDevice(dev) == cudaSuccess;
        if (!ok) cudaGetLastError();
    }
    ~DeviceGuard() {
        if (switched && prev >= 0) cudaSetDevice(prev);
    }
    DeviceGuard(const DeviceGuard&) = delete;
    DeviceGuard& operator=(const DeviceGuard&) = delete;
};
}

struct ab_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    ab::CellList cl;
    ab::Scratch sc;
    ab::BuildOptions build_opt;
    int coop_launch = 0;      // the device supports cooperative launches
    int table_mode = 0;       // testing: 0 automatic, 1 dense, 2 compact where allowed
    uint32_t* d_err = nullptr;
    std::string last_error;
};

namespace {

using ab::CellList;
using ab::Geom;

ab_status fail(ab_ctx* c, ab_status s, const char* fmt, ...) {
    if (c) {
        char buf[512];
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(buf, sizeof(buf), fmt, ap);
        va_end(ap);
        c->last_error = buf;
    }
    return s;
}

ab_status cuda_fail(ab_ctx* c, cudaError_t e, const char* where) {
    if (e == cudaErrorMemoryAllocation)
        return fail(c, AB_ERR_OOM, "%s: %s", where, cudaGetErrorString(e));
    return fail(c, AB_ERR_CUDA, "%s: %s", where, cudaGetErrorString(e));
}

// Stream-ordered growth: allocate the new buffer before freeing the old one,
// so a failed allocation leaves the previous workspace intact.
template <typename T>
cudaError_t grow(T** p, size_t* cap, size_t need, cudaStream_t st) {
    if (need <= *cap && *p) return cudaSuccess;
    size_t want = need + need / 4 + 64;
    void* q = nullptr;
    cudaError_t e = cudaMallocAsync(&q, want * sizeof(T), st);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return e;
    }
    if (*p) cudaFreeAsync(*p, st);
    *p = (T*)q;
    *cap = want;
    return cudaSuccess;
}

bool overlaps(const void* a, size_t na, const void* b, size_t nb) {
    if (!a || !b || na == 0 || nb == 0) return false;
    uintptr_t a0 = (uintptr_t)a, b0 = (uintptr_t)b;
    return a0 < b0 + nb && b0 < a0 + na;
}

bool aligned16(const void* p) { return ((uintptr_t)p & 15u) == 0; }

ab_status check_domain(ab_ctx* c, const ab_domain* d) {
    if (!d) return fail(c, AB_ERR_INVALID_ARG, "domain is NULL");
    if (d->dim != 2 && d->dim != 3) return fail(c, AB_ERR_INVALID_ARG, "dim must be 2 or 3 (got %d)", d->dim);
    if (!(d->radius > 0.0f) || !isfinite(d->radius))
        return fail(c, AB_ERR_INVALID_ARG, "radius must be finite and > 0");
    for (int k = 0; k < d->dim; ++k) {
        if (!isfinite(d->lo[k]) || !isfinite(d->hi[k]) || !(d->hi[k] > d->lo[k]))
            return fail(c, AB_ERR_INVALID_ARG, "axis %d: need finite lo < hi", k);
        float L = d->hi[k] - d->lo[k];
        if (!isfinite(L)) return fail(c, AB_ERR_INVALID_ARG, "axis %d: box too large", k);
    }
    return AB_OK;
}

// Cell geometry (see ab_build in the header for the width rule).
Geom make_geom(const ab_domain* d, int64_t n) {
    Geom g{};
    g.dim = d->dim;
    g.r = d->radius;
    g.r2 = d->radius * d->radius;
    int64_t nk[3] = {1, 1, 1};
    for (int k = 0; k < 3; ++k) {
        g.periodic[k] = 0;
        g.lo[k] = 0.0f;
        g.L[k] = 1.0f;
        g.halfL[k] = 0.5f;
        g.inv_w[k] = 0.0f;
    }
    for (int k = 0; k < d->dim; ++k) {
        g.periodic[k] = d->periodic[k] ? 1 : 0;
        g.lo[k] = d->lo[k];
        g.L[k] = d->hi[k] - d->lo[k];
        g.halfL[k] = 0.5f * g.L[k];
        const double L = (double)g.L[k];
        const double wmin = (double)d->radius * (1.0 + 0x1p-18) + L * 0x1p-18;
        double c = floor(L / wmin);
        if (c < 1.0) c = 1.0;
        if (c > (double)(1 << 21)) c = (double)(1 << 21);
        nk[k] = (int64_t)c;
    }
    const int64_t cap = n * 8 > (int64_t(1) << 22) ? n * 8 : (int64_t(1) << 22);
    for (;;) {
        int64_t t = nk[0] * nk[1] * nk[2];
        if (t <= cap) break;
        for (int k = 0; k < d->dim; ++k) nk[k] = nk[k] > 1 ? nk[k] / 2 : 1;
    }
    g.general = 0;
    for (int k = 0; k < d->dim; ++k)
        if (g.periodic[k] && nk[k] < 5) g.general = 1;
    // Sub-divide x: cells of 1/kx of the width along x, the stencil reaching
    // kx of them each way.  A stencil row then spans (2 kx + 1) / kx cut-off
    // widths instead of 3 (fewer candidates) and stays one contiguous range
    // of the sorted particles.  Needs >= 5 base cells on a periodic x axis
    // (the fast-path wrap rule then holds with 2 kx + 3 <= kx * n_x) and
    // room in the cell table.
    g.kx = g.ky = g.kz = 1;
    if (!g.general && nk[0] >= 5) {
        const int64_t rest = nk[1] * nk[2];
        for (int kx = 4; kx >= 2; --kx) {
            if (nk[0] * kx * rest <= cap && nk[0] * kx <= (int64_t(1) << 21)) {
                g.kx = kx;
                nk[0] *= kx;
                break;
            }
        }
    }
    // (splitting y or z as well was measured slower: 15 or 25 stencil rows
    // cost more than the candidates they save)
    g.n_cells = 1;
    for (int k = 0; k < 3; ++k) {
        g.n[k] = (int)nk[k];
        g.n_cells *= nk[k];
        if (k < d->dim) g.inv_w[k] = (float)((double)nk[k] / (double)g.L[k]);
    }
    return g;
}

ab_status ensure_sv(ab_ctx* c, int64_t n) {
    cudaError_t e = grow(&c->sc.sv, &c->sc.cap_sv, (size_t)(n > 0 ? n : 1), c->stream);
    return e == cudaSuccess ? AB_OK : cuda_fail(c, e, "workspace (variables)");
}

ab_status ensure_partial(ab_ctx* c, size_t count) {
    cudaError_t e = grow(&c->sc.partial, &c->sc.cap_partial, count > 0 ? count : 1, c->stream);
    return e == cudaSuccess ? AB_OK : cuda_fail(c, e, "workspace (partials)");
}

ab_status ensure_scan(ab_ctx* c, int64_t items) {
    size_t tiles = ab::scan_tiles(items) + 1;
    cudaError_t e = grow(&c->sc.scan_status, &c->sc.cap_tiles, tiles, c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "workspace (scan)");
    if (!c->sc.scan_ticket) {
        e = cudaMallocAsync((void**)&c->sc.scan_ticket, 16, c->stream);
        if (e != cudaSuccess) return cuda_fail(c, e, "workspace (scan ticket)");
    }
    return AB_OK;
}

ab_status require_cells(ab_ctx* c) {
    if (!c->cl.valid)
        return fail(c, AB_ERR_STALE, "no current cell list: call ab_build after creating the "
                                     "context or after moving the particles");
    return AB_OK;
}

size_t out_bytes(ab_op op, int64_t n) {
    return (op == AB_OP_EXPF || op == AB_OP_SOFT || op == AB_OP_SPH_FORCE) ? (size_t)n * 16
                                                                          : (size_t)n * 4;
}

}  // namespace

// The library is built with -fvisibility=hidden; only the C ABI is exported.
#pragma GCC visibility push(default)
extern "C" {

const char* ab_status_string(ab_status s) {
    switch (s) {
        case AB_OK: return "ok";
        case AB_ERR_INVALID_ARG: return "invalid argument";
        case AB_ERR_ALIAS: return "output overlaps an input";
        case AB_ERR_STALE: return "cell list missing or stale";
        case AB_ERR_OOM: return "out of device memory";
        case AB_ERR_CUDA: return "CUDA error";
        case AB_ERR_TIMEOUT: return "device-side wait timed out";
        case AB_ERR_UNSUPPORTED: return "unsupported request";
        case AB_ERR_CAPACITY: return "output capacity too small";
    }
    return "unknown status";
}

const char* ab_last_error(ab_ctx* c) { return c ? c->last_error.c_str() : ""; }

ab_status ab_create(ab_ctx** out, int device, void* stream) {
    if (!out) return AB_ERR_INVALID_ARG;
    *out = nullptr;
    int count = 0;
    if (cudaGetDeviceCount(&count) != cudaSuccess) {
        cudaGetLastError();
        return AB_ERR_CUDA;
    }
    if (device < 0 || device >= count) return AB_ERR_INVALID_ARG;
    ab::DeviceGuard dg(device);
    if (!dg.ok) return AB_ERR_CUDA;
    ab_ctx* c = new ab_ctx();
    c->device = device;
    c->stream = (cudaStream_t)stream;
    if (cudaDeviceGetAttribute(&c->coop_launch, cudaDevAttrCooperativeLaunch, device) != cudaSuccess) {
        cudaGetLastError();
        c->coop_launch = 0;
    }
    if (cudaMalloc((void**)&c->d_err, 16) != cudaSuccess ||
        cudaMemset(c->d_err, 0, 16) != cudaSuccess) {
        cudaGetLastError();
        delete c;
        return AB_ERR_OOM;
    }
    *out = c;
    return AB_OK;
}

ab_status ab_destroy(ab_ctx* c) {
    if (!c) return AB_OK;
    ab::DeviceGuard dg(c->device);
    cudaStreamSynchronize(c->stream);
    void* bufs[] = {c->cl.spos, c->cl.perm, c->cl.cell_rank, c->cl.tmp,
                    c->cl.cell_start, c->cl.occ, c->sc.sv, c->sc.scan_status, c->sc.scan_ticket,
                    c->sc.partial, c->sc.counts, c->sc.dense_ws, c->sc.solve_ws, c->sc.coop,
                    c->sc.rs_status, c->sc.rs_small};
    for (void* b : bufs)
        if (b) cudaFreeAsync(b, c->stream);
    cudaStreamSynchronize(c->stream);
    cudaFree(c->d_err);
    cudaGetLastError();
    delete c;
    return AB_OK;
}

ab_status ab_set_stream(ab_ctx* c, void* stream) {
    if (!c) return AB_ERR_INVALID_ARG;
    c->stream = (cudaStream_t)stream;
    return AB_OK;
}

ab_status ab_sync(ab_ctx* c) {
    if (!c) return AB_ERR_INVALID_ARG;
    ab::DeviceGuard dg(c->device);
    if (!dg.ok) return fail(c, AB_ERR_CUDA, "cannot make device %d current", c->device);
    cudaError_t e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "ab_sync");
    uint32_t h = 0;
    e = cudaMemcpy(&h, c->d_err, sizeof(h), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(c, e, "ab_sync (error word)");
    if (h) {
        cudaMemset(c->d_err, 0, sizeof(uint32_t));
        if (h & ab::DEVERR_SCAN_TIMEOUT)
            return fail(c, AB_ERR_TIMEOUT, "scan look-back wait exceeded its time limit");
        if (h & ab::DEVERR_TC_TIMEOUT)
            return fail(c, AB_ERR_TIMEOUT, "tensor-core pipeline wait exceeded its time limit");
    }
    return AB_OK;
}

static ab_status build_impl(ab_ctx* c, const ab_domain* dom, int64_t n, const float* pos,
                            bool packed) {
    if (!c) return AB_ERR_INVALID_ARG;
    ab_status s = check_domain(c, dom);
    if (s != AB_OK) return s;
    if (n < 0 || n >= (int64_t(1) << 31) - 1) return fail(c, AB_ERR_INVALID_ARG, "n out of range");
    if (!packed && n > 0 && (!pos || !aligned16(pos)))
        return fail(c, AB_ERR_INVALID_ARG, "pos4 must be a 16-byte aligned device pointer");
    if (packed && n > 0 && (!pos || ((uintptr_t)pos & 3)))
        return fail(c, AB_ERR_INVALID_ARG, "pos must be a 4-byte aligned device pointer");
    ab::DeviceGuard dg(c->device);
    if (!dg.ok) return fail(c, AB_ERR_CUDA, "cannot make device %d current", c->device);
    CellList& cl = c->cl;
    cl.valid = false;
    Geom g = make_geom(dom, n);
    // clustered inputs leave most cells empty: above 4 cells a particle the
    // table keeps offsets of the occupied cells only (needs the single-launch
    // build; the general path keeps the dense table)
    g.compact = 0;
    if (!g.general && c->coop_launch && c->table_mode != 1 &&
        (c->table_mode == 2 || g.n_cells > 4 * (n > 0 ? n : 1)))
        g.compact = 1;
    const size_t nn = (size_t)(n > 0 ? n : 1);
    cudaError_t e;
    if (nn > cl.cap_n || !cl.spos) {
        // all per-particle buffers share one capacity
        const size_t want = nn + nn / 4 + 64;
        void* fresh[4] = {nullptr, nullptr, nullptr, nullptr};
        // spos, perm, (cell, rank) per particle, tmp: (original index, cell) per slot
        const size_t bytes[4] = {16, 4, 8, 8};
        for (int t = 0; t < 4; ++t) {
            e = cudaMallocAsync(&fresh[t], want * bytes[t], c->stream);
            if (e != cudaSuccess) {
                cudaGetLastError();
                for (int u = 0; u < t; ++u) cudaFreeAsync(fresh[u], c->stream);
                return cuda_fail(c, e, "ab_build (particle buffers)");
            }
        }
        void* old[4] = {cl.spos, cl.perm, cl.cell_rank, cl.tmp};
        for (void* b : old)
            if (b) cudaFreeAsync(b, c->stream);
        cl.spos = (float4*)fresh[0];
        cl.perm = (uint32_t*)fresh[1];
        cl.cell_rank = (uint2*)fresh[2];
        cl.tmp = (uint32_t*)fresh[3];
        cl.cap_n = want;
    }
    const size_t table = g.compact ? (size_t)n + 1 : (size_t)g.n_cells + 1;
    if ((e = grow(&cl.cell_start, &cl.cap_cells, table, c->stream)) != cudaSuccess)
        return cuda_fail(c, e, "ab_build (cell table)");
    // the radix build finds the occupied cells' offsets first, for the dense
    // table too
    const int path = c->build_opt.path == ab::kPathAuto ? ab::auto_build_path(n, g)
                                                        : c->build_opt.path;
    const bool radix = path == ab::kPathRadix && ab::radix_supported(n, g.n_cells);
    if ((g.compact || radix) &&
        (e = grow(&cl.occ, &cl.cap_occ, (size_t)ab::occ_words(g.n_cells), c->stream)) != cudaSuccess)
        return cuda_fail(c, e, "ab_build (occupancy table)");
    if (radix) {
        uint64_t* before = c->sc.rs_status;
        if ((e = grow(&c->sc.rs_status, &c->sc.cap_rs_status,
                      ab::radix_status_words(n, g.n_cells), c->stream)) != cudaSuccess)
            return cuda_fail(c, e, "ab_build (radix look-back words)");
        if (c->sc.rs_status != before) c->sc.rs_epoch = 0;   // fresh memory: clear before use
        if (!c->sc.rs_small) {
            e = cudaMallocAsync((void**)&c->sc.rs_small, ab::radix_small_words() * sizeof(uint32_t),
                                c->stream);
            if (e != cudaSuccess) {
                cudaGetLastError();
                c->sc.rs_small = nullptr;
                return cuda_fail(c, e, "ab_build (radix counts)");
            }
        }
    }
    s = ensure_scan(c, g.n_cells + 1);
    if (s != AB_OK) return s;
    if (!c->sc.coop) {
        e = cudaMallocAsync((void**)&c->sc.coop, ab::coop_scratch_words() * sizeof(uint32_t), c->stream);
        if (e != cudaSuccess) {
            cudaGetLastError();
            c->sc.coop = nullptr;
            return cuda_fail(c, e, "ab_build (build scratch)");
        }
    }
    cl.n = n;
    cl.g = g;
    e = ab::launch_build(cl, pos, packed, c->sc, c->d_err, c->stream, c->build_opt);
    c->build_opt.skip_block = -1;   // the timeout hook applies to one build only
    c->build_opt.limit_ns = 0;
    if (e != cudaSuccess) return cuda_fail(c, e, "ab_build launch");
    cl.user_pos = pos;
    cl.valid = true;
    return AB_OK;
}

ab_status ab_build(ab_ctx* c, const ab_domain* dom, int64_t n, const float* pos4) {
    return build_impl(c, dom, n, pos4, false);
}

ab_status ab_build_packed(ab_ctx* c, const ab_domain* dom, int64_t n, const float* pos) {
    return build_impl(c, dom, n, pos, true);
}

ab_status ab_cell_shape(ab_ctx* c, int32_t* ncell, int64_t* n_cells, int32_t* reach) {
    if (!c) return AB_ERR_INVALID_ARG;
    ab_status s = require_cells(c);
    if (s != AB_OK) return s;
    if (ncell)
        for (int k = 0; k < 3; ++k) ncell[k] = c->cl.g.n[k];
    if (n_cells) *n_cells = c->cl.g.n_cells;
    if (reach) {
        reach[0] = c->cl.g.kx;
        reach[1] = c->cl.g.ky;
        reach[2] = c->cl.g.dim >= 3 ? c->cl.g.kz : 0;
    }
    return AB_OK;
}

ab_status ab_cell_export(ab_ctx* c, uint32_t* perm, uint32_t* cell_start) {
    if (!c) return AB_ERR_INVALID_ARG;
    ab_status s = require_cells(c);
    if (s != AB_OK) return s;
    ab::DeviceGuard dg(c->device);
    if (!dg.ok) return fail(c, AB_ERR_CUDA, "cannot make device %d current", c->device);
    cudaError_t e = cudaSuccess;
    if (perm && c->cl.n > 0)
        e = cudaMemcpyAsync(perm, c->cl.perm, (size_t)c->cl.n * 4, cudaMemcpyDeviceToDevice, c->stream);
    if (e == cudaSuccess && cell_start) {
        if (c->cl.g.compact)
            e = ab::launch_expand_cells(c->cl, cell_start, c->stream);
        else
            e = cudaMemcpyAsync(cell_start, c->cl.cell_start, (size_t)(c->cl.g.n_cells + 1) * 4,
                                cudaMemcpyDeviceToDevice, c->stream);
    }
    return e == cudaSuccess ? AB_OK : cuda_fail(c, e, "ab_cell_export");
}

ab_status ab_pair_sum(ab_ctx* c, ab_op op, const ab_op_params* prm, const float* w,
                      float* out, double* energy) {
    if (!c) return AB_ERR_INVALID_ARG;
    ab_status s = require_cells(c);
    if (s != AB_OK) return s;
    if ((int)op < AB_OP_COUNT || (int)op > AB_OP_SPH_FORCE)
        return fail(c, AB_ERR_INVALID_ARG, "unknown op");
    if (!prm) return fail(c, AB_ERR_INVALID_ARG, "params is NULL");
    const int64_t n = c->cl.n;
    const bool vec = (op == AB_OP_EXPF || op == AB_OP_SOFT || op == AB_OP_SPH_FORCE);
    const bool uses_w = (op == AB_OP_GAUSS || op == AB_OP_SPH_DENSITY || op == AB_OP_SPH_FORCE);
    const size_t wb = (size_t)n * (op == AB_OP_SPH_FORCE ? 8 : 4);
    if (n > 0 && !out) return fail(c, AB_ERR_INVALID_ARG, "out is NULL");
    if (vec && !aligned16(out)) return fail(c, AB_ERR_INVALID_ARG, "vector output must be 16-byte aligned");
    if (uses_w && n > 0 && !w) return fail(c, AB_ERR_INVALID_ARG, "this operator needs w");
    if (op == AB_OP_SPH_FORCE && n > 0 && ((uintptr_t)w & 7u))
        return fail(c, AB_ERR_INVALID_ARG, "SPH_FORCE w (float32[n][2]) must be 8-byte aligned");
    const size_t ob = out_bytes(op, n);
    // the positions were copied at build time; the inputs here are w only
    if ((uses_w && overlaps(out, ob, w, wb)) || (uses_w && overlaps(energy, 8, w, wb)) ||
        overlaps(energy, 8, out, ob))
        return fail(c, AB_ERR_ALIAS, "output overlaps an input");
    ab::DeviceGuard dg(c->device);
    if (!dg.ok) return fail(c, AB_ERR_CUDA, "cannot make device %d current", c->device);
    cudaError_t e;
    if (op == AB_OP_SPH_FORCE) {
        if ((s = ensure_sv(c, n)) != AB_OK) return s;
        e = ab::launch_gather_pairs(c->cl, (const float2*)w, c->sc.sv, c->stream);
        if (e != cudaSuccess) return cuda_fail(c, e, "ab_pair_sum gather");
    } else if (uses_w) {   // w rides in the pad component of the sorted positions
        e = ab::launch_gather_w_pos(c->cl, w, c->stream);
        if (e != cudaSuccess) return cuda_fail(c, e, "ab_pair_sum gather");
    }
    ab::PairOut o;
    o.out = vec ? nullptr : out;
    o.out4 = vec ? (float4*)out : nullptr;
    const int grid = ab::pair_grid(n);
    if (op == AB_OP_LJ && energy) {
        if ((s = ensure_partial(c, (size_t)grid)) != AB_OK) return s;
        o.partial = c->sc.partial;
        o.partial_count = grid;
    }
    e = ab::launch_pair_fwd(c->cl, op, *prm, c->sc.sv, o, c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "ab_pair_sum launch");
    if (op == AB_OP_LJ && energy) {
        if (n > 0) e = ab::launch_reduce_partials(o.partial, grid, energy, c->stream);
        else e = cudaMemsetAsync(energy, 0, sizeof(double), c->stream);
        if (e != cudaSuccess) return cuda_fail(c, e, "ab_pair_sum energy");
    }
    return AB_OK;
}

static ab_status energy_grad_impl(ab_ctx* c, ab_op op, const ab_op_params* prm, float* E,
                                  float* grad, bool packed, double* energy) {
    if (!c) return AB_ERR_INVALID_ARG;
    ab_status s = require_cells(c);
    if (s != AB_OK) return s;
    if (op != AB_OP_LJ) return fail(c, AB_ERR_UNSUPPORTED, "energy + gradient fused for LJ only");
    if (!prm) return fail(c, AB_ERR_INVALID_ARG, "params is NULL");
    const int64_t n = c->cl.n;
    if (!packed && grad && !aligned16(grad))
        return fail(c, AB_ERR_INVALID_ARG, "grad_pos4 must be 16-byte aligned");
    if (packed && grad && ((uintptr_t)grad & 3))
        return fail(c, AB_ERR_INVALID_ARG, "grad_pos must be 4-byte aligned");
    const size_t gbytes = (size_t)n * (packed ? 4 * (size_t)c->cl.g.dim : 16);
    if (overlaps(E, (size_t)n * 4, grad, gbytes) ||
        overlaps(energy, 8, E, (size_t)n * 4) || overlaps(energy, 8, grad, gbytes))
        return fail(c, AB_ERR_ALIAS, "outputs overlap");
    ab::DeviceGuard dg(c->device);
    if (!dg.ok) return fail(c, AB_ERR_CUDA, "cannot make device %d current", c->device);
    ab::PairOut o;
    o.out = E;
    if (packed) o.grad_packed = grad;
    else o.grad_pos = (float4*)grad;
    const int grid = ab::pair_grid(n);
    if (energy) {
        if ((s = ensure_partial(c, (size_t)grid)) != AB_OK) return s;
        o.partial = c->sc.partial;
        o.partial_count = grid;
    }
    cudaError_t e = ab::launch_pair_energy_grad(c->cl, op, *prm, o, c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "ab_pair_energy_grad launch");
    if (energy) {
        if (n > 0) e = ab::launch_reduce_partials(o.partial, grid, energy, c->stream);
        else e = cudaMemsetAsync(energy, 0, sizeof(double), c->stream);
        if (e != cudaSuccess) return cuda_fail(c, e, "ab_pair_energy_grad energy");
    }
    return AB_OK;
}

ab_status ab_pair_energy_grad(ab_ctx* c, ab_op op, const ab_op_params* prm, float* E,
                              float* grad_pos4, double* energy) {
    return energy_grad_impl(c, op, prm, E, grad_pos4, false, energy);
}

ab_status ab_pair_energy_grad_packed(ab_ctx* c, ab_op op, const ab_op_params* prm, float* E,
                                     float* grad_pos, double* energy) {
    return energy_grad_impl(c, op, prm, E, grad_pos, true, energy);
}

static ab_status pair_bwd_impl(ab_ctx* c, ab_op op, const ab_op_params* prm, const float* w,
                               const float* grad_out, float* out, double* energy,
                               float* grad_pos4, float* grad_w, double* grad_s, bool value) {
    if (!c) return AB_ERR_INVALID_ARG;
    ab_status s = require_cells(c);
    if (s != AB_OK) return s;
    if (op != AB_OP_GAUSS && op != AB_OP_LJ)
        return fail(c, AB_ERR_UNSUPPORTED, "adjoint implemented for GAUSS and LJ only");
    if (!prm) return fail(c, AB_ERR_INVALID_ARG, "params is NULL");
    const int64_t n = c->cl.n;
    if (n > 0 && !grad_out) return fail(c, AB_ERR_INVALID_ARG, "grad_out is NULL");
    if (op == AB_OP_GAUSS && n > 0 && !w) return fail(c, AB_ERR_INVALID_ARG, "GAUSS needs weights w");
    if (grad_pos4 && !aligned16(grad_pos4)) return fail(c, AB_ERR_INVALID_ARG, "grad_pos4 must be 16-byte aligned");
    if (op != AB_OP_LJ) energy = nullptr;      // the LJ total only
    const size_t n4 = (size_t)n * 4, n16 = (size_t)n * 16;
    const void* ins[2] = {w, grad_out};
    const size_t inb[2] = {n4, n4};
    const void* outs[5] = {grad_pos4, grad_w, grad_s, out, energy};
    const size_t outb[5] = {n16, n4, 8, n4, 8};
    for (int a = 0; a < 5; ++a) {
        for (int t = 0; t < 2; ++t)
            if (overlaps(outs[a], outb[a], ins[t], inb[t]))
                return fail(c, AB_ERR_ALIAS, "an output overlaps an input");
        for (int b = a + 1; b < 5; ++b)
            if (overlaps(outs[a], outb[a], outs[b], outb[b]))
                return fail(c, AB_ERR_ALIAS, "outputs overlap");
    }
    ab::DeviceGuard dg(c->device);
    if (!dg.ok) return fail(c, AB_ERR_CUDA, "cannot make device %d current", c->device);
    cudaError_t e;
    if ((s = ensure_sv(c, n)) != AB_OK) return s;
    // g into the pad of the sorted positions; GAUSS also needs w, as float[n]
    e = ab::launch_gather_w_pos(c->cl, grad_out, c->stream);
    if (e == cudaSuccess && op == AB_OP_GAUSS)
        e = ab::launch_gather_scalar(c->cl, w, reinterpret_cast<float*>(c->sc.sv), c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "adjoint gather");
    ab::PairOut o;
    o.grad_pos = (float4*)grad_pos4;
    o.grad_w = op == AB_OP_GAUSS ? grad_w : nullptr;
    o.out = value ? out : nullptr;
    const int grid = ab::pair_grid(n);
    double* red = op == AB_OP_GAUSS ? grad_s : (value ? energy : nullptr);
    if (red) {
        if ((s = ensure_partial(c, (size_t)grid)) != AB_OK) return s;
        o.partial = c->sc.partial;
        o.partial_count = grid;
    }
    e = ab::launch_pair_bwd(c->cl, op, *prm, c->sc.sv, o, c->stream, value);
    if (e != cudaSuccess) return cuda_fail(c, e, "adjoint launch");
    if (red) {
        if (n > 0) e = ab::launch_reduce_partials(o.partial, grid, red, c->stream);
        else e = cudaMemsetAsync(red, 0, sizeof(double), c->stream);
        if (e != cudaSuccess) return cuda_fail(c, e, "adjoint reduction");
    }
    return AB_OK;
}

ab_status ab_pair_sum_bwd(ab_ctx* c, ab_op op, const ab_op_params* prm, const float* w,
                          const float* grad_out, float* grad_pos4, float* grad_w,
                          double* grad_s) {
    return pair_bwd_impl(c, op, prm, w, grad_out, nullptr, nullptr, grad_pos4, grad_w, grad_s,
                         false);
}

ab_status ab_pair_sum_value_grad(ab_ctx* c, ab_op op, const ab_op_params* prm, const float* w,
                                 const float* grad_out, float* out, double* energy,
                                 float* grad_pos4, float* grad_w, double* grad_s) {
    return pair_bwd_impl(c, op, prm, w, grad_out, out, energy, grad_pos4, grad_w, grad_s, true);
}

ab_status ab_pair_list(ab_ctx* c, int64_t* offsets, int32_t* idx, int64_t cap, int64_t* nnz) {
    if (!c) return AB_ERR_INVALID_ARG;
    ab_status s = require_cells(c);
    if (s != AB_OK) return s;
    const int64_t n = c->cl.n;
    if (!offsets || !nnz || cap < 0 || (cap > 0 && !idx))
        return fail(c, AB_ERR_INVALID_ARG, "offsets, nnz required; idx required when cap > 0");
    if (overlaps(offsets, (size_t)(n + 1) * 8, idx, (size_t)cap * 4))
        return fail(c, AB_ERR_ALIAS, "offsets overlap idx");
    ab::DeviceGuard dg(c->device);
    if (!dg.ok) return fail(c, AB_ERR_CUDA, "cannot make device %d current", c->device);
    cudaError_t e = grow(&c->sc.counts, &c->sc.cap_counts, (size_t)n + 1, c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "ab_pair_list workspace");
    if ((s = ensure_scan(c, n + 1)) != AB_OK) return s;
    e = cudaMemsetAsync(c->sc.counts, 0, (size_t)(n + 1) * 4, c->stream);
    if (e == cudaSuccess) e = ab::launch_pair_count(c->cl, c->sc.counts, c->stream);
    if (e == cudaSuccess)
        e = ab::launch_scan_u32_to_i64(c->sc.counts, offsets, n + 1, c->sc.scan_status,
                                       c->sc.scan_ticket, c->d_err, c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "ab_pair_list count");
    int64_t total = 0;
    e = cudaMemcpyAsync(&total, offsets + n, sizeof(int64_t), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "ab_pair_list total");
    *nnz = total;
    if (total > cap) return fail(c, AB_ERR_CAPACITY, "need %lld index slots", (long long)total);
    e = ab::launch_pair_emit(c->cl, offsets, idx, c->stream);
    return e == cudaSuccess ? AB_OK : cuda_fail(c, e, "ab_pair_list emit");
}

static ab_status check_dense(ab_ctx* c, int64_t m, int64_t n, const float* X, const float* Y,
                             int32_t nrhs, const float* W, ab_prec prec) {
    if (m < 0 || n < 0 || m >= (int64_t(1) << 31) || n >= (int64_t(1) << 31))
        return fail(c, AB_ERR_INVALID_ARG, "m, n out of range");
    if (nrhs < 1 || nrhs > 64) return fail(c, AB_ERR_INVALID_ARG, "nrhs must be in [1, 64]");
    if ((int)prec < AB_PREC_FP32 || (int)prec > AB_PREC_BF16) return fail(c, AB_ERR_INVALID_ARG, "unknown precision");
    if ((m > 0 && (!X || !aligned16(X))) || (n > 0 && (!Y || !aligned16(Y))))
        return fail(c, AB_ERR_INVALID_ARG, "X, Y must be 16-byte aligned float32[.][4]");
    if (n > 0 && !W) return fail(c, AB_ERR_INVALID_ARG, "W is NULL");
    return AB_OK;
}

ab_status ab_kernel_matvec(ab_ctx* c, int64_t m, int64_t n, const float* X, const float* Y,
                           int32_t nrhs, const float* W, float s, ab_prec prec, float* out) {
    if (!c) return AB_ERR_INVALID_ARG;
    ab_status st = check_dense(c, m, n, X, Y, nrhs, W, prec);
    if (st != AB_OK) return st;
    if (m > 0 && !out) return fail(c, AB_ERR_INVALID_ARG, "out is NULL");
    const size_t ob = (size_t)m * nrhs * 4;
    if (overlaps(out, ob, X, (size_t)m * 16) || overlaps(out, ob, Y, (size_t)n * 16) ||
        overlaps(out, ob, W, (size_t)n * nrhs * 4))
        return fail(c, AB_ERR_ALIAS, "out overlaps an input");
    ab::DeviceGuard dg(c->device);
    if (!dg.ok) return fail(c, AB_ERR_CUDA, "cannot make device %d current", c->device);
    cudaError_t e;
    if (prec == AB_PREC_FP32) {
        e = ab::launch_dense_fwd(m, n, (const float4*)X, (const float4*)Y, nrhs, W, s, prec, out,
                                 c->stream);
    } else {
        if (nrhs != 64)
            return fail(c, AB_ERR_UNSUPPORTED, "tensor-core paths need nrhs == 64");
        e = grow(&c->sc.dense_ws, &c->sc.cap_dense_ws, ab::dense_tc_workspace_bytes(n), c->stream);
        if (e != cudaSuccess) return cuda_fail(c, e, "ab_kernel_matvec workspace");
        e = ab::launch_dense_tc_fwd(m, n, (const float4*)X, (const float4*)Y, nrhs, W, s, prec, out,
                                    c->sc.dense_ws, c->d_err, c->stream);
    }
    if (e == cudaErrorNotSupported)
        return fail(c, AB_ERR_UNSUPPORTED, "precision not available for this shape");
    return e == cudaSuccess ? AB_OK : cuda_fail(c, e, "ab_kernel_matvec");
}

ab_status ab_kernel_solve(ab_ctx* c, int64_t n, const float* X, int32_t nrhs, const float* B,
                          float s, float sigma2, ab_prec prec, float tol, int32_t max_iter, float* W,
                          int32_t* iters, float* relres) {
    if (!c) return AB_ERR_INVALID_ARG;
    ab_status st = check_dense(c, n, n, X, X, nrhs, B, prec);
    if (st != AB_OK) return st;
    if (n > 0 && !W) return fail(c, AB_ERR_INVALID_ARG, "W is NULL");
    if (!isfinite(s) || !isfinite(sigma2) || sigma2 < 0.0f || !(tol > 0.0f) || !isfinite(tol) ||
        max_iter < 0)
        return fail(c, AB_ERR_INVALID_ARG, "need finite s, sigma2 >= 0, tol > 0, max_iter >= 0");
    if (prec != AB_PREC_FP32 && nrhs != 64)
        return fail(c, AB_ERR_UNSUPPORTED, "tensor-core paths need nrhs == 64");
    const size_t vb = (size_t)n * nrhs * 4;
    if (overlaps(W, vb, X, (size_t)n * 16) || overlaps(W, vb, B, vb))
        return fail(c, AB_ERR_ALIAS, "W overlaps an input");
    if (iters) *iters = 0;
    if (relres) *relres = 0.0f;
    if (n == 0) return AB_OK;
    ab::DeviceGuard dg(c->device);
    if (!dg.ok) return fail(c, AB_ERR_CUDA, "cannot make device %d current", c->device);
    cudaError_t e = grow(&c->sc.solve_ws, &c->sc.cap_solve_ws, ab::solve_workspace_bytes(n, nrhs),
                         c->stream);
    if (e == cudaSuccess && prec != AB_PREC_FP32)
        e = grow(&c->sc.dense_ws, &c->sc.cap_dense_ws, ab::dense_tc_workspace_bytes(n), c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "ab_kernel_solve workspace");
    const float4* X4 = (const float4*)X;
    const ab::SolveMatvec mv = [&](const float* P, float* Q) -> cudaError_t {
        if (prec == AB_PREC_FP32) return ab::launch_dense_fwd(n, n, X4, X4, nrhs, P, s, prec, Q, c->stream);
        return ab::launch_dense_tc_fwd(n, n, X4, X4, nrhs, P, s, prec, Q, c->sc.dense_ws, c->d_err,
                                       c->stream);
    };
    int it = 0;
    float rr = 0.0f;
    e = ab::run_solve(n, nrhs, B, sigma2, tol, max_iter, W, c->sc.solve_ws, mv, &it, &rr, c->stream);
    if (e == cudaErrorNotSupported)
        return fail(c, AB_ERR_UNSUPPORTED, "precision not available for this shape");
    if (e != cudaSuccess) return cuda_fail(c, e, "ab_kernel_solve");
    if (iters) *iters = it;
    if (relres) *relres = rr;
    return AB_OK;
}

ab_status ab_kernel_matvec_bwd(ab_ctx* c, int64_t m, int64_t n, const float* X, const float* Y,
                               int32_t nrhs, const float* W, float s, ab_prec prec,
                               const float* G, float* dW, float* dX, float* dY, double* ds) {
    if (!c) return AB_ERR_INVALID_ARG;
    ab_status st = check_dense(c, m, n, X, Y, nrhs, W, prec);
    if (st != AB_OK) return st;
    if (m > 0 && !G) return fail(c, AB_ERR_INVALID_ARG, "G is NULL");
    if ((dX && !aligned16(dX)) || (dY && !aligned16(dY)))
        return fail(c, AB_ERR_INVALID_ARG, "dX, dY must be 16-byte aligned");
    const void* ins[4] = {X, Y, W, G};
    const size_t inb[4] = {(size_t)m * 16, (size_t)n * 16, (size_t)n * nrhs * 4, (size_t)m * nrhs * 4};
    const void* outs[4] = {dW, dX, dY, ds};
    const size_t outb[4] = {(size_t)n * nrhs * 4, (size_t)m * 16, (size_t)n * 16, 8};
    for (int a = 0; a < 4; ++a) {
        for (int b = 0; b < 4; ++b)
            if (overlaps(outs[a], outb[a], ins[b], inb[b]))
                return fail(c, AB_ERR_ALIAS, "an output overlaps an input");
        for (int b = a + 1; b < 4; ++b)
            if (overlaps(outs[a], outb[a], outs[b], outb[b]))
                return fail(c, AB_ERR_ALIAS, "outputs overlap");
    }
    ab::DeviceGuard dg(c->device);
    if (!dg.ok) return fail(c, AB_ERR_CUDA, "cannot make device %d current", c->device);
    double* partial = nullptr;
    if (ds) {
        // SIMT: one partial per 128-row block; tensor cores: up to two per block
        if ((st = ensure_partial(c, 2 * (size_t)ab::dense_partial_capacity(m, n) + 2)) != AB_OK) return st;
        partial = c->sc.partial;
    }
    int pc = 0;
    cudaError_t e;
    if (prec == AB_PREC_FP32) {
        e = ab::launch_dense_bwd(m, n, (const float4*)X, (const float4*)Y, nrhs, W, s, prec, G, dW,
                                 (float4*)dX, (float4*)dY, partial, &pc, c->stream);
    } else {
        if (nrhs != 64)
            return fail(c, AB_ERR_UNSUPPORTED, "tensor-core paths need nrhs == 64");
        // dW = K(Y, X) G: the forward kernel with the roles swapped;
        // dX (+ ds) and dY: the tensor-core gradient kernel
        size_t need = ab::dense_tc_workspace_bytes(m);
        const size_t g1 = ab::dense_tc_grad_workspace_bytes(m, n);
        const size_t g2 = ab::dense_tc_grad_workspace_bytes(n, m);
        if (g1 > need) need = g1;
        if (g2 > need) need = g2;
        e = grow(&c->sc.dense_ws, &c->sc.cap_dense_ws, need, c->stream);
        if (e == cudaSuccess && dW && n > 0)
            e = ab::launch_dense_tc_fwd(n, m, (const float4*)Y, (const float4*)X, nrhs, G, s, prec, dW,
                                        c->sc.dense_ws, c->d_err, c->stream);
        if (e == cudaSuccess && (dX || partial) && m > 0)
            e = ab::launch_dense_tc_gradx(m, n, (const float4*)X, (const float4*)Y, G, W, s, prec,
                                          (float4*)dX, partial, &pc, c->sc.dense_ws, c->d_err, c->stream);
        if (e == cudaSuccess && dY && n > 0) {
            int pc2 = 0;
            e = ab::launch_dense_tc_gradx(n, m, (const float4*)Y, (const float4*)X, W, G, s, prec,
                                          (float4*)dY, nullptr, &pc2, c->sc.dense_ws, c->d_err,
                                          c->stream);
        }
    }
    if (e == cudaErrorNotSupported)
        return fail(c, AB_ERR_UNSUPPORTED, "precision not available for this shape");
    if (e != cudaSuccess) return cuda_fail(c, e, "ab_kernel_matvec_bwd");
    if (ds) {
        e = pc > 0 ? ab::launch_reduce_partials(partial, pc, ds, c->stream)
                   : cudaMemsetAsync(ds, 0, sizeof(double), c->stream);
        if (e != cudaSuccess) return cuda_fail(c, e, "ab_kernel_matvec_bwd ds");
    }
    return AB_OK;
}

ab_status ab_bd_step(ab_ctx* c, const ab_domain* dom, int64_t n, float* pos4,
                     const float* force4, float dt, float D, uint64_t seed, uint64_t step) {
    if (!c) return AB_ERR_INVALID_ARG;
    ab_status s = check_domain(c, dom);
    if (s != AB_OK) return s;
    if (n < 0 || n >= (int64_t(1) << 31)) return fail(c, AB_ERR_INVALID_ARG, "n out of range");
    if (n > 0 && (!pos4 || !aligned16(pos4) || (force4 && !aligned16(force4))))
        return fail(c, AB_ERR_INVALID_ARG, "pos4/force4 must be 16-byte aligned");
    if (!isfinite(dt) || !isfinite(D) || D < 0.0f)
        return fail(c, AB_ERR_INVALID_ARG, "dt, D must be finite, D >= 0");
    if (overlaps(pos4, (size_t)n * 16, force4, (size_t)n * 16))
        return fail(c, AB_ERR_ALIAS, "force4 overlaps pos4");
    ab::DeviceGuard dg(c->device);
    if (!dg.ok) return fail(c, AB_ERR_CUDA, "cannot make device %d current", c->device);
    Geom g = make_geom(dom, 0);
    cudaError_t e = ab::launch_bd_step(g, n, (float4*)pos4, (const float4*)force4, dt, D, seed,
                                       step, c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "ab_bd_step");
    if (pos4 == c->cl.user_pos) c->cl.valid = false;
    return AB_OK;
}

ab_status ab_md_step(ab_ctx* c, const ab_domain* dom, int64_t n, float* pos4, float* vel4,
                     const float* acc4, float dt) {
    if (!c) return AB_ERR_INVALID_ARG;
    ab_status s = check_domain(c, dom);
    if (s != AB_OK) return s;
    if (n < 0 || n >= (int64_t(1) << 31)) return fail(c, AB_ERR_INVALID_ARG, "n out of range");
    if (n > 0 && (!pos4 || !vel4 || !acc4 || !aligned16(pos4) || !aligned16(vel4) || !aligned16(acc4)))
        return fail(c, AB_ERR_INVALID_ARG, "pos4/vel4/acc4 must be non-NULL and 16-byte aligned");
    if (!isfinite(dt)) return fail(c, AB_ERR_INVALID_ARG, "dt must be finite");
    const size_t b = (size_t)n * 16;
    if (overlaps(pos4, b, vel4, b) || overlaps(pos4, b, acc4, b) || overlaps(vel4, b, acc4, b))
        return fail(c, AB_ERR_ALIAS, "pos4, vel4 and acc4 must not overlap");
    ab::DeviceGuard dg(c->device);
    if (!dg.ok) return fail(c, AB_ERR_CUDA, "cannot make device %d current", c->device);
    Geom g = make_geom(dom, 0);
    cudaError_t e = ab::launch_md_step(g, n, (float4*)pos4, (float4*)vel4, (const float4*)acc4, dt,
                                       c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "ab_md_step");
    if (pos4 == c->cl.user_pos) c->cl.valid = false;
    return AB_OK;
}

// ---- testing hooks -------------------------------------------------------

ab_status ab_testing_cell_table(ab_ctx* c, int32_t mode) {
    if (!c || mode < 0 || mode > 2) return AB_ERR_INVALID_ARG;
    c->table_mode = mode;
    return AB_OK;
}

ab_status ab_testing_build_path(ab_ctx* c, int32_t path) {
    if (!c || path < ab::kPathSequence || path > ab::kPathAuto) return AB_ERR_INVALID_ARG;
    c->build_opt.path = path;
    return AB_OK;
}

ab_status ab_testing_build_timeout(ab_ctx* c, int32_t skip_block, int64_t limit_ns) {
    if (!c || skip_block < 0 || limit_ns <= 0 || limit_ns > 2000000000ll) return AB_ERR_INVALID_ARG;
    c->build_opt.skip_block = skip_block;
    c->build_opt.limit_ns = (long long)limit_ns;
    return AB_OK;
}

ab_status ab_testing_scan_timeout(ab_ctx* c, int64_t items, int32_t skip_tile,
                                  int64_t limit_ns) {
    if (!c || items < 1 || items >= (int64_t(1) << 30) || skip_tile < 0 || limit_ns <= 0 ||
        limit_ns > 2000000000ll)
        return AB_ERR_INVALID_ARG;
    ab::DeviceGuard dg(c->device);
    if (!dg.ok) return fail(c, AB_ERR_CUDA, "cannot make device %d current", c->device);
    cudaError_t e = grow(&c->sc.counts, &c->sc.cap_counts, (size_t)items, c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "testing scan workspace");
    ab_status s = ensure_scan(c, items);
    if (s != AB_OK) return s;
    e = cudaMemsetAsync(c->sc.counts, 0, (size_t)items * 4, c->stream);
    if (e == cudaSuccess)
        e = ab::launch_scan_u32(c->sc.counts, c->sc.counts, items, c->sc.scan_status,
                                c->sc.scan_ticket, c->d_err, skip_tile, (long long)limit_ns,
                                c->stream);
    return e == cudaSuccess ? AB_OK : cuda_fail(c, e, "testing scan");
}

}  // extern "C"
#pragma GCC visibility pop
