/*
 * aboria_gpu_testing.h -- test hooks of the aboria_gpu library.
 *
 * These entry points exist so that tests can exercise device-side error
 * paths without faulting or hanging a GPU.  They are not part of the
 * computational API and the paper has no counterpart for them.
 */
#ifndef ABORIA_GPU_TESTING_H
#define ABORIA_GPU_TESTING_H

#include <stdint.h>

#include "aboria_gpu.h"

#ifdef __cplusplus
extern "C" {
#endif

/* Run the cell-offset scan (the decoupled look-back prefix scan used by
 * ab_build) over `items` zeros on the context's scratch, with tile
 * `skip_tile` never publishing its status, so that the next tile's bounded
 * wait runs out after `limit_ns` nanoseconds (0 < limit_ns <= 2e9).  The
 * kernel then records the timeout in the context's error word and finishes;
 * the following ab_sync() returns AB_ERR_TIMEOUT and clears it.  Nothing
 * spins without a limit and no memory outside the scratch is touched.
 * Errors: AB_ERR_INVALID_ARG, AB_ERR_OOM, AB_ERR_CUDA. */
ab_status ab_testing_scan_timeout(ab_ctx* ctx, int64_t items, int32_t skip_tile,
                                  int64_t limit_ns);

/* Select the cell table of the following ab_build calls: mode 0 (the
 * default) keeps offsets of the occupied cells only when the lattice has
 * more than 4 cells a particle, 1 always keeps the dense table of every
 * cell, 2 always keeps the compact one (except on the general path, which
 * is always dense).  Every result is the same bit for bit; only memory and
 * time differ.  Errors: AB_ERR_INVALID_ARG. */
ab_status ab_testing_cell_table(ab_ctx* ctx, int32_t mode);

/* Select how the following ab_build calls run:
 *   0  the counting sort as a sequence of kernels (hash + atomic histogram,
 *      scan, scatter, stable finalize); a compact table has no sequence form
 *      and is built as in 1;
 *   1  the same counting sort in one cooperative launch whose phases are
 *      separated by bounded grid-wide barriers (above 2^21 particles with a
 *      dense table the kernel sequence is used);
 *   2  the stable radix sort of the cell ids (no per-particle global
 *      atomic; see ab_build);
 *   3  the automatic choice (the default).
 * Every path gives the same cell list bit for bit.
 * Errors: AB_ERR_INVALID_ARG. */
ab_status ab_testing_build_path(ab_ctx* ctx, int32_t path);

/* Make the next ab_build exercise its bounded wait.  On the cooperative
 * launch, block `skip_block` (clamped to none if the grid is smaller) never
 * arrives at the first grid barrier, so every other block's wait there gives
 * up after `limit_ns` nanoseconds (0 < limit_ns <= 2e9); all later waits of
 * that launch are bounded the same way, so it ends after at most one limit
 * per grid barrier (five for a dense table, eight for a compact one).  On the radix sort, tile `skip_block` of the scan of the first
 * digit's counts never publishes its sum, so the look-back of the scan tiles
 * after it gives up after `limit_ns`.  Either way the timeout is recorded as AB_ERR_TIMEOUT in the
 * context's error word, every access stays inside the library's buffers, the
 * cell list left behind is garbage, the following ab_sync() returns
 * AB_ERR_TIMEOUT, and a new ab_build restores a valid cell list.  Applies to
 * one build only.  Errors: AB_ERR_INVALID_ARG. */
ab_status ab_testing_build_timeout(ab_ctx* ctx, int32_t skip_block, int64_t limit_ns);

#ifdef __cplusplus
}
#endif

#endif /* ABORIA_GPU_TESTING_H */
