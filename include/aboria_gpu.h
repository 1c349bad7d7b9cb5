/*
 * aboria_gpu.h -- C ABI of the GB300 (sm_103a) particle-interaction library.
 *
 * The operations follow the problem statement of "Particle-based and Meshless
 * Methods with Aboria" (arXiv:1704.08907):
 *   - Sec. 1: N particles with positions in a d-dimensional hypercube, each
 *     axis periodic or not, and operators defined by positions and
 *     per-particle variables, typically sums over pairs of close particles;
 *   - Sec. 2.2.1: a cell-list search structure built in parallel by
 *     reordering the particles by cell;
 *   - Sec. 2.2.2: a box search over a particle's cell and the adjacent cells;
 *   - Sec. 3, Eq. 1 and the velocity-update listing: the radius-filtered sum
 *     over the shortest separation vector dx_ij = r_j - r_i;
 *   - Sec. 1 / 1.1: dense kernel operators of RBF interpolation and Gaussian
 *     processes (global operators named for fast summation in Sec. 2.2.2).
 *
 * Conventions for every entry point
 * ---------------------------------
 *  - All array arguments are DEVICE pointers on the context's device, unless
 *    a comment says "host".  The caller owns them; the library never frees
 *    or retains them past the call, except that ab_build records the
 *    positions pointer and size to detect stale use.
 *  - Positions are float32[n][4] (x, y, z, pad), 16-byte aligned; for d = 2
 *    the z and pad components are ignored.  The *_packed entry points take
 *    d floats per particle instead (4-byte aligned).  Per-particle scalars
 *    are float32[n].  Inputs and outputs are in the caller's particle order.
 *  - Every call is asynchronous on the context's CUDA stream.  Argument
 *    errors are returned immediately and launch nothing.  Errors detected on
 *    the device (a wait that timed out) are latched and returned by the next
 *    ab_sync().
 *  - Outputs must not overlap the call's inputs (the paper's aliasing rule,
 *    Sec. 2.2.3: an operator that writes what it reads goes through a
 *    temporary); an overlap returns AB_ERR_ALIAS.  ab_build copies the
 *    positions into the library's sorted workspace, so later pair sums do
 *    not read the caller's position array and may overwrite it.
 *  - The context owns its workspace (cell table, sorted copies, scan state)
 *    and grows it on demand with cudaMallocAsync on the context's stream
 *    (the device's default memory pool); AB_ERR_OOM leaves the context
 *    usable with its previous workspace.
 *  - Each call makes the context's device current while it runs and
 *    restores the caller's current device before it returns; a failure to
 *    select the device returns AB_ERR_CUDA.
 *  - A context is not thread-safe; use one per host thread / stream.
 */
#ifndef ABORIA_GPU_H
#define ABORIA_GPU_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ab_ctx ab_ctx;

typedef enum {
    AB_OK = 0,
    AB_ERR_INVALID_ARG = 1,  /* bad size, dimension, radius, box or pointer */
    AB_ERR_ALIAS = 2,        /* an output overlaps an input */
    AB_ERR_STALE = 3,        /* no cell list, or positions moved since build */
    AB_ERR_OOM = 4,          /* workspace allocation failed */
    AB_ERR_CUDA = 5,         /* a CUDA runtime call failed */
    AB_ERR_TIMEOUT = 6,      /* a bounded device-side wait gave up */
    AB_ERR_UNSUPPORTED = 7,  /* valid request this build does not implement */
    AB_ERR_CAPACITY = 8      /* caller's output buffer is too small */
} ab_status;

/* The hypercube domain (Sec. 1 property 1; Sec. 3 neighbour-search set-up):
 * [lo_k, hi_k) per axis k < dim, periodic[k] != 0 for a periodic axis, and
 * the interaction radius r_cut.  Positions on periodic axes must lie in
 * [lo, hi); on non-periodic axes they may lie anywhere (out-of-box particles
 * are indexed in the edge cells, distances use raw coordinates). */
typedef struct {
    int32_t dim;          /* 2 or 3 */
    int32_t periodic[3];
    float lo[3];
    float hi[3];
    float radius;         /* r > 0; pairs satisfy |dx|^2 < r*r (FP32) */
} ab_domain;

/* Built-in pair operators f (the paper's Level-3 expression is replaced by
 * this fixed set; each is evaluated for j != i with |dx_ij| < r):
 *   AB_OP_COUNT  y_i = number of neighbours                        (scalar)
 *   AB_OP_GAUSS  y_i = sum_j w_j exp(-s |dx|^2)                     (scalar)
 *   AB_OP_LJ     y_i = 1/2 sum_j eps((sig/|dx|)^12 - (sig/|dx|)^6)  (scalar;
 *                total energy = sum_i y_i; truncated, not shifted)
 *   AB_OP_EXPF   y_i = c sum_{j,|dx|>0} -exp(-|dx|) dx/|dx|  (Eq. 1; vector)
 *   AB_OP_SOFT   y_i = sum_{j,|dx|>0} -k (r - |dx|) dx/|dx|         (vector)
 * Scalar outputs are float32[n]; vector outputs float32[n][4] (pad = 0). */
typedef enum {
    AB_OP_COUNT = 0,
    AB_OP_GAUSS = 1,
    AB_OP_LJ = 2,
    AB_OP_EXPF = 3,
    AB_OP_SOFT = 4,
    /* SPH (Sec. 1 lists SPH among the particle methods), Wendland C2 kernel
     * with support r: W(d) = a (1 - d/r)^4 (1 + 4 d/r),
     * a = 21 / (2 pi r^3) in 3-D, 7 / (pi r^2) in 2-D (normalised). */
    AB_OP_SPH_DENSITY = 5,   /* rho_i = m_i W(0) + sum_j m_j W(d_ij); w = m */
    AB_OP_SPH_FORCE = 6      /* a_i = -sum_j m_j (A_i + A_j) grad_i W(d_ij),
                                w = (m, A = P / rho^2) per particle */
} ab_op;

typedef struct {
    float s;      /* GAUSS: exp(-s d^2), s = 1/h^2 */
    float eps;    /* LJ */
    float sigma;  /* LJ */
    float c;      /* EXPF (Eq. 1) */
    float k;      /* SOFT spring constant */
} ab_op_params;

/* Arithmetic of the dense kernel operator's two contractions. */
typedef enum {
    AB_PREC_FP32 = 0,    /* FP32 CUDA cores, direct |x - y|^2 */
    AB_PREC_TF32X3 = 1,  /* tensor cores, TF32 hi+lo split (3 products) */
    AB_PREC_BF16X3 = 2,  /* tensor cores, BF16 hi+lo split (3 products) */
    AB_PREC_TF32 = 3,    /* tensor cores, plain TF32 (reported, not exact) */
    AB_PREC_BF16 = 4     /* tensor cores, plain BF16 (reported, not exact) */
} ab_prec;

/* Create a context on CUDA device `device` issuing work on `stream`
 * (a cudaStream_t; NULL = the legacy default stream).  *ctx receives the
 * handle.  Errors: AB_ERR_INVALID_ARG (null ctx, bad device), AB_ERR_CUDA,
 * AB_ERR_OOM. */
ab_status ab_create(ab_ctx** ctx, int device, void* stream);

/* Synchronise the context's stream and release its workspace. */
ab_status ab_destroy(ab_ctx* ctx);

/* Issue subsequent work on `stream` (a cudaStream_t). */
ab_status ab_set_stream(ab_ctx* ctx, void* stream);

/* Wait for the context's stream; return AB_ERR_TIMEOUT if a device-side wait
 * gave up since the last ab_sync (the latch is then cleared), AB_ERR_CUDA on
 * a CUDA error, else AB_OK. */
ab_status ab_sync(ab_ctx* ctx);

/* Build the cell list (Sec. 2.2.1: a lattice of hypercube cells, filled in
 * parallel by reordering the particles; Sec. 3 sets the cell width to
 * r_cut).  Cell width per axis w_k = L_k / n_k with
 *   n_k = max(1, floor(L_k / (r (1 + 2^-18) + L_k 2^-18)))
 * (a width a hair above r, so rounding of the FP32 cell index can never hide
 * a pair from the 3^d stencil), coarsened uniformly if the table would
 * exceed max(2^22, 8n) cells; then, room permitting, the x cells are split
 * into kx = 2..4 parts (see ab_cell_shape).  Steps: cell hash + histogram, exclusive scan
 * of the counts (cell offsets), stable counting-sort scatter of the
 * positions.  The sort is stable: within a cell, particles keep ascending
 * original index, so every later result is deterministic.  When the lattice
 * has more than 4 cells a particle (clustered inputs leave most cells
 * empty), the library keeps offsets of the occupied cells only, with a
 * bitmap of occupied cells to find them (about 0.25 bytes a cell plus 4 a
 * particle instead of 4 bytes a cell); the order and every result are the
 * same bit for bit.  Up to 2^21 particles, and for every compact table, the
 * build runs as one cooperative launch whose phases are separated by grid
 * barriers with bounded waits (a wait that gives up is reported by ab_sync
 * as AB_ERR_TIMEOUT); larger dense builds run as a sequence of kernels.
 *   dom:  host pointer to the domain (copied).
 *   n:    number of particles, 0 <= n < 2^31.
 *   pos4: float32[n][4] device positions (16-byte aligned).
 * Errors: AB_ERR_INVALID_ARG (dim not 2/3, radius <= 0 or not finite,
 * hi <= lo, n out of range, misaligned or null pos4 with n > 0), AB_ERR_OOM,
 * AB_ERR_CUDA. */
ab_status ab_build(ab_ctx* ctx, const ab_domain* dom, int64_t n,
                   const float* pos4);

/* ab_build for positions packed as dom->dim floats per particle
 * (float32[n][3] in 3-D, float32[n][2] in 2-D, device, 4-byte aligned): the
 * layout arrays of coordinates usually have, a quarter (3-D) or half (2-D)
 * fewer bytes to bring to the device than pos4.  The cell list, and every
 * later result, is bit for bit that of ab_build on the same coordinates.
 * Errors as ab_build (AB_ERR_INVALID_ARG for a null or misaligned pos). */
ab_status ab_build_packed(ab_ctx* ctx, const ab_domain* dom, int64_t n,
                          const float* pos);

/* Shape of the last cell list: cells per axis (host int32[3]), the total
 * (host int64), and the stencil reach per axis (host int32[3]: the box
 * search visits cells c - reach .. c + reach).  Along x the cells may be a
 * fraction 1/reach[0] of the cut-off wide (reach[0] in 1..4): a stencil row
 * then covers (2 reach + 1) / reach cut-off widths instead of 3, with the
 * same 3^(d-1) rows.  Any pointer may be NULL.  Errors: AB_ERR_STALE if
 * nothing was built. */
ab_status ab_cell_shape(ab_ctx* ctx, int32_t* ncell, int64_t* n_cells,
                        int32_t* reach);

/* Copy out the last cell list for inspection: perm (device uint32[n],
 * perm[s] = original index of sorted slot s) and cell_start (device
 * uint32[n_cells + 1], particles of cell c occupy slots
 * [cell_start[c], cell_start[c+1]); a compact table is expanded to every
 * cell).  Either pointer may be NULL. */
ab_status ab_cell_export(ab_ctx* ctx, uint32_t* perm, uint32_t* cell_start);

/* Fixed-radius pair sum over the last cell list (Sec. 2.2.2 box search over
 * the cell and its adjacent cells; Sec. 3 Eq. 1 / velocity-update listing):
 *   y_i = sum_{j != i, |dx_ij|^2 < r^2} f(dx_ij, v_i, v_j)
 * with dx_ij the minimum-image separation.  The neighbour predicate is
 * evaluated in FP32 exactly as:
 *   dx = x_j - x_i; on a periodic axis: if dx > L/2: dx -= L,
 *                                       else if dx < -L/2: dx += L;
 *   d2 = (dx0*dx0 + dx1*dx1) + dx2*dx2 (round-to-nearest, no FMA);
 *   pair iff d2 < fl(r*r).
 * Values are accumulated in FP32.
 *   op, prm: operator and its parameters (host pointer).
 *   w:       float32[n] weights (GAUSS), masses m (SPH_DENSITY), or
 *            float32[n][2] pairs (m, P/rho^2) (SPH_FORCE); else ignored
 *            (may be NULL).
 *   out:     float32[n] (COUNT/GAUSS/LJ/SPH_DENSITY) or float32[n][4]
 *            (EXPF/SOFT/SPH_FORCE).
 *   energy:  optional device float64[1]; for LJ receives sum_i y_i
 *            (reduced in FP64 in a fixed order), else left unchanged.
 * Errors: AB_ERR_STALE (no build, or positions moved by ab_bd_step since),
 * AB_ERR_INVALID_ARG, AB_ERR_ALIAS, AB_ERR_OOM, AB_ERR_CUDA. */
ab_status ab_pair_sum(ab_ctx* ctx, ab_op op, const ab_op_params* prm,
                      const float* w, float* out, double* energy);

/* Adjoint of ab_pair_sum for a loss L with upstream gradient
 * grad_out = dL/dy (float32[n]).  Pairs are recomputed from the cell list;
 * no neighbour list is stored.
 *   GAUSS: grad_pos4 (float32[n][4]) = dL/dx_i
 *            = sum_j (g_i w_j + g_j w_i) 2 s exp(-s d^2) dx_ij,
 *          grad_w (float32[n]) = dL/dw_i = sum_j g_j exp(-s d^2),
 *          grad_s (device float64[1], optional) = dL/ds
 *            = -sum_i g_i sum_j w_j exp(-s d^2) d^2.
 *   LJ:    grad_pos4 = dL/dx_i = sum_j 1/2 (g_i + g_j) C_ij dx_ij,
 *          C = eps (12 (sig/d)^12 - 6 (sig/d)^6) / d^2; with g = 1 this is
 *          minus the force on particle i.  grad_w, grad_s unused.
 * Other operators return AB_ERR_UNSUPPORTED.  Optional outputs may be NULL.
 * Errors as ab_pair_sum. */
ab_status ab_pair_sum_bwd(ab_ctx* ctx, ab_op op, const ab_op_params* prm,
                          const float* w, const float* grad_out,
                          float* grad_pos4, float* grad_w, double* grad_s);

/* The forward of ab_pair_sum and its adjoint ab_pair_sum_bwd in one walk
 * over the pairs, for a loss L = sum_i g_i y_i whose upstream gradient
 * g = grad_out is known when the forward runs (a weighted sum of the
 * outputs, or any step that needs the value and the gradient together).
 * The pair terms and their derivatives share the predicate, the separation
 * and the kernel value; every output is bit for bit that of ab_pair_sum
 * followed by ab_pair_sum_bwd on the same cell list.
 *   GAUSS: out = y (float32[n]); grad_pos4, grad_w, grad_s as
 *          ab_pair_sum_bwd; energy unused.
 *   LJ:    out = E_i (float32[n]); energy (device float64[1]) = sum_i E_i;
 *          grad_pos4 as ab_pair_sum_bwd; grad_w, grad_s unused.
 * w, grad_out as ab_pair_sum_bwd.  Every output is optional (NULL).
 * Errors: AB_ERR_UNSUPPORTED (other operators), AB_ERR_ALIAS (an output
 * overlaps an input or another output), AB_ERR_STALE, AB_ERR_INVALID_ARG,
 * AB_ERR_OOM, AB_ERR_CUDA. */
ab_status ab_pair_sum_value_grad(ab_ctx* ctx, ab_op op, const ab_op_params* prm,
                                 const float* w, const float* grad_out, float* out,
                                 double* energy, float* grad_pos4, float* grad_w,
                                 double* grad_s);

/* A pair energy and the gradient of its total in one walk over the pairs:
 * the loss is L = sum_i E_i, so every upstream gradient is 1 and the forward
 * and the adjoint can share the predicate and the powers of sig/d (the
 * common molecular-dynamics step: energies and forces together).
 *   LJ only.  E (device float32[n], optional): E_i as ab_pair_sum;
 *   grad_pos4 (device float32[n][4], optional, 16-byte aligned):
 *     dL/dx_i as ab_pair_sum_bwd with grad_out = 1 (minus the force);
 *   energy (device float64[1], optional): sum_i E_i.
 * Bit for bit the results of ab_pair_sum (LJ) and of ab_pair_sum_bwd (LJ)
 * with a grad_out of ones.
 * Errors: AB_ERR_UNSUPPORTED (op other than LJ), AB_ERR_STALE,
 * AB_ERR_INVALID_ARG, AB_ERR_ALIAS (outputs overlap), AB_ERR_OOM,
 * AB_ERR_CUDA. */
ab_status ab_pair_energy_grad(ab_ctx* ctx, ab_op op, const ab_op_params* prm,
                              float* E, float* grad_pos4, double* energy);

/* ab_pair_energy_grad with the gradient packed as dim floats per particle:
 * grad_pos (device float32[n][dim], optional, 4-byte aligned), the same
 * values as the first dim components of grad_pos4.  Errors as
 * ab_pair_energy_grad. */
ab_status ab_pair_energy_grad_packed(ab_ctx* ctx, ab_op op, const ab_op_params* prm,
                                     float* E, float* grad_pos, double* energy);

/* Export the neighbour relation of the last cell list as CSR in the
 * caller's particle order: offsets (device int64[n+1]) and idx (device
 * int32[cap]) holding original indices of the neighbours of each particle,
 * in the library's deterministic traversal order (not sorted by j).
 * *nnz (host) receives the number of pairs (ordered, both directions).
 * This call synchronises the stream to read the pair count.
 * Errors: AB_ERR_CAPACITY if nnz > cap (offsets are still written),
 * AB_ERR_STALE, AB_ERR_INVALID_ARG, AB_ERR_OOM, AB_ERR_CUDA. */
ab_status ab_pair_list(ab_ctx* ctx, int64_t* offsets, int32_t* idx,
                       int64_t cap, int64_t* nnz);

/* Dense kernel operator (RBF interpolation / Gaussian processes, Sec. 1.1;
 * dense global operators, Sec. 2.2.2):
 *   out[i][c] = sum_j exp(-s |x_i - y_j|^2) W[j][c]
 *   X: float32[m][4] (x, y, z, pad; pad ignored), Y: float32[n][4],
 *   W: float32[n][nrhs] row-major, out: float32[m][nrhs].
 *   prec selects FP32 CUDA cores or a tensor-core split (see ab_prec).
 * Limits: 1 <= nrhs <= 64 for AB_PREC_FP32; nrhs == 64 for tensor-core
 * precisions.  Errors: AB_ERR_INVALID_ARG, AB_ERR_ALIAS, AB_ERR_UNSUPPORTED,
 * AB_ERR_CUDA. */
ab_status ab_kernel_matvec(ab_ctx* ctx, int64_t m, int64_t n, const float* X,
                           const float* Y, int32_t nrhs, const float* W,
                           float s, ab_prec prec, float* out);

/* Adjoint of ab_kernel_matvec for G = dL/dout (float32[m][nrhs]):
 *   dW[j][c] = sum_i K_ij G[i][c]                        (float32[n][nrhs])
 *   A_ij = (G_i . W_j) K_ij
 *   dX_i = -2 s sum_j A_ij (x_i - y_j)                   (float32[m][4])
 *   dY_j = +2 s sum_i A_ij (x_i - y_j)                   (float32[n][4])
 *   ds   = -sum_ij A_ij |x_i - y_j|^2                    (device float64[1])
 * Any output may be NULL.  For a lengthscale l with s = 1/(2 l^2) the
 * caller forms dl = ds * (-1/l^3).  Errors as ab_kernel_matvec. */
ab_status ab_kernel_matvec_bwd(ab_ctx* ctx, int64_t m, int64_t n,
                               const float* X, const float* Y, int32_t nrhs,
                               const float* W, float s, ab_prec prec,
                               const float* G, float* dW, float* dX,
                               float* dY, double* ds);

/* One Euler-Maruyama Brownian-dynamics step (Brownian dynamics, Sec. 1 and
 * Sec. 2.2.1), in place on pos4:
 *   x_k += dt F_k + sqrt(2 D dt) z_k
 * with z from Philox4x64-10 (Salmon et al., SC'11), counter
 * (i, step, 0, 0), key (seed, 0), and the Box-Muller transform of
 * u = ((word >> 40) + 1) 2^-24 (words 0,1 give z_0, z_1; words 2,3 give z_2).
 * Periodic axes wrap into [lo, hi); non-periodic axes reflect once at the
 * walls.  force4: float32[n][4] (may be NULL for free diffusion).  If pos4
 * is the array of the last ab_build, the cell list is marked stale.
 * Errors: AB_ERR_INVALID_ARG, AB_ERR_ALIAS (force4 overlaps pos4),
 * AB_ERR_CUDA. */
ab_status ab_bd_step(ab_ctx* ctx, const ab_domain* dom, int64_t n,
                     float* pos4, const float* force4, float dt, float D,
                     uint64_t seed, uint64_t step);

/* Solve (K(X, X) + sigma2 I) W = B for W, K_ij = exp(-s |x_i - x_j|^2): the
 * linear system of RBF interpolation with a nugget and of the Gaussian-
 * process posterior mean (paper Sec. 1.1; Rasmussen and Williams, Ch. 2).
 * Conjugate gradients (Hestenes and Stiefel), one independent iteration per
 * right-hand side, from W = 0; each iteration is one ab_kernel_matvec of the
 * chosen precision plus per-column FP64 inner products reduced in a fixed
 * order (run-to-run deterministic).  A column stops when
 * ||r|| <= tol ||b|| (r the recurrence residual); the call returns when all
 * have stopped or after max_iter iterations.
 *   n, X:   points, device float32[n][4] (16-byte aligned).
 *   nrhs, B: device float32[n][nrhs] right-hand sides; nrhs <= 64, and
 *           exactly 64 for the tensor-core precisions.
 *   s:      kernel scale; sigma2: the nugget sigma^2 >= 0 (sigma2 > 0 keeps
 *           the system well conditioned).
 *   W:      device float32[n][nrhs], the solution (overwritten).
 *   iters, relres: optional host outputs, the iterations run and the largest
 *           ||r||/||b|| over the columns.
 * Synchronises the context's stream once per iteration (the stopping test).
 * Errors: AB_ERR_INVALID_ARG, AB_ERR_ALIAS (W overlaps X or B),
 * AB_ERR_UNSUPPORTED, AB_ERR_OOM, AB_ERR_CUDA. */
ab_status ab_kernel_solve(ab_ctx* ctx, int64_t n, const float* X, int32_t nrhs,
                          const float* B, float s, float sigma2, ab_prec prec,
                          float tol, int32_t max_iter, float* W, int32_t* iters,
                          float* relres);

/* One step of the semi-implicit (symplectic) Euler integrator of the paper's
 * molecular-dynamics example (Sec. 3, Eqs. 2-3), with step dt (the paper
 * uses dt = 1 and folds the constant c into the force):
 *   v_i <- v_i + dt a_i,   x_i <- x_i + dt v_i   (the updated v_i),
 * a_i being for example the EXPF pair sum of ab_pair_sum (Eq. 1).
 *   dom:   the domain; periodic axes wrap into [lo, hi) (a value that rounds
 *          to hi becomes lo); on a non-periodic axis a particle that leaves
 *          [lo, hi] is reflected once at the wall and that component of its
 *          velocity reversed.
 *   pos4, vel4: device float32[n][4], updated in place (x, y, z; the fourth
 *          component and unused axes are left unchanged).
 *   acc4:  device float32[n][4], read only.
 * Arithmetic: FP32, each product and sum rounded separately (no FMA).
 * If pos4 is the array of the last ab_build, the cell list is marked stale.
 * Errors: AB_ERR_INVALID_ARG (NULL or unaligned arrays, non-finite dt,
 * bad domain), AB_ERR_ALIAS (any two arrays overlap), AB_ERR_CUDA. */
ab_status ab_md_step(ab_ctx* ctx, const ab_domain* dom, int64_t n,
                     float* pos4, float* vel4, const float* acc4, float dt);

/* Allocation-free exclusive prefix sum of n uint32 values (the paper has no
 * counterpart: this is a service for callers that cannot allocate device
 * memory).  out[k] = in[0] + ... + in[k-1] for 0 <= k < n, wrapping modulo
 * 2^32; in may equal out (in place), other overlaps return AB_ERR_ALIAS.
 * Scanning the n_cells + 1 cell counts of a cell list, the last one zero,
 * gives the cell_start table that ab_build computes.
 *
 * Who needs it: code that must not call cudaMalloc or any allocating routine
 * -- for example a caller whose device memory is entirely owned by its own
 * pool or a framework's caching allocator (a raw cudaMalloc would bypass the
 * pool's accounting and can synchronise the device), a real-time or
 * embedded loop with a fixed memory budget fixed at start-up, or code that
 * has no ab_ctx because creating one allocates.  The look-back state this
 * scan needs lives in a file-scope __device__ array of about 32 KB that every
 * GPU which loads the library keeps until the process exits; nothing is
 * allocated or freed by this call.
 *
 *   in, out: device uint32 pointers on the current device, 4-byte aligned.
 *   n:       0 <= n <= 16,777,216 (2^24); larger n returns
 *            AB_ERR_INVALID_ARG.
 *   stream:  cudaStream_t the work is issued on (NULL = legacy stream).
 * The first call on each device looks up the array's device address
 * (cudaGetSymbolAddress, with that device current); make that first call
 * before any stream capture.  Every call shares the one array and resets
 * the part it uses on its stream before the scan, so calls that overlap on
 * the GPU (different streams, no ordering between them) race and give
 * wrong results.  The call is asynchronous.  If a bounded device-side wait
 * gives up (not expected in practice: it waits at most one second for a
 * tile that is already running), out[0] is set to 0xFFFFFFFF, a value an
 * exclusive scan never produces there.  Errors: AB_ERR_INVALID_ARG,
 * AB_ERR_ALIAS, AB_ERR_CUDA. */
ab_status ab_exclusive_scan_u32_static(const uint32_t* in, uint32_t* out,
                                       int64_t n, void* stream);

/* Static description of a status code (never NULL). */
const char* ab_status_string(ab_status status);

/* Human-readable detail of the last error on this context ("" if none). */
const char* ab_last_error(ab_ctx* ctx);

#ifdef __cplusplus
}
#endif

#endif /* ABORIA_GPU_H */
